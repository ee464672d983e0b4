"""Pins for the FP64 oracle: each test ties the oracle to something other than
itself -- hand-worked values, brute force, closed forms, library routines
(LAPACK QR with column pivoting, torch autograd) or invariants the paper proves.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg

import css_inputs as ci
from oracle import css_oracle as O


def _load(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as fh:
        return json.load(fh)


# ----------------------------------------------------------------- golden ---
def test_hand_css_2x3(golden_dir):
    d = _load(golden_dir, "hand_css_2x3.json")
    A = np.array(d["A"])
    r = O.greedy_css(A, d["k"], keep_scores=True)
    assert r.S == d["S"]
    np.testing.assert_allclose(r.trace, d["trace"], atol=1e-12)
    np.testing.assert_allclose(r.scores[0], d["scores_t1"], rtol=1e-12)
    for i, v in d["scores_t2_candidates"].items():
        assert abs(r.scores[1][int(i)] - v) < 1e-12
    # residual-matrix form (Problem 3 + Lemma 2) gives the same
    r2 = O.greedy_css_residual(A, d["k"])
    assert r2.S == d["S"]
    np.testing.assert_allclose(r2.trace, d["trace"], atol=1e-12)


def test_hand_gcss_2x2(golden_dir):
    d = _load(golden_dir, "hand_gcss_2x2.json")
    A, B = np.array(d["A"]), np.array(d["B"])
    r = O.greedy_gcss(A, B, d["k"])
    assert r.S == d["S"]
    np.testing.assert_allclose(r.trace, d["trace"], atol=1e-12)
    r1 = O.greedy_gcss(A, B, 1)
    np.testing.assert_allclose(r1.f, d["f1"], atol=1e-12)


def test_hand_orthogonal(golden_dir):
    d = _load(golden_dir, "hand_orthogonal_3x3.json")
    A = np.array(d["A"])
    r = O.greedy_css(A, d["k"], keep_scores=True)
    assert r.S == d["S"]
    np.testing.assert_allclose(r.trace, d["trace"], atol=1e-12)
    g0 = np.sum(A * A, axis=0)
    np.testing.assert_allclose(r.scores[0] * g0, d["f0"], rtol=1e-12)


# ------------------------------------------------------------ brute force ---
@pytest.mark.parametrize("seed", [11, 12, 13])
def test_each_step_is_the_one_step_argmin(seed):
    """Problem 2: every greedy pick minimises F(S u {i}) over all candidates i,
    with F evaluated directly (Eq. Projection)."""
    A = ci.lowrank_uv(9, 14, 4, 0.05, seed)
    r = O.greedy_css(A, 7)
    for t, p in enumerate(r.S):
        prefix = r.S[:t]
        errs = {i: O.reconstruction_error(A, prefix + [i])
                for i in range(A.shape[1]) if i not in prefix}
        best = min(errs.values())
        assert errs[p] <= best * (1 + 1e-9) + 1e-12, (t, p, errs[p], best)


@pytest.mark.parametrize("seed", [21, 22])
def test_gcss_each_step_is_the_one_step_argmin(seed):
    """Problem 5: every GCSS pick minimises ||B - P^(S u {i}) B||^2."""
    A = ci.lowrank_uv(8, 13, 5, 0.1, seed)
    B = ci.lowrank_uv(8, 3, 2, 0.1, seed + 100)
    r = O.greedy_gcss(A, B, 6)
    for t, p in enumerate(r.S):
        prefix = r.S[:t]
        errs = {i: O.reconstruction_error(A, prefix + [i], B)
                for i in range(A.shape[1]) if i not in prefix}
        best = min(errs.values())
        assert errs[p] <= best * (1 + 1e-9) + 1e-12


def test_k_subset_brute_force_on_config_slice():
    """Rows 0-11, cols 0-15 of the 500 x 1000 FP64 workload, k = 3: the greedy
    set can never beat the optimum of Problem 1; equality when they coincide."""
    c = ci.CONFIGS["fp64_500x1000"]
    A = ci.lowrank_uv(c["m"], c["n"], c["rank"], c["noise"], c["seed"])[:12, :16]
    best_S, best_err = O.brute_force_css(A, 3)
    r = O.greedy_css(A, 3)
    g_err = O.reconstruction_error(A, r.S)
    assert g_err >= best_err * (1 - 1e-12)
    if tuple(sorted(r.S)) == best_S:
        assert abs(g_err - best_err) <= 1e-9 * best_err
    assert g_err / best_err < 2.0   # report-level sanity on this slice


# -------------------------------------------------------------- recursion ---
def test_recursive_error_equals_direct_error_every_step():
    """Theorem 1: the trace F^(t) = F^(t-1) - f_p/g_p equals ||A - P^(S)A||^2."""
    A = ci.lowrank_uv(60, 120, 10, 0.01, 3)
    r = O.greedy_css(A, 20)
    for t in range(len(r.S) + 1):
        d = O.reconstruction_error(A, r.S[:t])
        assert abs(r.trace[t] - d) <= 1e-8 * r.trace[0], t


@pytest.mark.slow
def test_recursive_error_fp64_config_full():
    """Theorem 1 on the full 500 x 1000 FP64 workload, k = 50, every step."""
    c = ci.CONFIGS["fp64_500x1000"]
    A = ci.lowrank_uv(c["m"], c["n"], c["rank"], c["noise"], c["seed"])
    r = O.greedy_css(A, c["k"])
    assert len(r.S) == c["k"]
    for t in range(0, c["k"] + 1):
        d = O.reconstruction_error(A, r.S[:t])
        assert abs(r.trace[t] - d) <= 1e-9 * r.trace[0], t
    # Eckart-Young: no rank-k column-based approximation beats the SVD tail
    sv = np.linalg.svd(A, compute_uv=False)
    tail = float(np.sum(sv[c["k"]:] ** 2))
    assert r.trace[-1] >= tail * (1 - 1e-9)
    assert r.trace[-1] < 1e-3 * r.trace[0]


def test_gcss_recursive_error_equals_direct():
    """Theorem 3: Fbar^(t) equals ||B - P^(S)B||^2 after every step."""
    A = ci.lowrank_uv(40, 90, 8, 0.02, 5)
    Om = ci.gaussian_omega(90, 6, 6, dtype=np.float64)
    B = A @ Om
    r = O.greedy_gcss(A, B, 12)
    for t in range(len(r.S) + 1):
        d = O.reconstruction_error(A, r.S[:t], B)
        assert abs(r.trace[t] - d) <= 1e-8 * r.trace[0] + 1e-12, t


def test_direct_error_two_ways():
    A = ci.lowrank_uv(30, 40, 30, 0.0, 8)
    S = [3, 7, 11, 19]
    a = O.reconstruction_error(A, S)
    b = O.reconstruction_error_normal_eq(A, S)
    assert abs(a - b) <= 1e-10 * a


# ------------------------------------------------------------- invariants ---
def test_invariants():
    A = ci.lowrank_uv(50, 80, 12, 0.01, 9)
    r = O.greedy_css(A, 25, keep_scores=True)
    tr = np.array(r.trace)
    assert np.all(np.diff(tr) <= 1e-9 * tr[0])                 # monotone
    W = r.W
    for t, p in enumerate(r.S):
        # omega^(r)_{p_s} = 0 for s < r  (W Pi upper triangular, Sec. 6)
        for s in range(t):
            assert abs(W[t, r.S[s]]) <= 1e-9 * np.abs(W[t]).max()
    # omega^(t)_p = sqrt(g_p) at selection: rebuild from the rows of W
    g0 = np.sum(A * A, axis=0)
    for t, p in enumerate(r.S):
        g_before = g0[p] - np.sum(W[:t, p] ** 2)
        assert abs(W[t, p] - np.sqrt(g_before)) <= 1e-9 * np.sqrt(g0[p])
    # f_i >= g_i^2 (Cauchy-Schwarz on G_:i) for the unselected columns; the
    # selected ones are zero up to rounding of f^(0)
    sel = np.zeros(A.shape[1], dtype=bool)
    sel[r.S] = True
    assert np.all(r.f[~sel] >= r.g[~sel] ** 2 * (1 - 1e-9))
    f0 = np.einsum("ij,ij->j", A, (A @ A.T) @ A)
    assert np.all(np.abs(r.f[sel]) <= 1e-12 * f0.max())


def test_rank_r_reaches_zero_at_k_equals_r():
    A = ci.lowrank_uv(40, 70, 9, 0.0, 10)
    r = O.greedy_css(A, 9)
    assert r.trace[-1] <= 1e-12 * r.trace[0]
    assert O.reconstruction_error(A, r.S) <= 1e-12 * r.trace[0]


def test_rank_exhaustion_stops_early():
    A = ci.lowrank_uv(20, 30, 4, 0.0, 14)
    r = O.greedy_css(A, 10, tau_rel=1e-10)
    assert len(r.S) == 4


# ---------------------------------------------------------- special cases ---
def test_norm_score_reproduces_qr_with_column_pivoting():
    """With the criterion replaced by g_i the recursion is QR with column
    pivoting (Businger-Golub); LAPACK dgeqp3 via scipy gives the order."""
    A = ci.lowrank_uv(30, 25, 25, 0.0, 15)
    _, _, piv = scipy.linalg.qr(A, pivoting=True, mode="economic")
    r = O.greedy_css(A, 10, score="norm")
    assert r.S == list(piv[:10])


def test_gcss_with_B_equal_A_is_css():
    A = ci.lowrank_uv(25, 40, 6, 0.05, 16)
    a = O.greedy_css(A, 10)
    b = O.greedy_gcss(A, A, 10)
    assert a.S == b.S
    np.testing.assert_allclose(a.trace, b.trace, rtol=1e-9)


def test_scale_invariance():
    A = ci.lowrank_uv(25, 40, 6, 0.05, 17)
    a = O.greedy_css(A, 8)
    b = O.greedy_css(3.0 * A, 8)
    assert a.S == b.S
    np.testing.assert_allclose(np.array(b.trace), 9.0 * np.array(a.trace), rtol=1e-9)
    B = ci.lowrank_uv(25, 5, 3, 0.1, 18)
    c = O.greedy_gcss(A, B, 8)
    d = O.greedy_gcss(A, 0.5 * B, 8)
    assert c.S == d.S


def test_permutation_equivariance():
    A = ci.lowrank_uv(25, 40, 6, 0.05, 19)
    perm = np.random.default_rng(0).permutation(40)
    a = O.greedy_css(A, 8)
    b = O.greedy_css(A[:, perm], 8)
    assert [int(perm[j]) for j in b.S] == a.S


def test_residual_form_matches_memory_efficient_form():
    A = ci.lowrank_uv(15, 22, 5, 0.05, 20)
    a = O.greedy_css(A, 10)
    b = O.greedy_css_residual(A, 10)
    assert a.S == b.S
    np.testing.assert_allclose(a.trace, b.trace, rtol=0, atol=1e-11 * a.trace[0])


def test_exact_scores_match_recursion():
    A = ci.lowrank_uv(30, 50, 7, 0.05, 23)
    r = O.greedy_css(A, 6, keep_scores=True)
    for t in range(len(r.S)):
        f, g = O.exact_scores(A, r.S[:t])
        cand = np.isfinite(r.scores[t])
        np.testing.assert_allclose(r.scores[t][cand],
                                   np.maximum(f[cand], 0) / g[cand], rtol=1e-8)


def test_exact_gcss_scores_match_recursion():
    """Theorem 4's recursive scores at every step equal Problem 5's definition
    for the prefix: ||B^T (I - P) a_i||^2 / ||(I - P) a_i||^2."""
    A = ci.lowrank_uv(30, 50, 7, 0.05, 26)
    B = ci.lowrank_uv(30, 9, 4, 0.05, 27)
    r = O.greedy_gcss(A, B, 6, keep_scores=True)
    assert len(r.S) == 6
    for t in range(len(r.S)):
        f, g = O.exact_gcss_scores(A, B, r.S[:t])
        cand = np.isfinite(r.scores[t])
        assert cand.sum() == 50 - t
        np.testing.assert_allclose(r.scores[t][cand],
                                   np.maximum(f[cand], 0) / g[cand], rtol=1e-8)


# ------------------------------------------------------- random projection ---
def test_random_projection_blocks_equal_product():
    A = ci.lowrank_uv(12, 50, 4, 0.1, 24)
    Om = ci.gaussian_omega(50, 5, 25, dtype=np.float64)
    B1 = O.random_projection(A, Om, [0, 7, 19, 50])
    # brute force: the per-column outer-product sum of Sec. 5.1
    B2 = np.zeros((12, 5))
    for i in range(50):
        B2 += np.outer(A[:, i], Om[i, :])
    np.testing.assert_allclose(B1, B2, rtol=1e-12, atol=1e-12)


def test_gaussian_omega_variance():
    Om = ci.gaussian_omega(20000, 40, 2, dtype=np.float64)
    assert abs(Om.var() * 40 - 1.0) < 0.02


# ------------------------------------------------------------ distributed ---
def test_distributed_single_block_is_gcss_set():
    A = ci.lowrank_uv(20, 60, 6, 0.05, 26)
    B = A @ ci.gaussian_omega(60, 8, 27, dtype=np.float64)
    final, per_block, _ = O.distributed_css(A, B, [0, 60], 10, 10)
    ref = O.greedy_gcss(A, B, 10)
    assert per_block[0] == ref.S
    assert sorted(final) == sorted(ref.S)


def test_distributed_union_order_and_ids():
    A = ci.lowrank_uv(20, 90, 6, 0.05, 28)
    B = A @ ci.gaussian_omega(90, 8, 29, dtype=np.float64)
    offs = [0, 25, 40, 90]
    final, per_block, r0 = O.distributed_css(A, B, offs, 4, 5)
    for b, ids in enumerate(per_block):
        assert all(offs[b] <= j < offs[b + 1] for j in ids)
        loc = O.greedy_gcss(A[:, offs[b]:offs[b + 1]], B, 4)
        assert [offs[b] + j for j in loc.S] == ids
    union = [j for ids in per_block for j in ids]
    assert set(final) <= set(union) and len(final) == 5
    # reading 8: the union step's f0/g0 equal the blocks' values
    f0 = np.sum((B.T @ A[:, union]) ** 2, axis=0)
    r_union = O.greedy_gcss(A[:, union], B, 0)
    assert r_union.f is not None
    np.testing.assert_allclose(r_union.f, f0, rtol=1e-12)


def test_lognormal_blocks():
    offs = ci.lognormal_blocks(262144, 64, 3000, 0.8, 3)
    w = np.diff(offs)
    assert offs[0] == 0 and offs[-1] == 262144 and len(w) == 64
    assert w.min() >= 100


# ---------------------------------------------------------------- adjoint ---
def test_residual_gradient_finite_differences():
    rng = np.random.default_rng(30)
    A = rng.standard_normal((9, 12))
    S = [1, 4, 7]
    L, G = O.residual_gradient(A, S)
    assert abs(L - O.reconstruction_error(A, S)) <= 1e-10 * L
    h = 1e-6
    for (i, j) in [(0, 1), (3, 4), (8, 7), (2, 0), (5, 11), (6, 3)]:
        Ap, Am = A.copy(), A.copy()
        Ap[i, j] += h
        Am[i, j] -= h
        fd = (O.reconstruction_error(Ap, S) - O.reconstruction_error(Am, S)) / (2 * h)
        assert abs(fd - G[i, j]) <= 1e-6 * max(1.0, abs(fd)), (i, j, fd, G[i, j])


def test_residual_gradient_against_torch_autograd():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(31)
    A = rng.standard_normal((16, 24))
    S = [0, 5, 9, 17, 23]
    _, G = O.residual_gradient(A, S)
    At = torch.tensor(A, requires_grad=True)
    AS = At[:, S]
    T = torch.linalg.solve(AS.T @ AS, AS.T @ At)
    L = ((At - AS @ T) ** 2).sum()
    L.backward()
    np.testing.assert_allclose(G, At.grad.numpy(), rtol=1e-9, atol=1e-9)


# ----------------------------------------------------------------- inputs ---
def test_bf16_rounding():
    x = np.array([1.0, 1.00390625, 1.005859375, -2.5, 3.1415927], dtype=np.float32)
    b = ci.round_bf16(x)
    # 1 + 2^-8 is the tie between 1 and 1 + 2^-7 -> even (1.0);
    # 1 + 1.5 * 2^-8 rounds up to 1 + 2^-7
    np.testing.assert_array_equal(b[:4], np.array([1.0, 1.0, 1.0078125, -2.5], np.float32))
    assert abs(b[4] - 3.140625) == 0


# --------------------------------------------------------------------------- #
# Omega from Philox4x32-10 (Sec. 5.1's random matrices)
# --------------------------------------------------------------------------- #
# Known-answer vectors published with the generator (Salmon et al., SC 2011,
# Random123 distribution): (counter, key) -> output.
PHILOX_KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF, 0xFFFFFFFF), (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,out", PHILOX_KAT)
def test_philox_known_answers(ctr, key, out):
    got = O.philox4x32_10(tuple(np.uint32(c) for c in ctr), key)
    assert tuple(int(x) for x in got) == out


def test_gaussian_omega_moments_and_independence():
    n, r = 4000, 50
    W = O.random_omega(n, r, 2024, O.OMEGA_GAUSSIAN)
    N = W.size
    # N(0, 1/r): mean within 5 standard errors, variance within 5 s.e. of 1/r
    assert abs(W.mean()) < 5 / np.sqrt(N * r)
    var_se = np.sqrt(2.0 / N) / r
    assert abs(W.var() - 1.0 / r) < 5 * var_se
    # fourth moment of a Gaussian: 3 sigma^4
    k4 = np.mean((W * np.sqrt(r)) ** 4)
    assert abs(k4 - 3.0) < 0.15
    # columns uncorrelated
    Cc = np.corrcoef(W[:, :8].T)
    assert np.max(np.abs(Cc - np.eye(8))) < 5 / np.sqrt(n)


def test_omega_entries_depend_only_on_position_and_seed():
    A = O.random_omega(300, 20, 7, O.OMEGA_GAUSSIAN)
    B = O.random_omega(500, 30, 7, O.OMEGA_GAUSSIAN)
    # the same draws; only the 1/sqrt(r) scale differs
    np.testing.assert_allclose(A * np.sqrt(20.0), B[:300, :20] * np.sqrt(30.0), rtol=1e-14, atol=0)
    C = O.random_omega(300, 20, 8, O.OMEGA_GAUSSIAN)
    assert np.mean(A == C) < 1e-3
    D = O.random_omega(300, 20, 7 + (1 << 32), O.OMEGA_GAUSSIAN)   # high key word matters
    assert np.mean(A == D) < 1e-3


def test_sparse_sign_omega():
    n, r = 40000, 60
    S = O.random_omega(n, r, 99, O.OMEGA_SPARSE_SIGN)
    assert set(np.unique(S)) <= {-1.0, 0.0, 1.0}
    p = 1.0 / np.sqrt(n)
    nnz = np.count_nonzero(S)
    assert abs(nnz - p * S.size) < 5 * np.sqrt(S.size * p * (1 - p))
    plus = np.count_nonzero(S > 0)
    assert abs(plus - nnz / 2) < 5 * np.sqrt(nnz / 4)
    # the threshold is floor(2^32 / sqrt n): for n = 4 exactly half of the draws
    assert O.sparse_sign_threshold(4) == 1 << 31
    assert O.sparse_sign_threshold(1) == 0xFFFFFFFF


def test_rnd_greedy_recovers_the_column_space_of_a_rank_l_matrix():
    """With r = l = rank(A), B = A Omega spans range(A) (almost surely), so the
    l columns RndGreedyCSS picks reconstruct A exactly (Theorem 3's trace
    reaches 0), for both random matrices of Sec. 5.1."""
    A = ci.lowrank_uv(40, 120, 6, 0.0, 3)
    for dist in (O.OMEGA_GAUSSIAN, O.OMEGA_SPARSE_SIGN):
        res = O.rnd_greedy_css(A, 6, seed=11, dist=dist)
        assert len(res.S) == 6
        assert O.reconstruction_error(A, res.S) <= 1e-18 * np.linalg.norm(A) ** 2


def test_relative_accuracy_end_points():
    assert O.relative_accuracy(5.0, 5.0, 2.0) == 0.0       # as good as uniform sampling
    assert O.relative_accuracy(2.0, 5.0, 2.0) == 100.0     # as good as the SVD
    assert O.relative_accuracy(3.5, 5.0, 2.0) == 50.0


# ------------------------------------------- Sec. 3.2: embedding, rank k ---
def test_embedding_rows_are_the_greedy_omegas():
    """W = Q^T A with Q from a Householder QR equals the omega history the
    greedy recursion builds (Eq. delta_omega): two unrelated computations of
    the same rows; W[:, S] is the upper-triangular R with a positive
    diagonal (the Q-less QR structure of the selection)."""
    A = ci.lowrank_uv(30, 50, 5, 0.05, 11)
    r = O.greedy_css(A, 8)
    Q, W, R = O.embedding(A, r.S)
    np.testing.assert_allclose(W, r.W, atol=1e-10 * np.abs(r.W).max())
    np.testing.assert_allclose(W[:, r.S], R, atol=1e-12 * np.abs(R).max())
    assert np.all(np.diag(R) > 0)
    assert np.allclose(np.tril(W[:, r.S], -1), 0.0, atol=1e-12 * np.abs(R).max())
    np.testing.assert_allclose(Q.T @ Q, np.eye(len(r.S)), atol=1e-13)


def test_embedding_projection_is_the_normal_equations_projection():
    """Q Q^T A = A_S (A_S^T A_S)^-1 A_S^T A (Eq. Projection), and
    ||A||^2 - ||W||^2 = F(S) from the normal equations."""
    A = ci.lowrank_uv(40, 70, 6, 0.1, 12)
    S = [3, 17, 5, 60, 41, 22, 9]
    Q, W, _ = O.embedding(A, S)
    AS = A[:, S]
    PA = AS @ np.linalg.solve(AS.T @ AS, AS.T @ A)
    np.testing.assert_allclose(Q @ W, PA, atol=1e-11 * np.abs(A).max())
    F = O.reconstruction_error_normal_eq(A, S)
    assert abs(np.sum(A * A) - np.sum(W * W) - F) <= 1e-10 * np.sum(A * A)


@pytest.mark.parametrize("k", [1, 3, 7])
def test_rank_k_is_the_best_rank_k_of_the_projection(k):
    """A~_{S,k} = Q W~_k is the best rank-k approximation of P^(S) A (Q has
    orthonormal columns), computed here by an SVD of the m x n matrix P^(S) A
    formed through the normal equations -- a different path -- and the error
    splits as ||A - A~_{S,k}||^2 = F(S) + sum_{i>=k} sigma_i(W)^2."""
    A = ci.lowrank_uv(35, 60, 8, 0.05, 13)
    S = O.greedy_css(A, 7).S
    Q, W, _ = O.embedding(A, S)
    out = O.rank_k_approximation(Q, W, k)
    AS = A[:, S]
    PA = AS @ np.linalg.solve(AS.T @ AS, AS.T @ A)
    U, s, Vt = np.linalg.svd(PA, full_matrices=False)
    best = (U[:, :k] * s[:k]) @ Vt[:k]
    Ak = Q @ out["Wk"]
    np.testing.assert_allclose(Ak, best, atol=1e-10 * np.abs(A).max())
    np.testing.assert_allclose(out["sigma"], s[:k], rtol=1e-12)
    err = np.sum((A - Ak) ** 2)
    assert abs(err - (O.reconstruction_error(A, S) + out["tail"])) <= 1e-10 * np.sum(A * A)


def test_rank_k_is_locally_optimal_over_rank_k_coefficients():
    """No rank-k coefficient matrix T near the optimum gives a smaller
    ||A - A_S T||_F (the minimisation Sec. 3.2 states): perturbations of T*
    kept at rank k by truncation never improve on it."""
    rng = np.random.default_rng(14)
    A = ci.lowrank_uv(20, 30, 6, 0.1, 14)
    S = [0, 4, 9, 13, 21]
    k = 2
    Q, W, _ = O.embedding(A, S)
    out = O.rank_k_approximation(Q, W, k)
    AS = A[:, S]
    T_star = np.linalg.lstsq(AS, Q @ out["Wk"], rcond=None)[0]
    best = np.sum((A - AS @ T_star) ** 2)
    for _ in range(200):
        T = T_star + 1e-3 * rng.standard_normal(T_star.shape)
        u, s, vt = np.linalg.svd(T, full_matrices=False)
        Tk = (u[:, :k] * s[:k]) @ vt[:k]
        assert np.sum((A - AS @ Tk) ** 2) >= best * (1 - 1e-12)


def test_approximate_svd_is_exact_when_the_selection_spans_A():
    """A of exact rank 4 and a selection spanning its range: P^(S) A = A, so
    Eq. (ApproxSVD) returns A's own leading singular triplets and
    A~_{S,k} is A's best rank-k approximation (Eckart-Young)."""
    U0 = np.linalg.qr(np.random.default_rng(15).standard_normal((25, 4)))[0]
    V0 = np.linalg.qr(np.random.default_rng(16).standard_normal((40, 4)))[0]
    A = (U0 * np.array([5.0, 3.0, 2.0, 0.5])) @ V0.T
    S = O.greedy_css(A, 4).S
    Q, W, _ = O.embedding(A, S)
    s_true = np.linalg.svd(A, compute_uv=False)
    for k in (2, 4):
        out = O.rank_k_approximation(Q, W, k)
        np.testing.assert_allclose(out["sigma"], s_true[:k], rtol=1e-12)
        Ua, sa, Vta = np.linalg.svd(A)
        best = (Ua[:, :k] * sa[:k]) @ Vta[:k]
        recon = (out["U"] * out["sigma"]) @ out["V"].T
        np.testing.assert_allclose(recon, best, atol=1e-12 * 5.0)
        np.testing.assert_allclose(out["U"].T @ out["U"], np.eye(k), atol=1e-13)
        np.testing.assert_allclose(out["V"].T @ out["V"], np.eye(k), atol=1e-13)


def test_approximate_singular_values_interlace():
    """W = Q^T A compresses A, so sigma_i(W) <= sigma_i(A) for every i
    (Cauchy interlacing); with k = l, A~_{S,l} = P^(S) A."""
    A = ci.lowrank_uv(30, 45, 10, 0.2, 17)
    S = O.greedy_css(A, 6).S
    Q, W, _ = O.embedding(A, S)
    out = O.rank_k_approximation(Q, W, len(S))
    sA = np.linalg.svd(A, compute_uv=False)
    assert np.all(out["sigma_all"] <= sA[:len(S)] * (1 + 1e-12))
    np.testing.assert_allclose(Q @ out["Wk"], Q @ (Q.T @ A), atol=1e-12 * np.abs(A).max())
    assert out["tail"] == 0.0 or out["tail"] < 1e-20
