"""Sec. 3.2 on the device against the oracle: the embedding Q = orth(A_S),
W = Q^T A (css_embed, and the basis / omega rows css_select returns), and the
rank-k approximation with the approximate SVD of Eq. (ApproxSVD)
(css_lowrank)."""
import numpy as np
import pytest
import torch

import css_inputs as ci
from oracle import css_oracle as O
from tests.gpu_helpers import dev_matrix

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def css():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_6838_gb300 import build, css as mod
    build.build()
    return mod


def _sel(n, l, seed):
    return [int(v) for v in np.random.default_rng(seed).choice(n, size=l, replace=False)]


def _sign_rule(U):
    """Each column signed so that its entry of largest magnitude (lowest index
    on ties) is positive -- the rule css_lowrank documents."""
    U = U.copy()
    for r in range(U.shape[1]):
        i = int(np.argmax(np.abs(U[:, r])))
        if U[i, r] < 0:
            U[:, r] = -U[:, r]
    return U


# ------------------------------------------------------------- css_embed ---
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("shape", [(130, 700, 9), (300, 2000, 33), (64, 64, 64), (1000, 500, 1),
                                   (257, 3001, 100), (400, 2500, 200), (520, 3000, 300)])
def test_embed_matches_oracle(css, dtype, shape):
    """l > 128 takes the blocked Cholesky (7 and 10 panels of 32 columns)."""
    m, n, l = shape
    A, vals = dev_matrix(ci.lowrank_uv(m, n, min(m, n, 2 * l + 5), 0.05, 300 + m), dtype)
    S = _sel(n, l, 17 + n)
    emb = css.embed(A, S)
    Qr, Wr, Rr = O.embedding(vals, S)
    Q = emb.Q.cpu().numpy()
    W = emb.W.cpu().numpy()
    # CholeskyQR2 against Householder: both orthonormal to ~1e-15
    np.testing.assert_allclose(Q, Qr, atol=1e-10)
    np.testing.assert_allclose(Q.T @ Q, np.eye(l), atol=1e-12)
    # W: FP64 products (FP64 input) or double-float (FP32/BF16): per column
    # within 1e-10 ||a_c||
    colnorm = np.linalg.norm(vals, axis=0)
    assert np.all(np.abs(W - Wr) <= 1e-10 * colnorm[None, :] + 1e-300)
    np.testing.assert_allclose(np.tril(W[:, S], -1), 0.0, atol=1e-10 * colnorm.max())
    assert np.all(np.diag(W[:, S]) > 0)


def test_embed_with_padded_leading_dimension(css):
    m, n, l = 100, 900, 12
    A, vals = dev_matrix(ci.lowrank_uv(m, n, 30, 0.05, 77), torch.float32, ld=136)
    assert A.stride(1) == 136
    S = _sel(n, l, 5)
    emb = css.embed(A, S)
    Qr, Wr, _ = O.embedding(vals, S)
    np.testing.assert_allclose(emb.Q.cpu().numpy(), Qr, atol=1e-10)
    colnorm = np.linalg.norm(vals, axis=0)
    assert np.all(np.abs(emb.W.cpu().numpy() - Wr) <= 1e-10 * colnorm[None, :])


def test_gcss_basis_is_the_embedding_of_its_selection(css):
    """gcss_select's basis (opts.basis) and omega rows: W = Q^T A also for
    Algorithm 3 (omega = A^T q whatever the target)."""
    m, n, r, k = 150, 1200, 20, 16
    A, vals = dev_matrix(ci.lowrank_uv(m, n, 2 * k, 0.05, 61), torch.float64)
    B = torch.from_numpy(ci.lowrank_uv(m, r, r, 0.0, 62)).cuda().t().contiguous().t()
    res = css.gcss_select(A, B, k, return_W=True, return_basis=True)
    S = res.indices.cpu().tolist()
    Qr, Wr, _ = O.embedding(vals, S)
    np.testing.assert_allclose(res.basis.cpu().numpy()[:, :len(S)], Qr, atol=1e-9)
    colnorm = np.linalg.norm(vals, axis=0)
    assert np.all(np.abs(res.W.cpu().numpy()[:len(S)] - Wr) <= 1e-9 * colnorm[None, :])


def test_embed_rejects_dependent_and_repeated_columns(css):
    A_np = ci.lowrank_uv(50, 80, 3, 0.0, 5)        # rank 3
    A, _ = dev_matrix(A_np, torch.float64)
    from paper_1312_6838_gb300._lib import CssError
    with pytest.raises(CssError):
        css.embed(A, [0, 1, 2, 3])                 # four columns of a rank-3 matrix
    with pytest.raises(CssError):
        css.embed(A, [4, 7, 4])


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
def test_select_basis_and_omega_rows_form_the_embedding(css, dtype):
    """css_select's own basis (opts.basis) and omega rows are Q and Q^T A of
    its selection (Gram-Schmidt in selection order), equal to css_embed's and
    to the oracle's up to the precision of the selection path."""
    m, n, k = 200, 1500, 24
    A, vals = dev_matrix(ci.lowrank_uv(m, n, 2 * k, 0.05, 41), dtype)
    res = css.select(A, k, return_W=True, return_basis=True)
    S = res.indices.cpu().tolist()
    assert len(S) == k
    Qr, Wr, _ = O.embedding(vals, S)
    Qb = res.basis.cpu().numpy()
    Ws = res.W.cpu().numpy()
    colnorm = np.linalg.norm(vals, axis=0)
    if dtype == torch.float64:
        q_tol, w_tol = 1e-9, 1e-9
    else:
        # FP32 dot products over m rows in the fused step (omega), the basis in
        # double-float from an FP32-accumulated pivot column
        q_tol, w_tol = 1e-4, 2e-5
    np.testing.assert_allclose(Qb, Qr, atol=q_tol)
    assert np.all(np.abs(Ws - Wr) <= w_tol * colnorm[None, :])
    emb = css.embed(A, S)
    np.testing.assert_allclose(emb.Q.cpu().numpy(), Qb, atol=q_tol)
    # columns past the selection are zero when the run stops early
    A0, _ = dev_matrix(ci.lowrank_uv(60, 90, 4, 0.0, 3), torch.float64)
    r0 = css.select(A0, 8, return_basis=True)
    assert r0.n_sel == 4
    assert torch.all(r0.basis[:, 4:] == 0)


# ----------------------------------------------------------- css_lowrank ---
def _lowrank_case(css, vals, S, k):
    Q, W, _ = O.embedding(vals, S)
    ref = O.rank_k_approximation(Q, W, k)
    Qd = torch.from_numpy(Q).cuda().t().contiguous().t()
    Wd = torch.from_numpy(W).cuda().contiguous()
    got = css.lowrank(Wd, k, Qd)
    return Q, W, ref, got


def _check_lowrank(vals, S, Q, W, ref, got, k):
    l, n = W.shape
    w2 = float(np.sum(W * W))
    res_tol = 4.0 * (n + l) * 2.0 ** -52 * w2       # the Gram route's resolution
    sig = got.sigma.cpu().numpy()
    assert np.all(np.diff(sig) <= 0) and np.all(sig >= 0)
    assert np.all(np.abs(sig ** 2 - ref["sigma"] ** 2) <= res_tol)
    assert abs(got.tail - ref["tail"]) <= res_tol * max(1, l - k)
    Uw = got.Uw.cpu().numpy()
    np.testing.assert_allclose(Uw.T @ Uw, np.eye(k), atol=1e-12)
    # the sign rule
    for r in range(k):
        i = int(np.argmax(np.abs(Uw[:, r])))
        assert Uw[i, r] > 0
    s_all = ref["sigma_all"]
    lam = np.concatenate([s_all ** 2, [0.0]])
    for r in range(k):
        gap = min(lam[r - 1] - lam[r] if r > 0 else np.inf, lam[r] - lam[r + 1])
        if gap > 1e-3 * lam[0]:
            # an isolated singular value: the vector itself (Davis-Kahan
            # sin(theta) <= ||dG|| / gap)
            ur = _sign_rule(ref["Uw"])[:, r]
            assert np.max(np.abs(Uw[:, r] - ur)) <= 1e-8 * lam[0] / gap
    if k < l and lam[k - 1] - lam[k] > 1e-3 * lam[0]:
        Pg = Uw @ Uw.T
        Pr = ref["Uw"] @ ref["Uw"].T
        assert np.max(np.abs(Pg - Pr)) <= 1e-8 * lam[0] / (lam[k - 1] - lam[k])
    U = got.U.cpu().numpy()
    np.testing.assert_allclose(U, Q @ Uw, atol=1e-12)
    V = got.V.cpu().numpy()
    keep = sig ** 2 > (n + l) * 2.0 ** -52 * w2
    assert np.all(V[:, ~keep] == 0)
    # V~ = W^T U^(W) / sigma is orthonormal up to ||dG|| / sigma^2
    well = sig ** 2 > 1e-6 * w2
    Vk = V[:, well]
    np.testing.assert_allclose(Vk.T @ Vk, np.eye(int(well.sum())), atol=1e-8)
    # the column-based rank-k approximation: ||A - U~ S~ V~^T||^2 = F(S) + tail
    Ak = (U * sig) @ V.T
    err = float(np.sum((vals - Ak) ** 2))
    want = O.reconstruction_error(vals, S) + ref["tail"]
    assert abs(err - want) <= 1e-9 * float(np.sum(vals * vals))


@pytest.mark.parametrize("shape", [(120, 900, 16, 5), (300, 2000, 33, 33), (200, 1200, 7, 1),
                                   (256, 4000, 100, 40), (80, 5000, 2, 2)])
def test_lowrank_matches_oracle(css, shape):
    m, n, l, k = shape
    vals = ci.lowrank_decaying(m, n, min(m, 3 * l + 4), 1e-3, 500 + l, dtype=np.float64)
    S = O.greedy_css(vals, l).S if l <= 40 else _sel(n, l, 9)
    Q, W, ref, got = _lowrank_case(css, vals, S, k)
    _check_lowrank(vals, S, Q, W, ref, got, k)


def test_lowrank_l_one(css):
    vals = ci.lowrank_uv(40, 300, 5, 0.1, 8)
    Q, W, ref, got = _lowrank_case(css, vals, [17], 1)
    w = W[0]
    assert abs(got.sigma.item() - np.linalg.norm(w)) <= 1e-12 * np.linalg.norm(w)
    assert got.Uw.item() == 1.0
    np.testing.assert_allclose(got.V.cpu().numpy()[:, 0], w / np.linalg.norm(w), atol=1e-13)


def test_lowrank_zero_rows_and_repeated_values(css):
    """Rows of zeros (an embedding of lower rank than l): sigma = 0 and zero
    V columns; equal singular values (orthogonal rows of one norm): every
    sigma equal and U^(W) orthogonal."""
    rng = np.random.default_rng(21)
    n = 700
    Wt = rng.standard_normal((6, n))
    W = np.vstack([Wt, np.zeros((3, n))])
    Wd = torch.from_numpy(W).cuda()
    got = css.lowrank(Wd, 9)
    s_ref = np.linalg.svd(W, compute_uv=False)
    np.testing.assert_allclose(got.sigma.cpu().numpy()[:6], s_ref[:6], rtol=1e-12)
    assert torch.all(got.sigma[6:] == 0)
    assert torch.all(got.V[:, 6:] == 0)
    O4 = np.linalg.qr(rng.standard_normal((n, 10)))[0].T * 2.0      # 10 x n, orthogonal rows
    got = css.lowrank(torch.from_numpy(O4).cuda().contiguous(), 10)
    np.testing.assert_allclose(got.sigma.cpu().numpy(), 2.0, rtol=1e-12)
    Uw = got.Uw.cpu().numpy()
    np.testing.assert_allclose(Uw.T @ Uw, np.eye(10), atol=1e-12)
    # W wider than tall the other way round: n < l, rank n
    W2 = rng.standard_normal((20, 5))
    got = css.lowrank(torch.from_numpy(W2).cuda().contiguous(), 20)
    s2 = np.linalg.svd(W2, compute_uv=False)
    np.testing.assert_allclose(got.sigma.cpu().numpy()[:5], s2, rtol=1e-10)
    assert np.all(got.sigma.cpu().numpy()[5:] <= 1e-6 * s2[0])


@pytest.mark.parametrize("l", [301, 512])
def test_lowrank_wide_embedding(css, l):
    """Several Jacobi CTAs and an odd l (one padding index)."""
    rng = np.random.default_rng(l)
    n = 6000
    W = rng.standard_normal((l, n)) * (1.0 / np.arange(1, l + 1))[:, None]
    got = css.lowrank(torch.from_numpy(W).cuda().contiguous(), 50)
    s_ref = np.linalg.svd(W, compute_uv=False)
    w2 = float(np.sum(W * W))
    assert np.all(np.abs(got.sigma.cpu().numpy() ** 2 - s_ref[:50] ** 2) <= 4 * (n + l) * 2.0 ** -52 * w2)
    assert abs(got.tail - float(np.sum(s_ref[50:] ** 2))) <= 4 * (n + l) * l * 2.0 ** -52 * w2
    Uw = got.Uw.cpu().numpy()
    np.testing.assert_allclose(Uw.T @ Uw, np.eye(50), atol=1e-11)


def test_lowrank_rejects_nonfinite(css):
    W = np.random.default_rng(2).standard_normal((8, 100))
    W[3, 40] = np.nan
    from paper_1312_6838_gb300._lib import CssError, CSS_ERR_NONFINITE
    with pytest.raises(CssError) as ei:
        css.lowrank(torch.from_numpy(W).cuda(), 4)
    assert ei.value.code == CSS_ERR_NONFINITE


def test_lowrank_without_U_or_V(css):
    W = np.random.default_rng(4).standard_normal((30, 2000)) * (1.0 / np.arange(1, 31))[:, None]
    Wd = torch.from_numpy(W).cuda()
    full = css.lowrank(Wd, 10)
    bare = css.lowrank(Wd, 10, want_V=False)
    assert bare.U is None and bare.V is None
    assert torch.equal(full.sigma, bare.sigma) and torch.equal(full.Uw, bare.Uw)
    assert full.tail == bare.tail


def test_lowrank_is_deterministic(css):
    W = np.random.default_rng(3).standard_normal((64, 3000))
    Wd = torch.from_numpy(W).cuda()
    a = css.lowrank(Wd, 20)
    b = css.lowrank(Wd, 20)
    assert torch.equal(a.sigma, b.sigma) and torch.equal(a.V, b.V) and torch.equal(a.Uw, b.Uw)


def test_select_then_lowrank_full_size(css):
    """The selection workload of the benchmark (4096 x 65536 BF16, 1/i
    spectrum of rank 256 plus 1e-3 noise, k = 256) followed by the rank-128
    approximation of its own basis and omega rows: sigma against the oracle's
    SVD of the same W, and ||A - U~ S~ V~^T||^2 = F(S) + tail evaluated on the
    device from the outputs (U~, V~ orthonormal, so it is
    ||A||^2 - 2 tr(S~ U~^T A V~) + ||S~||^2)."""
    m, n, k, kr = 4096, 65536, 256, 128
    A_np = ci.lowrank_decaying(m, n, 256, 1e-3, 0, dtype=np.float32)
    A, _ = dev_matrix(A_np, torch.bfloat16)
    del A_np
    res = css.select(A, k, return_W=True, return_basis=True)
    assert res.n_sel == k
    lr = css.lowrank(res.W, kr, res.basis)
    W = res.W.cpu().numpy()
    s_ref = np.linalg.svd(W, compute_uv=False)
    w2 = float(np.sum(W * W))
    sig = lr.sigma.cpu().numpy()
    assert np.all(np.abs(sig ** 2 - s_ref[:kr] ** 2) <= 4 * (n + k) * 2.0 ** -52 * w2)
    Ad = A.double()
    a2 = float((Ad * Ad).sum())
    UtAV = lr.U.t() @ Ad @ lr.V
    err = a2 - 2.0 * float((lr.sigma * torch.diagonal(UtAV)).sum()) + float((lr.sigma ** 2).sum())
    F = float(res.trace[k])
    # F(S) from the selection's trace (mixed path: 1e-4 relative) plus the tail
    assert abs(err - (F + lr.tail)) <= 2e-4 * a2
