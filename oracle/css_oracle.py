"""FP64 CPU oracle for greedy column subset selection (Farahat et al., arXiv:1312.6838).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  The CUDA library never
calls it and shares no code, header, table or helper with it; the two meet only
through the seeded input generators in ``css_inputs.py``, which hold none of the
method's arithmetic.

Everything here is plain numpy in float64, written to be checked against the
paper by eye.  Library primitives (matmul, QR, solve) serve as single steps; no
blocking, fusion or reordering is done beyond what the cited passage states.
Indices are 0-based; the paper counts from 1.

Functions and the passages they follow:

* ``reconstruction_error``   -- Problem 1 / Eq. (Projection), Sec. 3.1: the
  criterion F(S) = ||A - P^(S) A||_F^2 with P^(S) = A_S (A_S^T A_S)^-1 A_S^T.
* ``greedy_css``             -- Algorithm 1 with Eq. (delta_omega) and Theorem 2,
  Sec. 4.2: the memory-efficient recursion, three mat-vecs per iteration.
* ``greedy_css_residual``    -- Problem 3 with Lemma 2, Sec. 4.2: the explicit
  residual-matrix form (tiny inputs only).
* ``greedy_gcss``            -- Algorithm 3 with Theorem 4, Sec. 5.2.
* ``random_projection``      -- Algorithm 2, Sec. 5.1 (per-block partial sums, then
  the reducer's row sums).
* ``distributed_css``        -- Algorithm 4, Sec. 5.2.
* ``brute_force_css``        -- Problem 1 solved by enumeration (tiny inputs).
* ``exact_scores``           -- the greedy criterion of Problem 2 evaluated directly
  for a given selected prefix (used to check sampled outputs at large sizes).
* ``residual_gradient``      -- d||A - P^(S)A||_F^2 / dA at fixed S, derived from
  Eq. (Projection) by differentiating P^(S) (restated in the docstring).
* ``philox4x32_10``,
  ``random_omega``           -- the random matrix Omega of Sec. 5.1 drawn from a
  counter-based generator, Philox4x32-10 (Salmon, Moraes, Dror and Shaw,
  "Parallel random numbers: as easy as 1, 2, 3", SC 2011), written from that
  definition: the dense Gaussian matrix and the sparse random sign matrix
  (entries +-1 with probability 1/(2 sqrt n) each, 0 otherwise) that Sec. 5.1
  cites and Sec. 7 uses ("rnd" and "ssgn").
* ``rnd_greedy_css``         -- RndGreedyCSS of Sec. 7: Algorithm 3 with the
  target B = A Omega of Sec. 5.1, Omega n x l (r = l).
* ``relative_accuracy``      -- the evaluation measure of Sec. 7: the
  reconstruction error of a selection placed between that of uniform column
  sampling (0 %) and that of the best rank-l approximation by SVD (100 %).
* ``embedding``              -- Q = orth(A_:S) and W = Q^T A, Sec. 3.2
  (Eq. CSS_LowDim).
* ``rank_k_approximation``   -- the column-based rank-k approximation
  A~_{S,k} = Q W~_k and the approximate SVD of Eq. (ApproxSVD), Sec. 3.2.

Readings where the paper is silent (the same readings the CUDA path takes):

1. Alg. 1 initialises f^(0), g^(0) and reads f^(t) at t = 1: f^(1) = f^(0).
2. The candidate set excludes already-selected columns and every column whose
   residual norm g_i has fallen to tau_rel * g_i^(0) or below (and columns with
   g_i^(0) = 0).  If no candidate is left the run stops early (rank exhausted).
3. Ties in the argmax go to the lowest column index.
4. The stored f and g are never clamped; a negative f (rounding) scores as 0.
5. The error trace follows Theorem 1: F^(t) = F^(t-1) - f_p / g_p, with
   F^(0) = ||A||_F^2 (CSS) or ||B||_F^2 (GCSS).
"""
from __future__ import annotations

import itertools
import time

import numpy as np

__all__ = [
    "reconstruction_error",
    "reconstruction_error_normal_eq",
    "greedy_css",
    "greedy_css_residual",
    "greedy_gcss",
    "random_projection",
    "distributed_css",
    "brute_force_css",
    "exact_scores",
    "exact_gcss_scores",
    "residual_gradient",
    "philox4x32_10",
    "rnd_greedy_css",
    "relative_accuracy",
    "random_omega",
    "OMEGA_GAUSSIAN",
    "OMEGA_SPARSE_SIGN",
    "GreedyResult",
]


class GreedyResult:
    """Output of a greedy run, in selection order.

    ``S``      selected column indices (0-based), in selection order
    ``trace``  F^(0), F^(1), ..., F^(len(S)) from the recursion of Theorem 1/3
    ``W``      the omega vectors, one row per iteration (len(S) x n)
    ``gaps``   relative top-two score gap at each iteration (for the parity rule)
    ``scores`` the score vector f/g used at each iteration (only if requested)
    """

    def __init__(self):
        self.S: list[int] = []
        self.trace: list[float] = []
        self.W: np.ndarray | None = None
        self.gaps: list[float] = []
        self.scores: list[np.ndarray] = []
        self.fs: list[np.ndarray] = []     # f before each iteration (keep_scores)
        self.gs: list[np.ndarray] = []     # g before each iteration (keep_scores)
        self.f: np.ndarray | None = None
        self.g: np.ndarray | None = None
        # wall-clock instrumentation (time.perf_counter): after initialisation
        # and after each iteration; no effect on the arithmetic
        self.t_start: float = 0.0
        self.t_init: float = 0.0
        self.t_iter: list[float] = []


def _as64(X):
    return np.ascontiguousarray(np.asarray(X, dtype=np.float64))


# --------------------------------------------------------------------------- #
# Problem 1 / Eq. (Projection): the criterion evaluated directly.
# --------------------------------------------------------------------------- #
def reconstruction_error(A, S, B=None, chunk=None):
    """F(S) = ||T - P^(S) T||_F^2 with T = A (CSS) or T = B (GCSS, Problem 4).

    P^(S) projects onto span(A_:S) (Eq. Projection, Sec. 3.1).  It is applied
    through a Householder QR of A_:S (numpy/LAPACK), which spans the same space
    and stays accurate when A_:S is ill-conditioned; the residual is formed
    explicitly so that no cancellation against ||T||^2 occurs.  ``chunk``
    forms it ``chunk`` columns of T at a time (large inputs; same quantity).
    """
    A = _as64(A)
    T = A if B is None else _as64(B)
    S = list(S)
    if len(S) == 0:
        return float(np.sum(T * T))
    Q, _ = np.linalg.qr(A[:, S], mode="reduced")
    step = T.shape[1] if chunk is None else int(chunk)
    total = 0.0
    for c0 in range(0, T.shape[1], step):
        Tc = T[:, c0:c0 + step]
        R = Tc - Q @ (Q.T @ Tc)
        total += float(np.sum(R * R))
    return total


def reconstruction_error_normal_eq(A, S, B=None):
    """The same criterion through the normal equations exactly as Eq. (Projection)
    writes it: T - A_S (A_S^T A_S)^-1 A_S^T T.  Secondary check only."""
    A = _as64(A)
    T = A if B is None else _as64(B)
    S = list(S)
    AS = A[:, S]
    coeff = np.linalg.solve(AS.T @ AS, AS.T @ T)
    R = T - AS @ coeff
    return float(np.sum(R * R))


# --------------------------------------------------------------------------- #
# Candidate selection shared reading (points 2-4 of the module docstring).
# --------------------------------------------------------------------------- #
def _argmax_score(f, g, g0, selected, tau_rel):
    """Return (p, score vector, relative top-two gap) for  argmax_i f_i / g_i.

    Candidates: not selected, g0_i > 0 and g_i > tau_rel * g0_i.  A negative
    f_i scores 0.  Ties go to the lowest index (np.argmax returns the first).
    p is None when no candidate remains.
    """
    cand = (~selected) & (g0 > 0) & (g > tau_rel * g0)
    if not np.any(cand):
        return None, None, 0.0
    score = np.full(f.shape, -np.inf)
    score[cand] = np.maximum(f[cand], 0.0) / g[cand]
    p = int(np.argmax(score))
    best = score[p]
    rest = score.copy()
    rest[p] = -np.inf
    second = np.max(rest) if np.sum(cand) > 1 else -np.inf
    if not np.isfinite(second):
        gap = np.inf
    elif best > 0:
        gap = (best - second) / best
    else:
        gap = 0.0
    return p, score, float(gap)


# --------------------------------------------------------------------------- #
# Algorithm 1 (Sec. 4.2) with Eq. (delta_omega) and Theorem 2.
# --------------------------------------------------------------------------- #
def greedy_css(A, l, tau_rel=1e-12, forced=None, keep_scores=False,
               score="paper"):
    """Greedy CSS, memory-efficient form (Algorithm 1).

    Initialisation (Algorithm 1):
        f_i^(0) = ||A^T A_:i||^2,   g_i^(0) = A_:i^T A_:i .
    ||A^T A_:i||^2 is evaluated as A_:i^T (A A^T) A_:i (the same number; it
    avoids forming the n x n matrix A^T A).

    Iteration t:
        p       = argmax_i f_i / g_i
        delta   = A^T A_:p - sum_{r<t} omega_p^(r) omega^(r)        (Eq. delta_omega)
        omega   = delta / sqrt(delta_p)
        x       = A^T (A omega) - sum_{r<t} (omega^(r)^T omega) omega^(r)   (Thm 2)
        f      <- f - 2 omega o x + ||omega||^2 (omega o omega)          (Thm 2)
        g      <- g - omega o omega                                      (Thm 2)
    and the error recursion of Theorem 1 with R = {p}:
        F(S u {p}) = F(S) - f_p / g_p .

    ``forced``: optional list of column indices taken instead of the argmax at
    the first len(forced) iterations (teacher forcing / resume).
    ``score='norm'`` replaces the criterion by g_i alone (a test hook: the
    recursion then reproduces QR with column pivoting).
    """
    A = _as64(A)
    m, n = A.shape
    res = GreedyResult()
    res.t_start = time.perf_counter()
    g = np.einsum("ij,ij->j", A, A)
    g0 = g.copy()
    C = A @ A.T
    f = np.einsum("ij,ij->j", A, C @ A)
    selected = np.zeros(n, dtype=bool)
    F = float(np.sum(A * A))
    res.trace.append(F)
    omegas = np.zeros((0, n))
    forced = list(forced) if forced is not None else []
    res.t_init = time.perf_counter()
    for t in range(l):
        if score == "norm":
            p, sc, gap = _argmax_score(g * g, g, g0, selected, tau_rel)
        else:
            p, sc, gap = _argmax_score(f, g, g0, selected, tau_rel)
        if t < len(forced):
            p = int(forced[t])
        if p is None:
            break
        if keep_scores:
            res.scores.append(sc)
            res.fs.append(f.copy())
            res.gs.append(g.copy())
        res.gaps.append(gap)
        F = F - f[p] / g[p]
        selected[p] = True
        res.S.append(p)
        res.trace.append(F)
        delta = A.T @ A[:, p] - omegas.T @ omegas[:, p]
        omega = delta / np.sqrt(delta[p])
        x = A.T @ (A @ omega) - omegas.T @ (omegas @ omega)
        f = f - 2.0 * omega * x + np.dot(omega, omega) * omega * omega
        g = g - omega * omega
        omegas = np.vstack([omegas, omega])
        res.t_iter.append(time.perf_counter())
    res.W = omegas
    res.f, res.g = f, g
    return res


# --------------------------------------------------------------------------- #
# Problem 3 with Lemma 2 (Sec. 4.2): explicit residual matrix E.
# --------------------------------------------------------------------------- #
def greedy_css_residual(A, l, tau_rel=1e-12):
    """Greedy CSS keeping E explicitly (tiny inputs only).

    p = argmax_i ||E^T E_:i||^2 / (E_:i^T E_:i)                    (Problem 3)
    E <- E - E_:p E_:p^T E / (E_:p^T E_:p)                          (Lemma 2)
    F <- ||E||_F^2 after each update (Theorem 1 evaluated directly).
    """
    A = _as64(A)
    m, n = A.shape
    E = A.copy()
    g0 = np.einsum("ij,ij->j", A, A)
    selected = np.zeros(n, dtype=bool)
    res = GreedyResult()
    res.trace.append(float(np.sum(E * E)))
    for _ in range(l):
        G = E.T @ E
        f = np.sum(G * G, axis=0)
        g = np.diag(G).copy()
        p, _, gap = _argmax_score(f, g, g0, selected, tau_rel)
        if p is None:
            break
        res.gaps.append(gap)
        ep = E[:, p].copy()
        E = E - np.outer(ep, ep @ E) / np.dot(ep, ep)
        selected[p] = True
        res.S.append(p)
        res.trace.append(float(np.sum(E * E)))
    return res


# --------------------------------------------------------------------------- #
# Algorithm 3 (Sec. 5.2) with Theorem 4.
# --------------------------------------------------------------------------- #
def greedy_gcss(A, B, l, tau_rel=1e-12, forced=None, keep_scores=False):
    """Greedy generalized CSS: select columns of A to reconstruct B (Algorithm 3).

    Initialisation: f_i^(0) = ||B^T A_:i||^2,  g_i^(0) = A_:i^T A_:i.
    Iteration t:
        p       = argmax_i f_i / g_i
        delta   = A^T A_:p - sum_{r<t} omega_p^(r) omega^(r)
        gamma   = B^T A_:p - sum_{r<t} omega_p^(r) upsilon^(r)
        omega   = delta / sqrt(delta_p),  upsilon = gamma / sqrt(delta_p)
        x       = A^T (B upsilon) - sum_{r<t} (upsilon^(r)^T upsilon) omega^(r)   (Thm 4)
        f      <- f - 2 omega o x + ||upsilon||^2 (omega o omega)
        g      <- g - omega o omega
    Error recursion (Theorem 3): Fbar^(0) = ||B||_F^2, Fbar <- Fbar - f_p / g_p.
    """
    A = _as64(A)
    B = _as64(B)
    m, n = A.shape
    res = GreedyResult()
    g = np.einsum("ij,ij->j", A, A)
    g0 = g.copy()
    BtA = B.T @ A
    f = np.einsum("ij,ij->j", BtA, BtA)
    selected = np.zeros(n, dtype=bool)
    F = float(np.sum(B * B))
    res.trace.append(F)
    omegas = np.zeros((0, n))
    upsilons = np.zeros((0, B.shape[1]))
    forced = list(forced) if forced is not None else []
    for t in range(l):
        p, sc, gap = _argmax_score(f, g, g0, selected, tau_rel)
        if t < len(forced):
            p = int(forced[t])
        if p is None:
            break
        if keep_scores:
            res.scores.append(sc)
            res.fs.append(f.copy())
            res.gs.append(g.copy())
        res.gaps.append(gap)
        F = F - f[p] / g[p]
        selected[p] = True
        res.S.append(p)
        res.trace.append(F)
        delta = A.T @ A[:, p] - omegas.T @ omegas[:, p]
        gamma = B.T @ A[:, p] - upsilons.T @ omegas[:, p]
        omega = delta / np.sqrt(delta[p])
        upsilon = gamma / np.sqrt(delta[p])
        x = A.T @ (B @ upsilon) - omegas.T @ (upsilons @ upsilon)
        f = f - 2.0 * omega * x + np.dot(upsilon, upsilon) * omega * omega
        g = g - omega * omega
        omegas = np.vstack([omegas, omega])
        upsilons = np.vstack([upsilons, upsilon])
    res.W = omegas
    res.f, res.g = f, g
    return res


# --------------------------------------------------------------------------- #
# Omega (Sec. 5.1) from a counter-based generator.
# --------------------------------------------------------------------------- #
OMEGA_GAUSSIAN = 0
OMEGA_SPARSE_SIGN = 1

_PHILOX_M0, _PHILOX_M1 = 0xD2511F53, 0xCD9E8D57      # round multipliers
_PHILOX_W0, _PHILOX_W1 = 0x9E3779B9, 0xBB67AE85      # key increments (Weyl)


def philox4x32_10(ctr, key):
    """Philox4x32-10 (Salmon et al., SC 2011): ten rounds on a 4 x 32-bit
    counter with a 2 x 32-bit key.  Each round multiplies words 0 and 2 by the
    two constants (64-bit products split into high and low halves) and forms
    (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is bumped by the Weyl
    constants between rounds.  ``ctr`` is four uint32 arrays (broadcast), ``key``
    two ints; returns four uint32 arrays."""
    mask = np.uint64(0xFFFFFFFF)
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & mask for c in ctr)
    k0, k1 = np.uint64(key[0] & 0xFFFFFFFF), np.uint64(key[1] & 0xFFFFFFFF)
    for _ in range(10):
        p0 = np.uint64(_PHILOX_M0) * c0
        p1 = np.uint64(_PHILOX_M1) * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & mask
        hi1, lo1 = p1 >> np.uint64(32), p1 & mask
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + np.uint64(_PHILOX_W0)) & mask
        k1 = (k1 + np.uint64(_PHILOX_W1)) & mask
    return tuple(x.astype(np.uint32) for x in (c0, c1, c2, c3))


def sparse_sign_threshold(n):
    """A draw x0 (uniform 32-bit) marks a nonzero when x0 < floor(2^32 / sqrt n),
    i.e. with probability 1/sqrt(n) (the sparse random sign matrix of Sec. 5.1)."""
    return min(0xFFFFFFFF, int(np.floor(4294967296.0 / np.sqrt(float(n)))))


def random_omega(n, r, seed, dist):
    """Omega (n x r) of Sec. 5.1; entry (i, j) comes from the Philox block of
    counter (i, j, 0, 0) under key (seed mod 2^32, seed >> 32):
      Gaussian:    u1 = (x0 + 1) / 2^32, u2 = x1 / 2^32,
                   Omega_ij = sqrt(-2 ln u1) cos(2 pi u2) / sqrt(r)   (Box-Muller,
                   variance 1/r; the selection is invariant to the scale of B)
      sparse sign: Omega_ij = 0 unless x0 < floor(2^32 / sqrt n); then +1 if the
                   lowest bit of x1 is 0, else -1 (unscaled: the selection is
                   invariant to the scale of B)."""
    i = np.arange(n, dtype=np.uint64)[:, None]
    j = np.arange(r, dtype=np.uint64)[None, :]
    zero = np.zeros((1, 1), dtype=np.uint64)
    x0, x1, _, _ = philox4x32_10((i, j, zero, zero), (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF))
    if dist == OMEGA_GAUSSIAN:
        u1 = (x0.astype(np.float64) + 1.0) / 4294967296.0
        u2 = x1.astype(np.float64) / 4294967296.0
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2) / np.sqrt(float(r))
    if dist == OMEGA_SPARSE_SIGN:
        nz = x0.astype(np.uint64) < np.uint64(sparse_sign_threshold(n))
        sign = np.where((x1 & np.uint32(1)) == 0, 1.0, -1.0)
        return np.where(nz, sign, 0.0)
    raise ValueError("unknown distribution")


def rnd_greedy_css(A, l, seed, dist=OMEGA_GAUSSIAN, tau_rel=1e-12):
    """RndGreedyCSS (Sec. 7): greedy generalized CSS (Algorithm 3) of the
    columns of A for the random target B = A Omega with Omega = random_omega(
    n, l, seed, dist) -- the random projection of Sec. 5.1 with r = l."""
    A = _as64(A)
    B = random_projection(A, random_omega(A.shape[1], l, seed, dist))
    return greedy_gcss(A, B, l, tau_rel=tau_rel)


def relative_accuracy(err_S, err_uniform, err_svd):
    """Relative accuracy of Sec. 7 in percent, from Frobenius reconstruction
    errors (not squared): (||A - A_U|| - ||A - A_S||) / (||A - A_U|| - ||A - A_l||)
    x 100, where A_U is the approximation from a uniform random subset of l
    columns, A_S the one from the selected subset and A_l the best rank-l
    approximation (SVD)."""
    return 100.0 * (err_uniform - err_S) / (err_uniform - err_svd)


# --------------------------------------------------------------------------- #
# Algorithm 2 (Sec. 5.1): B = A Omega as per-block partial sums.
# --------------------------------------------------------------------------- #
def random_projection(A, Omega, block_offsets=None):
    """B = A Omega = sum_i A_:i Omega_i:  (Sec. 5.1).

    Each mapper (column block) accumulates its in-memory partial
    Bbar_(b) = sum_{i in block b} A_:i Omega_i: ; the reducers sum the c
    partials row by row (Algorithm 2).  ``block_offsets`` (c+1 increasing
    column offsets) defines the blocks; None means one block.
    """
    A = _as64(A)
    Omega = _as64(Omega)
    n = A.shape[1]
    if block_offsets is None:
        block_offsets = [0, n]
    partials = []
    for b in range(len(block_offsets) - 1):
        lo, hi = block_offsets[b], block_offsets[b + 1]
        partials.append(A[:, lo:hi] @ Omega[lo:hi, :])      # map: in-memory sum
    B = np.zeros((A.shape[0], Omega.shape[1]))
    for Bb in partials:                                      # reduce: row sums
        B += Bb
    return B


# --------------------------------------------------------------------------- #
# Algorithm 4 (Sec. 5.2): per-block GCSS, then GCSS on the union.
# --------------------------------------------------------------------------- #
def distributed_css(A, B, block_offsets, l_block, l, tau_rel=1e-12):
    """Distributed CSS (Algorithm 4) given the concise representation B.

    map:    each block b selects l_(b) = min(l_block, n_b) columns of A_(b) by
            greedy GCSS against B.
    reduce: A_(0) is the union in block order, each block's columns in their
            selection order; GCSS(A_(0), B, l) picks the final set.
    Returns (final global column ids in selection order, per-block global ids,
    the final GreedyResult on A_(0)).
    """
    A = _as64(A)
    B = _as64(B)
    per_block = []
    union = []
    for b in range(len(block_offsets) - 1):
        lo, hi = block_offsets[b], block_offsets[b + 1]
        lb = min(l_block, hi - lo)
        rb = greedy_gcss(A[:, lo:hi], B, lb, tau_rel=tau_rel)
        ids = [lo + j for j in rb.S]
        per_block.append(ids)
        union.extend(ids)
    r0 = greedy_gcss(A[:, union], B, l, tau_rel=tau_rel)
    final = [union[j] for j in r0.S]
    return final, per_block, r0


# --------------------------------------------------------------------------- #
# Problem 1 by enumeration.
# --------------------------------------------------------------------------- #
def brute_force_css(A, l, B=None):
    """argmin over |S| = l of F(S) by trying every subset (Problem 1).
    Returns (best subset as a sorted tuple, its error)."""
    A = _as64(A)
    n = A.shape[1]
    best, best_err = None, np.inf
    for S in itertools.combinations(range(n), l):
        if np.linalg.matrix_rank(A[:, S]) < l:
            continue
        err = reconstruction_error(A, S, B)
        if err < best_err:
            best, best_err = S, err
    return best, best_err


# --------------------------------------------------------------------------- #
# Problem 2 / Problem 5 criteria evaluated directly for a given prefix.
# --------------------------------------------------------------------------- #
def _residual_basis(A, S):
    A = _as64(A)
    if len(S) == 0:
        return np.zeros((A.shape[0], 0))
    Q, _ = np.linalg.qr(A[:, list(S)], mode="reduced")
    return Q


def exact_scores(A, S, cols=None, C=None):
    """f_i = ||E^T E_:i||^2 and g_i = E_:i^T E_:i with E = A - P^(S) A (Problem 2),
    for the columns ``cols`` (default: all).

    E^T E_:i = A^T (I - P) A_:i, so ||E^T E_:i||^2 = e_i^T (A A^T) e_i with
    e_i = (I - P) A_:i; ``C`` = A A^T may be passed in to reuse it.
    """
    A = _as64(A)
    n = A.shape[1]
    cols = np.arange(n) if cols is None else np.asarray(cols)
    Q = _residual_basis(A, S)
    Ec = A[:, cols]
    if Q.shape[1]:
        Ec = Ec - Q @ (Q.T @ Ec)
    if C is None:
        C = A @ A.T
    f = np.einsum("ij,ij->j", Ec, C @ Ec)
    g = np.einsum("ij,ij->j", Ec, Ec)
    return f, g


def exact_gcss_scores(A, B, S, cols=None):
    """f_i = ||F^T E_:i||^2, g_i = E_:i^T E_:i (Problem 5) for a given prefix S,
    where F = B - P^(S) B and E = A - P^(S) A.  F^T E_:i = B^T (I - P) A_:i."""
    A = _as64(A)
    B = _as64(B)
    n = A.shape[1]
    cols = np.arange(n) if cols is None else np.asarray(cols)
    Q = _residual_basis(A, S)
    Ec = A[:, cols]
    if Q.shape[1]:
        Ec = Ec - Q @ (Q.T @ Ec)
    H = B.T @ Ec
    return np.einsum("ij,ij->j", H, H), np.einsum("ij,ij->j", Ec, Ec)


# --------------------------------------------------------------------------- #
# Gradient of the criterion at a fixed selected set.
# --------------------------------------------------------------------------- #
def residual_gradient(A, S):
    """Gradient of L(A) = ||A - P^(S) A||_F^2 with respect to A, S fixed.

    With T = (A_S^T A_S)^-1 A_S^T A (the least-squares coefficients of
    Sec. 3.1) and R = A - A_S T:
        dL/dA      = 2 R                       for columns outside S,
        dL/dA_:S   = -2 R T^T                  (R_:S = 0, so only the
                                                dependence of P^(S) on A_S
                                                contributes).
    Derivation: dL = 2 tr(R^T dA) - tr(A^T dP A) and, differentiating
    Eq. (Projection), tr(A^T dP A) = 2 tr(T R^T dA_S).
    Returns (L, dL/dA).
    """
    A = _as64(A)
    S = list(S)
    AS = A[:, S]
    T = np.linalg.solve(AS.T @ AS, AS.T @ A)
    R = A - AS @ T
    G = 2.0 * R
    G[:, S] = -2.0 * (R @ T.T)
    return float(np.sum(R * R)), G


# --------------------------------------------------------------------------- #
# Sec. 3.2: embedding into the span of the selected columns, the column-based
# rank-k approximation and the approximate SVD (Eq. CSS_LowDim, Eq. ApproxSVD).
# --------------------------------------------------------------------------- #
def embedding(A, S):
    """Q = orth(A_:S) and W = Q^T A (Eq. CSS_LowDim).

    orth() is the thin QR factorisation A_:S = Q R (Householder, LAPACK) with
    each column of Q signed so that diag(R) > 0.  With that sign Q is the one
    orthonormal basis that Gram-Schmidt produces on the columns of A_:S taken
    in selection order: q_t is the normalised part of column S[t] outside the
    span of the earlier ones, the direction whose A^T q_t is the omega of
    iteration t (Eq. delta_omega).  Returns (Q m x l, W l x n, R l x l).
    """
    A = _as64(A)
    S = list(S)
    Q, R = np.linalg.qr(A[:, S], mode="reduced")
    sgn = np.where(np.diag(R) < 0.0, -1.0, 1.0)
    Q = Q * sgn
    R = R * sgn[:, None]
    return Q, Q.T @ A, R


def rank_k_approximation(Q, W, k):
    """Column-based rank-k approximation of Sec. 3.2 and the approximate SVD of
    Eq. (ApproxSVD), from an orthonormal Q (m x l) and W = Q^T A (l x n).

    1. Thin SVD W = U^(W) Sigma^(W) V^(W)^T (LAPACK), singular values
       descending; the best rank-k approximation of W is
       W~_k = U^(W)_k Sigma^(W)_k V^(W)_k^T.
    2. A~_{S,k} = Q W~_k.
    3. Eq. (ApproxSVD): U~ = Q U^(W)_k, Sigma~ = Sigma^(W)_k, V~ = V^(W)_k.

    Returns a dict: ``U`` (m x k), ``sigma`` (k), ``V`` (n x k), ``Uw``
    (l x k, U^(W)_k), ``Wk`` (l x n), ``sigma_all`` (all singular values of W)
    and ``tail`` = sum_{i >= k} sigma_i^2 = ||W - W~_k||_F^2.  A~_{S,k} itself
    is ``Q @ Wk``.
    """
    Q = _as64(Q)
    W = _as64(W)
    Uw, sw, Vwt = np.linalg.svd(W, full_matrices=False)
    Uk, sk, Vk = Uw[:, :k], sw[:k], Vwt[:k, :].T
    Wk = (Uk * sk) @ Vk.T
    return {"U": Q @ Uk, "sigma": sk, "V": Vk, "Uw": Uk, "Wk": Wk,
            "sigma_all": sw, "tail": float(np.sum(sw[k:] ** 2))}
