"""Shared helpers of the GPU parity tests (imported by tests only)."""
from dataclasses import dataclass, field

import numpy as np
import torch

import css_inputs as ci

GAP_TOL = 1e-6        # index agreement required where the oracle's top-two gap exceeds this


def dev_matrix(A_np, dtype, ld=None):
    """Column-major device copy of A_np in `dtype`; returns (tensor, the FP64
    values the device actually holds)."""
    from paper_1312_6838_gb300 import css
    A32 = np.asarray(A_np)
    if dtype == torch.bfloat16:
        vals = ci.round_bf16(A32.astype(np.float32)).astype(np.float64)
        t = torch.from_numpy(vals.astype(np.float32)).to(torch.bfloat16)
    elif dtype == torch.float32:
        vals = A32.astype(np.float32).astype(np.float64)
        t = torch.from_numpy(vals.astype(np.float32))
    else:
        vals = A32.astype(np.float64)
        t = torch.from_numpy(vals)
    return css.to_colmajor(t.cuda(), ld=ld), vals


def first_mismatch(a, b, start=0):
    for t in range(start, min(len(a), len(b))):
        if a[t] != b[t]:
            return t
    return None


# ------------------------------------------------------ the score error model
# Unit roundoff of the dot-product accumulation of each path: the mixed path
# (BF16 or FP32 stream) forms every dot product in FP32.
EPS = {torch.float64: 2.0 ** -53, torch.float32: 2.0 ** -24, torch.bfloat16: 2.0 ** -24}
P_FAIL = 1e-6         # allowed probability that any dot product of a run exceeds its bound


def hm_lambda(length, n_dots, p_fail=P_FAIL):
    """The constant lambda of the probabilistic rounding-error bound of Higham
    and Mary ("A new approach to probabilistic rounding error analysis", SIAM
    J. Sci. Comput. 41(5), 2019): with independent, mean-zero rounding errors
    an inner product of `length` terms computed with unit roundoff u is off by
    at most about lambda * sqrt(length) * u * sum_i |x_i y_i|, except with
    probability at most 2 * length * exp(-lambda^2 (1 - u)^2 / 2).  Taking the
    union over the `n_dots` products of a run, lambda is chosen so that none
    fails with probability above p_fail."""
    return float(np.sqrt(2.0 * np.log(2.0 * length * max(n_dots, 1) / p_fail)))


def _n_dots(ref, m):
    n = ref.fs[0].shape[0]
    return 2 * n * (len(ref.S) + 1) + m * m


def score_error_bound(ref, t, m, dtype):
    """Absolute error bound of every column's device score f_i / g_i at
    iteration t (an array over the columns; needs the oracle run with
    keep_scores=True).

    The device forms the initial scores and every update of Theorem 2/4 from
    dot products of length m with the original column a_i, each within
    lambda sqrt(m) u of its terms (hm_lambda).  The terms that make up
    f_i / g_i scale like f_i^(0) / g_i <= sc0_max g_i^(0) / g_i (sc0_max the
    largest initial score f^(0)/g^(0)), plus the score itself through g_i's
    own error, and t + 1 such contributions add with independent errors:
        |d sc_i| <= lambda u sqrt(m) sqrt(t + 1) (sc0_max g_i^(0) / g_i + sc_i).
    This is a first-order model, not a worst-case bound; the GPU tests
    measure the device's actual score errors against it
    (oracle_path_parity) and print the largest ratio they see."""
    f0, g0 = ref.fs[0], ref.gs[0]
    g = ref.gs[t]
    with np.errstate(divide="ignore", invalid="ignore"):
        sc0 = np.where(g0 > 0, np.maximum(f0, 0.0) / g0, 0.0)
        sc = np.maximum(ref.fs[t], 0.0) / g
        shrink = np.where(g > 0, g0 / g, np.inf)
    sc0_max = float(np.max(sc0)) if sc0.size else 0.0
    lam = hm_lambda(m, _n_dots(ref, m))
    return lam * EPS[dtype] * np.sqrt(m) * np.sqrt(t + 1) * (sc0_max * shrink + np.abs(sc))


def pair_error_bound(ref, t, m, dtype, cols=None):
    """The relative amount (against the best score of iteration t, as the
    oracle's gap is measured) by which two candidates' scores can be
    misjudged: the sum of their score error bounds over the best score.  By
    default the oracle's two best candidates."""
    sc = ref.scores[t]
    s = np.where(np.isfinite(sc), sc, -np.inf)
    order = np.argsort(-s, kind="stable")
    best = s[order[0]]
    top = order[:2] if cols is None else list(cols)
    if not np.isfinite(best) or best <= 0:
        return np.inf
    rho = score_error_bound(ref, t, m, dtype)
    return float(sum(rho[i] for i in top if np.isfinite(s[i])) / best)


def trace_error_bound(ref, m, dtype):
    """Absolute error bound of the device's recursive trace (Theorem 1/3) on
    the oracle's path, per iteration: F^(0) sums the columns' squared norms
    (each a dot product of length m), and every step subtracts the picked
    column's score f_p / g_p, whose error score_error_bound gives."""
    lam = hm_lambda(m, _n_dots(ref, m))
    out = [lam * EPS[dtype] * np.sqrt(m) * abs(ref.trace[0])]
    for t, p in enumerate(ref.S):
        out.append(out[-1] + float(score_error_bound(ref, t, m, dtype)[p]))
    return np.array(out)


def certify_selection(S_dev, ref_on_dev, m, dtype, gap_tol=GAP_TOL):
    """Checks that the device's own selection is a greedy selection within the
    path's arithmetic.  ref_on_dev is the oracle run teacher-forced on S_dev
    (keep_scores=True), so its score vector at iteration t is the exact one
    on the device's path.  Where the device's pick is not the oracle's argmax
    there, its relative score deficit against the best must be at most
    max(gap_tol, the two columns' score error bound).  Returns (the number of
    such steps, the largest deficit)."""
    n_off, worst = 0, 0.0
    for t, p in enumerate(S_dev):
        sc = ref_on_dev.scores[t]
        s = np.where(np.isfinite(sc), sc, -np.inf)
        best = int(np.argmax(s))
        if best == p:
            continue
        assert np.isfinite(s[p]), (t, p, "the device picked a column that is not a candidate")
        deficit = float((s[best] - s[p]) / s[best]) if s[best] > 0 else 0.0
        n_off += 1
        worst = max(worst, deficit)
        tol = max(gap_tol, pair_error_bound(ref_on_dev, t, m, dtype, cols=(best, p)))
        assert deficit <= tol, (t, p, best, deficit, tol)
    return n_off, worst


@dataclass
class ParityStats:
    """Step-by-step comparison of the device with the oracle along the oracle's
    own path (the device is teacher-forced to the oracle's picks, and reports
    its own argmax at every step).

    steps            iterations compared
    agree            steps where the device's argmax is the oracle's pick
    strict           mismatches where the oracle's top-two gap is <= 1e-6
                     (both picks correct under the spec rule)
    widened          mismatches with a gap above 1e-6, each explained by the
                     device's measured score errors, which lie within
                     score_error_bound
    max_widened_gap  the largest oracle gap among the widened steps
    measured_steps   iterations whose device score state was read back
    max_err_ratio    largest measured |score error| / score_error_bound over
                     the candidates at the measured steps (must be <= 1)
    """
    steps: int = 0
    agree: int = 0
    strict: int = 0
    widened: int = 0
    max_widened_gap: float = 0.0
    mismatch_steps: list = field(default_factory=list)
    measured_steps: list = field(default_factory=list)
    max_err_ratio: float = 0.0

    @property
    def restarts(self):
        return self.strict + self.widened

    def as_dict(self):
        return {"steps": self.steps, "agree": self.agree, "mismatch_gap_le_1e-6": self.strict,
                "mismatch_gap_gt_1e-6": self.widened, "max_gap_of_those": self.max_widened_gap,
                "mismatch_steps": self.mismatch_steps, "measured_steps": self.measured_steps,
                "max_score_err_over_bound": self.max_err_ratio}


def device_scores(run_state, t, tau, g0):
    """The device's score vector f/g at iteration t on the oracle's path: the
    state after t forced iterations (run_state(t) returns a Selection with
    diag_f, diag_g), with the candidate mask of the method (g > tau g0)."""
    r = run_state(t)
    f = r.diag_f.cpu().numpy()
    g = r.diag_g.cpu().numpy()
    with np.errstate(divide="ignore", invalid="ignore"):
        sc = np.maximum(f, 0.0) / g
    return sc, (g > tau * g0)


def oracle_path_parity(run_forced, ref, m, dtype, tau, sample_steps=(), gap_tol=GAP_TOL):
    """Compare the device with the oracle at every iteration of the oracle's
    path.

    run_forced(prefix, k, diag) runs the device with `prefix` forced and k
    iterations, with the diagnostics on.  One run with the oracle's whole
    sequence forced gives the device's own argmax at each step.  Where it
    differs from the oracle's pick and the oracle's gap exceeds gap_tol, the
    gap must lie within the two candidates' score error bound
    (pair_error_bound), and the device's score state at that step is read
    back: its pick must be the argmax of its own scores, and every
    candidate's measured score error must lie within score_error_bound.  The
    same measurement runs at `sample_steps`.  Returns ParityStats."""
    S = list(ref.S)
    k = len(S)
    st = ParityStats(steps=k)
    if k == 0:
        return st
    full = run_forced(S, k, True)
    da = full.diag_argmax.cpu().tolist()
    g0 = ref.gs[0]

    def measure(t):
        sc_dev, cand = device_scores(lambda tt: run_forced(S[:tt], tt, True), t, tau, g0)
        sc_ref = ref.scores[t]
        ok = np.isfinite(sc_ref) & cand
        rho = score_error_bound(ref, t, m, dtype)
        with np.errstate(divide="ignore", invalid="ignore"):
            ratio = np.abs(sc_dev - sc_ref) / rho
        ratio = ratio[ok]
        worst = float(np.max(ratio)) if ratio.size else 0.0
        st.max_err_ratio = max(st.max_err_ratio, worst)
        st.measured_steps.append(t)
        assert worst <= 1.0, (t, worst)
        return sc_dev

    for t in range(k):
        if da[t] == S[t]:
            st.agree += 1
            continue
        gap = ref.gaps[t]
        st.mismatch_steps.append((t, float(gap)))
        if gap <= gap_tol:
            st.strict += 1
            continue
        st.widened += 1
        st.max_widened_gap = max(st.max_widened_gap, float(gap))
        bound = pair_error_bound(ref, t, m, dtype)
        assert gap <= bound, (
            f"step {t}: device {da[t]}, oracle {S[t]}, gap {gap:.3e} beyond the score error bound {bound:.3e}")
        if t >= 1:
            sc_dev = measure(t)
            # the device's pick is the argmax of its own scores
            assert sc_dev[da[t]] >= sc_dev[S[t]], (t, sc_dev[da[t]], sc_dev[S[t]])
    for t in sample_steps:
        if 1 <= t < k and t not in st.measured_steps:
            measure(t)
    return st


def teacher_forced_parity(run_gpu, ref, gap_tol=GAP_TOL, max_rounds=64, m=None, dtype=None):
    """Compare the GPU's selection with the oracle step by step.  Where they
    differ the oracle's top-two gap must be below max(gap_tol, the path's
    score error bound for the two candidates) (both picks are then correct in
    the path's arithmetic); the GPU is re-run with the oracle's prefix forced
    and the comparison resumes after it.  Returns the number of forced
    restarts."""
    forced = []
    restarts = 0
    while True:
        got = run_gpu(forced)
        assert got[: len(forced)] == ref.S[: len(forced)]
        t = first_mismatch(got, ref.S, len(forced))
        if t is None:
            assert len(got) == len(ref.S), (len(got), len(ref.S))
            return restarts
        tol = gap_tol
        if m is not None and dtype is not None and ref.fs:
            tol = max(tol, pair_error_bound(ref, t, m, dtype))
        assert ref.gaps[t] <= tol, (
            f"step {t}: GPU picked {got[t]}, oracle {ref.S[t]}, oracle gap {ref.gaps[t]:.3e} "
            f"> allowed {tol:.3e}")
        forced = list(ref.S[: t + 1])
        restarts += 1
        assert restarts <= max_rounds


# ------------------------------------------------------ gradient, entry-wise
def gradient_entry_errors(G, G_ref, S, tol=None, tol_S=None):
    """Entry-wise error of a gradient against the oracle's, each entry scaled
    by the largest magnitude in its column of the oracle's gradient (and, if
    given, by that column's tolerance: `tol` for the columns outside S and
    `tol_S` for those in S, each an array over all columns or a number).  Returns (worst over the
    columns outside S, worst over the columns in S), so that a single wrong
    entry or column shows up at its own size instead of inside a norm of the
    whole matrix; with tolerances both must be <= 1."""
    G = np.asarray(G, dtype=np.float64)
    G_ref = np.asarray(G_ref, dtype=np.float64)
    colmax = np.max(np.abs(G_ref), axis=0)
    colmax = np.where(colmax > 0, colmax, 1e-300)
    scale = colmax if tol is None else colmax * np.broadcast_to(np.asarray(tol, dtype=np.float64), colmax.shape)
    ratio = np.abs(G - G_ref) / scale[None, :]
    inS = np.zeros(G.shape[1], dtype=bool)
    inS[list(S)] = True
    rest = float(np.max(ratio[:, ~inS])) if (~inS).any() else 0.0
    if tol_S is not None:
        tS = np.broadcast_to(np.asarray(tol_S, dtype=np.float64), colmax.shape)[inS]
        ratio_S = np.abs(G - G_ref)[:, inS] / (colmax[inS] * tS)[None, :]
    else:
        ratio_S = ratio[:, inS]
    sel = float(np.max(ratio_S)) if inS.any() else 0.0
    return rest, sel


def gradient_tolerances(vals, S, G_ref, dtype):
    """Entry-wise tolerances of the adjoint's dA, relative to each column's
    largest entry of the oracle's gradient.

    The device forms Q = A_S L^-T from the Cholesky factor L of A_S^T A_S
    (FP64), so Q's columns are orthonormal to about 4 k u_64 cond(A_S)^2
    (the normal-equations route squares the condition).  Columns outside S
    hold 2R with R = A - Q W: W = Q^T A (dot products of length m) and Q W
    (length k) are formed in FP64 (FP64 input) or in double-float (unit
    roundoff about 2^-48), so |dR_ij| <= ((m + k) u_acc + 4 k u_64
    cond(A_S)^2) ||a_j|| (|(QW)_ij| <= ||a_j||); then dA is rounded to A's
    own dtype (unit roundoff u_out: 2^-53, 2^-24, 2^-8 for BF16's 8-bit
    significand):
        tol_j = 2 u_out + 2 ((m + k) u_acc + 4 k u_64 cond^2) ||a_j|| / max_i |G_ij|.
    Columns in S hold -2 R T^T = -2 (R W^T) L^-1: R W^T sums over the n
    columns in FP64 (FP64 input) or FP32, each entry within lambda
    sqrt(n + m) u of its terms (hm_lambda), L^-1 multiplies by up to
    cond(A_S), and R carries the error above:
        tol_S,j = 2 u_out + lambda sqrt(n + m) u_sum cond + (the R term of tol_j).
    Returns (tol over all columns, tol_S over all columns)."""
    m, n = vals.shape
    k = len(S)
    u_out = {torch.float64: 2.0 ** -53, torch.float32: 2.0 ** -24, torch.bfloat16: 2.0 ** -8}[dtype]
    u_acc = 2.0 ** -53 if dtype == torch.float64 else 2.0 ** -48
    u_sum = 2.0 ** -53 if dtype == torch.float64 else 2.0 ** -24
    colmax = np.max(np.abs(G_ref), axis=0)
    colmax = np.where(colmax > 0, colmax, 1e-300)
    kappa = float(np.linalg.cond(vals[:, list(S)]))
    r_term = 2.0 * ((m + k) * u_acc + 4.0 * k * 2.0 ** -53 * kappa ** 2) * np.linalg.norm(vals, axis=0) / colmax
    tol = 2 * u_out + r_term
    lam = hm_lambda(n + m, m * k)
    tol_S = 2 * u_out + lam * np.sqrt(n + m) * u_sum * kappa + r_term
    return tol, tol_S
