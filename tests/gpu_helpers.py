"""Shared helpers of the GPU parity tests (imported by tests only)."""
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


# Unit roundoff of the dot-product accumulation of each path.
EPS = {torch.float64: 2.0 ** -53, torch.float32: 2.0 ** -24, torch.bfloat16: 2.0 ** -24}
SAFETY = 8.0


def score_error_bound(ref, t, m, dtype):
    """Relative error bound of the device scores of the oracle's two best
    candidates at iteration t (needs the oracle run with keep_scores=True).

    The device updates f_i by increments computed from dot products with the
    original column a_i, each accurate to about eps * sqrt(m) relative to
    f_i^(0); after t updates the error relative to the current f_i is
    eps * sqrt(m) * sqrt(t + 1) * f_i^(0) / f_i.  Below this gap both picks
    are correct in the path's arithmetic."""
    sc = ref.scores[t]
    f, f0 = ref.fs[t], ref.fs[0]
    s = np.where(np.isfinite(sc), sc, -np.inf)
    top = np.argsort(-s, kind="stable")[:2]
    b = 0.0
    for i in top:
        if np.isfinite(s[i]):
            b += abs(f0[i]) / max(abs(f[i]), 1e-300)
    return SAFETY * EPS[dtype] * np.sqrt(m) * np.sqrt(t + 1) * b


def teacher_forced_parity(run_gpu, ref, gap_tol=GAP_TOL, max_rounds=64, m=None, dtype=None):
    """Compare the GPU's selection with the oracle step by step.  Where they
    differ the oracle's top-two gap must be below max(gap_tol, the path's
    score error bound) (both picks are then correct); the GPU is re-run with
    the oracle's prefix forced and the comparison resumes after it.  Returns
    the number of forced restarts."""
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
            tol = max(tol, score_error_bound(ref, t, m, dtype))
        assert ref.gaps[t] <= tol, (
            f"step {t}: GPU picked {got[t]}, oracle {ref.S[t]}, oracle gap {ref.gaps[t]:.3e} "
            f"> allowed {tol:.3e}")
        forced = list(ref.S[: t + 1])
        restarts += 1
        assert restarts <= max_rounds
