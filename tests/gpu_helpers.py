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


def teacher_forced_parity(run_gpu, ref, gap_tol=GAP_TOL, max_rounds=64):
    """Compare the GPU's selection with the oracle step by step.  Where they
    differ the oracle's top-two gap must be below gap_tol (both picks are then
    correct); the GPU is re-run with the oracle's prefix forced and the
    comparison resumes after it.  Returns the number of forced restarts."""
    forced = []
    restarts = 0
    while True:
        got = run_gpu(forced)
        assert got[: len(forced)] == ref.S[: len(forced)]
        t = first_mismatch(got, ref.S, len(forced))
        if t is None:
            assert len(got) == len(ref.S), (len(got), len(ref.S))
            return restarts
        assert ref.gaps[t] <= gap_tol, (
            f"step {t}: GPU picked {got[t]}, oracle {ref.S[t]}, oracle gap {ref.gaps[t]:.3e}")
        forced = list(ref.S[: t + 1])
        restarts += 1
        assert restarts <= max_rounds
