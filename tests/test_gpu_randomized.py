"""RndGreedyCSS on the device (css_select_randomized) against the oracle:
Algorithm 3 for the target B = A Omega with the oracle's own Omega."""
import numpy as np
import pytest
import torch

import css_inputs as ci
from oracle import css_oracle as O
from tests.gpu_helpers import dev_matrix

pytestmark = pytest.mark.gpu

DISTS = [("gaussian", O.OMEGA_GAUSSIAN), ("sparse_sign", O.OMEGA_SPARSE_SIGN)]


@pytest.fixture(scope="module")
def css():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_6838_gb300 import build, css as mod
    build.build()
    return mod


def _oracle(vals, l, seed, code, tau):
    B = O.random_projection(vals, O.random_omega(vals.shape[1], l, seed, code))
    return O.greedy_gcss(vals, B, l, tau_rel=tau, keep_scores=True), B


@pytest.mark.parametrize("dist,code", DISTS)
@pytest.mark.parametrize("shape", [(120, 800, 10), (300, 2000, 16)])
def test_fp64_indices_match_the_oracle(css, dist, code, shape):
    """FP64: Omega to ~1e-13 and FP64 arithmetic throughout, so the picks agree
    wherever the oracle's top-two gap is above 1e-6 (compared up to the first
    pick that is closer)."""
    m, n, l = shape
    A_np = ci.lowrank_uv(m, n, 2 * l, 0.05, 1234 + m)
    A, vals = dev_matrix(A_np, torch.float64)
    seed = 99 + n
    ref, B = _oracle(vals, l, seed, code, 1e-12)
    got = css.select_randomized(A, l, seed, dist)
    assert got.n_sel == len(ref.S)
    S = got.indices.cpu().tolist()
    for t, gap in enumerate(ref.gaps):
        if gap <= 1e-6:
            break
        assert S[t] == ref.S[t], (t, S[t], ref.S[t])
    # Theorem 3's trace starts from ||B||_F^2
    assert abs(got.trace[0].item() - np.linalg.norm(B) ** 2) <= 1e-10 * np.linalg.norm(B) ** 2


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("dist,code", DISTS)
def test_mixed_selection_error(css, dtype, dist, code):
    """BF16/FP32: the device draws Omega in FP32 and accumulates in FP32; the
    reconstruction error of A by its selection stays within 1e-4 of the
    oracle's selection's (or below it)."""
    m, n, l = 256, 3000, 16
    A_np = ci.lowrank_uv(m, n, 2 * l, 0.05, 4321)
    A, vals = dev_matrix(A_np, dtype)
    seed = 7
    ref, _ = _oracle(vals, l, seed, code, 1e-6)
    got = css.select_randomized(A, l, seed, dist)
    e_gpu = O.reconstruction_error(vals, got.indices.cpu().tolist())
    e_ref = O.reconstruction_error(vals, ref.S)
    assert e_gpu <= e_ref * (1 + 1e-4)
