"""Omega drawn on the device (Philox4x32-10) against the oracle's independent
implementation, and B = A Omega with a generated Omega (css_project_random)
against the oracle's Algorithm 2 on the oracle's Omega."""
import numpy as np
import pytest
import torch

import css_inputs as ci
from oracle import css_oracle as O
from tests.gpu_helpers import dev_matrix

pytestmark = pytest.mark.gpu

DIST = {"gaussian": O.OMEGA_GAUSSIAN, "sparse_sign": O.OMEGA_SPARSE_SIGN}
EPS = {torch.float64: 2.0 ** -53, torch.float32: 2.0 ** -24, torch.bfloat16: 2.0 ** -24}


@pytest.fixture(scope="module")
def css():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_6838_gb300 import build, css as mod
    build.build()
    return mod


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("shape", [(1, 1), (777, 13), (4096, 100), (40000, 7)])
@pytest.mark.parametrize("seed", [0, 123456789, (7 << 32) + 5])
def test_omega_matches_oracle(css, dtype, shape, seed):
    n, r = shape
    for dist, code in DIST.items():
        got = css.random_omega(n, r, seed, dist, dtype).double().cpu().numpy()
        ref = O.random_omega(n, r, seed, code)
        if dist == "sparse_sign":
            np.testing.assert_array_equal(got, ref)       # integer decision, exact values
        elif dtype == torch.float64:
            np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-15)
        elif dtype == torch.float32:
            # FP32 Box-Muller: ln u1 to ~1e-7 relative, the angle to 2^-24 of a
            # turn (cos within 4e-7), sqrt(-2 ln u1) <= 6.7
            np.testing.assert_allclose(got, ref, rtol=2e-6, atol=6e-6 / np.sqrt(r))
        else:
            # then one rounding to BF16 (relative 2^-8 at worst)
            np.testing.assert_allclose(got, ref, rtol=2.0 ** -8 + 2e-6, atol=6e-6 / np.sqrt(r))


def test_omega_is_a_function_of_position_and_seed(css):
    a = css.random_omega(500, 20, 42, "gaussian")
    b = css.random_omega(800, 20, 42, "gaussian")
    assert torch.equal(a, b[:500])
    assert torch.equal(a, css.random_omega(500, 20, 42, "gaussian"))
    assert not torch.equal(a, css.random_omega(500, 20, 43, "gaussian"))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("shape", [(64, 700, 24), (300, 4096, 100), (2048, 16384, 400), (3000, 5000, 17)])
def test_sparse_sign_projection(css, dtype, shape):
    """No Omega is formed on the device: each column of B gathers the selected
    +-columns of A in row order.  FP32 sums (FP64 for FP64 input) against the
    FP64 product: error within n_terms * eps of sum |A| |Omega|."""
    m, n, r = shape
    A_np = ci.lowrank_uv(m, n, 8, 0.1, 900 + m)
    A, Av = dev_matrix(A_np, dtype)
    seed = 77 + n
    B = css.project_random(A, r, seed, "sparse_sign").double().cpu().numpy()
    Om = O.random_omega(n, r, seed, O.OMEGA_SPARSE_SIGN)
    ref = O.random_projection(Av, Om)
    bound = np.abs(Av) @ np.abs(Om)
    terms = max(1, int(np.max(np.count_nonzero(Om, axis=0))))
    assert np.all(np.abs(B - ref) <= 2 * terms * EPS[dtype] * bound + 1e-300)
    # reproducible bit for bit
    B2 = css.project_random(A, r, seed, "sparse_sign").double().cpu().numpy()
    np.testing.assert_array_equal(B, B2)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("shape", [(64, 700, 24), (256, 3000, 400), (2048, 16384, 400)])
def test_gaussian_projection(css, dtype, shape):
    """Omega generated in A's dtype, then css_project (tensor cores for BF16):
    the device Omega's own rounding (BF16: 2^-8 of each entry; FP32 Box-Muller
    as above) plus the product's accumulation bound."""
    m, n, r = shape
    A_np = ci.lowrank_uv(m, n, 8, 0.1, 950 + m)
    A, Av = dev_matrix(A_np, dtype)
    seed = 5 + m
    B = css.project_random(A, r, seed, "gaussian").double().cpu().numpy()
    Om = O.random_omega(n, r, seed, O.OMEGA_GAUSSIAN)
    ref = O.random_projection(Av, Om)
    bound = np.abs(Av) @ np.abs(Om)
    om_rel = {torch.float64: 1e-13, torch.float32: 2e-6, torch.bfloat16: 2.0 ** -8 + 2e-6}[dtype]
    om_abs = {torch.float64: 1e-15, torch.float32: 6e-6, torch.bfloat16: 6e-6}[dtype] / np.sqrt(r)
    tol = (om_rel + 4 * np.sqrt(n) * EPS[dtype]) * bound + om_abs * (np.abs(Av) @ np.ones((n, r)))
    assert np.all(np.abs(B - ref) <= tol + 1e-300)
