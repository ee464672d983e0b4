"""GPU checks of css_residual_backward: the loss ||A - P^(S) A||_F^2 and its
gradient at a fixed S, against the oracle's closed form, finite differences
(torch.autograd.gradcheck on the FP64 path) and the full 4096 x 16384 case."""
import numpy as np
import pytest
import torch

import css_inputs as ci
from oracle import css_oracle as O
from tests.gpu_helpers import dev_matrix, gradient_entry_errors, gradient_tolerances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def css():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_6838_gb300 import build, css as mod
    build.build()
    return mod


def _grad(css, A, S):
    Ag = A.detach().requires_grad_(True)
    L = css.residual(Ag, S)
    L.backward()
    return float(L.item()), Ag.grad


def test_gradcheck_fp64(css):
    """Finite differences of the device loss against the device adjoint."""
    A_np = ci.lowrank_uv(64, 128, 8, 0.05, 501)
    S = O.greedy_css(A_np, 8).S
    A, _ = dev_matrix(A_np, torch.float64)
    A.requires_grad_(True)
    assert torch.autograd.gradcheck(lambda X: css.residual(X, S), (A,), eps=1e-6, atol=1e-6,
                                    rtol=1e-5, fast_mode=True)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("shape", [(64, 128, 8), (257, 1000, 31), (500, 777, 64)])
def test_gradient_matches_oracle(css, dtype, shape):
    m, n, k = shape
    A_np = ci.lowrank_uv(m, n, k, 1e-3, 600 + m)
    A, vals = dev_matrix(A_np, dtype)
    S = O.greedy_css(vals, k, tau_rel=1e-10).S
    L_ref, G_ref = O.residual_gradient(vals, S)
    L, G = _grad(css, A, S)
    assert abs(L - L_ref) <= 1e-7 * L_ref, (L, L_ref)
    G = G.double().cpu().numpy()
    tol, tol_S = gradient_tolerances(vals, S, G_ref, dtype)
    rest, sel = gradient_entry_errors(G, G_ref, S, tol, tol_S)
    print(f"dA {dtype} {shape}: worst entry error / its tolerance: outside S {rest:.3e}, in S {sel:.3e}")
    assert rest <= 1.0, rest
    # the selected columns' block -2 R T^T separately
    assert sel <= 1.0, sel


def test_gradient_k_above_128_fp64(css):
    """k = 160 takes the blocked Cholesky of A_S^T A_S.  Going through the
    normal-equations matrix squares the condition of A_S, so the FP64 bound
    is c k u kappa(A_S)^2 (u = 2^-53): here kappa = 412, and a plain numpy
    evaluation of the same Cholesky route is itself 1.4e-10 from the
    oracle's (the device: 3.1e-10)."""
    m, n, k = 600, 900, 160
    A_np = ci.lowrank_uv(m, n, k, 1e-3, 600 + m)
    A, vals = dev_matrix(A_np, torch.float64)
    S = O.greedy_css(vals, k, tau_rel=1e-10).S
    L_ref, G_ref = O.residual_gradient(vals, S)
    L, G = _grad(css, A, S)
    assert abs(L - L_ref) <= 1e-7 * L_ref, (L, L_ref)
    kappa = np.linalg.cond(vals[:, S])
    tol = max(1e-10, 4.0 * k * 2.0 ** -53 * kappa ** 2)
    G = G.double().cpu().numpy()
    err = np.linalg.norm(G - G_ref) / np.linalg.norm(G_ref)
    assert err <= tol, (err, tol)
    # entry by entry, relative to each column's largest entry
    tol_c, tol_S = gradient_tolerances(vals, S, G_ref, torch.float64)
    rest, sel = gradient_entry_errors(G, G_ref, S, np.maximum(tol_c, tol), np.maximum(tol_S, tol))
    print(f"dA FP64 k = 160: worst entry error / its tolerance: outside S {rest:.3e}, in S {sel:.3e}")
    assert rest <= 1.0, rest
    assert sel <= 1.0, sel


def test_loss_only_and_grad_out_scaling(css):
    from paper_1312_6838_gb300 import _lib as L
    import ctypes as C
    A_np = ci.lowrank_uv(80, 300, 10, 1e-2, 700)
    A, vals = dev_matrix(A_np, torch.float32)
    S = O.greedy_css(vals, 10).S
    L_ref, G_ref = O.residual_gradient(vals, S)
    lib = L.load()
    m, n = A.shape
    sel = torch.tensor(S, dtype=torch.int32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    o = L.default_opts()
    nb = lib.css_workspace_size(L.CSS_OP_BACKWARD, L.CSS_F32, m, n, 0, len(S), 0, C.byref(o))
    ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    wp = ws.data_ptr() + (-ws.data_ptr()) % 256
    dA = css.empty_colmajor(m, n, torch.float32)
    code = lib.css_residual_backward(C.c_void_p(A.data_ptr()), L.CSS_F32, m, n, A.stride(1),
                                     C.c_void_p(sel.data_ptr()), len(S), 0.25,
                                     C.c_void_p(dA.data_ptr()), dA.stride(1),
                                     C.c_void_p(loss.data_ptr()), C.c_void_p(wp), nb, C.byref(o),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 0
    assert abs(loss.item() - L_ref) <= 1e-7 * L_ref
    tol, tol_S = gradient_tolerances(vals, S, 0.25 * G_ref, torch.float32)
    rest, sel = gradient_entry_errors(dA.double().cpu().numpy(), 0.25 * G_ref, S, tol, tol_S)
    assert rest <= 1.0, rest
    assert sel <= 1.0, sel


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
def test_residual_error_resolves_tiny_errors(css, dtype):
    """css.residual_error at an error of ~1e-8 of ||A||_F^2 (rank-k signal,
    1e-4 noise, the signal's own k columns selected): the direct residual
    keeps its accuracy where a recursion subtracting O(||A||^2) terms would
    not."""
    A_np = ci.lowrank_uv(200, 900, 12, 1e-4, 702)
    A, vals = dev_matrix(A_np, dtype)
    S = O.greedy_css(vals, 12).S
    e_ref = O.reconstruction_error(vals, S)
    # (BF16 rounding of the entries adds its own noise of ~2^-9 relative)
    assert e_ref <= (1e-4 if dtype == torch.bfloat16 else 1e-7) * float(np.sum(vals * vals))
    got = css.residual_error(A, S)
    tol = 1e-10 if dtype == torch.float64 else 1e-5
    assert abs(got - e_ref) <= tol * e_ref, (got, e_ref)


def test_rank_deficient_selection_rejected(css):
    from paper_1312_6838_gb300._lib import CssError
    A_np = ci.lowrank_uv(30, 60, 5, 0.0, 701)
    A_np[:, 7] = A_np[:, 3]
    A, _ = dev_matrix(A_np, torch.float64)
    with pytest.raises(CssError):
        css.residual(A, [3, 7, 9])
    with pytest.raises(CssError):
        css.residual(A, [3, 3])


@pytest.mark.slow
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float64])
def test_full_adjoint_workload(css, dtype):
    """4096 x 16384 (FP32 as configured; BF16 and FP64 too), rank 128 + 1e-3
    noise, S = the oracle's greedy set of 128 columns; the oracle's
    closed-form FP64 gradient of the same values on the host, compared entry
    by entry."""
    c = ci.CONFIGS["adjoint_4096x16384"]
    A_np = ci.lowrank_uv(c["m"], c["n"], c["rank"], c["noise"], c["seed"], dtype=np.float32)
    A, vals = dev_matrix(A_np, dtype)
    del A_np
    S = O.greedy_css(vals, c["k"], tau_rel=1e-6).S
    L_ref, G_ref = O.residual_gradient(vals, S)
    L, G = _grad(css, A, S)
    assert abs(L - L_ref) <= 1e-6 * L_ref, (L, L_ref)
    G = G.double().cpu().numpy()
    tol, tol_S = gradient_tolerances(vals, S, G_ref, dtype)
    rest, sel = gradient_entry_errors(G, G_ref, S, tol, tol_S)
    print(f"dA 4096 x 16384 {dtype}: worst entry error / its tolerance: outside S {rest:.3e}, in S {sel:.3e}")
    assert rest <= 1.0, rest
    assert sel <= 1.0, sel
