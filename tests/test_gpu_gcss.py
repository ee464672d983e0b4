"""GPU parity of gcss_select (Algorithm 3), gcss_distributed (Algorithm 4),
css_project (Algorithm 2) and css_select_batched against the FP64 oracle."""
import numpy as np
import pytest
import torch

import css_inputs as ci
from oracle import css_oracle as O
from tests.gpu_helpers import (certify_selection, dev_matrix, first_mismatch, oracle_path_parity,
                               pair_error_bound, trace_error_bound)

pytestmark = pytest.mark.gpu

TAU = {torch.float64: 1e-12, torch.float32: 1e-6, torch.bfloat16: 1e-6}
ERR_TOL = {torch.float64: 1e-10, torch.float32: 1e-4, torch.bfloat16: 1e-4}


@pytest.fixture(scope="module")
def css():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_6838_gb300 import build, css as mod
    build.build()
    return mod


def _target(B_np, dtype):
    from paper_1312_6838_gb300 import css
    bdt = torch.float64 if dtype == torch.float64 else torch.float32
    vals = B_np.astype(np.float64) if bdt == torch.float64 else B_np.astype(np.float32).astype(np.float64)
    return css.to_colmajor(torch.from_numpy(vals).to(bdt).cuda()), vals


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("shape", [(40, 90, 6, 10), (129, 700, 33, 20), (64, 333, 1, 8),
                                   (48, 257, 24, 10)])
def test_gcss_parity(css, dtype, shape):
    """Index parity within the path's error bound (k may exceed the target's
    rank: the late picks are then only defined up to that bound)."""
    m, n, r, k = shape
    A_np = ci.lowrank_uv(m, n, 8 if r < 24 else 40, 0.05, m + n)
    B_np = A_np @ ci.gaussian_omega(n, r, 7, dtype=np.float64)
    A, Av = dev_matrix(A_np, dtype)
    B, Bv = _target(B_np, dtype)
    ref = O.greedy_gcss(Av, Bv, k, tau_rel=TAU[dtype], keep_scores=True)
    # the initial scores ||B^T a_i||^2 are dot products of length m
    run = lambda prefix, kk, diag: css.gcss_select(A, B, kk, forced=prefix or None, diag=diag)
    stats = oracle_path_parity(run, ref, m, dtype, TAU[dtype],
                               sample_steps=(1, k // 2, k - 1))
    res = css.gcss_select(A, B, k)
    S = res.indices.cpu().tolist()
    e_gpu = O.reconstruction_error(Av, S, Bv)
    e_ref = O.reconstruction_error(Av, ref.S, Bv)
    if S == list(ref.S):
        assert abs(e_gpu - e_ref) <= ERR_TOL[dtype] * max(e_ref, 1e-12 * ref.trace[0])
    else:
        # parted at a near-tie: every pick of the device's own selection is a
        # greedy pick within the rule on its own path
        assert dtype != torch.float64 or stats.widened == 0
        ref_dev = O.greedy_gcss(Av, Bv, len(S), tau_rel=TAU[dtype], keep_scores=True, forced=S)
        certify_selection(S, ref_dev, m, dtype)
    full = css.gcss_select(A, B, len(ref.S), forced=list(ref.S))
    tr = full.trace.cpu().numpy()[: len(ref.S) + 1]
    bound = trace_error_bound(ref, m, dtype)
    assert np.all(np.abs(tr - np.asarray(ref.trace)) <= bound), np.max(np.abs(tr - ref.trace) / bound)


def test_gcss_with_B_equal_A_is_css(css):
    A_np = ci.lowrank_uv(50, 160, 7, 0.03, 21)
    A, Av = dev_matrix(A_np, torch.float64)
    B, _ = _target(A_np, torch.float64)
    a = css.select(A, 12).indices.cpu().tolist()
    b = css.gcss_select(A, B, 12).indices.cpu().tolist()
    assert a == b


def test_gcss_fp64_trace_and_W(css):
    A_np = ci.lowrank_uv(45, 110, 9, 0.02, 22)
    B_np = A_np @ ci.gaussian_omega(110, 12, 23, dtype=np.float64)
    A, Av = dev_matrix(A_np, torch.float64)
    B, Bv = _target(B_np, torch.float64)
    res = css.gcss_select(A, B, 14, return_W=True)
    ref = O.greedy_gcss(Av, Bv, 14)
    assert res.indices.cpu().tolist() == ref.S
    np.testing.assert_allclose(res.trace.cpu().numpy(), ref.trace, rtol=0, atol=1e-10 * ref.trace[0])
    np.testing.assert_allclose(res.W.cpu().numpy(), ref.W, rtol=1e-8, atol=1e-9 * np.abs(ref.W).max())


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
def test_distributed_parity(css, dtype):
    m, n, r = 48, 900, 10
    A_np = ci.lowrank_uv(m, n, 12, 0.05, 31)
    B_np = A_np @ ci.gaussian_omega(n, r, 32, dtype=np.float64)
    offs = ci.lognormal_blocks(n, 6, 150, 0.8, 33, min_w=20)
    A, Av = dev_matrix(A_np, dtype)
    B, Bv = _target(B_np, dtype)
    res = css.distributed(A, B, offs.tolist(), 8, 10)
    final, per_block, r0 = O.distributed_css(Av, Bv, offs.tolist(), 8, 10, tau_rel=TAU[dtype])
    bsel = res.block_sel.cpu().numpy()
    for b, ids in enumerate(per_block):
        got = [int(v) for v in bsel[b] if v >= 0]
        if dtype == torch.float64:
            assert got == ids
    if dtype == torch.float64:
        assert res.indices.cpu().tolist() == final
    else:
        e_gpu = O.reconstruction_error(Av, res.indices.cpu().tolist(), Bv)
        e_ref = O.reconstruction_error(Av, final, Bv)
        assert e_gpu <= e_ref * (1 + 1e-3)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("shape", [(64, 1000, 16), (100, 4097, 33), (2048, 8192, 400)])
def test_projection(css, dtype, shape):
    m, n, r = shape
    A_np = ci.lowrank_uv(m, n, 8, 0.1, 41).astype(np.float32)
    Om_np = ci.gaussian_omega(n, r, 42, dtype=np.float32)
    A, Av = dev_matrix(A_np, dtype)
    Om, Ov = dev_matrix(Om_np, dtype)
    B = css.project(A, Om).cpu().numpy().astype(np.float64)
    ref = O.random_projection(Av, Ov)
    # FP32 accumulation bound: |dB| <= c * K * 2^-24 * sum |a||omega|
    bound = np.abs(Av) @ np.abs(Ov)
    eps = 2.0 ** -52 if dtype == torch.float64 else 2.0 ** -24
    assert np.all(np.abs(B - ref) <= 4 * np.sqrt(n) * eps * bound + 1e-30)


def test_batched_matches_single(css):
    specs = [(37, 120, 5), (64, 500, 9), (200, 129, 12), (96, 1000, 16), (300, 300, 8), (17, 40, 3)]
    As, vals, ks = [], [], []
    for i, (m, n, k) in enumerate(specs):
        A_np = ci.batched_instance(m, n, k, 100 + i)
        A, Av = dev_matrix(A_np, torch.float32)
        As.append(A)
        vals.append(Av)
        ks.append(k)
    out = css.select_batched(As, ks)
    for A, Av, k, res in zip(As, vals, ks, out):
        ref = O.greedy_css(Av, k, tau_rel=1e-6, keep_scores=True)
        got = res.indices.cpu().tolist()
        t = first_mismatch(got, ref.S)
        e_gpu = O.reconstruction_error(Av, got)
        e_ref = O.reconstruction_error(Av, ref.S)
        if t is None:
            assert got == ref.S
            assert abs(e_gpu - e_ref) <= 1e-4 * e_ref
        else:
            assert ref.gaps[t] <= max(1e-6, pair_error_bound(ref, t, Av.shape[0], torch.float32))
            ref_dev = O.greedy_css(Av, len(got), tau_rel=1e-6, keep_scores=True, forced=got)
            certify_selection(got, ref_dev, Av.shape[0], torch.float32)


@pytest.mark.parametrize("grid", [3, 1000])
def test_batched_team_layouts(css, grid):
    specs = [(40 + 7 * i, 100 + 31 * i, 4 + i % 5) for i in range(24)]
    As, ks = [], []
    for i, (m, n, k) in enumerate(specs):
        A, _ = dev_matrix(ci.batched_instance(m, n, k, 200 + i), torch.float64)
        As.append(A)
        ks.append(k)
    out = css.select_batched(As, ks, grid_ctas=grid)
    for A, k, res in zip(As, ks, out):
        assert res.indices.cpu().tolist() == css.select(A, k).indices.cpu().tolist()
