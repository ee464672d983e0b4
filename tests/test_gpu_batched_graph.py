"""css_select_batched_prepare / css_select_batched_run: repeated runs and a
CUDA-graph replay of the device work give the selections of a direct
css_select_batched call (same kernels, so the same bits), including after the
matrices' values change in place; one problem is also checked against the
oracle."""
import numpy as np
import pytest
import torch

import css_inputs as ci
from oracle import css_oracle as O
from tests.gpu_helpers import dev_matrix

pytestmark = pytest.mark.gpu

SHAPES = [(64, 300, 8), (200, 1000, 16), (129, 777, 12), (512, 2048, 24), (1000, 500, 10),
          (300, 4096, 32)]


@pytest.fixture(scope="module")
def css():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_6838_gb300 import build, css as mod
    build.build()
    return mod


def _problems(seed, dtype):
    As, ks, vals = [], [], []
    for i, (m, n, k) in enumerate(SHAPES):
        A, v = dev_matrix(ci.lowrank_uv(m, n, 2 * k, 0.05, seed * 100 + i), dtype)
        As.append(A)
        ks.append(k)
        vals.append(v)
    return As, ks, vals


def _same(ref, got):
    for a, b in zip(ref, got):
        assert a.n_sel == b.n_sel
        assert torch.equal(a.indices, b.indices)
        assert torch.equal(a.trace, b.trace)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_prepared_runs_match_direct_call(css, dtype):
    As, ks, _ = _problems(3, dtype)
    ref = css.select_batched(As, ks)
    plan = css.BatchedPlan(As, ks)
    for _ in range(2):
        plan.run()
        assert plan.status() == 0
        _same(ref, plan.results())


def test_cuda_graph_replay(css):
    As, ks, _ = _problems(5, torch.float32)
    plan = css.BatchedPlan(As, ks)
    plan.run()                      # first launches outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.run()
    # new values in the same storage, then replay the captured work
    As2, _, vals2 = _problems(6, torch.float32)
    for A, A2 in zip(As, As2):
        A.copy_(A2)
    g.replay()
    torch.cuda.synchronize()
    assert plan.status() == 0
    got = plan.results()
    _same(css.select_batched(As, ks), got)
    # the replay selected on the new values: oracle parity for one problem
    # (signal rank 2k, so every pick is far from a tie)
    ref = O.greedy_css(vals2[1], ks[1], tau_rel=1e-6)
    assert got[1].indices.cpu().tolist() == list(ref.S)
    g.replay()
    torch.cuda.synchronize()
    _same(css.select_batched(As, ks), plan.results())


def test_run_rejects_another_workspace(css):
    from paper_1312_6838_gb300 import _lib as L
    import ctypes as C
    As, ks, _ = _problems(7, torch.float32)
    plan = css.BatchedPlan(As[:2], ks[:2])
    lib = L.load()
    other = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    code = lib.css_select_batched_run(C.byref(plan._plan), C.c_void_p(other.data_ptr()),
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == L.CSS_ERR_INVALID_ARG
