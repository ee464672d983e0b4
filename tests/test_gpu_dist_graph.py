"""gcss_distributed_prepare / gcss_distributed_run (Algorithm 4 with the union
of the blocks' picks built on the device): repeated runs and a CUDA-graph
replay of the whole pipeline give the bits of a direct gcss_distributed call,
including after A and B change in place, and the replay's selection matches
the oracle's Algorithm 4 on the new values."""
import numpy as np
import pytest
import torch

import css_inputs as ci
from oracle import css_oracle as O
from tests.gpu_helpers import dev_matrix

pytestmark = pytest.mark.gpu

M, N, R = 64, 1500, 12


@pytest.fixture(scope="module")
def css():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_6838_gb300 import build, css as mod
    build.build()
    return mod


def _inputs(seed, dtype):
    A_np = ci.lowrank_uv(M, N, 20, 0.05, seed)
    B_np = A_np @ ci.gaussian_omega(N, R, seed + 1, dtype=np.float64)
    A, Av = dev_matrix(A_np, dtype)
    bdt = torch.float64 if dtype == torch.float64 else torch.float32
    Bv = B_np if dtype == torch.float64 else B_np.astype(np.float32).astype(np.float64)
    from paper_1312_6838_gb300 import css
    B = css.to_colmajor(torch.from_numpy(Bv).to(bdt).cuda())
    return A, B, Av, Bv


OFFS = ci.lognormal_blocks(N, 7, 200, 0.8, 77, min_w=30).tolist()
LB, K = 10, 12


def _same(a, b):
    assert a.n_sel == b.n_sel
    assert torch.equal(a.sel[: a.n_sel], b.sel[: b.n_sel])
    assert torch.equal(a.trace[: a.n_sel + 1], b.trace[: b.n_sel + 1])
    assert torch.equal(a.block_sel, b.block_sel)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
def test_prepared_runs_match_direct_call(css, dtype):
    A, B, _, _ = _inputs(1001, dtype)
    ref = css.distributed(A, B, OFFS, LB, K)
    plan = css.DistributedPlan(A, B, OFFS, LB, K)
    for _ in range(2):
        plan.run()
        assert plan.status() == 0
        _same(ref, plan.result())


@pytest.mark.parametrize("dtype", [torch.float64, torch.bfloat16])
def test_cuda_graph_replay(css, dtype):
    A, B, _, _ = _inputs(1003, dtype)
    plan = css.DistributedPlan(A, B, OFFS, LB, K)
    plan.run()                      # first launches outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.run()
    # new values in the same storage, then replay the captured pipeline
    A2, B2, Av2, Bv2 = _inputs(1005, dtype)
    A.copy_(A2)
    B.copy_(B2)
    g.replay()
    torch.cuda.synchronize()
    assert plan.status() == 0
    got = plan.result()
    _same(css.distributed(A, B, OFFS, LB, K), got)
    final, per_block, _ = O.distributed_css(Av2, Bv2, OFFS, LB, K,
                                            tau_rel=1e-12 if dtype == torch.float64 else 1e-6)
    if dtype == torch.float64:
        assert got.indices.cpu().tolist() == list(final)
        bsel = got.block_sel.cpu().numpy()
        for b, ids in enumerate(per_block):
            assert [int(v) for v in bsel[b] if v >= 0] == ids
    else:
        e_gpu = O.reconstruction_error(Av2, got.indices.cpu().tolist(), Bv2)
        e_ref = O.reconstruction_error(Av2, final, Bv2)
        assert e_gpu <= e_ref * (1 + 1e-4)
    g.replay()
    torch.cuda.synchronize()
    _same(css.distributed(A, B, OFFS, LB, K), plan.result())


def test_union_smaller_than_k_reports_rank_exhausted(css):
    """Blocks of zero columns pick nothing, so the union holds fewer than k
    columns: the pipeline returns CSS_RANK_EXHAUSTED with n_sel = the union's
    size, and the picks it made are valid global ids."""
    from paper_1312_6838_gb300 import _lib as L
    A_np = ci.lowrank_uv(M, N, 20, 0.05, 1007)
    offs = [0, 400, 800, 1500]
    A_np[:, 400:1500] = 0.0
    A, _ = dev_matrix(A_np, torch.float64)
    B = css.to_colmajor(torch.from_numpy(A_np @ ci.gaussian_omega(N, R, 1008, dtype=np.float64)).cuda())
    plan = css.DistributedPlan(A, B, offs, 5, 8)
    plan.run()
    assert plan.status() == L.CSS_RANK_EXHAUSTED
    got = plan.result()
    assert got.n_sel == 5
    S = got.indices.cpu().tolist()
    assert all(0 <= j < 400 for j in S)
    assert got.sel[5:].cpu().tolist() == [-1] * 3
    bsel = got.block_sel.cpu().numpy()
    assert (bsel[1:] == -1).all()


def test_run_rejects_another_workspace(css):
    from paper_1312_6838_gb300 import _lib as L
    import ctypes as C
    A, B, _, _ = _inputs(1009, torch.float32)
    plan = css.DistributedPlan(A, B, OFFS, LB, K)
    other = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    code = L.load().gcss_distributed_run(C.byref(plan._plan), C.c_void_p(other.data_ptr()),
                                         C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == L.CSS_ERR_INVALID_ARG
