"""Bounded device waits running out, made to happen on purpose through the
library's test hook (css_opts.test_unmet_wait): a team barrier of the
persistent greedy kernel, or an mbarrier of the tensor-core initial-score
kernels, waits for an arrival that never comes.  The wait must end after
the caller's spin budget with CSS_ERR_TIMEOUT -- no trap, no fault -- and
the next call on the same context must give the same result as before."""
import ctypes as C

import numpy as np
import pytest
import torch

import css_inputs as ci
from tests.gpu_helpers import dev_matrix

pytestmark = pytest.mark.gpu

BUDGET_NS = 20_000_000   # 20 ms: far longer than any wait of these problems


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_6838_gb300 import _lib, build, css
    build.build()
    return _lib, css


def _problem(dtype):
    # 32 CTAs in the team (n / 128 and m / 16), so the barriers are real
    A, _ = dev_matrix(ci.lowrank_uv(512, 4096, 24, 0.05, 811), dtype)
    return A


@pytest.mark.parametrize("hook,dtype", [(1, torch.float32), (1, torch.bfloat16), (1, torch.float64),
                                        (2, torch.bfloat16)])
def test_select_wait_runs_out_then_context_is_usable(mods, hook, dtype):
    L, css = mods
    A = _problem(dtype)
    ref = css.select(A, 16)
    with pytest.raises(L.CssError) as ei:
        css.select(A, 16, spin_budget_ns=BUDGET_NS, test_unmet_wait=hook)
    assert ei.value.code == L.CSS_ERR_TIMEOUT
    again = css.select(A, 16)
    assert torch.equal(again.sel, ref.sel)
    assert torch.equal(again.trace, ref.trace)


@pytest.mark.parametrize("hook", [1, 2])
def test_gcss_wait_runs_out_then_context_is_usable(mods, hook):
    L, css = mods
    A = _problem(torch.bfloat16)
    B = css.to_colmajor(torch.from_numpy(
        ci.lowrank_uv(512, 4096, 24, 0.05, 811) @ ci.gaussian_omega(4096, 64, 812, dtype=np.float64)
    ).float().cuda())
    ref = css.gcss_select(A, B, 12)
    with pytest.raises(L.CssError) as ei:
        css.gcss_select(A, B, 12, spin_budget_ns=BUDGET_NS, test_unmet_wait=hook)
    assert ei.value.code == L.CSS_ERR_TIMEOUT
    again = css.gcss_select(A, B, 12)
    assert torch.equal(again.sel, ref.sel)
    assert torch.equal(again.trace, ref.trace)


@pytest.mark.parametrize("hook", [1, 2])
def test_async_call_reports_timeout_through_read_status(mods, hook):
    """sync = 0: the call returns CSS_OK once its work is queued, and
    css_read_status on the same workspace reports the wait that ran out,
    whether it was the greedy kernel's or the tensor-core kernel's."""
    L, css = mods
    A = _problem(torch.bfloat16)
    m, n = A.shape
    k = 16
    lib = L.load()
    o = L.default_opts()
    o.sync = 0
    o.spin_budget_ns = BUDGET_NS
    o.test_unmet_wait = hook
    nb = lib.css_workspace_size(L.CSS_OP_SELECT, L.CSS_BF16, m, n, 0, k, 0, C.byref(o))
    buf = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    wp = buf.data_ptr() + (-buf.data_ptr()) % 256
    sel = torch.empty(k, dtype=torch.int32, device="cuda")
    trace = torch.empty(k + 1, dtype=torch.float64, device="cuda")
    nsel = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = lib.css_select(C.c_void_p(A.data_ptr()), L.CSS_BF16, m, n, A.stride(1), k,
                          C.c_void_p(sel.data_ptr()), C.c_void_p(trace.data_ptr()),
                          C.c_void_p(nsel.data_ptr()), C.c_void_p(0), C.c_void_p(wp), nb, C.byref(o),
                          stream)
    assert code == L.CSS_OK
    assert lib.css_read_status(C.c_void_p(wp), stream) == L.CSS_ERR_TIMEOUT
    # the same workspace, without the hook: a clean status
    o.test_unmet_wait = 0
    code = lib.css_select(C.c_void_p(A.data_ptr()), L.CSS_BF16, m, n, A.stride(1), k,
                          C.c_void_p(sel.data_ptr()), C.c_void_p(trace.data_ptr()),
                          C.c_void_p(nsel.data_ptr()), C.c_void_p(0), C.c_void_p(wp), nb, C.byref(o),
                          stream)
    assert code == L.CSS_OK
    assert lib.css_read_status(C.c_void_p(wp), stream) == L.CSS_OK
    assert sel.cpu().tolist() == css.select(A, k).indices.cpu().tolist()


def test_hook_values_are_checked(mods):
    L, css = mods
    A = _problem(torch.float32)
    with pytest.raises(L.CssError) as ei:
        css.select(A, 4, test_unmet_wait=3)
    assert ei.value.code == L.CSS_ERR_INVALID_ARG
