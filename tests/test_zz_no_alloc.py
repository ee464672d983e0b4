"""css_select_noalloc: the allocation-free variant of css_select.

Some callers cannot allocate device memory (their host application has
reserved all of it, their framework forbids allocation calls, or they must
avoid the device-wide synchronisation cudaMalloc/cudaFree can cause).  This
entry point takes its scratch from a fixed array inside the library.  The
test calls it through the C ABI twice in a row and checks each result
against css_select with a caller workspace, within the tolerances the other
tests use.  It lives in a file of its own, collected last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import css_inputs as ci

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_6838_gb300 import _lib, build, css
    build.build()
    return _lib, css


def _noalloc(L, css, A, k, sync=True):
    m, n = A.shape
    lda = A.stride(1)
    dt = {torch.float64: L.CSS_F64, torch.float32: L.CSS_F32, torch.bfloat16: L.CSS_BF16}[A.dtype]
    sel = torch.full((k,), -1, dtype=torch.int32, device=A.device)
    trace = torch.zeros(k + 1, dtype=torch.float64, device=A.device)
    nsel = torch.zeros(1, dtype=torch.int32, device=A.device)
    o = L.default_opts()
    o.sync = 1 if sync else 0
    code = L.load().css_select_noalloc(
        C.c_void_p(A.data_ptr()), dt, m, n, lda, k, C.c_void_p(sel.data_ptr()),
        C.c_void_p(trace.data_ptr()), C.c_void_p(nsel.data_ptr()), C.c_void_p(0), C.byref(o),
        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return code, sel, trace, int(nsel.item())


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
def test_noalloc_matches_css_select_twice(mods, dtype):
    L, css = mods
    A_np = ci.lowrank_uv(300, 2000, 40, 0.05, 123)
    A = css.to_colmajor(torch.from_numpy(A_np).to(dtype).cuda())
    k = 20
    ref = css.select(A, k)
    tol = 1e-10 if dtype == torch.float64 else 1e-6
    for _ in range(2):
        code, sel, trace, ns = _noalloc(L, css, A, k)
        assert code == 0, L.status_string(code)
        assert ns == ref.n_sel == k
        assert sel.cpu().tolist() == ref.indices.cpu().tolist()
        np.testing.assert_allclose(trace.cpu().numpy(), ref.trace.cpu().numpy(), rtol=0,
                                   atol=tol * ref.trace[0].item())


def test_noalloc_rejects_sizes_beyond_its_scratch(mods):
    L, css = mods
    m, n, k = 4096, 16384, 128    # workspace > CSS_NOALLOC_SCRATCH_BYTES
    o = L.default_opts()
    need = L.load().css_workspace_size(L.CSS_OP_SELECT, L.CSS_F32, m, n, 0, k, 0, C.byref(o))
    assert need > L.CSS_NOALLOC_SCRATCH_BYTES
    A = css.empty_colmajor(m, n, torch.float32)
    code, _, _, _ = _noalloc(L, css, A, k)
    assert code == L.CSS_ERR_WORKSPACE


def test_noalloc_stale_scratch_from_a_larger_problem(mods):
    """The array keeps whatever the previous call left in it.  A call on a
    larger problem of another dtype (more columns, more picks, so more split
    slots, counters and descriptors in use) runs between two calls on a small
    problem; the small problem's result must still equal css_select's."""
    L, css = mods
    small = css.to_colmajor(torch.from_numpy(ci.lowrank_uv(120, 700, 12, 0.05, 321)).float().cuda())
    big = css.to_colmajor(torch.from_numpy(ci.lowrank_uv(512, 6000, 80, 0.05, 322)).to(torch.bfloat16).cuda())
    k_small, k_big = 10, 60
    ref = css.select(small, k_small)
    ref_big = css.select(big, k_big)
    for big_between in (False, True):
        if big_between:
            code, sel_b, _, ns_b = _noalloc(L, css, big, k_big)
            assert code == 0, L.status_string(code)
            assert ns_b == k_big
            assert sel_b.cpu().tolist() == ref_big.indices.cpu().tolist()
        code, sel, trace, ns = _noalloc(L, css, small, k_small)
        assert code == 0, L.status_string(code)
        assert ns == k_small
        assert sel.cpu().tolist() == ref.indices.cpu().tolist()
        assert torch.equal(trace, ref.trace)


def test_noalloc_rejects_asynchronous_calls(mods):
    """The call's device status lives in the library's array, which the caller
    cannot pass to css_read_status: sync = 0 is refused before any work."""
    L, css = mods
    A = css.to_colmajor(torch.from_numpy(ci.lowrank_uv(64, 200, 8, 0.05, 323)).float().cuda())
    code, sel, _, _ = _noalloc(L, css, A, 4, sync=False)
    assert code == L.CSS_ERR_INVALID_ARG
    assert sel.cpu().tolist() == [-1] * 4
