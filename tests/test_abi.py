"""Host-side checks of the C ABI: the library builds/loads, exports every
function include/css.h declares, and rejects bad arguments before touching
the GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1312_6838_gb300 import _lib, build
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    return _lib.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "css.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z_0-9]*\s*\*?\s*([a-z_][a-z_0-9]*)\s*\(",
                       src, flags=re.M)
    return sorted(set(n for n in names if n.startswith(("css_", "gcss_"))))


def test_every_declared_symbol_is_exported(lib):
    from paper_1312_6838_gb300 import _lib
    names = _declared()
    assert len(names) >= 14, names
    for n in names:
        assert hasattr(lib, n), f"libcss.so does not export {n}"
    assert set(names) == set(_lib.EXPORTED)


def test_version_and_status_strings(lib):
    assert b"libcss" in lib.css_version()
    names = {0: b"CSS_OK", 1: b"CSS_RANK_EXHAUSTED", -1: b"CSS_ERR_INVALID_ARG", -2: b"CSS_ERR_CUDA",
             -3: b"CSS_ERR_NO_MEMORY", -4: b"CSS_ERR_WORKSPACE", -5: b"CSS_ERR_TIMEOUT",
             -6: b"CSS_ERR_NONFINITE", -7: b"CSS_ERR_UNSUPPORTED", -8: b"CSS_ERR_NOT_CONVERGED"}
    for code, name in names.items():
        assert lib.css_status_string(code).startswith(name), (code, lib.css_status_string(code))


def test_workspace_size_is_host_only(lib):
    from paper_1312_6838_gb300 import _lib as L
    o = L.default_opts()
    a = lib.css_workspace_size(L.CSS_OP_SELECT, L.CSS_BF16, 4096, 65536, 0, 256, 0, C.byref(o))
    b = lib.css_workspace_size(L.CSS_OP_SELECT, L.CSS_F32, 4096, 65536, 0, 256, 0, C.byref(o))
    assert a > 0 and b > 0
    # C = A A^T (m x m FP32, plus its BF16 split for the tensor-core initial
    # scores) dominates; W (k x n FP64) is an optional caller output, so the
    # workspace grows with k only through Q and Z (m x k each)
    assert a >= 4096 * 4096 * 4 and b >= 4096 * 4096 * 4
    a4 = lib.css_workspace_size(L.CSS_OP_SELECT, L.CSS_BF16, 4096, 65536, 0, 1024, 0, C.byref(o))
    assert 0 < a4 - a < 4 * 4096 * (1024 - 256) * 8
    assert lib.css_workspace_size(L.CSS_OP_SELECT, L.CSS_F32, 0, 10, 0, 1, 0, None) == 0
    assert lib.css_workspace_size(L.CSS_OP_GCSS, L.CSS_F32, 100, 1000, 0, 10, 0, None) == 0
    assert lib.css_workspace_size(L.CSS_OP_PROJECT, L.CSS_BF16, 2048, 262144, 400, 0, 0, None) > 0
    offs = (C.c_int64 * 4)(0, 10, 25, 40)
    assert lib.gcss_distributed_workspace_size(L.CSS_F32, 8, 40, 3, offs, 3, 4, 5) > 0
    bad = (C.c_int64 * 4)(0, 10, 10, 40)
    assert lib.gcss_distributed_workspace_size(L.CSS_F32, 8, 40, 3, bad, 3, 4, 5) == 0


def test_invalid_arguments_rejected_on_host(lib):
    from paper_1312_6838_gb300 import _lib as L
    o = L.default_opts()
    P = C.c_void_p
    fake = P(0x10000)  # never dereferenced: validation fails first
    # NULL A
    r = lib.css_select(P(0), L.CSS_F32, 10, 20, 10, 3, fake, fake, fake, P(0), fake, 1 << 20,
                       C.byref(o), P(0))
    assert r == L.CSS_ERR_INVALID_ARG
    # k > n
    r = lib.css_select(fake, L.CSS_F32, 10, 2, 10, 3, fake, fake, fake, P(0), fake, 1 << 20,
                       C.byref(o), P(0))
    assert r == L.CSS_ERR_INVALID_ARG
    # lda < m
    r = lib.css_select(fake, L.CSS_F32, 10, 20, 9, 3, fake, fake, fake, P(0), fake, 1 << 20,
                       C.byref(o), P(0))
    assert r == L.CSS_ERR_INVALID_ARG
    # misaligned workspace
    r = lib.css_select(fake, L.CSS_F32, 10, 20, 10, 3, fake, fake, fake, P(0), P(0x10008), 1 << 20,
                       C.byref(o), P(0))
    assert r == L.CSS_ERR_WORKSPACE
    # workspace too small
    r = lib.css_select(fake, L.CSS_F32, 10, 20, 10, 3, fake, fake, fake, P(0), fake, 16,
                       C.byref(o), P(0))
    assert r == L.CSS_ERR_WORKSPACE
    # bad score mode
    o.score_mode = 7
    r = lib.css_select(fake, L.CSS_F32, 10, 20, 10, 3, fake, fake, fake, P(0), fake, 1 << 20,
                       C.byref(o), P(0))
    assert r == L.CSS_ERR_INVALID_ARG
    o.score_mode = 0
    # GCSS: B rows / ldb
    r = lib.gcss_select(fake, L.CSS_F32, 10, 20, 10, fake, 3, 9, 3, fake, fake, fake, P(0), fake,
                        1 << 20, C.byref(o), P(0))
    assert r == L.CSS_ERR_INVALID_ARG
    # distributed: offsets that do not end at n
    offs = (C.c_int64 * 3)(0, 5, 19)
    r = lib.gcss_distributed(fake, L.CSS_F32, 10, 20, 10, fake, 3, 10, offs, 2, 2, 2, fake, fake,
                             fake, P(0), fake, 1 << 20, C.byref(o), P(0))
    assert r == L.CSS_ERR_INVALID_ARG
    # projection: ldo < n
    r = lib.css_project(fake, L.CSS_BF16, 10, 20, 10, fake, 4, 19, fake, 10, fake, 1 << 20,
                        C.byref(o), P(0))
    assert r == L.CSS_ERR_INVALID_ARG


def test_opts_layout_matches_header(lib):
    from paper_1312_6838_gb300 import _lib as L
    o = L.default_opts()
    assert o.tau_rel < 0 and o.sync == 1 and o.n_forced == 0 and o.grid_ctas == 0


def test_embed_and_lowrank_host_checks(lib):
    """Sec. 3.2 entry points: workspace sizes need no device, and argument
    errors are found on the host before anything is enqueued."""
    from paper_1312_6838_gb300 import _lib as L
    o = L.default_opts()
    P = C.c_void_p
    fake = P(0x10000)
    assert lib.css_workspace_size(L.CSS_OP_EMBED, L.CSS_BF16, 4096, 65536, 0, 256, 0, None) > 0
    assert lib.css_workspace_size(L.CSS_OP_EMBED, L.CSS_BF16, 100, 65536, 0, 101, 0, None) == 0
    assert lib.css_workspace_size(L.CSS_OP_EMBED, L.CSS_F64, 4096, 65536, 0, 1025, 0, None) == 0
    a = lib.css_workspace_size(L.CSS_OP_LOWRANK, L.CSS_F64, 4096, 65536, 256, 128, 0, None)
    b = lib.css_workspace_size(L.CSS_OP_LOWRANK, L.CSS_F64, 0, 65536, 256, 128, 0, None)
    assert a > 0 and a == b                       # m is not needed for the workspace
    assert lib.css_workspace_size(L.CSS_OP_LOWRANK, L.CSS_F64, 0, 65536, 256, 257, 0, None) == 0
    assert lib.css_workspace_size(L.CSS_OP_LOWRANK, L.CSS_F64, 0, 65536, 1025, 10, 0, None) == 0
    # css_embed: NULL A, no output requested, l > m, repeated check needs a device (not here)
    r = lib.css_embed(P(0), L.CSS_F32, 10, 20, 10, fake, 3, fake, 10, fake, 20, fake, 1 << 20, C.byref(o), P(0))
    assert r == L.CSS_ERR_INVALID_ARG
    r = lib.css_embed(fake, L.CSS_F32, 10, 20, 10, fake, 3, P(0), 10, P(0), 20, fake, 1 << 20, C.byref(o), P(0))
    assert r == L.CSS_ERR_INVALID_ARG
    r = lib.css_embed(fake, L.CSS_F32, 10, 20, 10, fake, 11, fake, 10, fake, 20, fake, 1 << 20, C.byref(o), P(0))
    assert r == L.CSS_ERR_INVALID_ARG
    r = lib.css_embed(fake, L.CSS_F32, 10, 20, 10, fake, 3, fake, 9, P(0), 20, fake, 1 << 20, C.byref(o), P(0))
    assert r == L.CSS_ERR_INVALID_ARG              # ldq < m
    # css_lowrank: NULL W, k > l, ldw < n, U without Q, workspace too small
    r = lib.css_lowrank(P(0), 20, P(0), 0, 0, 20, 4, 2, fake, P(0), 1, P(0), 20, P(0), P(0), fake, 1 << 30,
                        C.byref(o), P(0))
    assert r == L.CSS_ERR_INVALID_ARG
    r = lib.css_lowrank(fake, 20, P(0), 0, 0, 20, 4, 5, fake, P(0), 1, P(0), 20, P(0), P(0), fake, 1 << 30,
                        C.byref(o), P(0))
    assert r == L.CSS_ERR_INVALID_ARG
    r = lib.css_lowrank(fake, 19, P(0), 0, 0, 20, 4, 2, fake, P(0), 1, P(0), 20, P(0), P(0), fake, 1 << 30,
                        C.byref(o), P(0))
    assert r == L.CSS_ERR_INVALID_ARG
    r = lib.css_lowrank(fake, 20, P(0), 0, 10, 20, 4, 2, fake, fake, 10, P(0), 20, P(0), P(0), fake, 1 << 30,
                        C.byref(o), P(0))
    assert r == L.CSS_ERR_INVALID_ARG
    r = lib.css_lowrank(fake, 20, P(0), 0, 0, 20, 4, 2, fake, P(0), 1, P(0), 20, P(0), P(0), fake, 64,
                        C.byref(o), P(0))
    assert r == L.CSS_ERR_WORKSPACE


def test_batch_descriptors_match_the_struct(lib):
    """css.select_batched fills css_problem[count] as a numpy record array:
    every field must land where the C struct has it (read back through
    ctypes), the outputs of problem i are views at the running offsets, and
    the host-only workspace query sees the same batch as a field-by-field
    fill."""
    import torch
    from paper_1312_6838_gb300 import _lib as L, css
    As = [torch.empty((7, 5)).t(), torch.empty((40, 33)).t()[:30], torch.empty((9, 4)).t()]
    ks = [2, 3, 4]
    b = css._Batch(As, ks)
    arr = (L.css_problem * len(As)).from_address(b.rec.ctypes.data)
    ref = (L.css_problem * len(As))()
    for i, (A, k) in enumerate(zip(As, ks)):
        p = arr[i]
        m, n, lda = css._colmajor(A)
        assert (p.A, p.m, p.n, p.lda, p.k) == (A.data_ptr(), m, n, lda, k)
        assert p.sel == b.sel.data_ptr() + 4 * sum(ks[:i])
        assert p.trace == b.trace.data_ptr() + 8 * sum(v + 1 for v in ks[:i])
        assert p.n_sel == b.n_sel.data_ptr() + 4 * i and not p.W
        ref[i].A, ref[i].m, ref[i].n, ref[i].lda, ref[i].k = A.data_ptr(), m, n, lda, k
        ref[i].sel, ref[i].trace, ref[i].n_sel = p.sel, p.trace, p.n_sel
    o = L.default_opts()
    for dt in (L.CSS_F32, L.CSS_BF16, L.CSS_F64):
        got = lib.css_batched_workspace_size(b.probs(), len(As), dt, C.byref(o))
        assert got > 0 and got == lib.css_batched_workspace_size(ref, len(As), dt, C.byref(o))
    res = b.results()
    assert [tuple(r.sel.shape) + tuple(r.trace.shape) for r in res] == [(2, 3), (3, 4), (4, 5)]
    with pytest.raises(ValueError):
        css._Batch(As, [2, 0, 4])
    with pytest.raises(TypeError):
        css._Batch([As[0], As[1].double()], [2, 3])


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of css_opts, css_problem and the two plan structs
    (paper_1312_6838_gb300/_lib.py) against include/css.h as a C compiler
    lays it out: every field's offset and size, and each struct's size."""
    import shutil
    import subprocess
    from paper_1312_6838_gb300 import _lib as L
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [L.css_opts, L.css_problem, L.css_batched_plan, L.css_distributed_plan]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "css.h"', "int main(void) {"]
    for S in structs:
        name = S.__name__
        lines.append(f'  printf("{name} . %zu %zu\\n", (size_t)0, sizeof({name}));')
        for f, _ in S._fields_:
            lines.append(f'  printf("{name} {f} %zu %zu\\n", offsetof({name}, {f}), '
                         f'sizeof((({name}*)0)->{f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = 0
    for line in filter(None, out):
        name, field, off, size = line.split()
        S = getattr(L, name)
        if field == ".":
            assert C.sizeof(S) == int(size), (name, C.sizeof(S), size)
        else:
            d = getattr(S, field)
            assert (d.offset, d.size) == (int(off), int(size)), (name, field, d.offset, d.size, off, size)
        seen += 1
    assert seen == sum(len(S._fields_) + 1 for S in structs)
