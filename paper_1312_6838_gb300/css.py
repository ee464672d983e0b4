"""Python front end of libcss: torch tensors in, C-ABI calls out.

Every function here only checks shapes, allocates the caller-side buffers
(outputs and the workspace, through torch's allocator) and calls the C ABI;
all arithmetic runs in the CUDA library.  Matrices are column-major: pass a
tensor whose ``stride(0) == 1`` (for example ``X.t()`` of a row-major n x m
tensor X whose rows are the columns of A).

Functions mirror include/css.h:

* ``select``            Algorithm 1 (greedy CSS)
* ``gcss_select``       Algorithm 3 (greedy generalized CSS, target B)
* ``distributed``       Algorithm 4 (per-block GCSS, then GCSS on the union)
* ``project``           B = A Omega (Sec. 5.1, Algorithm 2)
* ``select_batched``    independent Algorithm 1 instances in one launch
* ``residual``          ||A - P^(S) A||_F^2 with a hand-written adjoint
* ``select_host``       Algorithm 1 from host memory (copies included)
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib as L

_DT = {torch.float64: L.CSS_F64, torch.float32: L.CSS_F32, torch.bfloat16: L.CSS_BF16}
_ACC = {torch.float64: torch.float64, torch.float32: torch.float32, torch.bfloat16: torch.float32}


def _check(code, where):
    if code < 0:
        raise L.CssError(code, where)
    return code


def _colmajor(A: torch.Tensor, name="A"):
    if A.dim() != 2:
        raise ValueError(f"{name} must be 2-D")
    if A.dtype not in _DT:
        raise TypeError(f"{name}: dtype {A.dtype} not supported (float64, float32, bfloat16)")
    m, n = A.shape
    if m > 1 and A.stride(0) != 1:
        raise ValueError(f"{name} must be column-major (stride(0) == 1); pass X.t() "
                         "for a row-major tensor X holding the columns as rows")
    lda = A.stride(1) if n > 1 else m
    return m, n, max(lda, m)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor]):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _workspace(nbytes, device):
    # 256-byte aligned device buffer from torch's allocator
    buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    off = (-buf.data_ptr()) % 256
    return buf, buf[off:off + nbytes]


def empty_colmajor(m, n, dtype, device="cuda", ld=None):
    """A column-major m x n tensor (leading dimension ld >= m)."""
    ld = ld or m
    storage = torch.empty((n, ld), dtype=dtype, device=device)
    return storage[:, :m].t()


def to_colmajor(X: torch.Tensor, ld=None):
    """Copy X (m x n) into a column-major tensor with leading dimension ld."""
    m, n = X.shape
    out = empty_colmajor(m, n, X.dtype, X.device, ld)
    out.copy_(X)
    return out


@dataclass
class Selection:
    sel: torch.Tensor            # int32[k] selected columns, selection order (first n_sel valid)
    trace: torch.Tensor          # float64[k+1] error trace (Theorem 1 / 3)
    n_sel: int
    status: int
    W: Optional[torch.Tensor] = None        # float64[k, n] omega rows
    diag_argmax: Optional[torch.Tensor] = None
    diag_f: Optional[torch.Tensor] = None
    diag_g: Optional[torch.Tensor] = None
    timing_ms: Optional[tuple] = None       # (initial scores, greedy iterations)
    trace_ns: Optional[torch.Tensor] = None  # int64[k, 16] phase timestamps
    basis: Optional[torch.Tensor] = None    # float64 (m, k) column-major: Q, W = Q^T A

    @property
    def indices(self):
        return self.sel[: self.n_sel]


def _opts(tau_rel=None, forced=None, score_mode=0, grid_ctas=0, tile_cols=0, spin_budget_ns=0,
          sync=True, diag=None, init_path=0, test_unmet_wait=0, split_share=0, pivot_cost=0):
    o = L.default_opts()
    o.init_path = int(init_path)
    o.test_unmet_wait = int(test_unmet_wait)
    o.split_share = int(split_share)
    o.pivot_cost = int(pivot_cost)
    if tau_rel is not None:
        o.tau_rel = float(tau_rel)
    if forced is not None:
        o.forced = forced.data_ptr()
        o.n_forced = int(forced.numel())
    o.score_mode = int(score_mode)
    o.grid_ctas = int(grid_ctas)
    o.tile_cols = int(tile_cols)
    o.spin_budget_ns = int(spin_budget_ns)
    o.sync = 1 if sync else 0
    if diag is not None:
        o.diag_argmax = diag[0].data_ptr()
        o.diag_f = diag[1].data_ptr()
        o.diag_g = diag[2].data_ptr()
    return o


def _prep_forced(forced, device):
    if forced is None:
        return None
    return torch.as_tensor(list(forced) if not torch.is_tensor(forced) else forced,
                           dtype=torch.int32).to(device).contiguous()


def select(A: torch.Tensor, k: int, *, tau_rel=None, forced=None, return_W=False, diag=False,
           score_mode=0, grid_ctas=0, tile_cols=0, spin_budget_ns=0, stream=None,
           timing=False, phase_trace=False, init_path=0, return_basis=False,
           test_unmet_wait=0, split_share=0) -> Selection:
    """Greedy CSS (Algorithm 1) of the columns of A (column-major, on the GPU).
    ``test_unmet_wait`` is the test hook of the bounded device waits (css.h)."""
    m, n, lda = _colmajor(A)
    dev = A.device
    dt = _DT[A.dtype]
    lib = L.load()
    sel = torch.empty(k, dtype=torch.int32, device=dev)
    trace = torch.empty(k + 1, dtype=torch.float64, device=dev)
    nsel = torch.zeros(1, dtype=torch.int32, device=dev)
    W = torch.empty((k, n), dtype=torch.float64, device=dev) if return_W else None
    fz = _prep_forced(forced, dev)
    dg = None
    if diag:
        dg = (torch.full((k,), -1, dtype=torch.int32, device=dev),
              torch.empty(n, dtype=torch.float64, device=dev),
              torch.empty(n, dtype=torch.float64, device=dev))
    o = _opts(tau_rel, fz, score_mode, grid_ctas, tile_cols, spin_budget_ns, True, dg, init_path,
              test_unmet_wait, split_share)
    tms = (C.c_double * 2)() if timing else None
    if tms is not None:
        o.timing_ms = C.cast(tms, C.c_void_p)
    tr = torch.zeros((k, 16), dtype=torch.int64, device=dev) if phase_trace else None
    if tr is not None:
        o.trace_ns = tr.data_ptr()
    Qb = torch.empty((k, m), dtype=torch.float64, device=dev).t() if return_basis else None
    if Qb is not None:
        o.basis = Qb.data_ptr()
    nbytes = lib.css_workspace_size(L.CSS_OP_SELECT, dt, m, n, 0, k, 0, C.byref(o))
    if nbytes == 0:
        raise ValueError("invalid sizes for css_select")
    _keep, ws = _workspace(nbytes, dev)
    code = lib.css_select(_ptr(A), dt, m, n, lda, k, _ptr(sel), _ptr(trace), _ptr(nsel), _ptr(W),
                          _ptr(ws), nbytes, C.byref(o), _stream(stream))
    _check(code, "css_select")
    ns = int(nsel.item())
    res = Selection(sel, trace, ns, code, W, *(dg if dg else (None, None, None)))
    if tms is not None:
        res.timing_ms = (tms[0], tms[1])
    res.trace_ns = tr
    res.basis = Qb
    return res


def gcss_select(A: torch.Tensor, B: torch.Tensor, k: int, *, tau_rel=None, forced=None,
                return_W=False, diag=False, grid_ctas=0, tile_cols=0, spin_budget_ns=0,
                stream=None, init_path=0, return_basis=False, test_unmet_wait=0) -> Selection:
    """Greedy generalized CSS (Algorithm 3): columns of A reconstructing B.
    B must be float64 when A is float64, float32 otherwise (column-major)."""
    m, n, lda = _colmajor(A)
    mb, r, ldb = _colmajor(B, "B")
    if mb != m:
        raise ValueError("A and B must have the same number of rows")
    if B.dtype != _ACC[A.dtype]:
        raise TypeError(f"B must be {_ACC[A.dtype]} for A of dtype {A.dtype}")
    dev = A.device
    dt = _DT[A.dtype]
    lib = L.load()
    sel = torch.empty(k, dtype=torch.int32, device=dev)
    trace = torch.empty(k + 1, dtype=torch.float64, device=dev)
    nsel = torch.zeros(1, dtype=torch.int32, device=dev)
    W = torch.empty((k, n), dtype=torch.float64, device=dev) if return_W else None
    fz = _prep_forced(forced, dev)
    dg = None
    if diag:
        dg = (torch.full((k,), -1, dtype=torch.int32, device=dev),
              torch.empty(n, dtype=torch.float64, device=dev),
              torch.empty(n, dtype=torch.float64, device=dev))
    o = _opts(tau_rel, fz, 0, grid_ctas, tile_cols, spin_budget_ns, True, dg, init_path,
              test_unmet_wait)
    Qb = torch.empty((k, m), dtype=torch.float64, device=dev).t() if return_basis else None
    if Qb is not None:
        o.basis = Qb.data_ptr()
    nbytes = lib.css_workspace_size(L.CSS_OP_GCSS, dt, m, n, r, k, 0, C.byref(o))
    if nbytes == 0:
        raise ValueError("invalid sizes for gcss_select")
    _keep, ws = _workspace(nbytes, dev)
    code = lib.gcss_select(_ptr(A), dt, m, n, lda, _ptr(B), r, ldb, k, _ptr(sel), _ptr(trace),
                           _ptr(nsel), _ptr(W), _ptr(ws), nbytes, C.byref(o), _stream(stream))
    _check(code, "gcss_select")
    res = Selection(sel, trace, int(nsel.item()), code, W, *(dg if dg else (None, None, None)))
    res.basis = Qb
    return res


@dataclass
class Embedding:
    Q: torch.Tensor      # float64 (m, l), column-major: orth(A_:S)
    W: torch.Tensor      # float64 (l, n), row t contiguous: Q^T A


def embed(A: torch.Tensor, S, *, stream=None) -> Embedding:
    """Q = orth(A_:S) and W = Q^T A (Sec. 3.2, Eq. CSS_LowDim) on the GPU."""
    m, n, lda = _colmajor(A)
    dev = A.device
    dt = _DT[A.dtype]
    lib = L.load()
    sel = torch.as_tensor(list(S) if not torch.is_tensor(S) else S, dtype=torch.int32).to(dev).contiguous()
    l = int(sel.numel())
    Q = torch.empty((l, m), dtype=torch.float64, device=dev).t()
    W = torch.empty((l, n), dtype=torch.float64, device=dev)
    o = L.default_opts()
    nbytes = lib.css_workspace_size(L.CSS_OP_EMBED, dt, m, n, 0, l, 0, C.byref(o))
    if nbytes == 0:
        raise ValueError("invalid sizes for css_embed")
    _keep, ws = _workspace(nbytes, dev)
    code = lib.css_embed(_ptr(A), dt, m, n, lda, _ptr(sel), l, _ptr(Q), m, _ptr(W), n, _ptr(ws), nbytes,
                         C.byref(o), _stream(stream))
    _check(code, "css_embed")
    return Embedding(Q, W)


@dataclass
class LowRank:
    sigma: torch.Tensor                  # float64 (k,), descending
    Uw: torch.Tensor                     # float64 (l, k) column-major: U^(W)_k
    tail: float                          # sum_{i >= k} sigma_i(W)^2
    U: Optional[torch.Tensor] = None     # float64 (m, k) column-major: Q U^(W)_k
    V: Optional[torch.Tensor] = None     # float64 (n, k) column-major: V^(W)_k
    timing_ms: Optional[tuple] = None    # (Gram, eigendecomposition, products, sweeps)


def lowrank(W: torch.Tensor, k: int, Q: Optional[torch.Tensor] = None, *, want_V=True,
            stream=None, timing=False) -> LowRank:
    """Rank-k approximation / approximate SVD from an embedding (Sec. 3.2,
    Eq. ApproxSVD).  W: float64 (l, n) with unit column stride; Q: float64
    (m, l) column-major or None (then U is not formed)."""
    if W.dtype != torch.float64 or W.dim() != 2 or W.stride(1) != 1 or not W.is_cuda:
        raise TypeError("W must be a CUDA float64 (l, n) tensor with unit column stride")
    l, n = W.shape
    ldw = W.stride(0) if l > 1 else n
    dev = W.device
    m, ldq = 0, 1
    if Q is not None:
        m, lq, ldq = _colmajor(Q, "Q")
        if Q.dtype != torch.float64 or lq != l:
            raise TypeError("Q must be float64 (m, l) column-major")
    lib = L.load()
    sigma = torch.empty(k, dtype=torch.float64, device=dev)
    Uw = torch.empty((k, l), dtype=torch.float64, device=dev).t()
    tail = torch.empty(1, dtype=torch.float64, device=dev)
    U = torch.empty((k, m), dtype=torch.float64, device=dev).t() if Q is not None else None
    V = torch.empty((k, n), dtype=torch.float64, device=dev).t() if want_V else None
    o = L.default_opts()
    tms = (C.c_double * 4)() if timing else None
    if tms is not None:
        o.timing_ms = C.cast(tms, C.c_void_p)
    nbytes = lib.css_workspace_size(L.CSS_OP_LOWRANK, L.CSS_F64, m, n, l, k, 0, C.byref(o))
    if nbytes == 0:
        raise ValueError("invalid sizes for css_lowrank")
    _keep, ws = _workspace(nbytes, dev)
    code = lib.css_lowrank(_ptr(W), ldw, _ptr(Q), ldq, m, n, l, k, _ptr(sigma), _ptr(U), max(m, 1),
                           _ptr(V), n, _ptr(Uw), _ptr(tail), _ptr(ws), nbytes, C.byref(o),
                           _stream(stream))
    _check(code, "css_lowrank")
    return LowRank(sigma, Uw, float(tail.item()), U, V, tuple(tms) if tms is not None else None)


@dataclass
class Distributed:
    sel: torch.Tensor
    trace: torch.Tensor
    n_sel: int
    block_sel: torch.Tensor      # int32[nblocks, l_block], global ids, -1 padded
    status: int

    @property
    def indices(self):
        return self.sel[: self.n_sel]


def distributed(A: torch.Tensor, B: torch.Tensor, block_offsets: Sequence[int], l_block: int,
                k: int, *, tau_rel=None, grid_ctas=0, tile_cols=0, stream=None,
                init_path=0, timing=None, pivot_cost=0) -> Distributed:
    """Distributed CSS (Algorithm 4) with the concise representation B."""
    m, n, lda = _colmajor(A)
    mb, r, ldb = _colmajor(B, "B")
    if mb != m or B.dtype != _ACC[A.dtype]:
        raise ValueError("B must be m x r of dtype float32 (float64 for float64 A)")
    dev = A.device
    dt = _DT[A.dtype]
    lib = L.load()
    offs = (C.c_int64 * len(block_offsets))(*[int(v) for v in block_offsets])
    nb = len(block_offsets) - 1
    sel = torch.empty(k, dtype=torch.int32, device=dev)
    trace = torch.empty(k + 1, dtype=torch.float64, device=dev)
    nsel = torch.zeros(1, dtype=torch.int32, device=dev)
    bsel = torch.empty((nb, l_block), dtype=torch.int32, device=dev)
    o = _opts(tau_rel, None, 0, grid_ctas, tile_cols, init_path=init_path, pivot_cost=pivot_cost)
    tms = (C.c_double * 2)() if timing is not None else None
    if tms is not None:
        o.timing_ms = C.cast(tms, C.c_void_p)
    nbytes = lib.gcss_distributed_workspace_size(dt, m, n, r, offs, nb, l_block, k)
    if nbytes == 0:
        raise ValueError("invalid block partition or sizes")
    _keep, ws = _workspace(nbytes, dev)
    code = lib.gcss_distributed(_ptr(A), dt, m, n, lda, _ptr(B), r, ldb, offs, nb, l_block, k,
                                _ptr(sel), _ptr(trace), _ptr(nsel), _ptr(bsel), _ptr(ws), nbytes,
                                C.byref(o), _stream(stream))
    _check(code, "gcss_distributed")
    if tms is not None:
        # (initial scores, the blocks' persistent launch) in ms
        timing.extend([tms[0], tms[1]])
    return Distributed(sel, trace, int(nsel.item()), bsel, code)


class DistributedPlan:
    """Algorithm 4 prepared once (gcss_distributed_prepare) whose device work,
    run(), can be repeated or captured in a CUDA graph: it reads A and B given
    here (their storage must stay allocated; their values may change between
    runs) and writes the selection into the tensors held here."""

    def __init__(self, A: torch.Tensor, B: torch.Tensor, block_offsets: Sequence[int], l_block: int,
                 k: int, *, tau_rel=None, grid_ctas=0, tile_cols=0, stream=None, init_path=0):
        m, n, lda = _colmajor(A)
        mb, r, ldb = _colmajor(B, "B")
        if mb != m or B.dtype != _ACC[A.dtype]:
            raise ValueError("B must be m x r of dtype float32 (float64 for float64 A)")
        dev = A.device
        dt = _DT[A.dtype]
        self._lib = L.load()
        offs = (C.c_int64 * len(block_offsets))(*[int(v) for v in block_offsets])
        nb = len(block_offsets) - 1
        self.sel = torch.empty(k, dtype=torch.int32, device=dev)
        self.trace = torch.empty(k + 1, dtype=torch.float64, device=dev)
        self.nsel = torch.zeros(1, dtype=torch.int32, device=dev)
        self.block_sel = torch.empty((nb, l_block), dtype=torch.int32, device=dev)
        self._A, self._B = A, B
        o = _opts(tau_rel, None, 0, grid_ctas, tile_cols, init_path=init_path)
        nbytes = self._lib.gcss_distributed_workspace_size(dt, m, n, r, offs, nb, l_block, k)
        if nbytes == 0:
            raise ValueError("invalid block partition or sizes")
        self._keep, self._ws = _workspace(nbytes, dev)
        self._plan = L.css_distributed_plan()
        code = self._lib.gcss_distributed_prepare(
            _ptr(A), dt, m, n, lda, _ptr(B), r, ldb, offs, nb, l_block, k, _ptr(self.sel),
            _ptr(self.trace), _ptr(self.nsel), _ptr(self.block_sel), _ptr(self._ws), nbytes, C.byref(o),
            C.byref(self._plan), _stream(stream))
        _check(code, "gcss_distributed_prepare")

    def run(self, stream=None):
        """Enqueue the whole pipeline (device work only)."""
        code = self._lib.gcss_distributed_run(C.byref(self._plan), _ptr(self._ws), _stream(stream))
        _check(code, "gcss_distributed_run")

    def status(self, stream=None):
        """Status of the last run (synchronises the stream)."""
        return self._lib.css_read_status(_ptr(self._ws), _stream(stream))

    def result(self):
        return Distributed(self.sel, self.trace, int(self.nsel.item()), self.block_sel, 0)


def project(A: torch.Tensor, Omega: torch.Tensor, *, out=None, stream=None, sync=True,
            init_path=0):
    """B = A Omega (Sec. 5.1).  Omega is n x r column-major of A's dtype.
    Returns B (m x r, column-major) in float32 (float64 for float64 input)."""
    m, n, lda = _colmajor(A)
    no, r, ldo = _colmajor(Omega, "Omega")
    if no != n or Omega.dtype != A.dtype:
        raise ValueError("Omega must be n x r with A's dtype")
    dev = A.device
    dt = _DT[A.dtype]
    lib = L.load()
    B = out if out is not None else empty_colmajor(m, r, _ACC[A.dtype], dev)
    _, _, ldb = _colmajor(B, "B")
    o = _opts(sync=sync, init_path=init_path)
    nbytes = lib.css_workspace_size(L.CSS_OP_PROJECT, dt, m, n, r, 0, 0, C.byref(o))
    _keep, ws = _workspace(nbytes, dev)
    code = lib.css_project(_ptr(A), dt, m, n, lda, _ptr(Omega), r, ldo, _ptr(B), ldb, _ptr(ws),
                           nbytes, C.byref(o), _stream(stream))
    _check(code, "css_project")
    return B


OMEGA = {"gaussian": L.CSS_OMEGA_GAUSSIAN, "sparse_sign": L.CSS_OMEGA_SPARSE_SIGN}


def random_omega(n: int, r: int, seed: int, dist="gaussian", dtype=torch.float32, device="cuda",
                 stream=None) -> torch.Tensor:
    """Omega (n x r, column-major) drawn on the device from Philox4x32-10
    (css_random_omega): "gaussian" N(0, 1/r) or "sparse_sign"."""
    lib = L.load()
    Om = empty_colmajor(n, r, dtype, device)
    _, _, ldo = _colmajor(Om, "Omega")
    code = lib.css_random_omega(n, r, int(seed), OMEGA[dist], _DT[dtype], _ptr(Om), ldo, _stream(stream))
    _check(code, "css_random_omega")
    return Om


def project_random(A: torch.Tensor, r: int, seed: int, dist="gaussian", *, out=None, stream=None,
                   sync=True, init_path=0):
    """B = A Omega with Omega drawn on the device (css_project_random)."""
    m, n, lda = _colmajor(A)
    dev = A.device
    dt = _DT[A.dtype]
    lib = L.load()
    B = out if out is not None else empty_colmajor(m, r, _ACC[A.dtype], dev)
    _, _, ldb = _colmajor(B, "B")
    o = _opts(sync=sync, init_path=init_path)
    nbytes = lib.css_workspace_size(L.CSS_OP_PROJECT_RANDOM, dt, m, n, r, 0, 0, C.byref(o))
    _keep, ws = _workspace(nbytes, dev)
    code = lib.css_project_random(_ptr(A), dt, m, n, lda, r, int(seed), OMEGA[dist], _ptr(B), ldb,
                                  _ptr(ws), nbytes, C.byref(o), _stream(stream))
    _check(code, "css_project_random")
    return B


def select_randomized(A: torch.Tensor, l: int, seed: int, dist="gaussian", *, tau_rel=None,
                      stream=None) -> Selection:
    """RndGreedyCSS (Sec. 7): Algorithm 3 for the target B = A Omega with Omega
    n x l drawn on the device (css_select_randomized)."""
    m, n, lda = _colmajor(A)
    dev = A.device
    dt = _DT[A.dtype]
    lib = L.load()
    sel = torch.empty(l, dtype=torch.int32, device=dev)
    trace = torch.empty(l + 1, dtype=torch.float64, device=dev)
    nsel = torch.zeros(1, dtype=torch.int32, device=dev)
    o = _opts(tau_rel)
    nbytes = lib.css_workspace_size(L.CSS_OP_RANDOMIZED, dt, m, n, 0, l, 0, C.byref(o))
    _keep, ws = _workspace(nbytes, dev)
    code = lib.css_select_randomized(_ptr(A), dt, m, n, lda, l, int(seed), OMEGA[dist], _ptr(sel),
                                     _ptr(trace), _ptr(nsel), _ptr(ws), nbytes, C.byref(o),
                                     _stream(stream))
    _check(code, "css_select_randomized")
    return Selection(sel, trace, int(nsel.item()), code)


# css_problem as a numpy record (same field offsets), so that a batch's
# descriptors are filled by array operations rather than field by field
_PROBLEM = np.dtype({"names": [f for f, _ in L.css_problem._fields_],
                     "formats": ["<u8", "<i8", "<i8", "<i8", "<i4", "<i4", "<u8", "<u8", "<u8", "<u8"],
                     "offsets": [getattr(L.css_problem, f).offset for f, _ in L.css_problem._fields_],
                     "itemsize": C.sizeof(L.css_problem)})


class _Batch:
    """The css_problem descriptors of a batch and its outputs: one tensor each
    for every problem's indices, traces and counts (problem i's are views)."""

    def __init__(self, As: Sequence[torch.Tensor], ks: Sequence[int]):
        if len(As) != len(ks) or not As:
            raise ValueError("need one k per matrix")
        self.dtype = As[0].dtype
        self.device = As[0].device
        count = len(As)
        _colmajor(As[0])   # the dtype and layout checks' messages
        rows = []
        for A in As:
            if A.dtype != self.dtype:
                raise TypeError("all matrices must share one dtype")
            if A.dim() != 2:
                raise ValueError("A must be 2-D")
            m, n = A.shape
            s0, s1 = A.stride()
            if m > 1 and s0 != 1:
                raise ValueError("A must be column-major (stride(0) == 1)")
            rows.append((m, n, max(s1 if n > 1 else m, m), A.data_ptr()))
        tab = np.array(rows, dtype=np.uint64).reshape(count, 4)
        shape = tab[:, :3].astype(np.int64)
        ptr = tab[:, 3]
        k = np.asarray([int(v) for v in ks], dtype=np.int64)
        if (k < 1).any() or (k > np.iinfo(np.int32).max).any():
            raise ValueError("every k must be a positive int32")
        self.sel_off = np.concatenate(([0], np.cumsum(k)))
        self.trace_off = np.concatenate(([0], np.cumsum(k + 1)))
        self.sel = torch.empty(int(self.sel_off[-1]), dtype=torch.int32, device=self.device)
        self.trace = torch.empty(int(self.trace_off[-1]), dtype=torch.float64, device=self.device)
        self.n_sel = torch.zeros(count, dtype=torch.int32, device=self.device)
        rec = np.zeros(count, dtype=_PROBLEM)
        rec["A"] = ptr
        rec["m"], rec["n"], rec["lda"] = shape[:, 0], shape[:, 1], shape[:, 2]
        rec["k"] = k
        rec["sel"] = np.uint64(self.sel.data_ptr()) + 4 * self.sel_off[:-1].astype(np.uint64)
        rec["trace"] = np.uint64(self.trace.data_ptr()) + 8 * self.trace_off[:-1].astype(np.uint64)
        rec["n_sel"] = np.uint64(self.n_sel.data_ptr()) + 4 * np.arange(count, dtype=np.uint64)
        self.rec = rec
        self.count = count
        self.k = k.tolist()

    def probs(self):
        return self.rec.ctypes.data_as(C.POINTER(L.css_problem))

    def results(self, code=0):
        ns = self.n_sel.tolist()
        sels = self.sel.split(self.k)
        traces = self.trace.split([v + 1 for v in self.k])
        return [Selection(s, t, v, code) for s, t, v in zip(sels, traces, ns)]


def select_batched(As: Sequence[torch.Tensor], ks: Sequence[int], *, grid_ctas=0, tile_cols=0,
                   tau_rel=None, stream=None, timing=None, init_path=0):
    """Independent greedy CSS problems in one persistent launch.  Returns a list
    of Selection.  ``init_path=1`` keeps the initial scores on the SIMT
    kernels (css_opts.init_path)."""
    b = _Batch(As, ks)
    dt = _DT[b.dtype]
    lib = L.load()
    o = _opts(tau_rel, None, 0, grid_ctas, tile_cols, init_path=init_path)
    tms = (C.c_double * 2)() if timing is not None else None
    if tms is not None:
        o.timing_ms = C.cast(tms, C.c_void_p)
    nbytes = lib.css_batched_workspace_size(b.probs(), b.count, dt, C.byref(o))
    if nbytes == 0:
        raise ValueError("invalid batch")
    _keep, ws = _workspace(nbytes, b.device)
    code = lib.css_select_batched(b.probs(), b.count, dt, _ptr(ws), nbytes, C.byref(o), _stream(stream))
    _check(code, "css_select_batched")
    if tms is not None:
        timing.extend([tms[0], tms[1]])
    return b.results(code)


class BatchedPlan:
    """A batch prepared once (css_select_batched_prepare) whose device work,
    run(), can be repeated or captured in a CUDA graph: it reads the matrices
    given here (their storage must stay allocated; their values may change
    between runs) and writes the selections into the tensors held here."""

    def __init__(self, As: Sequence[torch.Tensor], ks: Sequence[int], *, grid_ctas=0,
                 tile_cols=0, tau_rel=None, stream=None, init_path=0):
        b = _Batch(As, ks)
        dt = _DT[b.dtype]
        self._lib = L.load()
        self._batch = b
        self._As = list(As)
        o = _opts(tau_rel, None, 0, grid_ctas, tile_cols, init_path=init_path)
        nbytes = self._lib.css_batched_workspace_size(b.probs(), b.count, dt, C.byref(o))
        if nbytes == 0:
            raise ValueError("invalid batch")
        self._keep, self._ws = _workspace(nbytes, b.device)
        self._plan = L.css_batched_plan()
        code = self._lib.css_select_batched_prepare(b.probs(), b.count, dt, _ptr(self._ws), nbytes,
                                                    C.byref(o), C.byref(self._plan), _stream(stream))
        _check(code, "css_select_batched_prepare")

    def run(self, stream=None):
        """Enqueue the initial scores and the persistent launch (device work only)."""
        code = self._lib.css_select_batched_run(C.byref(self._plan), _ptr(self._ws), _stream(stream))
        _check(code, "css_select_batched_run")

    def status(self, stream=None):
        """Status of the last run (synchronises the stream)."""
        return self._lib.css_read_status(_ptr(self._ws), _stream(stream))

    def results(self):
        return self._batch.results()


def autotune_distributed(A: torch.Tensor, B: torch.Tensor, block_offsets: Sequence[int], l_block: int,
                         k: int, *, stream=None):
    """Time Algorithm 4's planner pivot costs (300, 700, 1500, 3000 columns) on
    this problem and record the fastest for this device and shape bucket
    (css_autotune_distributed).  Returns (best cost, {cost: block-launch ms})."""
    m, n, lda = _colmajor(A)
    mb, r, ldb = _colmajor(B, "B")
    dt = _DT[A.dtype]
    lib = L.load()
    dev = A.device
    offs = (C.c_int64 * len(block_offsets))(*[int(v) for v in block_offsets])
    nb = len(block_offsets) - 1
    sel = torch.empty(k, dtype=torch.int32, device=dev)
    trace = torch.empty(k + 1, dtype=torch.float64, device=dev)
    nsel = torch.zeros(1, dtype=torch.int32, device=dev)
    nbytes = lib.gcss_distributed_workspace_size(dt, m, n, r, offs, nb, l_block, k)
    _keep, ws = _workspace(nbytes, dev)
    best = C.c_int32(0)
    times = (C.c_double * 4)()
    code = lib.css_autotune_distributed(_ptr(A), dt, m, n, lda, _ptr(B), r, ldb, offs, nb, l_block, k,
                                        _ptr(sel), _ptr(trace), _ptr(nsel), _ptr(ws), nbytes, C.byref(best),
                                        C.cast(times, C.c_void_p), _stream(stream))
    _check(code, "css_autotune_distributed")
    return best.value, {c: times[i] for i, c in enumerate((300, 700, 1500, 3000))}


def autotune(A: torch.Tensor, k: int, *, stream=None):
    """Time the fused step's tile widths (2, 4, 8) on A and record the fastest
    for this device and shape bucket (css_autotune_select).  Returns
    (best width, {width: greedy-iteration ms})."""
    m, n, lda = _colmajor(A)
    dt = _DT[A.dtype]
    lib = L.load()
    dev = A.device
    sel = torch.empty(k, dtype=torch.int32, device=dev)
    trace = torch.empty(k + 1, dtype=torch.float64, device=dev)
    nsel = torch.zeros(1, dtype=torch.int32, device=dev)
    o = L.default_opts()
    nbytes = lib.css_workspace_size(L.CSS_OP_SELECT, dt, m, n, 0, k, 0, C.byref(o))
    _keep, ws = _workspace(nbytes, dev)
    best = C.c_int32(0)
    times = (C.c_double * 3)()
    code = lib.css_autotune_select(_ptr(A), dt, m, n, lda, k, _ptr(sel), _ptr(trace), _ptr(nsel),
                                   _ptr(ws), nbytes, C.byref(best), C.cast(times, C.c_void_p),
                                   _stream(stream))
    _check(code, "css_autotune_select")
    return best.value, {2: times[0], 4: times[1], 8: times[2]}


def select_host(A_host: torch.Tensor, k: int, A_dev: torch.Tensor, *, ws=None, stream=None):
    """Algorithm 1 from host memory: copies A_host (column-major, ideally pinned)
    into the device staging tensor A_dev, selects, copies the results back.
    Returns (sel int32[k], trace float64[k+1], n_sel) as host tensors."""
    m, n, lda = _colmajor(A_host)
    dt = _DT[A_host.dtype]
    lib = L.load()
    sel = torch.empty(k, dtype=torch.int32)
    trace = torch.empty(k + 1, dtype=torch.float64)
    nsel = torch.zeros(1, dtype=torch.int32)
    o = L.default_opts()
    nbytes = lib.css_workspace_size(L.CSS_OP_HOST_SELECT, dt, m, n, 0, k, 0, C.byref(o))
    if ws is None:
        _keep, ws = _workspace(nbytes, A_dev.device)
    code = lib.css_select_host(C.c_void_p(A_host.data_ptr()), dt, m, n, lda, k,
                               C.c_void_p(sel.data_ptr()), C.c_void_p(trace.data_ptr()),
                               C.c_void_p(nsel.data_ptr()), _ptr(A_dev), _ptr(ws), nbytes,
                               C.byref(o), _stream(stream))
    _check(code, "css_select_host")
    return sel, trace, int(nsel.item())


def host_workspace_bytes(m, n, k, dtype):
    lib = L.load()
    o = L.default_opts()
    return lib.css_workspace_size(L.CSS_OP_HOST_SELECT, _DT[dtype], m, n, 0, k, 0, C.byref(o))


class _Residual(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, sel):
        m, n, lda = _colmajor(A)
        dt = _DT[A.dtype]
        lib = L.load()
        loss = torch.empty(1, dtype=torch.float64, device=A.device)
        o = L.default_opts()
        k = int(sel.numel())
        nbytes = lib.css_workspace_size(L.CSS_OP_BACKWARD, dt, m, n, 0, k, 0, C.byref(o))
        _keep, ws = _workspace(nbytes, A.device)
        code = lib.css_residual_backward(_ptr(A), dt, m, n, lda, _ptr(sel), k, 1.0,
                                         C.c_void_p(0), 0, _ptr(loss), _ptr(ws), nbytes,
                                         C.byref(o), _stream(None))
        _check(code, "css_residual_backward(loss)")
        ctx.save_for_backward(A, sel)
        return loss[0].to(A.dtype if A.dtype != torch.bfloat16 else torch.float32)

    @staticmethod
    def backward(ctx, grad):
        A, sel = ctx.saved_tensors
        m, n, lda = _colmajor(A)
        dt = _DT[A.dtype]
        lib = L.load()
        dA = empty_colmajor(m, n, A.dtype, A.device, lda)
        _, _, ldd = _colmajor(dA)
        o = L.default_opts()
        k = int(sel.numel())
        nbytes = lib.css_workspace_size(L.CSS_OP_BACKWARD, dt, m, n, 0, k, 0, C.byref(o))
        _keep, ws = _workspace(nbytes, A.device)
        code = lib.css_residual_backward(_ptr(A), dt, m, n, lda, _ptr(sel), k, float(grad.item()),
                                         _ptr(dA), ldd, C.c_void_p(0), _ptr(ws), nbytes,
                                         C.byref(o), _stream(None))
        _check(code, "css_residual_backward")
        return dA, None


def residual_error(A: torch.Tensor, S) -> float:
    """||A - P^(S) A||_F^2 for a fixed selected set S as an FP64 number, from
    the residual R = A - Q (Q^T A) formed on the device (the forward half of
    css_residual_backward, no gradient).  Unlike the selection's recursive
    trace it keeps its accuracy when the error is a tiny fraction of
    ||A||_F^2."""
    m, n, lda = _colmajor(A)
    dt = _DT[A.dtype]
    lib = L.load()
    sel = torch.as_tensor(list(S) if not torch.is_tensor(S) else S, dtype=torch.int32).to(A.device).contiguous()
    loss = torch.empty(1, dtype=torch.float64, device=A.device)
    o = L.default_opts()
    k = int(sel.numel())
    nbytes = lib.css_workspace_size(L.CSS_OP_BACKWARD, dt, m, n, 0, k, 0, C.byref(o))
    if nbytes == 0:
        raise ValueError("invalid sizes for css_residual_backward")
    _keep, ws = _workspace(nbytes, A.device)
    code = lib.css_residual_backward(_ptr(A), dt, m, n, lda, _ptr(sel), k, 1.0, C.c_void_p(0), 0,
                                     _ptr(loss), _ptr(ws), nbytes, C.byref(o), _stream(None))
    _check(code, "css_residual_backward(loss)")
    return float(loss.item())


def residual(A: torch.Tensor, S) -> torch.Tensor:
    """||A - P^(S) A||_F^2 (Eq. Projection) for a fixed selected set S, as an
    autograd function whose backward is the hand-written adjoint kernel."""
    sel = torch.as_tensor(S, dtype=torch.int32, device=A.device).contiguous()
    return _Residual.apply(A, sel)
