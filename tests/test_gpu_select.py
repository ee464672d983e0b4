"""GPU parity of css_select (Algorithm 1) against the FP64 oracle, through the
C ABI (paper_1312_6838_gb300.css is argument marshalling only)."""
import numpy as np
import pytest
import scipy.linalg
import torch

import css_inputs as ci
from oracle import css_oracle as O
from tests.gpu_helpers import (GAP_TOL, certify_selection, dev_matrix, first_mismatch, oracle_path_parity,
                               pair_error_bound, teacher_forced_parity, trace_error_bound)

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


def _run(css, A, k, forced=None, **kw):
    r = css.select(A, k, forced=forced if forced else None, **kw)
    return r


def _check_case(css, A_np, k, dtype, ld=None, sample_steps=(), **kw):
    """The parity rule of the tests, on one matrix:
    * every iteration of the oracle's path: the device's argmax against the
      oracle's pick; mismatches are allowed only where the oracle's top-two
      gap is <= 1e-6, or within the derived score error bound with the
      device's measured score errors inside that bound (oracle_path_parity);
    * the device's own selection: identical to the oracle's, with the final
      error within ERR_TOL; or, where it parted at a near-tie, every one of
      its picks within the same rule on its own path (certify_selection);
    * Theorem 1's recursive trace on the oracle's path against the oracle's.
    Returns (result, oracle result, ParityStats)."""
    A, vals = dev_matrix(A_np, dtype, ld)
    m = vals.shape[0]
    ref = O.greedy_css(vals, k, tau_rel=TAU[dtype], keep_scores=True)
    run = lambda prefix, kk, diag: _run(css, A, kk, prefix, diag=diag, **kw)
    stats = oracle_path_parity(run, ref, m, dtype, TAU[dtype], sample_steps=sample_steps)
    res = _run(css, A, k, **kw)
    S = res.indices.cpu().tolist()
    e_gpu = O.reconstruction_error(vals, S)
    e_ref = O.reconstruction_error(vals, ref.S)
    if S == list(ref.S):
        assert abs(e_gpu - e_ref) <= ERR_TOL[dtype] * e_ref + 1e-300, (e_gpu, e_ref)
    else:
        assert dtype != torch.float64 or stats.widened == 0
        ref_dev = O.greedy_css(vals, len(S), tau_rel=TAU[dtype], keep_scores=True, forced=S)
        certify_selection(S, ref_dev, m, dtype)
    # Theorem 1's recursive trace on the oracle's own path (teacher-forced)
    # against the oracle's trace: absolute error of the device recursion
    full = _run(css, A, len(ref.S), list(ref.S), **kw)
    tr = full.trace.cpu().numpy()[: len(ref.S) + 1]
    bound = trace_error_bound(ref, m, dtype)
    assert np.all(np.abs(tr - np.asarray(ref.trace)) <= bound), np.max(np.abs(tr - ref.trace) / bound)
    return res, ref, stats


def test_fp64_workload_500x1000(css):
    c = ci.CONFIGS["fp64_500x1000"]
    A_np = ci.lowrank_uv(c["m"], c["n"], c["rank"], c["noise"], c["seed"])
    res, ref, stats = _check_case(css, A_np, c["k"], torch.float64, sample_steps=(1, 25, 49))
    assert stats.agree == c["k"]
    tr = res.trace.cpu().numpy()
    np.testing.assert_allclose(tr, ref.trace, rtol=0, atol=1e-10 * ref.trace[0])
    assert res.indices.cpu().tolist() == ref.S


def test_fp64_brute_force_slice(css):
    c = ci.CONFIGS["fp64_500x1000"]
    A_np = ci.lowrank_uv(c["m"], c["n"], c["rank"], c["noise"], c["seed"])[:12, :16]
    A, _ = dev_matrix(A_np, torch.float64)
    res = css.select(A, 3)
    ref = O.greedy_css(A_np, 3)
    assert res.indices.cpu().tolist() == ref.S
    best_S, best_err = O.brute_force_css(A_np, 3)
    assert O.reconstruction_error(A_np, ref.S) >= best_err * (1 - 1e-12)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("shape", [(37, 203, 9), (129, 1000, 24), (64, 64, 64), (300, 77, 30)])
def test_ragged_shapes(css, dtype, shape):
    """Ragged sizes.  The signal rank is 2k, so every pick is made while the
    scores are far above the FP32 accumulation floor."""
    m, n, k = shape
    A_np = ci.lowrank_uv(m, n, min(2 * k, m, n), 0.05, m * 1000 + n)
    _check_case(css, A_np, k, dtype, sample_steps=(1, k // 2, k - 1))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("shape", [(37, 203, 9), (129, 1000, 24), (64, 64, 64), (300, 77, 30)])
def test_ragged_shapes_beyond_rank(css, dtype, shape):
    """The same shapes with a signal of rank max(2, k // 2) below k: the
    later picks are made among noise-level scores, where the mixed path's
    score errors are comparable to the oracle's gaps.  Same rule, with the
    device's measured score errors checked against the bound at three
    iterations."""
    m, n, k = shape
    A_np = ci.lowrank_uv(m, n, max(2, k // 2), 0.05, m * 1000 + n)
    _check_case(css, A_np, k, dtype, sample_steps=(1, k // 2, k - 1))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
def test_beyond_numerical_rank(css, dtype):
    """k larger than the signal rank (60 x 400, rank 5, k = 14): the late
    scores are differences of O(f0) quantities, so the mixed path's picks are
    only defined up to its score error (FP64 resolves them).  The rule of
    _check_case, with the device's measured score errors checked against the
    bound at every iteration."""
    A_np = ci.lowrank_uv(60, 400, 5, 0.05, 77)
    _, _, stats = _check_case(css, A_np, 14, dtype, sample_steps=range(1, 14))
    if dtype == torch.float64:
        assert stats.agree == 14


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_padded_and_unaligned_leading_dimension(css, dtype):
    A_np = ci.lowrank_uv(50, 300, 24, 0.05, 3)
    _check_case(css, A_np, 12, dtype, ld=64)      # aligned padding
    _check_case(css, A_np, 12, dtype, ld=51)      # forces the scalar load path
    # a signal of rank 6 < k: picks beyond the numerical rank on both paths
    A_lo = ci.lowrank_uv(50, 300, 6, 0.05, 3)
    _check_case(css, A_lo, 12, dtype, ld=64, sample_steps=range(1, 12))
    _check_case(css, A_lo, 12, dtype, ld=51, sample_steps=range(1, 12))


@pytest.mark.parametrize("tile", [2, 4, 8])
def test_tile_widths_agree(css, tile):
    """Every tile width (which changes which tiles the fused step splits by
    rows, and so the FP32 summation order of their dots) meets the oracle
    under the mixed-path rule within the numerical rank (10)."""
    A_np = ci.lowrank_uv(200, 777, 10, 0.02, 5)
    _check_case(css, A_np, 10, torch.float32, tile_cols=tile)


@pytest.mark.parametrize("grid", [1, 2, 7, 64])
def test_team_sizes_agree(css, grid):
    A_np = ci.lowrank_uv(96, 1500, 8, 0.02, 6)
    A, vals = dev_matrix(A_np, torch.float64)
    ref = O.greedy_css(vals, 16)
    res = css.select(A, 16, grid_ctas=grid)
    assert res.indices.cpu().tolist() == ref.S
    np.testing.assert_allclose(res.trace.cpu().numpy(), ref.trace, rtol=0, atol=1e-10 * ref.trace[0])


def test_W_and_score_state(css):
    A_np = ci.lowrank_uv(40, 120, 6, 0.03, 8)
    A, vals = dev_matrix(A_np, torch.float64)
    k = 10
    res = css.select(A, k, return_W=True, diag=True)
    ref = O.greedy_css(vals, k)
    assert res.indices.cpu().tolist() == ref.S
    np.testing.assert_allclose(res.W.cpu().numpy(), ref.W, rtol=1e-9, atol=1e-9 * np.abs(ref.W).max())
    f = res.diag_f.cpu().numpy()
    g = res.diag_g.cpu().numpy()
    sel = np.zeros(120, bool)
    sel[ref.S] = True
    # f and g are differences of O(f0) and O(g0) terms: compare on that scale
    f0 = np.einsum("ij,ij->j", vals, (vals @ vals.T) @ vals)
    g0 = np.sum(vals * vals, axis=0)
    np.testing.assert_allclose(g[~sel], ref.g[~sel], rtol=0, atol=1e-13 * g0.max())
    np.testing.assert_allclose(f[~sel], ref.f[~sel], rtol=0, atol=1e-13 * f0.max())
    assert res.diag_argmax.cpu().tolist() == ref.S
    # Q-less QR structure: W Pi upper triangular (Sec. 6)
    W = res.W.cpu().numpy()
    for t in range(k):
        for s in range(t):
            assert abs(W[t, ref.S[s]]) <= 1e-10 * np.abs(W[t]).max()


def test_edge_k_equals_one_and_full(css):
    A_np = ci.lowrank_uv(20, 20, 20, 0.0, 9)
    for k in (1, 20):
        A, vals = dev_matrix(A_np, torch.float64)
        res = css.select(A, k)
        ref = O.greedy_css(vals, k)
        assert res.indices.cpu().tolist() == ref.S
    # k = m = n: the error reaches zero
    assert res.trace[-1].item() <= 1e-10 * res.trace[0].item()


def test_rank_exhaustion(css):
    A_np = ci.lowrank_uv(30, 80, 4, 0.0, 10)
    A, vals = dev_matrix(A_np, torch.float64)
    res = css.select(A, 10, tau_rel=1e-10)
    ref = O.greedy_css(vals, 10, tau_rel=1e-10, keep_scores=True)
    assert res.status == 1  # CSS_RANK_EXHAUSTED
    assert res.n_sel == len(ref.S) == 4
    # the last pick is an exact tie (the residual has rank one), so any column
    # is correct there; the prefix before it is unique
    teacher_forced_parity(
        lambda forced: css.select(A, 10, tau_rel=1e-10, forced=forced or None).indices.cpu().tolist(),
        ref, m=30, dtype=torch.float64)
    assert O.reconstruction_error(vals, res.indices.cpu().tolist()) <= 1e-12 * ref.trace[0]


def test_zero_and_duplicate_columns(css):
    rng = np.random.default_rng(11)
    A_np = rng.standard_normal((25, 40))
    A_np[:, 5] = 0.0
    A_np[:, 17] = A_np[:, 3]
    A_np[:, 30] = 2.0 * A_np[:, 3]
    A, vals = dev_matrix(A_np, torch.float64)
    res = css.select(A, 12)
    ref = O.greedy_css(vals, 12)
    S = res.indices.cpu().tolist()
    assert 5 not in S
    assert S == ref.S
    assert len({3, 17, 30} & set(S)) <= 1


def test_single_column_and_single_row(css):
    A, _ = dev_matrix(np.arange(1.0, 8.0).reshape(7, 1), torch.float64)
    res = css.select(A, 1)
    assert res.indices.cpu().tolist() == [0]
    assert abs(res.trace[1].item()) <= 1e-12 * res.trace[0].item()
    # one row: every column scores the same (sum of squares of the row), so
    # the tie goes to the lowest index
    A2, _ = dev_matrix(np.array([[1.0, -3.0, 2.0, 0.5]]), torch.float64)
    res2 = css.select(A2, 1)
    assert res2.indices.cpu().tolist() == O.greedy_css(np.array([[1.0, -3.0, 2.0, 0.5]]), 1).S == [0]


def test_forced_prefix(css):
    A_np = ci.lowrank_uv(60, 200, 7, 0.02, 12)
    A, vals = dev_matrix(A_np, torch.float64)
    forced = [11, 150, 3]
    res = css.select(A, 9, forced=forced)
    ref = O.greedy_css(vals, 9, forced=forced)
    assert res.indices.cpu().tolist() == ref.S
    assert ref.S[:3] == forced
    np.testing.assert_allclose(res.trace.cpu().numpy(), ref.trace, rtol=0, atol=1e-10 * ref.trace[0])


def test_forced_prefix_rejects_bad_indices(css):
    from paper_1312_6838_gb300._lib import CssError
    A, _ = dev_matrix(ci.lowrank_uv(10, 30, 3, 0.1, 13), torch.float64)
    with pytest.raises(CssError):
        css.select(A, 4, forced=[1, 1])
    with pytest.raises(CssError):
        css.select(A, 4, forced=[40])


def test_norm_score_is_qr_with_column_pivoting(css):
    A_np = ci.lowrank_uv(30, 25, 25, 0.0, 15)
    _, _, piv = scipy.linalg.qr(A_np, pivoting=True, mode="economic")
    A, _ = dev_matrix(A_np, torch.float64)
    res = css.select(A, 10, score_mode=1)
    assert res.indices.cpu().tolist() == list(piv[:10])


def test_nonfinite_input_reported(css):
    from paper_1312_6838_gb300._lib import CssError, CSS_ERR_NONFINITE
    A_np = ci.lowrank_uv(16, 40, 3, 0.1, 16)
    A_np[4, 7] = np.nan
    A, _ = dev_matrix(A_np, torch.float32)
    with pytest.raises(CssError) as ei:
        css.select(A, 3)
    assert ei.value.code == CSS_ERR_NONFINITE
    # the context stays usable
    A2, _ = dev_matrix(ci.lowrank_uv(16, 40, 3, 0.1, 17), torch.float32)
    assert css.select(A2, 3).n_sel == 3


def test_rows_and_columns_are_permutation_equivariant(css):
    A_np = ci.lowrank_uv(48, 300, 6, 0.03, 18)
    perm = np.random.default_rng(1).permutation(300)
    A, _ = dev_matrix(A_np, torch.float64)
    Ap, _ = dev_matrix(A_np[:, perm], torch.float64)
    a = css.select(A, 10).indices.cpu().tolist()
    b = css.select(Ap, 10).indices.cpu().tolist()
    assert [int(perm[j]) for j in b] == a


@pytest.mark.parametrize("tile", [2, 4, 8])
def test_repeat_is_bitwise_identical(css, tile):
    """The fused step hands out whole tiles, then row chunks of the last tiles
    whose sums are finished by whichever warp adds the last chunk: the result
    must not depend on that timing.  n is large enough for both kinds of unit
    (more tiles than the team has warps)."""
    A_np = ci.lowrank_uv(256, 24576, 16, 0.01, 91)
    A, _ = dev_matrix(A_np, torch.float32)
    runs = [css.select(A, 24, tile_cols=tile, diag=True, return_W=True) for _ in range(3)]
    for r in runs[1:]:
        assert torch.equal(r.sel, runs[0].sel)
        assert torch.equal(r.trace, runs[0].trace)
        assert torch.equal(r.diag_f, runs[0].diag_f)
        assert torch.equal(r.diag_g, runs[0].diag_g)
        assert torch.equal(r.W, runs[0].W)


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float32, torch.float64])
@pytest.mark.parametrize("shape", [(304, 5000, 24), (300, 2000, 16), (128, 700, 10)])
def test_select_from_host_memory(css, dtype, shape):
    """css_select_host: A copied from pinned host memory in column chunks
    whose arrival starts the initial scores' K chunks (BF16), then the same
    selection, trace and error as css_select on the device copy, bit for bit,
    and parity with the oracle."""
    m, n, k = shape
    A_np = ci.lowrank_uv(m, n, 2 * k, 0.05, 910 + m)
    A, vals = dev_matrix(A_np, dtype)
    host = A.t().contiguous().cpu().pin_memory().t()   # column-major, pinned
    A_dev = css.empty_colmajor(m, n, dtype)
    for _ in range(2):   # the second call reuses the copy stream and events
        sel, trace, ns = css.select_host(host, k, A_dev)
        ref = css.select(A, k)
        assert ns == ref.n_sel
        assert sel.tolist() == ref.indices.cpu().tolist()
        assert torch.equal(trace, ref.trace.cpu())
    assert torch.equal(A_dev.cpu(), A.cpu())
    oref = O.greedy_css(vals, k, tau_rel=1e-6)
    assert abs(O.reconstruction_error(vals, sel.tolist()) - oref.trace[-1]) <= 1e-4 * oref.trace[0]


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("init_path", [0, 1])
def test_tiny_and_degenerate_shapes_mixed(css, dtype, init_path):
    """The mixed paths (tensor-core or SIMT initial scores) on the degenerate
    cases: one column, one row (every column ties: lowest index), k = m = n,
    a zero column and duplicated columns; picks as the oracle's on the values
    the device holds."""
    A, vals = dev_matrix(np.arange(1.0, 8.0).reshape(7, 1), dtype)
    assert css.select(A, 1, init_path=init_path).indices.cpu().tolist() == [0]
    row = np.array([[1.0, -3.0, 2.0, 0.5]])
    A, vals = dev_matrix(row, dtype)
    assert css.select(A, 1, init_path=init_path).indices.cpu().tolist() == [0]
    A_np = ci.lowrank_uv(12, 12, 12, 0.0, 19)
    A, vals = dev_matrix(A_np, dtype)
    res = css.select(A, 12, init_path=init_path)
    assert sorted(res.indices.cpu().tolist()) == list(range(12))
    assert O.reconstruction_error(vals, res.indices.cpu().tolist()) <= 1e-10 * float(np.sum(vals * vals))
    rng = np.random.default_rng(21)
    A_np = rng.standard_normal((25, 40))
    A_np[:, 5] = 0.0
    A_np[:, 17] = A_np[:, 3]
    A_np[:, 30] = 2.0 * A_np[:, 3]
    A, vals = dev_matrix(A_np, dtype)
    res = css.select(A, 12, init_path=init_path)
    S = res.indices.cpu().tolist()
    assert 5 not in S
    assert len({3, 17, 30} & set(S)) <= 1
    ref = O.greedy_css(vals, 12, tau_rel=1e-6, keep_scores=True)
    t = first_mismatch(S, list(ref.S))
    if t is not None:
        assert ref.gaps[t] <= max(GAP_TOL, pair_error_bound(ref, t, 25, dtype)), (t, ref.gaps[t])
