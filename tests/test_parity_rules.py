"""CPU checks of the parity rules the GPU tests apply (tests/gpu_helpers.py),
run against the oracle itself standing in for the device: the oracle's own
run passes every rule, and a planted mistake in its output fails the rule
meant to catch it."""
import numpy as np
import pytest
import torch

import css_inputs as ci
from oracle import css_oracle as O
from tests.gpu_helpers import (certify_selection, gradient_entry_errors, hm_lambda, oracle_path_parity,
                               score_error_bound)


class _FakeSel:
    """What oracle_path_parity reads from a device run, made by the oracle."""

    def __init__(self, diag_argmax, f, g):
        self.diag_argmax = torch.tensor(diag_argmax, dtype=torch.int32)
        self.diag_f = torch.from_numpy(f)
        self.diag_g = torch.from_numpy(g)


def _oracle_device(A, tau, plant=None):
    """run_forced(prefix, k, diag) served by the FP64 oracle: its own argmax
    at each step (the argmax of its kept scores) and its state after k steps.
    `plant` = (step, column): report that column as the argmax there."""
    def run(prefix, k, diag):
        r = O.greedy_css(A, k, tau_rel=tau, keep_scores=True, forced=prefix)
        own = [int(np.argmax(np.where(np.isfinite(s), s, -np.inf))) for s in r.scores]
        if plant is not None and plant[0] < len(own):
            own[plant[0]] = plant[1]
        return _FakeSel(own, r.f, r.g)
    return run


def test_lambda_of_the_probabilistic_bound():
    # 2 * length * exp(-lambda^2 / 2) * n_dots = p_fail
    lam = hm_lambda(4096, 2 * 65536 * 256, 1e-6)
    assert abs(2 * 4096 * 2 * 65536 * 256 * np.exp(-lam ** 2 / 2) - 1e-6) < 1e-12
    assert 8.9 < lam < 9.0
    assert hm_lambda(64, 100) < hm_lambda(4096, 100) < hm_lambda(4096, 10 ** 6)


def test_oracle_passes_its_own_path():
    A = ci.lowrank_uv(40, 150, 5, 0.05, 901)
    ref = O.greedy_css(A, 10, tau_rel=1e-12, keep_scores=True)
    st = oracle_path_parity(_oracle_device(A, 1e-12), ref, 40, torch.float64, 1e-12,
                            sample_steps=range(1, 10))
    assert st.agree == 10 and st.restarts == 0
    assert st.max_err_ratio == 0.0


def test_planted_wrong_pick_at_a_wide_gap_fails():
    A = ci.lowrank_uv(40, 150, 5, 0.05, 901)
    ref = O.greedy_css(A, 10, tau_rel=1e-12, keep_scores=True)
    t = int(np.argmax(ref.gaps[:5]))
    assert ref.gaps[t] > 1e-3
    wrong = [j for j in range(150) if j not in ref.S][0]
    with pytest.raises(AssertionError):
        oracle_path_parity(_oracle_device(A, 1e-12, plant=(t, wrong)), ref, 40, torch.float64, 1e-12)


def test_certify_selection():
    A = ci.lowrank_uv(40, 150, 5, 0.05, 902)
    ref = O.greedy_css(A, 8, tau_rel=1e-12, keep_scores=True)
    on_own = O.greedy_css(A, 8, tau_rel=1e-12, keep_scores=True, forced=ref.S)
    assert certify_selection(ref.S, on_own, 40, torch.float64) == (0, 0.0)
    # a selection whose third pick is a poor column is not a greedy selection
    sc = ref.scores[2]
    worst = int(np.argmin(np.where(np.isfinite(sc) & (sc > 0), sc, np.inf)))
    bad = ref.S[:2] + [worst]
    on_bad = O.greedy_css(A, 3, tau_rel=1e-12, keep_scores=True, forced=bad)
    with pytest.raises(AssertionError):
        certify_selection(bad, on_bad, 40, torch.float64)


def test_score_error_bound_scale():
    """The bound is at least lambda u sqrt(m) sqrt(t + 1) times the largest
    initial score (a column's residual never grows: g_i <= g_i^(0)), and it
    grows as a column's residual shrinks."""
    A = ci.lowrank_uv(40, 150, 5, 0.05, 903)
    ref = O.greedy_css(A, 8, tau_rel=1e-12, keep_scores=True)
    sc0_max = np.max(ref.fs[0] / ref.gs[0])
    lam = hm_lambda(40, 2 * 150 * 9 + 40 * 40)
    for t in (1, 4, 7):
        b = score_error_bound(ref, t, 40, torch.float32)
        cand = np.isfinite(ref.scores[t])
        assert np.all(b[cand] >= lam * 2.0 ** -24 * np.sqrt(40 * (t + 1)) * sc0_max * (1 - 1e-12))
        i = int(np.argmin(np.where(cand, ref.gs[t] / ref.gs[0], np.inf)))
        j = int(np.argmax(np.where(cand, ref.gs[t] / ref.gs[0], -np.inf)))
        assert b[i] >= b[j] or ref.scores[t][j] > ref.scores[t][i]


def test_entrywise_gradient_check_catches_one_wrong_column():
    A = ci.lowrank_uv(60, 140, 6, 1e-3, 904)
    S = O.greedy_css(A, 6).S
    _, G = O.residual_gradient(A, S)
    assert gradient_entry_errors(G, G, S) == (0.0, 0.0)
    # one column of -2 R T^T off by 0.1 percent
    G1 = G.copy()
    G1[:, S[3]] *= 1.001
    rest, sel = gradient_entry_errors(G1, G, S)
    assert rest == 0.0 and 9e-4 < sel < 1.1e-3
    # one entry of 2R off by 0.1 percent of its column's largest entry
    G2 = G.copy()
    j = [c for c in range(140) if c not in S][5]
    G2[7, j] += 1e-3 * np.max(np.abs(G[:, j]))
    rest, sel = gradient_entry_errors(G2, G, S)
    assert sel == 0.0 and abs(rest - 1e-3) < 1e-9


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
def test_gradient_tolerances_reject_one_wrong_column(dtype):
    """With the derived tolerances, the oracle's own gradient passes and a
    single column of -2 R T^T off by one percent (or a single column of 2R
    off by one percent) fails; for BF16 output, whose rounding alone is
    0.4 percent, by two percent."""
    from tests.gpu_helpers import gradient_tolerances
    A = ci.lowrank_uv(80, 300, 8, 1e-3, 905)
    S = O.greedy_css(A, 8).S
    _, G = O.residual_gradient(A, S)
    tol, tol_S = gradient_tolerances(A, S, G, dtype)
    off = 1.02 if dtype == torch.bfloat16 else 1.01
    assert gradient_entry_errors(G, G, S, tol, tol_S) == (0.0, 0.0)
    G1 = G.copy()
    G1[:, S[5]] *= off
    assert gradient_entry_errors(G1, G, S, tol, tol_S)[1] > 1.0
    G2 = G.copy()
    j = [c for c in range(300) if c not in S][11]
    G2[:, j] *= off
    assert gradient_entry_errors(G2, G, S, tol, tol_S)[0] > 1.0
