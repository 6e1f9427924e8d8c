"""Pins of the oracle's fluence-rate bounds (Eq. 2, 6; reading R11).

The bounds are pinned against (1) a case worked out by hand from Eq. 2,
(2) an independent linear program over Eq. 2's constraints as stated (the
largest and smallest gantry speed each placed CP can take), (3) special cases
(no machine, no leaf motion, one aperture) and (4) a whole plan, whose fluence
rates must respect the bounds of its final aperture set.
"""
import numpy as np
import pytest
from scipy.optimize import linprog

import oracle
import synth


def _mlc(K, n_rows, n_cols, arcs=(0,), travel=3, machine=None):
    return synth.MLC(K, n_rows, n_cols, np.array(arcs, np.int32), travel, False, machine)


def test_hand_worked_case():
    # one arc of 8 CPs at 45 degrees; apertures at CP 2 and CP 5 (m = 3 steps)
    mach = synth.Machine(cp_step_deg=45.0, speed_min=0.5, speed_max=4.0, speed_step_max=0.5,
                         rate_min=0.03, rate_max=0.04, leaf_speed_cols=0.05)
    mlc = _mlc(8, 2, 8, machine=mach)
    lv2 = np.array([[1, 4], [2, 6]])
    lv5 = np.array([[3, 4], [2, 3]])
    # largest leaf move 3 columns (row 1, right leaf 6 -> 3) over 3 * 45 degrees at 0.05 columns/s:
    # the interval takes at least 60 s, so s_2 <= 135 / 60 = 2.25 deg/s; CP 5 is the last: s_5 <= 4,
    # and the speed-change limit gives s_5 <= 2.25 + 3 * 0.5 = 3.75
    S_hat, S_U = oracle.gantry_speed_bounds(mlc, mach, [5, 2], [lv5, lv2])
    assert S_hat.tolist() == [4.0, 2.25]
    assert S_U.tolist() == [3.75, 2.25]
    lo, hi = oracle.fluence_bounds(mlc, mach, [5, 2], [lv5, lv2])
    assert lo.tolist() == [np.float32(0.03 / 3.75), np.float32(0.03 / 2.25)]
    assert hi.tolist() == [np.float32(0.08)] * 2


def _random_sequence(mlc, n, seed):
    """n distinct CPs with leaves that move at most 2 columns between any two CPs
    of an arc (within every travel window of 3 columns per step)."""
    rng = np.random.default_rng(seed)
    cps = rng.choice(mlc.K, size=n, replace=False)
    base = {}
    for a in range(mlc.n_arcs):
        L = rng.integers(2, mlc.n_cols // 2 - 1, size=mlc.n_rows)
        R = rng.integers(mlc.n_cols // 2 + 1, mlc.n_cols - 2, size=mlc.n_rows)
        base[a] = (L, R)
    leaves = []
    for k in cps:
        a = int(np.searchsorted(mlc.arc_first_cp, k, side="right") - 1)
        L, R = base[a]
        dl = rng.integers(-1, 2, size=mlc.n_rows)
        dr = rng.integers(-1, 2, size=mlc.n_rows)
        leaves.append(np.stack([L + dl, R + dr], axis=1))
    return [int(k) for k in cps], leaves


def _lp_speed_range(mlc, mach, cps, leaves):
    """Extreme speeds of each placed CP over the constraints of Eq. 2, written out
    one by one: box, leaf-motion limit of each interval, speed-change limit."""
    n = len(cps)
    A, b = [], []
    order = sorted(range(n), key=lambda t: cps[t])
    for i, t in enumerate(order):
        k = cps[t]
        nxt = [u for u in order[i + 1:] if oracle.arc_of(mlc, cps[u]) == oracle.arc_of(mlc, k)]
        if not nxt:
            continue
        u = nxt[0]
        m = cps[u] - k
        d = max(abs(int(leaves[t][r][s]) - int(leaves[u][r][s])) for r in range(mlc.n_rows) for s in (0, 1))
        if d > 0:  # time of the interval (m step / s_k) >= time of the largest leaf move (d / v)
            row = np.zeros(n)
            row[t] = 1.0
            A.append(row)
            b.append(m * mach.cp_step_deg * mach.leaf_speed_cols / d)
        for sgn in (1.0, -1.0):  # |s_k - s_k'| <= m Delta S
            row = np.zeros(n)
            row[t], row[u] = sgn, -sgn
            A.append(row)
            b.append(m * mach.speed_step_max)
    bounds = [(mach.speed_min, mach.speed_max)] * n
    smax, smin = np.empty(n), np.empty(n)
    for t in range(n):
        c = np.zeros(n)
        c[t] = -1.0
        r = linprog(c, A_ub=np.array(A) if A else None, b_ub=np.array(b) if b else None, bounds=bounds,
                    method="highs")
        assert r.status == 0
        smax[t] = r.x[t]
        c[t] = 1.0
        r = linprog(c, A_ub=np.array(A) if A else None, b_ub=np.array(b) if b else None, bounds=bounds,
                    method="highs")
        assert r.status == 0
        smin[t] = r.x[t]
    return smin, smax


@pytest.mark.parametrize("seed", range(6))
def test_bounds_are_the_extreme_speeds_of_eq2(seed):
    arcs = (0,) if seed % 2 == 0 else (0, 13)
    mlc = _mlc(26, 5, 16, arcs=arcs)
    mach = synth.make_machine(mlc, speed_step_max=[0.05, 0.5, 3.0][seed % 3])
    mach.leaf_speed_cols *= [1.0, 1.6, 3.0][seed % 3]
    mlc.machine = mach
    cps, leaves = _random_sequence(mlc, [3, 7, 12, 20, 9, 16][seed], seed)
    smin, smax = _lp_speed_range(mlc, mach, cps, leaves)
    _, S_U = oracle.gantry_speed_bounds(mlc, mach, cps, leaves)
    np.testing.assert_allclose(S_U, smax, rtol=1e-9)
    np.testing.assert_allclose(smin, mach.speed_min, rtol=1e-9)
    lo, hi = oracle.fluence_bounds(mlc, mach, cps, leaves)
    np.testing.assert_allclose(lo, mach.rate_min / smax, rtol=1e-6)
    np.testing.assert_allclose(hi, mach.rate_max / smin, rtol=1e-6)
    assert np.all(lo <= hi)
    if seed % 3 == 0:  # a tight speed-change limit couples the CPs: not every S_U is its own interval's
        S_hat, _ = oracle.gantry_speed_bounds(mlc, mach, cps, leaves)
        assert np.any(S_U < S_hat)


def test_special_cases():
    mlc = _mlc(12, 3, 10)
    lv = [np.array([[2, 7]] * 3)] * 3
    lo, hi = oracle.fluence_bounds(mlc, None, [4, 1, 9], lv)
    assert lo.tolist() == [0.0] * 3 and np.all(np.isinf(hi))
    mach = synth.make_machine(mlc)
    # leaves that never move: no interval limits the speed
    S_hat, S_U = oracle.gantry_speed_bounds(mlc, mach, [4, 1, 9], lv)
    assert S_hat.tolist() == [mach.speed_max] * 3 and S_U.tolist() == [mach.speed_max] * 3
    # one aperture
    lo, hi = oracle.fluence_bounds(mlc, mach, [6], [np.array([[0, 10]] * 3)])
    assert lo[0] == np.float32(mach.rate_min / mach.speed_max)
    assert hi[0] == np.float32(mach.rate_max / mach.speed_min)
    # a zero slowest speed: no upper bound on the fluence rate
    mach0 = synth.make_machine(mlc, speed_min=0.0)
    mach0.leaf_speed_cols = 1.0
    lo, hi = oracle.fluence_bounds(mlc, mach0, [6], [np.array([[0, 10]] * 3)])
    assert np.isinf(hi[0])
    # arcs do not couple: CP 5 is the last of arc 0, CP 6 the first of arc 1
    mlc2 = _mlc(12, 3, 10, arcs=(0, 6))
    mach2 = synth.make_machine(mlc2, speed_step_max=0.0)
    S_hat, S_U = oracle.gantry_speed_bounds(mlc2, mach2, [5, 6, 8],
                                            [np.array([[1, 5]] * 3), np.array([[2, 6]] * 3),
                                             np.array([[4, 8]] * 3)])
    assert S_hat[0] == mach2.speed_max  # no later CP in arc 0
    assert S_U[0] == mach2.speed_max
    assert S_hat[1] == min(mach2.speed_max, 2 * mach2.cp_step_deg * mach2.leaf_speed_cols / 2)


def test_plan_respects_bounds_and_they_bind():
    c = synth.make_case("cfg1", seed=0)
    mlc = synth.MLC(c.mlc.K, c.mlc.n_rows, c.mlc.n_cols, c.mlc.arc_first_cp, c.mlc.travel_cols)
    mlc.machine = synth.make_machine(mlc)
    D = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, c.val)
    r = oracle.cg_plan(D, mlc, c.structs, 12)
    lo, hi = oracle.fluence_bounds(mlc, mlc.machine, r.cps, r.leaves)
    y = np.asarray(r.y)
    assert np.all(y >= lo.astype(np.float64)) and np.all(y <= hi.astype(np.float64))
    assert np.any(y == lo.astype(np.float64)) and np.any(y == hi.astype(np.float64))
    assert len(set(lo.tolist())) > 1  # the leaf motion makes the lower bounds differ
    # the same plan without a machine is not bounded that way
    r0 = oracle.cg_plan(D, c.mlc, c.structs, 12)
    assert np.max(r0.y) > hi[0]
