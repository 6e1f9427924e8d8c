"""Pins of the column-generation loop (Section 2.1) and of the aperture maps
(Eq. 5; x = A y and its adjoint)."""
import itertools

import numpy as np

import oracle
import synth


def test_first_aperture_is_global_best(tiny_case):
    c = tiny_case
    D = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, c.val)
    s = c.structs
    _, g = oracle.objective_grad(np.zeros(c.V), s.struct_id, s.T, s.w_over, s.w_under)
    pi = oracle.beamlet_price(D, g)
    k, lv, price = oracle.price_apertures(c.mlc, pi, np.zeros(c.mlc.K, bool), np.zeros((c.mlc.K, c.mlc.n_rows, 2)))
    N = c.mlc.n_cols
    best = -np.inf
    for kk in range(c.mlc.K):
        tot = 0.0
        for r in range(c.mlc.n_rows):
            base = (kk * c.mlc.n_rows + r) * N
            tot += max(float(np.sum(pi[base + L: base + R])) for L in range(N + 1) for R in range(L, N + 1))
        best = max(best, tot)
    assert abs(price - best) <= 1e-12 * abs(best)
    plan = oracle.cg_plan(D, c.mlc, s, 1)
    assert plan.cps == [k]


def test_plan_objective_decreases(ragged_case):
    c = ragged_case
    D = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, c.val)
    s = c.structs
    F0 = oracle.objective_grad(np.zeros(c.V), s.struct_id, s.T, s.w_over, s.w_under)[0]
    Fs = [F0]
    for n in range(1, 5):
        plan = oracle.cg_plan(D, c.mlc, s, n)
        Fs.append(plan.F)
        assert len(set(plan.cps)) == len(plan.cps)          # occupied CPs never repeat
        assert all(p > 0 for p in plan.prices)
    assert all(b <= a * (1 + 1e-6) for a, b in zip(Fs, Fs[1:]))
    assert Fs[-1] < 0.9 * F0


def test_final_dose_is_D_of_A_y(ragged_case):
    c = ragged_case
    D = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, c.val)
    plan = oracle.cg_plan(D, c.mlc, c.structs, 3)
    x = oracle.aperture_fluence(c.mlc, plan.cps, plan.leaves, plan.y)
    np.testing.assert_allclose(plan.dose, D @ x, rtol=1e-12)
    cols = np.stack([oracle.aperture_dose(D, c.mlc, k, lv) for k, lv in zip(plan.cps, plan.leaves)], 1)
    np.testing.assert_allclose(plan.dose, cols @ plan.y, rtol=1e-10, atol=1e-14)


def test_stops_when_no_price_is_positive(tiny_case):
    c = tiny_case
    D = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, c.val)
    s = c.structs
    zero = synth.Structures(s.struct_id, np.zeros_like(s.T), s.w_over, s.w_under, s.names)
    plan = oracle.cg_plan(D, c.mlc, zero, 5)
    assert plan.cps == [] and plan.stop == "price" and plan.F == 0.0


def test_aperture_dose_is_column_sum(ragged_case):
    c = ragged_case
    D = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, c.val)
    lv = np.array([[1, 5], [0, 0], [2, 7]])
    want = np.zeros(c.V)
    inside = set(oracle.aperture_beamlets(c.mlc, 3, lv).tolist())
    assert len(inside) == 4 + 0 + 5
    for i, j, v in zip(c.vox.tolist(), c.blt.tolist(), c.val.tolist()):
        if j in inside:
            want[i] += v
    np.testing.assert_allclose(oracle.aperture_dose(D, c.mlc, 3, lv), want, rtol=1e-13)


def test_fluence_map_adjoint():
    mlc = synth.MLC(7, 5, 9, np.array([0], np.int32), 3)
    cps, leaves, y = synth.random_apertures(mlc, 11, 3, 2, 7)
    pi = synth.random_vector(mlc.K * 5 * 9, 4).astype(np.float64)
    x = oracle.aperture_fluence(mlc, cps, leaves, y)
    gy = oracle.aperture_grad(mlc, cps, leaves, pi)
    assert abs(float(x @ pi) - float(y.astype(np.float64) @ gy)) < 1e-12 * float(np.abs(x) @ np.abs(pi))
    # explicit incidence matrix
    A = np.zeros((mlc.K * 5 * 9, len(cps)))
    for n, k in enumerate(cps):
        for r, c in itertools.product(range(5), range(9)):
            if leaves[n][r][0] <= c < leaves[n][r][1]:
                A[(k * 5 + r) * 9 + c, n] = 1
    np.testing.assert_allclose(x, A @ y, rtol=1e-15)


def test_refine_plan_pins(ragged_case):
    """refine_plan (reading R12): on a plan chosen with E4M3 values, the refined
    y is a KKT point of the master problem on the float32 DA built column by
    column from unit aperture indicators, no worse than the plan's own y scored
    on the float32 matrix; on an FP32 plan it changes nothing."""
    c = ragged_case
    s = c.structs
    tight = oracle.BBOptions(max_iter=3000, rel_tol5=1e-12, step_tol=1e-14)
    D = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, c.val)
    Dq = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, oracle.quantize_ddc(c.J, c.blt, c.val, "fp8")[0])
    plan = oracle.cg_plan(Dq, c.mlc, s, 4, tight)
    y_r, dose, F_r, _ = oracle.refine_plan(D, c.mlc, s, plan.cps, plan.leaves, plan.y, tight)
    # DA from indicator vectors written out beamlet by beamlet
    n = len(plan.cps)
    DA = np.zeros((c.V, n))
    for a, (k, lv) in enumerate(zip(plan.cps, plan.leaves)):
        ind = np.zeros(c.J)
        for r in range(c.mlc.n_rows):
            for col in range(int(lv[r][0]), int(lv[r][1])):
                ind[(k * c.mlc.n_rows + r) * c.mlc.n_cols + col] = 1.0
        DA[:, a] = D @ ind
    assert np.allclose(dose, DA @ y_r, rtol=1e-12, atol=1e-14)
    F_chk, g = oracle.objective_grad(DA @ y_r, s.struct_id, s.T, s.w_over, s.w_under)
    assert abs(F_chk - F_r) <= 1e-12 * F_r
    G = -(DA.T @ g)  # gradient of F in y
    scale = np.max(np.abs(DA.T @ np.abs(g))) + 1e-30
    assert np.all(np.where(y_r > 0, np.abs(G), np.maximum(-G, 0.0)) <= 1e-6 * scale)
    F_plan_y, _ = oracle.objective_grad(DA @ np.asarray(plan.y), s.struct_id, s.T, s.w_over, s.w_under)
    assert F_r <= F_plan_y * (1 + 1e-12)
    # an FP32 plan is already optimal for its own columns
    p32 = oracle.cg_plan(D, c.mlc, s, 4, tight)
    _, _, F32r, _ = oracle.refine_plan(D, c.mlc, s, p32.cps, p32.leaves, p32.y, tight)
    assert abs(F32r - p32.F) <= 1e-9 * p32.F
