"""Pins of the objective (Eq. 1) and g = -grad F (Eq. 4)."""
import numpy as np

import oracle

T = np.array([1.0, 0.5], np.float32)        # 0: target (T = prescription), 1: OAR (T = limit)
WO = np.array([1.0, 0.3], np.float32)       # overdose weights
WU = np.array([1.0, 0.0], np.float32)       # underdose weight; zero for the OAR


def test_hand_values():
    sid = np.array([0, 0, 0, 1, 1], np.uint8)
    z = np.array([1.5, 0.5, 1.0, 0.2, 1.0])
    F, g = oracle.objective_grad(z, sid, T, WO, WU)
    # target over by 0.5: 0.25, g = -1; under by 0.5: 0.25, g = +1; on target: 0
    # OAR below its limit: 0; OAR over by 0.5: 0.3 * 0.25 = 0.075, g = -0.3
    w = float(np.float32(0.3))
    assert abs(F - (0.25 + 0.25 + 0.0 + 0.0 + w * 0.25)) < 1e-15
    np.testing.assert_allclose(g, [-1.0, 1.0, 0.0, 0.0, -w], rtol=0, atol=1e-15)


def test_zero_at_prescription():
    sid = np.array([0, 1, 0, 1], np.uint8)
    z = T[sid].astype(np.float64)
    F, g = oracle.objective_grad(z, sid, T, WO, WU)
    assert F == 0.0 and not np.any(g)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    sid = rng.integers(0, 2, 200).astype(np.uint8)
    z = rng.uniform(0, 2, 200)
    z[np.abs(z - T[sid]) < 0.01] += 0.05      # keep away from the kinks
    _, g = oracle.objective_grad(z, sid, T, WO, WU)
    h = 1e-3
    for i in range(0, 200, 7):
        zp, zm = z.copy(), z.copy()
        zp[i] += h
        zm[i] -= h
        fd = (oracle.objective_grad(zp, sid, T, WO, WU)[0] - oracle.objective_grad(zm, sid, T, WO, WU)[0]) / (2 * h)
        assert abs(fd + g[i]) < 1e-9


def test_active_weight():
    sid = np.array([0, 0, 0, 1, 1], np.uint8)
    z = np.array([1.5, 0.5, 1.0, 0.2, 1.0])
    np.testing.assert_allclose(oracle.active_weight(z, sid, T, WO, WU), [1.0, 1.0, 0.0, 0.0, 0.3], rtol=1e-7)
