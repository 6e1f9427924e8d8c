"""Parity of the non-SpMV steps with the FP64 oracle: objective and gradient
(Eq. 1, 4), pricing (Section 2.2.2; bit-exact given the same float32 prices),
aperture maps (Eq. 5, x = A y, A^T pi) and the master problem (Eq. 6-10)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import U32, dev, host, make_ddc, require_cuda, spmv_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()
    import __graft_entry__
    __graft_entry__.build()


# ---------------------------------------------------------------------------- objective

@pytest.mark.parametrize("name", ["ragged", "cfg1"])
def test_objective_grad(name):
    from paper_1503_01721_gb300 import api
    c = synth.make_case(name, seed=0)
    s = c.structs
    rng = np.random.default_rng(1)
    z = rng.uniform(0, 1.3, c.V).astype(np.float32)
    z[::7] = s.T[s.struct_id[::7]]          # exactly at the threshold
    vox = api.VoxelParams.from_numpy(s)
    g = torch.empty(c.V, device="cuda")
    F = torch.empty(1, dtype=torch.float64, device="cuda")
    api.objective_grad(dev(z, torch.float32), vox, g, F)
    F_ref, g_ref = oracle.objective_grad(z, s.struct_id, s.T, s.w_over, s.w_under)
    assert abs(F.item() - F_ref) <= 1e-12 * F_ref
    np.testing.assert_allclose(host(g), g_ref, rtol=4 * U32, atol=1e-30)
    F2 = torch.empty(1, dtype=torch.float64, device="cuda")
    api.objective_grad(dev(z, torch.float32), vox, None, F2)
    assert F2.item() == F.item()             # same order of additions


# ---------------------------------------------------------------------------- pricing

def random_state(mlc, rng, frac):
    occupied = (rng.random(mlc.K) < frac).astype(np.uint8)
    leaves = np.zeros((mlc.K, mlc.n_rows, 2), np.int16)
    for k in np.nonzero(occupied)[0]:
        a = rng.integers(0, mlc.n_cols + 1, size=(mlc.n_rows, 2))
        leaves[k] = np.sort(a, axis=1)
    return occupied, leaves


def gpu_price(mlc, pi, occupied, leaves):
    from paper_1503_01721_gb300 import api
    bk = torch.empty(1, dtype=torch.int32, device="cuda")
    bl = torch.empty(mlc.n_rows * 2, dtype=torch.int16, device="cuda")
    bp = torch.empty(1, dtype=torch.float64, device="cuda")
    api.price_apertures(mlc, dev(pi, torch.float32), dev(occupied, torch.uint8), dev(leaves, torch.int16), bk, bl, bp)
    torch.cuda.synchronize()
    return int(bk.item()), host(bl).reshape(mlc.n_rows, 2), bp.item()


@pytest.mark.parametrize("geom,seed,ints", [((5, 3, 4, 1, (0,)), 0, True), ((12, 4, 9, 2, (0, 6)), 1, True),
                                            ((36, 20, 20, 3, (0,)), 2, False), ((180, 64, 64, 3, (0,)), 3, False),
                                            ((40, 8, 80, 2, (0, 20)), 4, True)])
def test_price_apertures_bit_exact(geom, seed, ints):
    K, nr, nc, travel, arcs = geom
    mlc = synth.MLC(K, nr, nc, np.array(arcs, np.int32), travel)
    rng = np.random.default_rng(seed)
    for frac in (0.0, 0.3, 0.8):
        if ints:
            pi = rng.integers(-3, 4, K * nr * nc).astype(np.float32)
        else:
            pi = (rng.normal(size=K * nr * nc) * 10.0 ** rng.uniform(-3, 3)).astype(np.float32)
            pi[rng.random(pi.size) < 0.2] = 0.0
        occupied, leaves = random_state(mlc, rng, frac)
        k, lv, price = gpu_price(mlc, pi, occupied, leaves)
        k_ref, lv_ref, price_ref = oracle.price_apertures(mlc, pi, occupied, leaves)
        assert k == k_ref
        if k_ref >= 0:
            assert price == price_ref                      # bitwise: same float64 operations
            assert np.array_equal(lv, np.asarray(lv_ref))


@pytest.mark.parametrize("geom,seed,ints", [((5, 3, 4, 1, (0,)), 10, True), ((12, 4, 9, 2, (0, 6)), 11, True),
                                            ((36, 20, 20, 3, (0,)), 12, False), ((36, 20, 20, 3, (0,)), 13, True),
                                            ((40, 8, 80, 2, (0, 20)), 14, False),
                                            # 64 rows of 65 x 65 windows (no CP occupied), and the 88-column limit
                                            ((45, 64, 64, 3, (0,)), 15, True), ((24, 16, 88, 4, (0, 12)), 16, False),
                                            # more unoccupied CPs than chains that run at once: two rounds
                                            ((400, 4, 10, 2, (0, 200)), 17, True), ((300, 6, 14, 3, (0,)), 18, False)])
def test_price_apertures_interdigitation_bit_exact(geom, seed, ints):
    """Interdigitation (Section 2.2.2): the GPU chain DP and the oracle's give the
    same CP, the same float64 price and the same leaves."""
    K, nr, nc, travel, arcs = geom
    mlc = synth.MLC(K, nr, nc, np.array(arcs, np.int32), travel, interdigitation=True)
    rng = np.random.default_rng(seed)
    for frac in (0.0, 0.3, 0.8):
        if ints:
            pi = rng.integers(-3, 4, K * nr * nc).astype(np.float32)
        else:
            pi = (rng.normal(size=K * nr * nc) * 10.0 ** rng.uniform(-3, 3)).astype(np.float32)
            pi[rng.random(pi.size) < 0.2] = 0.0
        occupied, leaves = random_state(mlc, rng, frac)
        k, lv, price = gpu_price(mlc, pi, occupied, leaves)
        k_ref, lv_ref, price_ref = oracle.price_apertures(mlc, pi, occupied, leaves)
        assert k == k_ref
        if k_ref >= 0:
            assert price == price_ref
            assert np.array_equal(lv, np.asarray(lv_ref))
            assert all(lv[r][0] <= min(lv[q][1] for q in (r - 1, r + 1) if 0 <= q < nr) for r in range(nr))


def test_price_all_occupied():
    mlc = synth.MLC(4, 2, 3, np.array([0], np.int32), 1)
    occupied = np.ones(4, np.uint8)
    k, _, price = gpu_price(mlc, np.ones(24, np.float32), occupied, np.zeros((4, 2, 2), np.int16))
    assert k == -1 and price == -np.inf


# ---------------------------------------------------------------------------- apertures

def test_aperture_maps():
    from paper_1503_01721_gb300 import api
    c = synth.make_case("cfg1", seed=0)
    ddc = make_ddc(c)
    D = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, c.val)
    cps, leaves, y = synth.random_apertures(c.mlc, 60, 0)
    for n in (0, 17, 59):
        da = torch.full((c.V,), float("nan"), device="cuda")
        api.aperture_dose(ddc.h, c.mlc, int(cps[n]), dev(leaves[n], torch.int16), da)
        ref = oracle.aperture_dose(D, c.mlc, int(cps[n]), leaves[n])
        ind = oracle.aperture_indicator(c.mlc, int(cps[n]), leaves[n])
        assert np.all(np.abs(host(da) - ref) <= spmv_bound(abs(D) @ ind))
    x = torch.empty(c.J, device="cuda")
    api.aperture_fluence(c.mlc, dev(cps, torch.int32), dev(leaves, torch.int16), dev(y, torch.float32), x)
    x_ref = oracle.aperture_fluence(c.mlc, cps, leaves, y)
    np.testing.assert_allclose(host(x), x_ref, rtol=64 * U32, atol=0)
    pi = synth.random_vector(c.J, 8)
    gy = torch.empty(60, device="cuda")
    api.aperture_grad(c.mlc, dev(cps, torch.int32), dev(leaves, torch.int16), dev(pi, torch.float32), gy)
    gy_ref = oracle.aperture_grad(c.mlc, cps, leaves, pi)
    absg = oracle.aperture_grad(c.mlc, cps, leaves, np.abs(pi))
    assert np.all(np.abs(host(gy) - gy_ref) <= U32 * absg + 1e-12 * absg)


# ---------------------------------------------------------------------------- master problem

def random_mp(seed, V=5000, n=8):
    rng = np.random.default_rng(seed)
    DA = (rng.uniform(0, 1, size=(V, n)) * (rng.random((V, n)) < 0.4)).astype(np.float32)
    sid = rng.integers(0, 3, V).astype(np.uint8)
    s = synth.Structures(sid, np.array([1.0, 0.5, 0.3], np.float32), np.array([1.0, 0.3, 0.05], np.float32),
                         np.array([1.0, 0.0, 0.0], np.float32), ["t", "o", "n"])
    return DA, s


@pytest.mark.parametrize("seed,upper,V,n", [(0, None, 5000, 8), (1, None, 5000, 8), (2, 0.05, 5000, 8),
                                            (3, None, 5000, 37),
                                            (4, None, 4999, 8),      # ld not a multiple of 4: global-load pass
                                            (5, None, 3000, 120)])   # too many columns for two staged tiles
def test_mp_bb_solve(seed, upper, V, n):
    from paper_1503_01721_gb300 import api
    DA, s = random_mp(seed, V=V, n=n)
    V, n = DA.shape
    hi = None if upper is None else np.full(n, upper, np.float32)
    y = torch.zeros(n, device="cuda")
    z = torch.empty(V, device="cuda")
    rep = api.mp_bb_solve(dev(DA.T, torch.float32), api.VoxelParams.from_numpy(s), y, z,
                          hi=None if hi is None else dev(hi, torch.float32))
    yg = host(y).astype(np.float64)
    DA64 = DA.astype(np.float64)
    F_gpu, g = oracle.objective_grad(DA64 @ yg, s.struct_id, s.T, s.w_over, s.w_under)
    # the returned z is DA y in float32 and the reported F is its objective
    assert np.max(np.abs(host(z) - DA64 @ yg)) <= 1e-5 * max(1.0, np.max(np.abs(DA64 @ yg)))
    assert abs(rep["F"] - F_gpu) <= 1e-5 * F_gpu
    # optimum from the oracle with tight tolerances
    tight = oracle.BBOptions(max_iter=20000, rel_tol5=1e-15, step_tol=1e-16)
    _, _, F_opt, _, _, _ = oracle.mp_bb_solve(DA64, s.struct_id, s.T, s.w_over, s.w_under, np.zeros(n), hi=hi,
                                              opts=tight)
    assert F_opt <= F_gpu * (1 + 1e-9)
    assert F_gpu <= F_opt * (1 + 1e-4)
    # KKT in float64 at the GPU's y
    G = -(DA64.T @ g)
    scale = np.max(np.abs(DA64.T @ np.abs(g)))
    hib = np.full(n, np.inf) if hi is None else hi
    for k in range(n):
        if yg[k] <= 0:
            assert G[k] >= -2e-3 * scale
        elif yg[k] >= hib[k]:
            assert G[k] <= 2e-3 * scale
        else:
            assert abs(G[k]) <= 2e-3 * scale
    assert rep["stop"] in ("rel", "step")
