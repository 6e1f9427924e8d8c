"""Parity at the full sizes of the benchmarked workloads, in the launch
configuration bench.py times (autotuned SpMV configurations, the default master
problem options, 60 apertures).

The oracle cannot run a whole 968M-nonzero plan, so it checks what it can
compute one by one and what must hold at any size:
  * sampled rows of D^T g and D x against float64 sums of the COO entries;
  * the plan's first aperture against the oracle's pricing of the zero-dose state
    (equal CP, or a near tie within float32 price error);
  * every aperture inside its leaf-travel windows at the time it was placed;
  * the final dose D (A y) at sampled voxels within 1e-5 relative L-inf of the
    float64 product, and F equal to the objective of the returned dose;
  * for the two-arc case stored as BF16 and FP8, sampled products against the
    float64 product of the dequantised values, and a BF16 plan's dose within the
    format's relative precision of the float32 matrix's dose.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import host, require_cuda, spmv_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()
    import __graft_entry__
    __graft_entry__.build()


def _ddc(c, dtype="f32"):
    from paper_1503_01721_gb300 import api
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dt)
    # host COO, autotuned configuration: the bench's build
    return api.Ddc(c.V, c.J, t(c.vox, torch.int32), t(c.blt, torch.int32), t(c.val, torch.float32), dtype=dtype,
                   autotune=True)


def _beamlet_offsets(c):
    assert np.all(np.diff(c.blt) >= 0)  # beamlet-major COO
    return np.searchsorted(c.blt, np.arange(c.J + 1))


def _entries_of_voxels(c, voxels):
    flag = np.zeros(c.V, bool)
    flag[voxels] = True
    return np.flatnonzero(flag[c.vox])


def _products(ddc, c, g, x):
    from paper_1503_01721_gb300 import api
    pi = torch.empty(c.J, device="cuda")
    d = torch.empty(c.V, device="cuda")
    api.beamlet_price(ddc.h, torch.from_numpy(g).cuda(), pi)
    api.dose_forward(ddc.h, torch.from_numpy(x).cuda(), d)
    torch.cuda.synchronize()
    return host(pi), host(d)


def _stored(c, dtype):
    """Stored value (float64) of COO entries idx, as the oracle's quantiser defines it
    (computed for the sampled entries only)."""
    if dtype == "f32":
        return lambda idx: c.val[idx].astype(np.float64)
    if dtype == "bf16":
        return lambda idx: oracle.bf16_values(oracle.bf16_codes(c.val[idx])).astype(np.float64)
    off = _beamlet_offsets(c)
    colmax = np.zeros(c.J, np.float64)
    nz = off[1:] > off[:-1]
    colmax[nz] = np.maximum.reduceat(np.abs(c.val), off[:-1][nz])
    scale = oracle.e4m3_scale(colmax)
    return lambda idx: oracle.e4m3_values(oracle.e4m3_codes(c.val[idx].astype(np.float64) / scale[c.blt[idx]])) * \
        scale[c.blt[idx]]


def _check_sampled(c, stored, pi, d, g, x, rng, n=256):
    """pi and d against float64 sums over the COO entries of sampled beamlets / voxels;
    stored(idx): the stored values of entries idx read back as float64."""
    off = _beamlet_offsets(c)
    for j in rng.choice(c.J, n, replace=False):
        s, e = off[j], off[j + 1]
        terms = stored(np.arange(s, e)) * g[c.vox[s:e]].astype(np.float64)
        assert abs(pi[j] - terms.sum()) <= spmv_bound(np.abs(terms).sum(), e - s), f"beamlet {j}"
    voxels = rng.choice(c.V, n, replace=False)
    sel = _entries_of_voxels(c, voxels)
    w = stored(sel) * x[c.blt[sel]].astype(np.float64)
    ref = np.bincount(c.vox[sel], weights=w, minlength=c.V)[voxels]
    mag = np.bincount(c.vox[sel], weights=np.abs(w), minlength=c.V)[voxels]
    lens = np.bincount(c.vox[sel], minlength=c.V)[voxels]
    assert np.all(np.abs(d[voxels] - ref) <= spmv_bound(mag, lens))


@pytest.fixture(scope="module")
def cfg2():
    c = synth.make_case("cfg2", seed=0, cache=False)
    ddc = _ddc(c)
    yield c, ddc
    ddc.close()


def test_cfg2_sampled_products(cfg2):
    c, ddc = cfg2
    g = synth.random_vector(c.V, 11)
    x = synth.random_vector(c.J, 12, 0.0, 1.0)
    pi, d = _products(ddc, c, g, x)
    _check_sampled(c, _stored(c, "f32"), pi, d, g, x, np.random.default_rng(3))


def test_cfg2_plan(cfg2):
    from paper_1503_01721_gb300 import api
    c, ddc = cfg2
    m, s, n = c.mlc, c.structs, c.n_apertures
    assert n == 60
    vox = api.VoxelParams.from_numpy(s)
    cps = torch.empty(n, dtype=torch.int32)
    lv = torch.empty(n * m.n_rows * 2, dtype=torch.int16)
    y = torch.empty(n, dtype=torch.float32)
    dose = torch.empty(c.V, dtype=torch.float32)
    F, st = api.cg_plan(ddc.h, m, vox, n, cps_out=cps, leaves_out=lv, y_out=y, dose_out=dose)
    cps, y, dose = cps.numpy(), y.numpy().astype(np.float64), dose.numpy()
    lv = lv.numpy().reshape(n, m.n_rows, 2).astype(np.int64)
    assert st["n_apertures"] == n and len(set(cps.tolist())) == n and np.all(y >= 0.0)
    # every aperture inside the travel windows set by the apertures placed before it
    occupied = np.zeros(m.K, bool)
    leaves_all = np.zeros((m.K, m.n_rows, 2), np.int64)
    for t in range(n):
        k = int(cps[t])
        Lmin, Lmax, Rmin, Rmax = (np.asarray(a) for a in oracle.leaf_windows(m, occupied, leaves_all, k))
        L, R = lv[t, :, 0], lv[t, :, 1]
        assert np.all((L <= R) & (L >= Lmin) & (L <= Lmax) & (R >= Rmin) & (R <= Rmax)), f"aperture {t}"
        occupied[k] = True
        leaves_all[k] = lv[t]
    # the first aperture: the oracle's pricing of the zero-dose state
    _, g0 = oracle.objective_grad(np.zeros(c.V), s.struct_id, s.T, s.w_over, s.w_under)
    pi0 = np.bincount(c.blt, weights=c.val.astype(np.float64) * g0[c.vox], minlength=c.J).astype(np.float32)
    none = np.zeros(m.K, bool)
    k_ref, _, p_ref = oracle.price_apertures(m, pi0, none, np.zeros((m.K, m.n_rows, 2), np.int64))
    if int(cps[0]) != k_ref:
        p_gpu, _ = oracle.price_cp(m, pi0, none, np.zeros((m.K, m.n_rows, 2), np.int64), int(cps[0]))
        assert p_ref - p_gpu <= 1e-4 * abs(p_ref), f"first CP {cps[0]} vs oracle {k_ref}"
    # final dose D (A y) at sampled voxels, and F of the returned dose
    x = oracle.aperture_fluence(m, cps, lv, y)
    voxels = np.random.default_rng(5).choice(c.V, 4096, replace=False)
    sel = _entries_of_voxels(c, voxels)
    ref = np.bincount(c.vox[sel], weights=c.val[sel].astype(np.float64) * x[c.blt[sel]], minlength=c.V)[voxels]
    assert np.max(np.abs(dose[voxels] - ref)) <= 1e-5 * np.max(np.abs(ref))
    F_ref, _ = oracle.objective_grad(dose.astype(np.float64), s.struct_id, s.T, s.w_over, s.w_under)
    assert abs(F - F_ref) <= 1e-6 * F_ref
    F0, _ = oracle.objective_grad(np.zeros(c.V), s.struct_id, s.T, s.w_over, s.w_under)
    assert F < F0


@pytest.fixture(scope="module")
def cfg3():
    return synth.make_case("cfg3", seed=0, cache=False)


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_cfg3_low_precision_sampled_products(cfg3, dtype):
    c = cfg3
    ddc = _ddc(c, dtype)
    g = synth.random_vector(c.V, 21)
    x = synth.random_vector(c.J, 22, 0.0, 1.0)
    pi, d = _products(ddc, c, g, x)
    ddc.close()
    _check_sampled(c, _stored(c, dtype), pi, d, g, x, np.random.default_rng(9))


def test_cfg3_bf16_plan_dose_error(cfg3):
    """A BF16 plan's final dose against the float64 product with the float32 matrix:
    within the format's relative precision (2^-8) at sampled voxels."""
    from paper_1503_01721_gb300 import api
    c = cfg3
    m, s, n = c.mlc, c.structs, 60
    ddc = _ddc(c, "bf16")
    vox = api.VoxelParams.from_numpy(s)
    cps = torch.empty(n, dtype=torch.int32)
    lv = torch.empty(n * m.n_rows * 2, dtype=torch.int16)
    y = torch.empty(n, dtype=torch.float32)
    dose = torch.empty(c.V, dtype=torch.float32)
    F, st = api.cg_plan(ddc.h, m, vox, n, cps_out=cps, leaves_out=lv, y_out=y, dose_out=dose)
    ddc.close()
    k = int(st["n_apertures"])
    x = oracle.aperture_fluence(m, cps.numpy()[:k], lv.numpy().reshape(n, m.n_rows, 2)[:k].astype(np.int64),
                                y.numpy()[:k].astype(np.float64))
    voxels = np.random.default_rng(13).choice(c.V, 4096, replace=False)
    sel = _entries_of_voxels(c, voxels)
    ref = np.bincount(c.vox[sel], weights=c.val[sel].astype(np.float64) * x[c.blt[sel]], minlength=c.V)[voxels]
    err = np.max(np.abs(dose.numpy()[voxels] - ref)) / np.max(np.abs(ref))
    assert err <= 2.0 ** -8, err
