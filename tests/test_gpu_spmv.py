"""Parity of the two hot sparse products with the FP64 oracle:
beamlet_price pi = D^T g (Eq. 3) and dose_forward d = D x (Section 2.1).

Bound: each output within c * 2^-24 * sum_i |D_ij g_i| of the float64 result on
the same stored values (the float32 accumulation bound of the tile reduction);
the dose also within 1e-5 relative L-infinity.  Lower-precision storage is
compared with the oracle on the dequantised values (same bound) and its total
error against the float32 matrix is checked against the format's rounding.
"""
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import INDEX16_TWIN, N_SPMV_CFG, dev, host, make_ddc, require_cuda, spmv_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()
    import __graft_entry__
    __graft_entry__.build()


def run_products(ddc, V, J, g, x, cp_active=None, bpc=0):
    from paper_1503_01721_gb300 import api
    pi = torch.full((J,), float("nan"), device="cuda")
    d = torch.full((V,), float("nan"), device="cuda")
    api.beamlet_price(ddc.h, dev(g, torch.float32), pi, None if cp_active is None else dev(cp_active, torch.uint8), bpc)
    api.dose_forward(ddc.h, dev(x, torch.float32), d)
    torch.cuda.synchronize()
    return host(pi), host(d)


def check_products(V, J, vox, blt, val, dtype="f32", tile_cfg=-1, seed=0):
    ddc = make_ddc((vox, blt, val), dtype, tile_cfg, V, J)
    g = synth.random_vector(V, seed + 1)
    x = synth.random_vector(J, seed + 2, 0.0, 1.0)
    pi, d = run_products(ddc, V, J, g, x)
    vq, _ = oracle.quantize_ddc(J, blt, val, dtype)
    Dq = oracle.ddc_matrix(V, J, vox, blt, vq)
    absD = abs(Dq)
    pi_ref = oracle.beamlet_price(Dq, g)
    d_ref = oracle.dose_forward(Dq, x)
    len_t = np.bincount(blt, minlength=J)
    len_d = np.bincount(vox, minlength=V)
    assert np.all(np.abs(pi - pi_ref) <= spmv_bound(absD.T @ np.abs(g.astype(np.float64)), len_t))
    assert np.all(np.abs(d - d_ref) <= spmv_bound(absD @ np.abs(x.astype(np.float64)), len_d))
    if d_ref.size and np.max(np.abs(d_ref)) > 0:
        assert np.max(np.abs(d - d_ref)) <= 1e-5 * np.max(np.abs(d_ref))
    return ddc, pi, d


@pytest.mark.parametrize("name", ["tiny", "ragged", "cfg1"])
def test_products_f32(name):
    c = synth.make_case(name, seed=0)
    check_products(c.V, c.J, c.vox, c.blt, c.val)


@pytest.mark.parametrize("cfg", list(range(N_SPMV_CFG)))
def test_every_tile_config(cfg):
    c = synth.make_case("ragged", seed=1)
    check_products(c.V, c.J, c.vox, c.blt, c.val, tile_cfg=cfg)
    c = synth.make_case("cfg1", seed=0)
    check_products(c.V, c.J, c.vox, c.blt, c.val, tile_cfg=cfg, seed=5)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
def test_index16_configs_match_their_32bit_twins_bit_for_bit(dtype):
    """The 16-bit column index changes the bytes read, not the arithmetic: each
    configuration that reads it gives the same bits as the consecutive-lane
    configuration with the same launch shape."""
    cases = [synth.make_case("ragged", seed=1), synth.make_case("cfg1", seed=0)]
    for c in cases:
        g = synth.random_vector(c.V, 11)
        x = synth.random_vector(c.J, 12, 0.0, 1.0)
        for z, twin in INDEX16_TWIN.items():
            dz = make_ddc(c, dtype, z)
            info = dz.info()
            assert info["index16_Dt"] == 1 and info["index16_D"] == 1 and info["cfg_Dt"] == z
            assert info["bytes16_Dt"] == 2 * c.nnz + 4 * _chunks(c.blt, c.J) + 8 * (c.J + 1)
            dc = make_ddc(c, dtype, twin)
            a = run_products(dz, c.V, c.J, g, x)
            b = run_products(dc, c.V, c.J, g, x)
            assert all(np.array_equal(u.view(np.uint32), v.view(np.uint32)) for u, v in zip(a, b))


def _chunks(rows, n_rows):
    return int(np.sum((np.bincount(rows, minlength=n_rows) + 127) // 128))


def test_index16_chunk_span_limit():
    """A chunk whose columns span 65,535 fits 16 bits; 65,537 does not, and then the
    matrix keeps 32-bit indices only (the 16-bit configurations are refused)."""
    from paper_1503_01721_gb300 import _lib
    V = 140000
    rows = [np.array([0, 65535]),                                         # span 65,535: fits
            np.concatenate([np.arange(128), 100000 + np.arange(172)]),    # 3 chunks, a jump between chunks
            np.arange(7, 7 + 128 * 40, 40)]                               # 128 entries spanning 5,080
    def coo(rs):
        vox = np.concatenate(rs).astype(np.int32)
        blt = np.concatenate([np.full(len(r), j) for j, r in enumerate(rs)]).astype(np.int32)
        val = np.random.default_rng(1).uniform(0.1, 1.0, len(vox)).astype(np.float32)
        return vox, blt, val
    vox, blt, val = coo(rows)
    ddc, _, _ = check_products(V, len(rows), vox, blt, val, tile_cfg=12)
    assert ddc.info()["index16_Dt"] == 1
    bad = rows + [np.array([5, 65542])]                                  # span 65,537: does not fit
    vox, blt, val = coo(bad)
    with pytest.raises(_lib.VmatError) as e:
        make_ddc((vox, blt, val), "f32", 12, V, len(bad))
    assert e.value.status == _lib.VMAT_EUNSUPPORTED
    ddc = make_ddc((vox, blt, val), "f32", -1, V, len(bad), index16=True)
    info = ddc.info()
    assert info["index16_Dt"] == 0 and info["bytes16_Dt"] == 0 and info["index16_D"] == 1
    # the autotuner times the 16-bit configurations only where the index exists
    from paper_1503_01721_gb300 import api
    ddc = api.Ddc(V, len(bad), dev(vox, torch.int32), dev(blt, torch.int32), dev(val, torch.float32),
                  autotune=True, index16=True)
    assert ddc.info()["cfg_Dt"] not in INDEX16_TWIN
    g = synth.random_vector(V, 1)
    pi, _ = run_products(ddc, V, len(bad), g, np.ones(len(bad), np.float32))
    D = oracle.ddc_matrix(V, len(bad), vox, blt, val)
    pi_ref = oracle.beamlet_price(D, g)
    assert np.all(np.abs(pi - pi_ref) <= spmv_bound(abs(D).T @ np.abs(g.astype(np.float64)),
                                                     np.bincount(blt, minlength=len(bad))))


def test_separate_configurations_per_matrix():
    """tile_cfg_Dt sets CSR(D^T)'s configuration apart from CSR(D)'s (an autotuned pair
    reused without tuning again): the handle reports both and the products are right."""
    from paper_1503_01721_gb300 import _lib, api
    c = synth.make_case("cfg1", seed=0)
    coo = (dev(c.vox, torch.int32), dev(c.blt, torch.int32), dev(c.val, torch.float32))
    tuned = api.Ddc(c.V, c.J, *coo, autotune=True)
    info = tuned.info()
    ddc = api.Ddc(c.V, c.J, *coo, tile_cfg=info["cfg_D"], tile_cfg_Dt=info["cfg_Dt"])
    assert (ddc.info()["cfg_D"], ddc.info()["cfg_Dt"]) == (info["cfg_D"], info["cfg_Dt"])
    ddc = api.Ddc(c.V, c.J, *coo, tile_cfg=1, tile_cfg_Dt=11)
    assert (ddc.info()["cfg_D"], ddc.info()["cfg_Dt"]) == (1, 11)
    g = synth.random_vector(c.V, 21)
    x = synth.random_vector(c.J, 22, 0.0, 1.0)
    a = run_products(ddc, c.V, c.J, g, x)
    b = run_products(make_ddc(c, "f32", 11), c.V, c.J, g, x)
    assert np.array_equal(a[0].view(np.uint32), b[0].view(np.uint32))  # D^T g by configuration 11 in both
    b = run_products(make_ddc(c, "f32", 1), c.V, c.J, g, x)
    assert np.array_equal(a[1].view(np.uint32), b[1].view(np.uint32))  # D x by configuration 1 in both
    with pytest.raises(_lib.VmatError) as e:
        api.Ddc(c.V, c.J, *coo, tile_cfg_Dt=N_SPMV_CFG)
    assert e.value.status == _lib.VMAT_EINVAL


def test_kept_coo_builds_the_same_matrices():
    """Keeping the COO changes where the column-ordered build sorts (its own temporaries
    instead of the COO's arrays), not the result: the same products, bit for bit, and
    the kept COO builds again."""
    from paper_1503_01721_gb300 import api
    c = synth.make_case("cfg1", seed=0)
    g = synth.random_vector(c.V, 31)
    x = synth.random_vector(c.J, 32, 0.0, 1.0)
    ref = run_products(make_ddc(c, "f32", 9), c.V, c.J, g, x)
    h = api.ddc_load_coo(c.V, c.J, dev(c.vox, torch.int32), dev(c.blt, torch.int32), dev(c.val, torch.float32))
    try:
        for _ in range(2):  # the second build reads the kept COO
            api.ddc_build(h, "f32", tile_cfg=9, keep_coo=True)
            pi = torch.empty(c.J, device="cuda")
            d = torch.empty(c.V, device="cuda")
            api.beamlet_price(h, dev(g, torch.float32), pi)
            api.dose_forward(h, dev(x, torch.float32), d)
            torch.cuda.synchronize()
            assert np.array_equal(host(pi).view(np.uint32), ref[0].view(np.uint32))
            assert np.array_equal(host(d).view(np.uint32), ref[1].view(np.uint32))
    finally:
        api.ddc_free(h)


def test_shuffled_coo_gives_identical_bits():
    c = synth.make_case("cfg1", seed=0)
    _, pi1, d1 = check_products(c.V, c.J, c.vox, c.blt, c.val)
    v2, b2, a2 = synth.shuffled_coo(c.vox, c.blt, c.val, 9)
    _, pi2, d2 = check_products(c.V, c.J, v2, b2, a2)
    assert np.array_equal(pi1.view(np.uint32), pi2.view(np.uint32))
    assert np.array_equal(d1.view(np.uint32), d2.view(np.uint32))


def test_repeat_is_bitwise_deterministic():
    c = synth.make_case("ragged", seed=1)
    ddc = make_ddc(c)
    g = synth.random_vector(c.V, 3)
    x = synth.random_vector(c.J, 4)
    a = run_products(ddc, c.V, c.J, g, x)
    b = run_products(ddc, c.V, c.J, g, x)
    assert all(np.array_equal(u.view(np.uint32), v.view(np.uint32)) for u, v in zip(a, b))


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_low_precision_storage(dtype):
    c = synth.make_case("cfg1", seed=0)
    _, pi, d = check_products(c.V, c.J, c.vox, c.blt, c.val, dtype=dtype)
    # total error against the float32 matrix: elementwise storage error <= 2^-8 (bf16), 2^-4 (fp8)
    D = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, c.val)
    x = synth.random_vector(c.J, 2, 0.0, 1.0).astype(np.float64)
    d_ref = oracle.dose_forward(D, x)
    rel = np.max(np.abs(d - d_ref)) / np.max(np.abs(d_ref))
    assert rel <= {"bf16": 2.0 ** -8, "fp8": 2.0 ** -4}[dtype] + 1e-5


def test_cp_active_restricts_rows():
    c = synth.make_case("cfg1", seed=0)
    ddc = make_ddc(c)
    rng = np.random.default_rng(3)
    active = (rng.random(c.mlc.K) < 0.5).astype(np.uint8)
    bpc = c.mlc.n_rows * c.mlc.n_cols
    g = synth.random_vector(c.V, 6)
    pi, _ = run_products(ddc, c.V, c.J, g, np.zeros(c.J, np.float32), active, bpc)
    D = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, c.val)
    pi_ref = oracle.beamlet_price(D, g)
    rows = np.repeat(active.astype(bool), bpc)
    bound = spmv_bound(abs(D).T @ np.abs(g.astype(np.float64)), np.bincount(c.blt, minlength=c.J))
    assert np.all(np.abs(pi[rows] - pi_ref[rows]) <= bound[rows])


def _placed_state(mlc, rng, n_placed):
    """n_placed occupied CPs with random openings (L <= R) on every row."""
    occupied = np.zeros(mlc.K, bool)
    occupied[rng.choice(mlc.K, n_placed, replace=False)] = True
    L = rng.integers(0, mlc.n_cols + 1, size=(mlc.K, mlc.n_rows))
    W = rng.integers(0, mlc.n_cols // 2 + 1, size=(mlc.K, mlc.n_rows))
    leaves = np.stack([L, np.minimum(L + W, mlc.n_cols)], axis=2) * occupied[:, None, None]
    return occupied, leaves.astype(np.int64)


@pytest.mark.parametrize("cfg", list(range(N_SPMV_CFG)))
def test_windowed_price_every_config(cfg):
    """beamlet_price_windowed: inside the leaf-travel windows of the unoccupied CPs
    (the oracle's windows) bit-identical to the full pass of the same
    configuration; the row configurations leave every other entry unwritten."""
    from paper_1503_01721_gb300 import api
    for name, seed, n_placed in (("ragged", 1, 3), ("cfg1", 0, 9)):
        c = synth.make_case(name, seed=seed)
        m = c.mlc
        ddc = make_ddc(c, tile_cfg=cfg)
        rng = np.random.default_rng(40 + cfg)
        occupied, leaves = _placed_state(m, rng, n_placed)
        need = np.zeros((m.K, m.n_rows, m.n_cols), bool)
        for k in range(m.K):
            if occupied[k]:
                continue
            Lmin, _, _, Rmax = oracle.leaf_windows(m, occupied, leaves, k)
            for r in range(m.n_rows):
                need[k, r, Lmin[r]:max(Rmax[r], Lmin[r])] = True
        need = need.reshape(-1)
        assert 0 < need.sum() < c.J
        g = dev(synth.random_vector(c.V, 7 + cfg), torch.float32)
        full = torch.empty(c.J, device="cuda")
        api.beamlet_price(ddc.h, g, full)
        pw = torch.full((c.J,), float("nan"), device="cuda")
        api.beamlet_price_windowed(ddc.h, m, dev(occupied, torch.uint8), dev(leaves, torch.int16), g, pw)
        torch.cuda.synchronize()
        full, pw = host(full), host(pw)
        assert np.array_equal(pw[need].view(np.uint32), full[need].view(np.uint32)), f"{name} cfg {cfg}"
        if cfg >= 4:  # warp-row families: rows outside the windows are skipped
            assert np.all(np.isnan(pw[~need])), f"{name} cfg {cfg}"
        ddc.close()


def test_empty_matrix():
    V, J = 7, 12
    e = np.zeros(0, np.int32)
    ddc = make_ddc((e, e, np.zeros(0, np.float32)), V=V, J=J)
    pi, d = run_products(ddc, V, J, synth.random_vector(V, 1), synth.random_vector(J, 2))
    assert np.array_equal(pi, np.zeros(J, np.float32)) and np.array_equal(d, np.zeros(V, np.float32))


def test_tile_boundaries_long_rows_and_empty_rows():
    # beamlet rows of 4096, 0, 1, 8191, 0, 20000 entries (several full tiles, a row
    # longer than the shared-memory sort limit) and voxels without entries
    V = 21000
    lens = [4096, 0, 1, 8191, 0, 20000, 0]
    rng = np.random.default_rng(0)
    vox, blt = [], []
    for j, n in enumerate(lens):
        vv = rng.choice(V - 100, size=n, replace=False) + 50
        vox.append(vv)
        blt.append(np.full(n, j))
    vox = np.concatenate(vox).astype(np.int32)
    blt = np.concatenate(blt).astype(np.int32)
    val = rng.uniform(0.01, 1, len(vox)).astype(np.float32)
    for cfg in range(N_SPMV_CFG):
        check_products(V, len(lens), vox, blt, val, tile_cfg=cfg)


def test_long_row_sort_path(monkeypatch):
    monkeypatch.setenv("VMAT_SORT_SMEM_CAP", "32")
    c = synth.make_case("ragged", seed=1)
    v2, b2, a2 = synth.shuffled_coo(c.vox, c.blt, c.val, 2)
    check_products(c.V, c.J, v2, b2, a2)


def test_invalid_coo_rejected():
    from paper_1503_01721_gb300 import _lib, api
    vox = np.array([0, 1, 5], np.int32)   # 5 is out of range for V = 4
    blt = np.array([0, 1, 1], np.int32)
    val = np.ones(3, np.float32)
    with pytest.raises(_lib.VmatError) as e:
        make_ddc((vox, blt, val), V=4, J=2)
    assert e.value.status == _lib.VMAT_EINVAL
    vox = np.array([0, 1, 1], np.int32)   # duplicate (1, 1)
    with pytest.raises(_lib.VmatError) as e:
        make_ddc((vox, blt, val), V=4, J=2)
    assert e.value.status == _lib.VMAT_EINVAL and "duplicate" in str(e.value)
    assert api.device_status(reset=True) in (0, 4)


def test_host_coo_input_and_info():
    from paper_1503_01721_gb300 import api
    c = synth.make_case("ragged", seed=1)
    h = api.ddc_load_coo(c.V, c.J, torch.from_numpy(c.vox), torch.from_numpy(c.blt), torch.from_numpy(c.val))
    api.ddc_build(h, "f32")
    info = api.ddc_info(h)
    assert info["nnz"] == c.nnz and info["V"] == c.V and info["J"] == c.J
    assert info["n_active_vox"] == len(np.unique(c.vox))
    assert info["bytes_Dt"] == c.nnz * 8 + (c.J + 1) * 8
    api.ddc_free(h)
