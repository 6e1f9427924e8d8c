"""CSR(D^T) with its columns in brick order (build option vox_grid).

The brick order renumbers the voxels inside CSR(D^T) only (4 x 4 x 2 bricks,
the grid padded up to whole bricks) so that the gathers of g in D^T g (Eq. 3)
touch fewer cache lines.  It changes no result beyond float32 rounding order:
beamlet_price and its windowed form still take g in voxel order and are
checked against the FP64 oracle with the same componentwise bound as voxel
order; plans and batches built on such a matrix (which write g in brick order
directly) are checked against the oracle's plan and against each other.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import N_SPMV_CFG, dev, host, make_ddc, require_cuda, spmv_bound
from test_gpu_cg import TIGHT, gpu_plan, near_tie_at

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()
    import __graft_entry__
    __graft_entry__.build()


def _price_check(c, ddc, dtype, seed):
    from paper_1503_01721_gb300 import api
    g = synth.random_vector(c.V, seed)
    pi = torch.full((c.J,), float("nan"), device="cuda")
    api.beamlet_price(ddc.h, dev(g, torch.float32), pi)
    torch.cuda.synchronize()
    vq, _ = oracle.quantize_ddc(c.J, c.blt, c.val, dtype)
    Dq = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, vq)
    pi_ref = oracle.beamlet_price(Dq, g)
    bound = spmv_bound(abs(Dq).T @ np.abs(g.astype(np.float64)), np.bincount(c.blt, minlength=c.J))
    assert np.all(np.abs(host(pi) - pi_ref) <= bound)
    return host(pi)


@pytest.mark.parametrize("name", ["tiny", "ragged", "cfg1"])
@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
def test_brick_beamlet_price(name, dtype):
    """ragged (13 x 11 x 9) pads every axis up to whole bricks; voxels without entries get dose 0."""
    c = synth.make_case(name, seed=0)
    ddc = make_ddc(c, dtype, brick=True)
    assert ddc.info()["vox_brick"] == 1
    _price_check(c, ddc, dtype, 3)
    # CSR(D)'s rows (the compact voxels) are in brick order too; the dose comes back in voxel order
    from paper_1503_01721_gb300 import api
    x = synth.random_vector(c.J, 4, 0.0, 1.0)
    d = torch.full((c.V,), float("nan"), device="cuda")
    api.dose_forward(ddc.h, dev(x, torch.float32), d)
    torch.cuda.synchronize()
    vq, _ = oracle.quantize_ddc(c.J, c.blt, c.val, dtype)
    Dq = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, vq)
    d_ref = oracle.dose_forward(Dq, x)
    bound = spmv_bound(abs(Dq) @ np.abs(x.astype(np.float64)), np.bincount(c.vox, minlength=c.V))
    assert np.all(np.abs(host(d) - d_ref) <= bound)


@pytest.mark.parametrize("cfg", list(range(N_SPMV_CFG)))
def test_brick_every_config(cfg):
    for name, seed in (("ragged", 1), ("cfg1", 0)):
        c = synth.make_case(name, seed=seed)
        _price_check(c, make_ddc(c, tile_cfg=cfg, brick=True), "f32", 7)


@pytest.mark.parametrize("cfg", [0, 5, 6, 9, 11])
def test_brick_windowed_equals_full_pass_inside_windows(cfg):
    from paper_1503_01721_gb300 import api
    from test_gpu_spmv import _placed_state
    for name, seed, n_placed in (("ragged", 1, 3), ("cfg1", 0, 9)):
        c = synth.make_case(name, seed=seed)
        m = c.mlc
        ddc = make_ddc(c, tile_cfg=cfg, brick=True)
        occupied, leaves = _placed_state(m, np.random.default_rng(60 + cfg), n_placed)
        need = np.zeros((m.K, m.n_rows, m.n_cols), bool)
        for k in range(m.K):
            if occupied[k]:
                continue
            Lmin, _, _, Rmax = oracle.leaf_windows(m, occupied, leaves, k)
            for r in range(m.n_rows):
                need[k, r, Lmin[r]:max(Rmax[r], Lmin[r])] = True
        need = need.reshape(-1)
        g = dev(synth.random_vector(c.V, 17 + cfg), torch.float32)
        full = torch.empty(c.J, device="cuda")
        api.beamlet_price(ddc.h, g, full)
        pw = torch.full((c.J,), float("nan"), device="cuda")
        api.beamlet_price_windowed(ddc.h, m, dev(occupied, torch.uint8), dev(leaves, torch.int16), g, pw)
        torch.cuda.synchronize()
        assert np.array_equal(host(pw)[need].view(np.uint32), host(full)[need].view(np.uint32)), f"{name} cfg {cfg}"


def test_brick_long_rows():
    """Rows longer than the shared-memory sort (20,000 entries) are sorted again by
    brick position through the global-memory path."""
    from paper_1503_01721_gb300 import api
    nx, ny, nz = 30, 35, 20
    V = nx * ny * nz
    lens = [4096, 0, 1, 8191, 0, 20000, 0]
    rng = np.random.default_rng(0)
    vox = np.concatenate([rng.choice(V, size=n, replace=False) for n in lens]).astype(np.int32)
    blt = np.concatenate([np.full(n, j) for j, n in enumerate(lens)]).astype(np.int32)
    val = rng.uniform(0.01, 1, len(vox)).astype(np.float32)
    J = len(lens)
    g = synth.random_vector(V, 2)
    D = oracle.ddc_matrix(V, J, vox, blt, val)
    pi_ref = oracle.beamlet_price(D, g)
    bound = spmv_bound(abs(D).T @ np.abs(g.astype(np.float64)), np.asarray(lens))
    for cfg in (0, 5, 11):
        ddc = api.Ddc(V, J, dev(vox, torch.int32), dev(blt, torch.int32), dev(val, torch.float32), tile_cfg=cfg,
                      vox_grid=(nx, ny, nz))
        pi = torch.empty(J, device="cuda")
        api.beamlet_price(ddc.h, dev(g, torch.float32), pi)
        torch.cuda.synchronize()
        assert np.all(np.abs(host(pi) - pi_ref) <= bound)
        ddc.close()


@pytest.mark.parametrize("name,n", [("ragged", 4), ("cfg1", 20)])
def test_brick_plan_matches_oracle(name, n):
    c = synth.make_case(name, seed=0)
    ddc = make_ddc(c, brick=True)
    D = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, c.val)
    s = c.structs
    F, st, cps, lv, y, dose = gpu_plan(ddc, c, n, TIGHT)
    d_ref = oracle.dose_forward(D, oracle.aperture_fluence(c.mlc, cps, lv, y))
    assert np.max(np.abs(dose - d_ref)) <= 1e-5 * max(np.max(np.abs(d_ref)), 1e-30)
    ref = oracle.cg_plan(D, c.mlc, s, n, oracle.BBOptions(**TIGHT))
    if list(cps) == ref.cps:
        assert abs(F - ref.F) <= 1e-4 * ref.F
    else:
        t = next(i for i, (a, b) in enumerate(zip(list(cps), ref.cps)) if a != b)
        assert near_tie_at(ddc, c, D, t, cps[t], TIGHT), \
            f"aperture sequence differs at step {t}: gpu {list(cps)} oracle {ref.cps}"


def test_brick_batch_equals_single_plans():
    """A batch of brick-ordered plans (the batched gradient writes g in brick order)
    against the same plans through cg_plan, bit for bit in F."""
    from paper_1503_01721_gb300 import api
    cases = [(synth.make_case("ragged", seed=0), 4), (synth.make_case("cfg1", seed=0), 10),
             (synth.make_case("cfg1", seed=2), 6)]
    ddcs = [make_ddc(c, brick=True) for c, _ in cases]
    voxs = [api.VoxelParams.from_numpy(c.structs) for c, _ in cases]
    batch = api.Batch([(d.h, c.mlc, v, n) for d, v, (c, n) in zip(ddcs, voxs, cases)], api.BBOptions(**TIGHT))
    F, st = batch.run()
    for i, (c, n) in enumerate(cases):
        F1, _, cps1, _, _, _ = gpu_plan(ddcs[i], c, n, TIGHT)
        assert st[i]["n_apertures"] == n
        assert F1 == F[i]
    batch.close()


def test_brick_grid_must_match_V():
    from paper_1503_01721_gb300 import api, _lib
    c = synth.make_case("tiny", seed=0)
    args = (c.V, c.J, dev(c.vox, torch.int32), dev(c.blt, torch.int32), dev(c.val, torch.float32))
    for grid in ((8, 8, 7), (8, 8, 0), (-8, -8, 8)):
        with pytest.raises(_lib.VmatError) as e:
            api.Ddc(*args, vox_grid=grid)
        assert e.value.status == _lib.VMAT_EINVAL


def test_autotuned_window_config_is_the_plans():
    """An autotuned handle times the warp-row configurations once on a pass over half
    of every MLC row and runs the plan's windowed D^T g passes with the fastest: the
    plan is bit for bit the plan of a handle built with that configuration."""
    from paper_1503_01721_gb300 import api
    c = synth.make_case("cfg1", seed=0)
    g = c.geom
    args = (c.V, c.J, dev(c.vox, torch.int32), dev(c.blt, torch.int32), dev(c.val, torch.float32))
    tuned = api.Ddc(*args, autotune=True, vox_grid=(g.nx, g.ny, g.nz))
    vox = api.VoxelParams.from_numpy(c.structs)
    F1, st1 = api.cg_plan(tuned.h, c.mlc, vox, 8)
    cfg = int(st1["pp1_spmv_cfg"])
    assert 0 <= cfg < N_SPMV_CFG
    F2, st2 = api.cg_plan(tuned.h, c.mlc, vox, 8)
    assert st2["pp1_spmv_cfg"] == cfg and F2 == F1
    fixed = api.Ddc(*args, tile_cfg=tuned.info()["cfg_D"], tile_cfg_Dt=cfg, vox_grid=(g.nx, g.ny, g.nz))
    F3, st3 = api.cg_plan(fixed.h, c.mlc, vox, 8)
    assert st3["pp1_spmv_cfg"] == cfg and F3 == F1
