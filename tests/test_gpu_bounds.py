"""Fluence-rate bounds from the delivery limits (Eq. 2, 6) on the GPU.

fluence_bounds is bit-exact against the oracle (the same float64 expressions,
rounded to float32) on random aperture sequences, multi-arc MLCs, unplaced
slots and long sequences.  Plans with a machine (cg_plan and batches) follow the
oracle's plan with the same bounds: aperture sequence equal up to near ties,
objective within the plan tolerances, every fluence rate inside the bounds of
its final aperture set, and both bounds binding somewhere.
"""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import make_ddc, require_cuda
from test_gpu_cg import TIGHT, gpu_plan, near_tie_at
from test_oracle_bounds import _mlc, _random_sequence

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()
    import __graft_entry__
    __graft_entry__.build()


def _gpu_bounds(mlc, cps, leaves):
    from paper_1503_01721_gb300 import api
    n = len(cps)
    c = torch.tensor(np.asarray(cps, np.int32), device="cuda")
    lv = torch.tensor(np.asarray(leaves, np.int16).reshape(-1), device="cuda")
    lo = torch.full((n,), -1.0, device="cuda")
    hi = torch.full((n,), -1.0, device="cuda")
    api.fluence_bounds(mlc, c, lv, lo, hi)
    torch.cuda.synchronize()
    return lo.cpu().numpy(), hi.cpu().numpy()


@pytest.mark.parametrize("seed", range(8))
def test_bounds_bit_exact(seed):
    arcs = [(0,), (0, 13), (0, 5, 11, 20)][seed % 3]
    mlc = _mlc(26, 5, 16, arcs=arcs)
    mach = synth.make_machine(mlc, speed_step_max=[0.05, 0.5, 3.0, 0.0][seed % 4])
    mach.leaf_speed_cols *= [1.0, 1.7, 3.1][seed % 3]
    mlc.machine = mach
    cps, leaves = _random_sequence(mlc, [1, 3, 7, 12, 20, 26, 9, 16][seed], seed)
    lo, hi = _gpu_bounds(mlc, cps, leaves)
    lo_r, hi_r = oracle.fluence_bounds(mlc, mach, cps, leaves)
    assert np.array_equal(lo, lo_r) and np.array_equal(hi, hi_r)


def test_bounds_unplaced_slots_long_sequences_and_no_machine():
    mlc = _mlc(360, 8, 40, arcs=(0, 180))
    mlc.machine = synth.make_machine(mlc, speed_step_max=0.02)
    cps, leaves = _random_sequence(mlc, 300, 7)
    lo, hi = _gpu_bounds(mlc, cps, leaves)
    lo_r, hi_r = oracle.fluence_bounds(mlc, mlc.machine, cps, leaves)
    assert np.array_equal(lo, lo_r) and np.array_equal(hi, hi_r)
    # slots not yet placed (cps < 0) get [0, +inf) and do not act as neighbours
    cps2 = list(cps[:40]) + [-1] * 10
    leaves2 = list(leaves[:40]) + [np.zeros((8, 2), np.int64)] * 10
    lo, hi = _gpu_bounds(mlc, cps2, leaves2)
    lo_r, hi_r = oracle.fluence_bounds(mlc, mlc.machine, cps[:40], leaves[:40])
    assert np.array_equal(lo[:40], lo_r) and np.array_equal(hi[:40], hi_r)
    assert np.all(lo[40:] == 0.0) and np.all(np.isinf(hi[40:]))
    # a zero slowest speed: no upper bound
    mlc.machine = synth.make_machine(mlc, speed_min=0.0)
    mlc.machine.leaf_speed_cols = 1.0
    lo, hi = _gpu_bounds(mlc, cps[:20], leaves[:20])
    lo_r, hi_r = oracle.fluence_bounds(mlc, mlc.machine, cps[:20], leaves[:20])
    assert np.array_equal(lo, lo_r) and np.all(np.isinf(hi))
    # no machine: the fixed box
    mlc.machine = None
    lo, hi = _gpu_bounds(mlc, cps[:5], leaves[:5])
    assert np.all(lo == 0.0) and np.all(np.isinf(hi))


def _machine_case(name, seed=0, **kw):
    c = synth.make_case(name, seed=seed)
    mlc = dataclasses.replace(c.mlc)
    mlc.machine = synth.make_machine(mlc, **kw)
    return dataclasses.replace(c, mlc=mlc)


@pytest.mark.parametrize("name,n", [("tiny", 4), ("ragged", 4), ("cfg1", 12)])
@pytest.mark.parametrize("tight", [False, True])
def test_plan_with_machine_matches_oracle(name, n, tight):
    c = _machine_case(name)
    ddc = make_ddc(c)
    D = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, c.val)
    s = c.structs
    opts = TIGHT if tight else None
    F, st, cps, lv, y, dose = gpu_plan(ddc, c, n, opts)
    # every fluence rate lies within the bounds of the final aperture set (float32 compares)
    lo, hi = oracle.fluence_bounds(c.mlc, c.mlc.machine, list(cps), list(lv))
    assert np.all(y >= lo) and np.all(y <= hi)
    x = oracle.aperture_fluence(c.mlc, cps, lv, y)
    d_ref = oracle.dose_forward(D, x)
    assert np.max(np.abs(dose - d_ref)) <= 1e-5 * max(np.max(np.abs(d_ref)), 1e-30)
    ref = oracle.cg_plan(D, c.mlc, s, n, oracle.BBOptions(**TIGHT) if tight else None)
    if list(cps) == ref.cps:
        assert abs(F - ref.F) <= (1e-4 if tight else 1e-2) * ref.F
        if tight:
            np.testing.assert_allclose(y, ref.y, atol=1e-4 * max(np.max(ref.y), 1e-30))
    else:
        t = next(i for i, (a, b) in enumerate(zip(list(cps), ref.cps)) if a != b)
        assert near_tie_at(ddc, c, D, t, cps[t], opts), f"sequence differs at {t}: gpu {list(cps)} oracle {ref.cps}"
    if name == "cfg1" and tight:  # converged master problems end on the bounds they hit
        assert np.any(y == lo) and np.any(y == hi), "both bounds bind on this plan"


def test_batch_with_machines():
    from paper_1503_01721_gb300 import api
    from test_gpu_batch import _batch_outputs
    cases = [(_machine_case("tiny"), 3), (synth.make_case("ragged", seed=0), 4), (_machine_case("cfg1"), 12),
             (_machine_case("cfg1", seed=2, speed_step_max=0.1), 10)]
    ddcs = [make_ddc(c) for c, _ in cases]
    voxs = [api.VoxelParams.from_numpy(c.structs) for c, _ in cases]
    batch = api.Batch([(d.h, c.mlc, v, n) for d, v, (c, n) in zip(ddcs, voxs, cases)], api.BBOptions(**TIGHT))
    F, stats = batch.run()
    outs = _batch_outputs(batch, cases)
    for i, (c, n) in enumerate(cases):
        cps, lv, y, dose = outs[i]
        assert stats[i]["n_apertures"] == n
        lo, hi = oracle.fluence_bounds(c.mlc, c.mlc.machine, list(cps), list(lv))
        assert np.all(y >= lo) and np.all(y <= hi)
        D = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, c.val)
        ref = oracle.cg_plan(D, c.mlc, c.structs, n, oracle.BBOptions(**TIGHT))
        if list(cps) == ref.cps:
            assert abs(F[i] - ref.F) <= 1e-4 * ref.F
        else:
            t = next(k for k, (a, b) in enumerate(zip(list(cps), ref.cps)) if a != b)
            assert near_tie_at(ddcs[i], c, D, t, cps[t], TIGHT), \
                f"plan {i}: sequence differs at {t}: batch {list(cps)} oracle {ref.cps}"
        F1, _, cps1, _, _, _ = gpu_plan(ddcs[i], c, n, TIGHT)
        if list(cps1) == list(cps):
            assert abs(F1 - F[i]) <= 1e-4 * F1
    batch.close()


def test_plan_with_machine_and_interdigitation():
    """Both constraints at once: the delivery-limit bounds on y and the interdigitation
    constraint on the apertures, against the oracle with the same two."""
    c = _machine_case("cfg1")
    c = dataclasses.replace(c, mlc=dataclasses.replace(c.mlc, interdigitation=True))
    ddc = make_ddc(c)
    D = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, c.val)
    F, st, cps, lv, y, dose = gpu_plan(ddc, c, 12, TIGHT)
    lo, hi = oracle.fluence_bounds(c.mlc, c.mlc.machine, list(cps), list(lv))
    assert np.all(y >= lo) and np.all(y <= hi)
    for t in range(len(cps)):  # adjacent rows never interdigitate
        L, R = lv[t, :, 0], lv[t, :, 1]
        assert np.all(L[1:] <= R[:-1]) and np.all(L[:-1] <= R[1:])
    ref = oracle.cg_plan(D, c.mlc, c.structs, 12, oracle.BBOptions(**TIGHT))
    if list(cps) == ref.cps:
        assert abs(F - ref.F) <= 1e-4 * ref.F
    else:
        t = next(i for i, (a, b) in enumerate(zip(list(cps), ref.cps)) if a != b)
        assert near_tie_at(ddc, c, D, t, cps[t], TIGHT), f"sequence differs at {t}: gpu {list(cps)} oracle {ref.cps}"
