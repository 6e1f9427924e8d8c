"""Batched plans (vmat_batch_*): independent plans of different sizes advanced
together in shared launches, the run recorded as one CUDA graph.

Every plan of a batch is checked against the FP64 oracle as a single plan is
(aperture sequence equal up to near ties, objective close, final dose = D (A y)
to float32 accuracy), against the library's own single-plan cg_plan, and a
second run of the same graph must reproduce the first bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import make_ddc, require_cuda
from test_gpu_cg import TIGHT, gpu_plan, near_tie_at

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()
    import __graft_entry__
    __graft_entry__.build()


def _cases():
    # different grids, CP counts, MLC shapes and aperture counts in one batch
    return [(synth.make_case("tiny", seed=0), 3), (synth.make_case("ragged", seed=0), 4),
            (synth.make_case("cfg1", seed=0), 12), (synth.make_case("tiny", seed=1), 2),
            (synth.make_case("cfg1", seed=2), 20)]


def _batch_outputs(batch, cases):
    out = []
    for i, (c, n) in enumerate(cases):
        cps = torch.empty(max(n, 1), dtype=torch.int32)
        lv = torch.empty(max(n, 1) * c.mlc.n_rows * 2, dtype=torch.int16)
        y = torch.empty(max(n, 1), dtype=torch.float32)
        dose = torch.empty(c.V, dtype=torch.float32)
        batch.result(i, cps, lv, y, dose)
        out.append((cps.numpy()[:n].copy(), lv.numpy()[:n * c.mlc.n_rows * 2].reshape(n, c.mlc.n_rows, 2).copy(),
                    y.numpy()[:n].copy(), dose.numpy().copy()))
    return out


def _check_batch(batch, ddcs, cases, tight):
    """Every plan against the oracle and against cg_plan alone; a second replay of
    the graph equal bit for bit."""
    F, stats = batch.run()
    outs = _batch_outputs(batch, cases)
    for i, (c, n) in enumerate(cases):
        cps, lv, y, dose = outs[i]
        st = stats[i]
        assert st["n_apertures"] == n and st["stop"] == "count" and st["bb_iters_total"] > 0
        if c.mlc.interdigitation:  # the left leaf of a row never passes an adjacent row's right leaf
            for a in lv:
                assert np.all(a[1:, 0] <= a[:-1, 1]) and np.all(a[:-1, 0] <= a[1:, 1])
        D = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, c.val)
        s = c.structs
        x = oracle.aperture_fluence(c.mlc, cps, lv, y)
        d_ref = oracle.dose_forward(D, x)
        assert np.max(np.abs(dose - d_ref)) <= 1e-5 * max(np.max(np.abs(d_ref)), 1e-30)
        F_at, _ = oracle.objective_grad(d_ref, s.struct_id, s.T, s.w_over, s.w_under)
        assert abs(F[i] - F_at) <= 1e-5 * F_at
        ref = oracle.cg_plan(D, c.mlc, s, n, oracle.BBOptions(**TIGHT) if tight else None)
        if list(cps) == ref.cps:
            assert abs(F[i] - ref.F) <= (1e-4 if tight else 1e-2) * ref.F
        else:
            t = next(k for k, (a, b) in enumerate(zip(list(cps), ref.cps)) if a != b)
            assert near_tie_at(ddcs[i], c, D, t, cps[t], TIGHT if tight else None), \
                f"plan {i}: sequence differs at {t}: batch {list(cps)} oracle {ref.cps}"
        # the same plan alone through cg_plan
        F1, _, cps1, _, _, _ = gpu_plan(ddcs[i], c, n, TIGHT if tight else None)
        if list(cps1) == list(cps):
            assert abs(F1 - F[i]) <= (1e-4 if tight else 1e-2) * F1
    # a second run of the recorded graph reproduces the first bit for bit
    F2, stats2 = batch.run()
    assert F2 == F
    outs2 = _batch_outputs(batch, cases)
    for a, b in zip(outs, outs2):
        for u, v in zip(a, b):
            assert np.array_equal(u, v)


@pytest.mark.parametrize("tight", [False, True])
def test_batch_matches_oracle_and_single_plans(tight):
    from paper_1503_01721_gb300 import api
    cases = _cases()
    ddcs = [make_ddc(c) for c, _ in cases]
    voxs = [api.VoxelParams.from_numpy(c.structs) for c, _ in cases]
    opts = api.BBOptions(**TIGHT) if tight else None
    batch = api.Batch([(d.h, c.mlc, v, n) for d, v, (c, n) in zip(ddcs, voxs, cases)], opts)
    info = batch.info()
    assert info["n_plans"] == len(cases) and info["max_apertures"] == 20
    assert info["graph"] == 1 and info["graph_nodes"] > 0
    assert info["spmv_cfg"] in info["autotune_ms"]
    _check_batch(batch, ddcs, cases, tight)
    batch.close()


def test_batch_with_interdigitation_plans():
    """Plans with the interdigitation constraint (Section 2.2.2) mixed with plain ones
    in one batch: each priced by the row-chain program on its own, the others by the
    shared pricing launch, all in the same graph."""
    import dataclasses
    from paper_1503_01721_gb300 import api

    def interdig(c):
        return dataclasses.replace(c, mlc=dataclasses.replace(c.mlc, interdigitation=True))
    cases = [(interdig(synth.make_case("tiny", seed=0)), 3), (synth.make_case("cfg1", seed=0), 8),
             (interdig(synth.make_case("ragged", seed=0)), 4), (interdig(synth.make_case("cfg1", seed=2)), 10)]
    ddcs = [make_ddc(c) for c, _ in cases]
    voxs = [api.VoxelParams.from_numpy(c.structs) for c, _ in cases]
    batch = api.Batch([(d.h, c.mlc, v, n) for d, v, (c, n) in zip(ddcs, voxs, cases)], api.BBOptions(**TIGHT))
    assert batch.info()["graph"] == 1
    _check_batch(batch, ddcs, cases, True)
    batch.close()


def test_batch_stops_and_empty_plans():
    from paper_1503_01721_gb300 import api
    c = synth.make_case("tiny", seed=0)
    s = c.structs
    zero = synth.Structures(s.struct_id, np.zeros_like(s.T), s.w_over, s.w_under, s.names)
    ddc = make_ddc(c)
    v_ok = api.VoxelParams.from_numpy(s)
    v_zero = api.VoxelParams.from_numpy(zero)
    batch = api.Batch([(ddc.h, c.mlc, v_ok, 3), (ddc.h, c.mlc, v_zero, 3), (ddc.h, c.mlc, v_ok, 0)])
    F, st = batch.run()
    assert st[0]["n_apertures"] == 3 and st[0]["stop"] == "count"
    assert st[1]["n_apertures"] == 0 and st[1]["stop"] == "price" and F[1] == 0.0
    assert st[2]["n_apertures"] == 0 and st[2]["stop"] == "count"
    # no apertures: the dose is 0 and F is the objective of zero dose
    F0, _ = oracle.objective_grad(np.zeros(c.V), s.struct_id, s.T, s.w_over, s.w_under)
    assert abs(F[2] - F0) <= 1e-12 * F0
    # the one plan that ran matches cg_plan's F closely
    F1, _ = api.cg_plan(ddc.h, c.mlc, v_ok, 3)
    assert abs(F[0] - F1) <= 1e-2 * F1
    batch.close()


def test_batch_rejects_bad_input():
    from paper_1503_01721_gb300 import api, _lib
    c = synth.make_case("tiny", seed=0)
    v = api.VoxelParams.from_numpy(c.structs)
    a = make_ddc(c)
    b = make_ddc(c, dtype="bf16")
    with pytest.raises(_lib.VmatError) as e:
        api.Batch([(a.h, c.mlc, v, 2), (b.h, c.mlc, v, 2)])
    assert e.value.status == _lib.VMAT_EINVAL
    with pytest.raises(_lib.VmatError) as e:
        api.Batch([(a.h, c.mlc, v, c.mlc.K + 1)])
    assert e.value.status == _lib.VMAT_EINVAL
    with pytest.raises(_lib.VmatError):
        api.Batch([])
