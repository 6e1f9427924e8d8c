"""DDC truncation (the paper's method S1, Section 2.4): the plan is optimised on
a matrix truncated to a radius about each beamlet axis and its dose is then
evaluated on the full matrix.  The GPU plan on the truncated matrix follows the
oracle's, and its full-matrix dose and objective match the oracle's evaluation
of the same apertures and intensities."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import dev, host, make_ddc, require_cuda, spmv_bound
from test_gpu_cg import TIGHT, gpu_plan, near_tie_at

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()
    import __graft_entry__
    __graft_entry__.build()


def test_truncated_plan_evaluated_on_full_matrix():
    from paper_1503_01721_gb300 import api
    full = synth.make_case("cfg1", seed=0)
    tr = synth.make_truncated_case("cfg1", 1.25, seed=0)
    assert 0.2 < tr.nnz / full.nnz < 0.3
    n = 12
    d_tr = make_ddc(tr)
    d_full = make_ddc(full)
    Dt = oracle.ddc_matrix(tr.V, tr.J, tr.vox, tr.blt, tr.val)
    Df = oracle.ddc_matrix(full.V, full.J, full.vox, full.blt, full.val)
    s = tr.structs
    F_model, st, cps, lv, y, dose_model = gpu_plan(d_tr, tr, n, TIGHT)
    ref = oracle.cg_plan(Dt, tr.mlc, s, n, oracle.BBOptions(**TIGHT))
    if list(cps) == ref.cps:
        assert abs(F_model - ref.F) <= 1e-4 * ref.F
    else:
        t = next(i for i, (a, b) in enumerate(zip(list(cps), ref.cps)) if a != b)
        assert near_tie_at(d_tr, tr, Dt, t, cps[t], TIGHT)
    # the same apertures and intensities on the full matrix
    x = torch.empty(full.J, device="cuda")
    api.aperture_fluence(full.mlc, dev(cps, torch.int32), dev(lv, torch.int16), dev(y, torch.float32), x)
    dose_true = torch.empty(full.V, device="cuda")
    api.dose_forward(d_full.h, x, dose_true)
    F_true = torch.empty(1, dtype=torch.float64, device="cuda")
    vox = api.VoxelParams.from_numpy(s)
    api.objective_grad(dose_true, vox, None, F_true)
    x_ref = oracle.aperture_fluence(full.mlc, cps, lv, y)
    d_ref = oracle.dose_forward(Df, x_ref)
    lens = np.bincount(full.vox, minlength=full.V)
    assert np.all(np.abs(host(dose_true) - d_ref) <= spmv_bound(abs(Df) @ np.abs(x_ref), lens) + 1e-6 * np.abs(d_ref))
    F_ref, _ = oracle.objective_grad(d_ref, s.struct_id, s.T, s.w_over, s.w_under)
    assert abs(F_true.item() - F_ref) <= 1e-5 * F_ref
    # the dropped penumbra only adds dose: the full-matrix dose is never lower
    assert np.all(host(dose_true) >= dose_model - 1e-6 * np.max(dose_model))
