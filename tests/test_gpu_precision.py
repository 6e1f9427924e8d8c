"""Precision form: DDC values stored as BF16, or FP8 E4M3 with per-beamlet
power-of-two scales, FP32 accumulation, FP64 step lengths and objective.

The plan objective of the lower-precision DDC must stay within 0.5% of the
FP64 oracle's plan on the float32 matrix, and the final dose (recomputed in
FP32 from the stored values) is reported against both the FP64 oracle on the
float32 values (total error) and on the dequantised values (accumulation only).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import host, make_ddc, require_cuda, spmv_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_low_precision_plan_objective(dtype):
    from paper_1503_01721_gb300 import api
    c = synth.make_case("cfg1", seed=0)
    n = 20
    ddc = make_ddc(c, dtype=dtype)
    vox = api.VoxelParams.from_numpy(c.structs)
    cps = torch.empty(n, dtype=torch.int32)
    lv = torch.empty(n * c.mlc.n_rows * 2, dtype=torch.int16)
    y = torch.empty(n, dtype=torch.float32)
    dose = torch.empty(c.V, device="cuda")
    F, st = api.cg_plan(ddc.h, c.mlc, vox, n, cps_out=cps, leaves_out=lv, y_out=y, dose_out=dose)
    m = st["n_apertures"]
    D = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, c.val)
    ref = oracle.cg_plan(D, c.mlc, c.structs, n)
    assert abs(F - ref.F) <= 5e-3 * ref.F, f"{dtype} plan F {F} vs FP64 oracle {ref.F}"
    # the final dose is D_q (A y) in FP32: exact to accumulation error on the stored values
    x = oracle.aperture_fluence(c.mlc, cps.numpy()[:m], lv.numpy().reshape(n, -1, 2)[:m], y.numpy()[:m])
    vq, _ = oracle.quantize_ddc(c.J, c.blt, c.val, dtype)
    Dq = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, vq)
    d_q = oracle.dose_forward(Dq, x)
    lens = np.bincount(c.vox, minlength=c.V)
    assert np.all(np.abs(host(dose) - d_q) <= spmv_bound(abs(Dq) @ np.abs(x), lens))
    # total error of the stored format against the float32 matrix
    d_ref = oracle.dose_forward(D, x)
    rel = np.max(np.abs(host(dose) - d_ref)) / np.max(np.abs(d_ref))
    assert rel <= {"bf16": 2.0 ** -8, "fp8": 2.0 ** -4}[dtype] + 1e-5
