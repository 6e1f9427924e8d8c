"""Precision form: DDC values stored as BF16, or FP8 E4M3 with per-beamlet
power-of-two scales; FP32 accumulation.

Parity: a low-precision plan is the FP64 oracle's plan on the dequantised
matrix (the stored values read back as float64): same aperture sequence up to
near ties, objective within 1e-4.  The final dose is D_q (A y) in FP32 and
matches the FP64 product of the dequantised matrix to accumulation error; its
total error against the float32 matrix is bounded by the format's relative
precision (2^-8 for BF16, 2^-4 for E4M3).

Distance to the FP32 plan (the oracle on the float32 values): BF16 stays within
0.5%.  E4M3's 3-bit mantissa moves the plan objective by about 1% on the
40^3 case (the oracle alone, run on the dequantised matrix, gives +0.93%,
and +0.65% when its plan is scored on the float32 matrix); the test bounds it
by 1.5%.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import make_ddc, require_cuda, spmv_bound
from test_gpu_cg import TIGHT, gpu_plan, near_tie_at

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()
    import __graft_entry__
    __graft_entry__.build()


_REF = {}


def _oracle_plan(c, n, dtype):
    key = (c.name, n, dtype)
    if key not in _REF:
        v = c.val if dtype == "f32" else oracle.quantize_ddc(c.J, c.blt, c.val, dtype)[0]
        D = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, v)
        _REF[key] = (D, oracle.cg_plan(D, c.mlc, c.structs, n, oracle.BBOptions(**TIGHT)))
    return _REF[key]


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_low_precision_plan(dtype):
    c = synth.make_case("cfg1", seed=0)
    n = 20
    D, ref32 = _oracle_plan(c, n, "f32")
    Dq, refq = _oracle_plan(c, n, dtype)
    ddc = make_ddc(c, dtype=dtype)
    F, st, cps, lv, y, dose = gpu_plan(ddc, c, n, TIGHT)
    assert st["n_apertures"] == n
    # parity with the oracle on the dequantised matrix
    if list(cps) == refq.cps:
        assert abs(F - refq.F) <= 1e-4 * refq.F
    else:
        t = next(i for i, (a, b) in enumerate(zip(list(cps), refq.cps)) if a != b)
        assert near_tie_at(ddc, c, Dq, t, cps[t], TIGHT), \
            f"aperture sequence differs at step {t}: gpu {list(cps)} oracle {refq.cps}"
    # the stated distance to the FP32 plan
    assert abs(F - ref32.F) <= {"bf16": 5e-3, "fp8": 1.5e-2}[dtype] * ref32.F, \
        f"{dtype} plan F {F} vs FP32-matrix oracle {ref32.F}"
    # final dose: accumulation error on the stored values, and total error of the format
    x = oracle.aperture_fluence(c.mlc, cps, lv, y)
    d_q = oracle.dose_forward(Dq, x)
    lens = np.bincount(c.vox, minlength=c.V)
    assert np.all(np.abs(dose - d_q) <= spmv_bound(abs(Dq) @ np.abs(x), lens))
    d_ref = oracle.dose_forward(D, x)
    rel = np.max(np.abs(dose - d_ref)) / np.max(np.abs(d_ref))
    assert rel <= {"bf16": 2.0 ** -8, "fp8": 2.0 ** -4}[dtype]
