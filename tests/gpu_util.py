"""Helpers for the -m gpu parity tests (device marshalling and error bounds)."""
import numpy as np
import pytest
import torch

U32 = 2.0 ** -24  # float32 unit roundoff
# Depth of the float32 summation tree of one row in the tile SpMV: at most
# E (16) serial adds in a thread, log2(512) = 9 levels of the keyed scan, one add
# per spanned tile and the products' own rounding; 64 covers every row length
# in the tests with margin.
SPMV_C = 64


def require_cuda():
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")


def dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)


def host(t):
    return t.detach().cpu().numpy()


def spmv_bound(abs_terms_sum):
    """Componentwise float32 accumulation bound c * u * sum_i |a_i b_i|."""
    return SPMV_C * U32 * abs_terms_sum + 1e-37


def make_ddc(case_or_coo, dtype="f32", tile_cfg=-1, V=None, J=None):
    from paper_1503_01721_gb300 import api
    if hasattr(case_or_coo, "vox"):
        c = case_or_coo
        V, J, vox, blt, val = c.V, c.J, c.vox, c.blt, c.val
    else:
        vox, blt, val = case_or_coo
    return api.Ddc(V, J, dev(vox, torch.int32), dev(blt, torch.int32), dev(val, torch.float32), dtype=dtype,
                   tile_cfg=tile_cfg)
