"""Helpers for the -m gpu parity tests (device marshalling and error bounds)."""
import numpy as np
import pytest
import torch

U32 = 2.0 ** -24  # float32 unit roundoff
# Depth of the float32 summation of one row of n entries: the tile kernel adds
# at most E (16) serially in a thread, log2(512) = 9 levels of keyed scan and one
# add per spanned tile; the warp-per-row kernel adds n/128 per accumulator, 2
# levels to join the 4 accumulators and 5 butterfly levels.  (64 + n/64) units
# of roundoff bound both, for every row length.
SPMV_C = 64
# SpMV configurations the library offers (tile_cfg 0 .. N_SPMV_CFG - 1)
N_SPMV_CFG = 15
# configurations that read the 16-bit column index, and their consecutive-lane twins (same products,
# same order)
INDEX16_TWIN = {12: 9, 13: 10, 14: 11}


def require_cuda():
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")


def dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)


def host(t):
    return t.detach().cpu().numpy()


def spmv_bound(abs_terms_sum, row_len=0):
    """Componentwise float32 accumulation bound (64 + n/64) * u * sum_i |a_i b_i|."""
    return (SPMV_C + np.asarray(row_len, np.float64) / 64.0) * U32 * abs_terms_sum + 1e-37


def make_ddc(case_or_coo, dtype="f32", tile_cfg=-1, V=None, J=None, index16=None, refine=False, brick=False):
    """index16 None: build the 16-bit column index when tile_cfg reads it.  brick: CSR(D^T)
    columns in brick order (a case's own grid)."""
    from paper_1503_01721_gb300 import api
    if hasattr(case_or_coo, "vox"):
        c = case_or_coo
        V, J, vox, blt, val = c.V, c.J, c.vox, c.blt, c.val
    else:
        vox, blt, val = case_or_coo
    if index16 is None:
        index16 = tile_cfg in INDEX16_TWIN
    grid = None
    if brick:
        g = case_or_coo.geom
        grid = (g.nx, g.ny, g.nz)
    return api.Ddc(V, J, dev(vox, torch.int32), dev(blt, torch.int32), dev(val, torch.float32), dtype=dtype,
                   tile_cfg=tile_cfg, index16=index16, refine=refine, vox_grid=grid)
