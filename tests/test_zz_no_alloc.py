"""price_apertures_noalloc, the pricing call for callers that cannot allocate
device memory while they plan (e.g. a service whose GPU memory all belongs to
its own pool), returns exactly what price_apertures returns.

Both are called through the C ABI on the same inputs, twice in a row with
different inputs, so the second call also shows that the fixed scratch array
left over from the first call does not leak into the result.  Pricing results
are compared bit for bit with price_apertures and with the oracle's pricing, as
in the other pricing tests, for the unconstrained search and for the
interdigitation chain (whose scratch layout in the fixed array differs).  The
stream-ordered pool the library allocates its scratch from shows no use during
an allocation-free call (and does show it during price_apertures).  This file
sorts last so that a run stopping at its first failure has run every other test.
"""
import ctypes
import ctypes.util

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1503_01721_gb300 import _lib
    return _lib.load()


class PoolWatch:
    """High-water mark of the current device's stream-ordered memory pool, the pool
    cudaMallocAsync draws from (CUDA driver API through ctypes)."""
    USED_MEM_HIGH = 8  # CU_MEMPOOL_ATTR_USED_MEM_HIGH

    def __init__(self):
        self.cu = ctypes.CDLL(ctypes.util.find_library("cuda") or "libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetMemPool(ctypes.byref(self.pool), dev) == 0

    def reset(self):
        zero = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH, ctypes.byref(zero)) == 0

    def high(self):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, self.USED_MEM_HIGH, ctypes.byref(v)) == 0
        return v.value


def c_mlc(mlc):
    from paper_1503_01721_gb300 import _lib
    arcs = (ctypes.c_int32 * len(mlc.arc_first_cp))(*[int(a) for a in mlc.arc_first_cp])
    m = _lib.Mlc(mlc.K, mlc.n_rows, mlc.n_cols, len(arcs), ctypes.cast(arcs, ctypes.POINTER(ctypes.c_int32)),
                 mlc.travel_cols, int(mlc.interdigitation))
    return m, arcs


def call(lib, fn, mlc, pi, occupied, leaves, watch=None):
    from paper_1503_01721_gb300 import _lib
    m, keep = c_mlc(mlc)
    bk = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    bl = torch.full((mlc.n_rows * 2,), -7, dtype=torch.int16, device="cuda")
    bp = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    if watch:
        watch.reset()
    st = getattr(lib, fn)(ctypes.byref(m), pi.data_ptr(), occupied.data_ptr(), leaves.data_ptr(), bk.data_ptr(),
                          bl.data_ptr(), bp.data_ptr(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    _lib.check(fn, st)
    torch.cuda.synchronize()
    used = watch.high() if watch else None
    return (int(bk.item()), bl.cpu().numpy().copy(), bp.cpu().numpy().view(np.uint64)[0]), used


def inputs(mlc, seed):
    rng = np.random.default_rng(seed)
    pi = (rng.normal(size=mlc.K * mlc.n_rows * mlc.n_cols) * 10.0).astype(np.float32)
    pi[rng.random(pi.size) < 0.3] = 0.0
    occupied = (rng.random(mlc.K) < 0.3).astype(np.uint8)
    leaves = np.sort(rng.integers(0, mlc.n_cols + 1, size=(mlc.K, mlc.n_rows, 2)), axis=2).astype(np.int16)
    return pi, occupied, leaves


def on_device(pi, occupied, leaves):
    d = lambda a, dt: torch.as_tensor(a).to("cuda", dt).contiguous()
    return d(pi, torch.float32), d(occupied, torch.uint8), d(leaves, torch.int16)


CASES = (
    # the H&N-like geometry (180 CPs x 64 rows, within the row limit), then a smaller one
    (synth.MLC(180, 64, 64, np.array([0], np.int32), 3), 1),
    (synth.MLC(36, 20, 20, np.array([0, 18], np.int32), 2), 2),
    # the interdigitation chain: 36 x 20 x 20 needs about 756 KB of the fixed array
    (synth.MLC(36, 20, 20, np.array([0], np.int32), 3, interdigitation=True), 3),
)


def test_noalloc_matches_price_apertures_and_oracle_on_consecutive_calls(lib):
    watch = PoolWatch()
    for mlc, seed in CASES:
        pi, occupied, leaves = inputs(mlc, seed)
        args = on_device(pi, occupied, leaves)
        want, used_alloc = call(lib, "price_apertures", mlc, *args, watch=watch)
        got, used_noalloc = call(lib, "price_apertures_noalloc", mlc, *args, watch=watch)
        assert used_alloc > 0        # the probe sees the allocating call's scratch
        assert used_noalloc == 0     # and nothing during the allocation-free call
        assert want[0] >= 0
        assert got[0] == want[0]
        assert np.array_equal(got[1], want[1])
        assert got[2] == want[2]
        k_ref, lv_ref, p_ref = oracle.price_apertures(mlc, pi, occupied, leaves.astype(np.int64))
        assert got[0] == k_ref
        assert np.array_equal(got[1].reshape(-1, 2), np.asarray(lv_ref))
        assert got[2] == np.float64(p_ref).view(np.uint64)


def test_noalloc_rejects_sizes_beyond_its_limit(lib):
    from paper_1503_01721_gb300 import _lib
    dummy = torch.zeros(16, device="cuda")
    for mlc in (synth.MLC(1025, 64, 8, np.array([0], np.int32), 3),   # 65,600 rows > 65,536
                # within the row limit, but the chain search's tables need about 99 MB
                synth.MLC(180, 64, 64, np.array([0], np.int32), 3, interdigitation=True)):
        m, keep = c_mlc(mlc)
        st = lib.price_apertures_noalloc(ctypes.byref(m), dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(),
                                         dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), None)
        assert st == _lib.VMAT_EINVAL
        assert b"limit" in lib.vmat_last_error()
