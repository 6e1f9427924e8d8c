"""Python binding of libvmat with the C ABI's names (argument marshalling only).

Every array argument is a torch tensor on the current CUDA device (the COO
input of ``ddc_load_coo`` may also be on the host).  Work runs in libvmat's
kernels on the current torch stream unless ``stream`` is given.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import check

_DT = {torch.float32: "float32", torch.int32: "int32", torch.int16: "int16", torch.uint8: "uint8",
       torch.float64: "float64"}


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t, dtype, n=None, name="tensor", device=True, allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if device and not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if n is not None and t.numel() < n:
        raise ValueError(f"{name} has {t.numel()} elements, needs {n}")
    return ctypes.c_void_p(t.data_ptr())


@dataclass
class VoxelParams:
    """Eq. 1 parameters on the device: structure label per voxel and per-structure T, w+, w-."""
    struct_id: torch.Tensor  # uint8 [V]
    T: torch.Tensor          # float32 [n_struct]
    w_over: torch.Tensor
    w_under: torch.Tensor

    @classmethod
    def from_numpy(cls, s, device="cuda"):
        f = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(device=device, dtype=dt)
        return cls(f(s.struct_id, torch.uint8), f(s.T, torch.float32), f(s.w_over, torch.float32),
                   f(s.w_under, torch.float32))

    def c(self) -> _lib.Voxels:
        n = self.T.numel()
        for name in ("T", "w_over", "w_under"):
            _ptr(getattr(self, name), torch.float32, n, name)
        return _lib.Voxels(_ptr(self.struct_id, torch.uint8, None, "struct_id").value, n,
                           self.T.data_ptr(), self.w_over.data_ptr(), self.w_under.data_ptr())


class _MlcC:
    """Holds the ctypes MLC struct, its host arc array and machine limits alive for a call."""

    def __init__(self, mlc):
        arcs = np.ascontiguousarray(np.asarray(mlc.arc_first_cp, np.int32))
        self._arcs = (ctypes.c_int32 * len(arcs))(*arcs.tolist())
        m = getattr(mlc, "machine", None)
        self._machine = None if m is None else _lib.Machine(
            float(m.cp_step_deg), float(m.speed_min), float(m.speed_max), float(m.speed_step_max),
            float(m.rate_min), float(m.rate_max), float(m.leaf_speed_cols))
        self.s = _lib.Mlc(int(mlc.K), int(mlc.n_rows), int(mlc.n_cols), len(arcs),
                          ctypes.cast(self._arcs, ctypes.POINTER(ctypes.c_int32)), int(mlc.travel_cols),
                          int(bool(getattr(mlc, "interdigitation", False))),
                          ctypes.pointer(self._machine) if self._machine is not None else None)


def _bb_opts(opts):
    if opts is None:
        return None
    return _lib.BBOpts(int(opts.max_iter), float(opts.rel_tol5), float(opts.step_tol), float(opts.delta_min),
                       float(opts.delta_max))


@dataclass
class BBOptions:
    max_iter: int = 500
    rel_tol5: float = 1e-6
    step_tol: float = 1e-9
    delta_min: float = 1e-12
    delta_max: float = 1e12


# ---------------------------------------------------------------------------- DDC matrix

def ddc_load_coo(V: int, J: int, vox: torch.Tensor, blt: torch.Tensor, val: torch.Tensor, stream=None) -> int:
    """Copy a COO DDC (host or device tensors) into a new library handle."""
    nnz = val.numel()
    on_dev = val.is_cuda
    for t, dt, nm in ((vox, torch.int32, "vox"), (blt, torch.int32, "blt"), (val, torch.float32, "val")):
        _ptr(t, dt, nnz, nm, device=on_dev)
        if t.is_cuda != on_dev:
            raise ValueError("vox, blt and val must all be on the host or all on the device")
    h = ctypes.c_void_p()
    check("ddc_load_coo", _lib.load().ddc_load_coo(int(V), int(J), int(nnz), vox.data_ptr(), blt.data_ptr(),
                                                    val.data_ptr(), int(on_dev), _stream(stream), ctypes.byref(h)))
    return h.value


def ddc_build(h: int, dtype: str = "f32", build_D: bool = True, build_Dt: bool = True, tile_cfg: int = -1,
              autotune: bool = False, keep_coo: bool = False, stream=None, index16: bool = False,
              tile_cfg_Dt: int = -1, refine: bool = False, vox_grid=None) -> None:
    """Build CSR(D) / CSR(D^T); index16 also stores 16-bit chunk-relative column indices where they fit.
    tile_cfg sets the SpMV configuration of CSR(D) (and of CSR(D^T) unless tile_cfg_Dt >= 0).
    refine (BF16 / FP8): keep CSR(D)'s FP32 values too, for cg_plan's FP32 refinement.
    vox_grid (nx, ny, nz), voxel i = (z ny + y) nx + x: CSR(D^T) columns in 4x4x2 brick order."""
    grid = (0, 0, 0) if vox_grid is None else tuple(int(v) for v in vox_grid)
    o = _lib.BuildOpts(_lib.DTYPES[dtype], int(build_D), int(build_Dt), int(tile_cfg), int(autotune), int(keep_coo),
                       int(index16), int(tile_cfg_Dt), int(refine), (ctypes.c_int32 * 3)(*grid))
    check("ddc_build", _lib.load().ddc_build(ctypes.c_void_p(h), ctypes.byref(o), _stream(stream)))


def ddc_free(h: int) -> None:
    check("ddc_free", _lib.load().ddc_free(ctypes.c_void_p(h)))


def ddc_info(h: int) -> dict:
    info = _lib.DdcInfo()
    check("ddc_info", _lib.load().ddc_info(ctypes.c_void_p(h), ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in info._fields_}


# ---------------------------------------------------------------------------- products

def dose_forward(h: int, x: torch.Tensor, d: torch.Tensor, stream=None) -> None:
    """d = D x (Section 2.1)."""
    check("dose_forward", _lib.load().dose_forward(ctypes.c_void_p(h), _ptr(x, torch.float32, None, "x"),
                                                   _ptr(d, torch.float32, None, "d"), _stream(stream)))


def beamlet_price(h: int, g: torch.Tensor, pi: torch.Tensor, cp_active: torch.Tensor | None = None,
                  beamlets_per_cp: int = 0, stream=None) -> None:
    """pi = D^T g (Eq. 3), optionally only for CPs with cp_active != 0."""
    check("beamlet_price", _lib.load().beamlet_price(
        ctypes.c_void_p(h), _ptr(g, torch.float32, None, "g"), _ptr(pi, torch.float32, None, "pi"),
        _ptr(cp_active, torch.uint8, None, "cp_active", allow_none=True), int(beamlets_per_cp), _stream(stream)))


def beamlet_price_windowed(h: int, mlc, occupied: torch.Tensor, leaves: torch.Tensor, g: torch.Tensor,
                           pi: torch.Tensor, stream=None) -> None:
    """pi = D^T g (Eq. 3) on the beamlets inside the leaf-travel windows of the
    unoccupied CPs (the entries price_apertures reads); other entries unspecified."""
    m = _MlcC(mlc)
    check("beamlet_price_windowed", _lib.load().beamlet_price_windowed(
        ctypes.c_void_p(h), ctypes.byref(m.s), _ptr(occupied, torch.uint8, mlc.K, "occupied"),
        _ptr(leaves, torch.int16, mlc.K * mlc.n_rows * 2, "leaves"), _ptr(g, torch.float32, None, "g"),
        _ptr(pi, torch.float32, None, "pi"), _stream(stream)))


def objective_grad(z: torch.Tensor, vox: VoxelParams, g: torch.Tensor | None = None,
                   F: torch.Tensor | None = None, stream=None) -> None:
    """F(z) (Eq. 1) into F (float64 [1]) and g = -grad F (Eq. 4) into g."""
    vc = vox.c()
    check("objective_grad", _lib.load().objective_grad(
        z.numel(), _ptr(z, torch.float32, None, "z"), ctypes.byref(vc), _ptr(g, torch.float32, z.numel(), "g", allow_none=True),
        _ptr(F, torch.float64, 1, "F", allow_none=True), _stream(stream)))


def price_apertures(mlc, pi, occupied, leaves, best_cp, best_leaves, best_price, stream=None) -> None:
    """Best opening per MLC row and best CP (Section 2.2.2)."""
    m = _MlcC(mlc)
    check("price_apertures", _lib.load().price_apertures(
        ctypes.byref(m.s), _ptr(pi, torch.float32, None, "pi"), _ptr(occupied, torch.uint8, mlc.K, "occupied"),
        _ptr(leaves, torch.int16, mlc.K * mlc.n_rows * 2, "leaves"), _ptr(best_cp, torch.int32, 1, "best_cp"),
        _ptr(best_leaves, torch.int16, mlc.n_rows * 2, "best_leaves"),
        _ptr(best_price, torch.float64, 1, "best_price"), _stream(stream)))


def aperture_dose(h: int, mlc, cp: int, leaves: torch.Tensor, da: torch.Tensor, stream=None) -> None:
    """DA of one aperture (Eq. 5)."""
    m = _MlcC(mlc)
    check("aperture_dose", _lib.load().aperture_dose(
        ctypes.c_void_p(h), ctypes.byref(m.s), int(cp), _ptr(leaves, torch.int16, mlc.n_rows * 2, "leaves"),
        _ptr(da, torch.float32, None, "da"), _stream(stream)))


def aperture_fluence(mlc, cps, leaves, y, x, stream=None) -> None:
    """x = A y."""
    m = _MlcC(mlc)
    n = cps.numel()
    check("aperture_fluence", _lib.load().aperture_fluence(
        ctypes.byref(m.s), n, _ptr(cps, torch.int32, n, "cps"), _ptr(leaves, torch.int16, n * mlc.n_rows * 2, "leaves"),
        _ptr(y, torch.float32, n, "y"), _ptr(x, torch.float32, None, "x"), _stream(stream)))


def aperture_grad(mlc, cps, leaves, pi, gy, stream=None) -> None:
    """gy = A^T pi."""
    m = _MlcC(mlc)
    n = cps.numel()
    check("aperture_grad", _lib.load().aperture_grad(
        ctypes.byref(m.s), n, _ptr(cps, torch.int32, n, "cps"), _ptr(leaves, torch.int16, n * mlc.n_rows * 2, "leaves"),
        _ptr(pi, torch.float32, None, "pi"), _ptr(gy, torch.float32, n, "gy"), _stream(stream)))


def fluence_bounds(mlc, cps: torch.Tensor, leaves: torch.Tensor, lo: torch.Tensor, hi: torch.Tensor,
                   stream=None) -> None:
    """Fluence-rate bounds of Eq. 6 from the delivery limits of Eq. 2 (``mlc.machine``)
    for the placed apertures (cps < 0: slots not placed)."""
    m = _MlcC(mlc)
    n = cps.numel()
    check("fluence_bounds", _lib.load().fluence_bounds(
        ctypes.byref(m.s), n, _ptr(cps, torch.int32, n, "cps"), _ptr(leaves, torch.int16, n * mlc.n_rows * 2, "leaves"),
        _ptr(lo, torch.float32, n, "lo"), _ptr(hi, torch.float32, n, "hi"), _stream(stream)))


def mp_bb_solve(DA: torch.Tensor, vox: VoxelParams, y: torch.Tensor, z: torch.Tensor, lo=None, hi=None,
                opts: BBOptions | None = None, stream=None) -> dict:
    """Master problem (Eq. 6-10).  DA: float32 [n_ap, ld] (row n = aperture n's dose vector over V voxels)."""
    n_ap, ld = DA.shape
    V = z.numel()
    vc = vox.c()
    o = _bb_opts(opts)
    rep = _lib.BBReport()
    check("mp_bb_solve", _lib.load().mp_bb_solve(
        _ptr(DA, torch.float32, None, "DA"), V, n_ap, ld, ctypes.byref(vc),
        _ptr(lo, torch.float32, n_ap, "lo", allow_none=True), _ptr(hi, torch.float32, n_ap, "hi", allow_none=True),
        _ptr(y, torch.float32, n_ap, "y"), _ptr(z, torch.float32, V, "z"),
        ctypes.byref(o) if o is not None else None, ctypes.byref(rep), _stream(stream)))
    return {"iters": rep.iters, "stop": _lib.STOP_NAMES.get(rep.stop_reason, rep.stop_reason), "F": rep.F}


def cg_plan(h: int, mlc, vox: VoxelParams, n_apertures: int, opts: BBOptions | None = None, cps_out=None,
            leaves_out=None, y_out=None, dose_out=None, stream=None):
    """Column generation (Section 2.1).  Outputs may be host or device tensors.  Returns (F, stats)."""
    m = _MlcC(mlc)
    vc = vox.c()
    o = _bb_opts(opts)
    F = ctypes.c_double()
    st = _lib.PlanStats()

    def anyp(t, dt, n, name):
        return None if t is None else _ptr(t, dt, n, name, device=False)
    check("cg_plan", _lib.load().cg_plan(
        ctypes.c_void_p(h), ctypes.byref(m.s), ctypes.byref(vc), int(n_apertures),
        ctypes.byref(o) if o is not None else None,
        anyp(cps_out, torch.int32, n_apertures, "cps_out"),
        anyp(leaves_out, torch.int16, n_apertures * mlc.n_rows * 2, "leaves_out"),
        anyp(y_out, torch.float32, n_apertures, "y_out"), anyp(dose_out, torch.float32, None, "dose_out"),
        ctypes.byref(F), ctypes.byref(st), _stream(stream)))
    stats = {f: getattr(st, f) for f, _ in st._fields_}
    stats["stop"] = _lib.STOP_NAMES.get(stats["stop_reason"], stats["stop_reason"])
    return F.value, stats


class Batch:
    """Independent plans advanced together (vmat_batch_*): one CUDA graph per run.

    ``plans`` is a list of (ddc_handle, mlc, VoxelParams, n_apertures).  The
    handles, MLC arrays and voxel tensors must outlive the batch.
    """

    def __init__(self, plans, opts: BBOptions | None = None, stream=None):
        self._keep = []
        descs = (_lib.PlanDesc * len(plans))()
        for i, (h, mlc, vox, n_ap) in enumerate(plans):
            m = _MlcC(mlc)
            vc = vox.c()
            self._keep += [m, vc, vox]
            descs[i] = _lib.PlanDesc(ctypes.c_void_p(h), ctypes.pointer(m.s), ctypes.pointer(vc), int(n_ap))
        self._descs = descs
        self.n = len(plans)
        self._V = [int(v.struct_id.numel()) for _, _, v, _ in plans]
        self._ap = [int(p[3]) for p in plans]
        self._rows = [int(p[1].n_rows) for p in plans]
        o = _bb_opts(opts)
        hb = ctypes.c_void_p()
        check("vmat_batch_create", _lib.load().vmat_batch_create(
            len(plans), descs, ctypes.byref(o) if o is not None else None, _stream(stream), ctypes.byref(hb)))
        self.h = hb.value

    def run(self, stream=None):
        """Run every plan once; returns (F list, stats list)."""
        F = (ctypes.c_double * self.n)()
        st = (_lib.PlanStats * self.n)()
        check("vmat_batch_run", _lib.load().vmat_batch_run(ctypes.c_void_p(self.h), F, st, _stream(stream)))
        stats = []
        for i in range(self.n):
            d = {f: getattr(st[i], f) for f, _ in st[i]._fields_}
            d["stop"] = _lib.STOP_NAMES.get(d["stop_reason"], d["stop_reason"])
            stats.append(d)
        return list(F), stats

    def result(self, i: int, cps_out=None, leaves_out=None, y_out=None, dose_out=None, stream=None):
        n, nr, V = self._ap[i], self._rows[i], self._V[i]

        def anyp(t, dt, k, name):
            return None if t is None else _ptr(t, dt, k, name, device=False)
        check("vmat_batch_result", _lib.load().vmat_batch_result(
            ctypes.c_void_p(self.h), int(i), anyp(cps_out, torch.int32, n, "cps_out"),
            anyp(leaves_out, torch.int16, n * nr * 2, "leaves_out"), anyp(y_out, torch.float32, n, "y_out"),
            anyp(dose_out, torch.float32, V, "dose_out"), _stream(stream)))

    def info(self) -> dict:
        inf = _lib.BatchInfo()
        check("vmat_batch_info_get", _lib.load().vmat_batch_info_get(ctypes.c_void_p(self.h), ctypes.byref(inf)))
        d = {f: getattr(inf, f) for f, _ in inf._fields_ if f != "autotune_ms"}
        d["autotune_ms"] = {c: inf.autotune_ms[c] for c in range(16) if inf.autotune_ms[c] > 0}
        return d

    def close(self):
        if getattr(self, "h", None):
            _lib.load().vmat_batch_free(ctypes.c_void_p(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def device_status(reset: bool = False) -> int:
    return int(_lib.load().vmat_device_status(int(reset)))


def launch_count() -> int:
    """Kernels libvmat has launched in this process."""
    return int(_lib.load().vmat_launch_count())


def spmv_config_count() -> int:
    """Number of SpMV configurations (tile_cfg values 0 .. count - 1)."""
    return int(_lib.load().vmat_spmv_config_count())


def version() -> str:
    return _lib.load().vmat_version().decode()


class Ddc:
    """Owning wrapper of a DDC handle (frees it when garbage-collected)."""

    def __init__(self, V, J, vox, blt, val, dtype="f32", build_D=True, build_Dt=True, tile_cfg=-1,
                 autotune=False, stream=None, index16=False, tile_cfg_Dt=-1, refine=False, vox_grid=None):
        self.V, self.J = int(V), int(J)
        self.h = ddc_load_coo(V, J, vox, blt, val, stream)
        try:
            ddc_build(self.h, dtype, build_D, build_Dt, tile_cfg, autotune, False, stream, index16, tile_cfg_Dt,
                      refine, vox_grid)
        except Exception:
            ddc_free(self.h)
            self.h = None
            raise
        self.dtype = dtype

    def info(self):
        return ddc_info(self.h)

    def close(self):
        if getattr(self, "h", None):
            ddc_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
