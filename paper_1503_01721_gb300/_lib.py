"""ctypes view of libvmat's C ABI (include/vmat.h): structs, signatures, loader.

Loading fails loudly when libvmat.so has not been built; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvmat.so")

c_i32, c_i64, c_f64, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p

VMAT_OK, VMAT_EINVAL, VMAT_ENOMEM, VMAT_ECUDA, VMAT_ESTATE, VMAT_ETIMEOUT, VMAT_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
DTYPES = {"f32": 0, "bf16": 1, "fp8": 2}
STOP_NAMES = {1: "rel", 2: "step", 3: "maxit", 4: "grad0", 5: "flat", 10: "price", 11: "count"}


class Machine(ctypes.Structure):
    _fields_ = [("cp_step_deg", c_f64), ("speed_min", c_f64), ("speed_max", c_f64), ("speed_step_max", c_f64),
                ("rate_min", c_f64), ("rate_max", c_f64), ("leaf_speed_cols", c_f64)]


class Mlc(ctypes.Structure):
    _fields_ = [("K", c_i32), ("n_rows", c_i32), ("n_cols", c_i32), ("n_arcs", c_i32),
                ("arc_first_cp", ctypes.POINTER(c_i32)), ("travel_cols", c_i32), ("interdigitation", c_i32),
                ("machine", ctypes.POINTER(Machine))]


class Voxels(ctypes.Structure):
    _fields_ = [("struct_id", c_vp), ("n_struct", c_i32), ("T", c_vp), ("w_over", c_vp), ("w_under", c_vp)]


class BuildOpts(ctypes.Structure):
    _fields_ = [("dtype", c_i32), ("build_D", c_i32), ("build_Dt", c_i32), ("tile_cfg", c_i32),
                ("autotune", c_i32), ("keep_coo", c_i32), ("index16", c_i32), ("tile_cfg_Dt", c_i32),
                ("refine_f32", c_i32), ("vox_grid", c_i32 * 3)]


class BBOpts(ctypes.Structure):
    _fields_ = [("max_iter", c_i32), ("rel_tol5", c_f64), ("step_tol", c_f64), ("delta_min", c_f64),
                ("delta_max", c_f64)]


class BBReport(ctypes.Structure):
    _fields_ = [("iters", c_i32), ("stop_reason", c_i32), ("F", c_f64)]


class DdcInfo(ctypes.Structure):
    _fields_ = [("V", c_i32), ("J", c_i32), ("nnz", c_i64), ("n_active_vox", c_i32), ("dtype", c_i32),
                ("built_D", c_i32), ("built_Dt", c_i32), ("tile_nnz_D", c_i32), ("tile_nnz_Dt", c_i32),
                ("bytes_D", c_i64), ("bytes_Dt", c_i64), ("build_ms", c_f64), ("cfg_D", c_i32), ("cfg_Dt", c_i32),
                ("index16_D", c_i32), ("index16_Dt", c_i32), ("bytes16_D", c_i64), ("bytes16_Dt", c_i64),
                ("refine_f32", c_i32), ("vox_brick", c_i32)]


class PlanStats(ctypes.Structure):
    _fields_ = [("t_total_ms", c_f64), ("t_pp1_ms", c_f64), ("t_pp2_ms", c_f64), ("t_da_ms", c_f64),
                ("t_mp_ms", c_f64), ("t_final_ms", c_f64), ("pp1_spmv_ms", c_f64), ("pp1_spmv_launches", c_i64),
                ("pp1_spmv_bytes", c_f64), ("other_spmv_bytes", c_f64), ("n_apertures", c_i32),
                ("bb_iters_total", c_i32), ("stop_reason", c_i32), ("kernel_launches", c_i64),
                ("pp1_full_bytes", c_f64), ("refined", c_i32), ("refine_bb_iters", c_i32), ("t_refine_ms", c_f64),
                ("F_before_refine", c_f64), ("mp_bytes", c_f64), ("pp1_spmv_cfg", c_i32)]


class PlanDesc(ctypes.Structure):
    _fields_ = [("ddc", c_vp), ("mlc", ctypes.POINTER(Mlc)), ("vox", ctypes.POINTER(Voxels)), ("n_apertures", c_i32)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("n_plans", c_i32), ("max_apertures", c_i32), ("spmv_cfg", c_i32), ("graph", c_i32),
                ("graph_nodes", c_i64), ("device_bytes", c_i64), ("autotune_ms", c_f64 * 32)]


# name -> (restype, argtypes); every entry point declared in include/vmat.h
SIGNATURES = {
    "ddc_load_coo": (c_i32, [c_i32, c_i32, c_i64, c_vp, c_vp, c_vp, c_i32, c_vp, ctypes.POINTER(c_vp)]),
    "ddc_build": (c_i32, [c_vp, ctypes.POINTER(BuildOpts), c_vp]),
    "ddc_free": (c_i32, [c_vp]),
    "ddc_info": (c_i32, [c_vp, ctypes.POINTER(DdcInfo)]),
    "dose_forward": (c_i32, [c_vp, c_vp, c_vp, c_vp]),
    "beamlet_price": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_i32, c_vp]),
    "beamlet_price_windowed": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "objective_grad": (c_i32, [c_i32, c_vp, ctypes.POINTER(Voxels), c_vp, c_vp, c_vp]),
    "price_apertures": (c_i32, [ctypes.POINTER(Mlc), c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "price_apertures_noalloc": (c_i32, [ctypes.POINTER(Mlc), c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "aperture_dose": (c_i32, [c_vp, ctypes.POINTER(Mlc), c_i32, c_vp, c_vp, c_vp]),
    "aperture_fluence": (c_i32, [ctypes.POINTER(Mlc), c_i32, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "aperture_grad": (c_i32, [ctypes.POINTER(Mlc), c_i32, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "fluence_bounds": (c_i32, [ctypes.POINTER(Mlc), c_i32, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "mp_bb_solve": (c_i32, [c_vp, c_i32, c_i32, c_i64, ctypes.POINTER(Voxels), c_vp, c_vp, c_vp, c_vp,
                            ctypes.POINTER(BBOpts), ctypes.POINTER(BBReport), c_vp]),
    "cg_plan": (c_i32, [c_vp, ctypes.POINTER(Mlc), ctypes.POINTER(Voxels), c_i32, ctypes.POINTER(BBOpts),
                        c_vp, c_vp, c_vp, c_vp, ctypes.POINTER(c_f64), ctypes.POINTER(PlanStats), c_vp]),
    "vmat_batch_create": (c_i32, [c_i32, ctypes.POINTER(PlanDesc), ctypes.POINTER(BBOpts), c_vp,
                                  ctypes.POINTER(c_vp)]),
    "vmat_batch_run": (c_i32, [c_vp, ctypes.POINTER(c_f64), ctypes.POINTER(PlanStats), c_vp]),
    "vmat_batch_result": (c_i32, [c_vp, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "vmat_batch_info_get": (c_i32, [c_vp, ctypes.POINTER(BatchInfo)]),
    "vmat_batch_free": (c_i32, [c_vp]),
    "vmat_last_error": (ctypes.c_char_p, []),
    "vmat_device_status": (c_i32, [c_i32]),
    "vmat_version": (ctypes.c_char_p, []),
    "vmat_launch_count": (c_i64, []),
    "vmat_spmv_config_count": (c_i32, []),
}

_lock = threading.Lock()
_lib = None


class VmatError(RuntimeError):
    def __init__(self, fn: str, status: int, msg: str):
        super().__init__(f"{fn} failed with status {status}: {msg}")
        self.status = status


def load() -> ctypes.CDLL:
    """Load libvmat.so once.  Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is not built: run __graft_entry__.build() "
                                   "(nvcc for sm_103a); there is no CPU fallback")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def check(fn: str, status: int) -> None:
    if status != VMAT_OK:
        raise VmatError(fn, status, load().vmat_last_error().decode(errors="replace"))
