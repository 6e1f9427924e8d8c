"""The C ABI library loads on any host and exports every entry point that
include/vmat.h declares; host-side argument checks reject bad calls before any
CUDA work (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vmat.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1503_01721_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_header_parses():
    names = declared_functions()
    for must in ("ddc_load_coo", "ddc_build", "dose_forward", "beamlet_price", "price_apertures",
                 "mp_bb_solve", "cg_plan"):
        assert must in names


def test_every_declared_symbol_is_exported_and_bound(lib):
    from paper_1503_01721_gb300 import _lib
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} not exported"
        assert name in _lib.SIGNATURES, f"{name} has no ctypes signature"


def test_version(lib):
    assert b"sm_103a" in lib.vmat_version()


def test_spmv_config_count(lib):
    from gpu_util import N_SPMV_CFG
    assert lib.vmat_spmv_config_count() == N_SPMV_CFG


def test_host_validation_errors(lib):
    from paper_1503_01721_gb300 import _lib
    h = ctypes.c_void_p()
    assert lib.ddc_load_coo(0, 5, 0, None, None, None, 0, None, ctypes.byref(h)) == _lib.VMAT_EINVAL
    assert b"V > 0" in lib.vmat_last_error()
    assert lib.ddc_load_coo(4, 5, 3, None, None, None, 0, None, ctypes.byref(h)) == _lib.VMAT_EINVAL
    assert lib.ddc_build(None, None, None) == _lib.VMAT_EINVAL
    assert lib.dose_forward(None, None, None, None) == _lib.VMAT_EINVAL
    assert lib.beamlet_price(None, None, None, None, 0, None) == _lib.VMAT_EINVAL
    assert lib.beamlet_price_windowed(None, None, None, None, None, None, None) == _lib.VMAT_EINVAL
    assert lib.ddc_free(None) == _lib.VMAT_OK
    # MLC checks: arcs must start at CP 0 and increase
    arcs = (ctypes.c_int32 * 2)(1, 3)
    m = _lib.Mlc(6, 2, 4, 2, ctypes.cast(arcs, ctypes.POINTER(ctypes.c_int32)), 1)
    assert lib.price_apertures(ctypes.byref(m), None, None, None, None, None, None, None) == _lib.VMAT_EINVAL
    assert b"arc" in lib.vmat_last_error()
    arcs = (ctypes.c_int32 * 2)(0, 3)
    m = _lib.Mlc(6, 2, 2000, 2, ctypes.cast(arcs, ctypes.POINTER(ctypes.c_int32)), 1)
    assert lib.price_apertures(ctypes.byref(m), None, None, None, None, None, None, None) == _lib.VMAT_EINVAL
    assert b"n_cols" in lib.vmat_last_error()
    # machine checks (Eq. 2 limits): finite, ordered, travel window reachable at the slowest speed
    arcs = (ctypes.c_int32 * 1)(0)
    good = dict(cp_step_deg=10.0, speed_min=0.5, speed_max=4.0, speed_step_max=0.5, rate_min=0.02,
                rate_max=0.025, leaf_speed_cols=0.1875)
    for bad, msg in (({"speed_min": 5.0}, b"speed_min <= speed_max"), ({"rate_min": 0.03}, b"rate_min <= rate_max"),
                     ({"leaf_speed_cols": 0.1}, b"travel_cols * speed_min"), ({"cp_step_deg": 0.0}, b"> 0"),
                     ({"speed_step_max": float("inf")}, b"finite"), ({"speed_step_max": -1.0}, b"speed_step_max")):
        mach = _lib.Machine(**{**good, **bad})
        m = _lib.Mlc(6, 2, 4, 1, ctypes.cast(arcs, ctypes.POINTER(ctypes.c_int32)), 3, 0, ctypes.pointer(mach))
        assert lib.fluence_bounds(ctypes.byref(m), 1, 8, 8, 8, 8, None) == _lib.VMAT_EINVAL, bad
        assert msg in lib.vmat_last_error(), (bad, lib.vmat_last_error())
    mach = _lib.Machine(**good)
    m = _lib.Mlc(6, 2, 4, 1, ctypes.cast(arcs, ctypes.POINTER(ctypes.c_int32)), 3, 0, ctypes.pointer(mach))
    assert lib.fluence_bounds(ctypes.byref(m), -1, None, None, None, None, None) == _lib.VMAT_EINVAL
    assert lib.fluence_bounds(ctypes.byref(m), 9000, 8, 8, 8, 8, None) == _lib.VMAT_EINVAL
    assert lib.fluence_bounds(ctypes.byref(m), 2, None, 8, 8, 8, None) == _lib.VMAT_EINVAL
    assert lib.fluence_bounds(ctypes.byref(m), 0, None, None, None, None, None) == _lib.VMAT_OK
    # voxel parameter checks
    v = _lib.Voxels(None, 0, None, None, None)
    assert lib.objective_grad(10, None, ctypes.byref(v), None, None, None) == _lib.VMAT_EINVAL
    assert lib.mp_bb_solve(None, 0, 0, 0, None, None, None, None, None, None, None, None) == _lib.VMAT_EINVAL


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1503_01721_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load()
