"""Seeded synthetic inputs for the column-generation VMAT hot path.

This module serves both the FP64 oracle and the CUDA library and holds none of
the method's arithmetic: it only writes inputs (a pencil-beam DDC matrix in COO
form, voxel structure labels with per-structure dose parameters, the MLC
geometry, and random apertures for the differentiation workload).

Workload recipes (voxel units unless noted):

* ``tiny``  8x8x8 @ 5 mm, 4 CPs, 4x4 beamlets: brute-force scale.
* ``ragged`` 13x11x9 @ 5 mm, 5 CPs, 3x7 beamlets: odd sizes, ragged tails.
* ``cfg1``  40x40x40 @ 5 mm, one arc of 36 CPs, 20x20 beamlets (14,400),
  spherical target r=8 (prescription 1.0) at the centre + U[-2,2]^3 and two
  spherical OARs r=5 (limit 0.5) at distance r_t + r_o + 2 in seeded
  directions; 20 apertures.
* ``cfg2``  128x128x96 @ 2.5 mm, one arc of 180 CPs at 2 deg, 64x64 beamlets
  (737,280), three ellipsoidal targets (1.0/0.9/0.8, semi-axes U[6,16]) and
  six ellipsoidal OARs (limit 0.5, semi-axes U[4,10]); 60 apertures.
* ``cfg3``  cfg2 geometry with two arcs (360 CPs, second arc offset by 1 deg).
* ``cfg5``  a batch of 24 prostate-like plans of uneven size (``batch_specs``):
  grids from 80x80x60 to 160x160x120, 90-360 CPs (one arc up to 180, else two),
  40-80 leaf pairs, 16-80 columns chosen so that each DDC has 2e8-1.2e9
  nonzeros (1.14e10 in all); 60 apertures each.  ``cfg5q`` is the same batch
  with a quarter of the CPs (profiling), ``batch_small`` four small plans.

Pencil-beam value exp(-0.05 * depth) * exp(-rho^2/2), depth and lateral
distance rho both in voxel units (sigma = 1 voxel), dropped below 1% of the
unit peak; see ``gen.c`` for the geometry.  Depth in voxels keeps every target
voxel within reach (the 1% depth reach is 92 voxels); a millimetre depth would
stop cfg2 beams 37 voxels in, short of its central targets.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None


class _Geom(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("h_mm", ctypes.c_double),
        ("n_cp", ctypes.c_int32), ("n_arcs", ctypes.c_int32),
        ("arc_offset_deg", ctypes.c_double),
        ("n_rows", ctypes.c_int32), ("n_cols", ctypes.c_int32),
        ("pitch_vox", ctypes.c_double),
        ("mu_per_vox", ctypes.c_double),
        ("sigma_vox", ctypes.c_double),
        ("cutoff", ctypes.c_double),
        ("trunc_vox", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile ``gen.c`` into ``libsynth.so`` (gcc, OpenMP, no FP contraction)."""
    src = os.path.join(_HERE, "gen.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            lib.synth_count.restype = ctypes.c_int64
            lib.synth_count.argtypes = [ctypes.POINTER(_Geom), ctypes.c_void_p]
            lib.synth_fill.restype = ctypes.c_int
            lib.synth_fill.argtypes = [ctypes.POINTER(_Geom), ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.synth_n_beamlets.restype = ctypes.c_int64
            lib.synth_n_beamlets.argtypes = [ctypes.POINTER(_Geom)]
            lib.synth_count_list.restype = ctypes.c_int64
            lib.synth_count_list.argtypes = [ctypes.POINTER(_Geom), ctypes.c_void_p, ctypes.c_int64,
                                             ctypes.c_void_p]
            lib.synth_fill_list.restype = ctypes.c_int
            lib.synth_fill_list.argtypes = [ctypes.POINTER(_Geom), ctypes.c_void_p, ctypes.c_int64,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            _lib = lib
    return _lib


@dataclasses.dataclass(frozen=True)
class Geometry:
    nx: int
    ny: int
    nz: int
    h_mm: float
    n_cp: int
    n_rows: int
    n_cols: int
    n_arcs: int = 1
    arc_offset_deg: float = 1.0
    pitch_vox: float = 1.0
    mu_per_vox: float = 0.05
    sigma_vox: float = 1.0
    cutoff: float = 0.01
    trunc_vox: float = 0.0  # > 0: truncation radius about each beamlet axis (the paper's S1 matrix)

    @property
    def V(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def K(self) -> int:
        return self.n_cp * self.n_arcs

    @property
    def J(self) -> int:
        return self.K * self.n_rows * self.n_cols

    def _c(self) -> _Geom:
        return _Geom(self.nx, self.ny, self.nz, self.h_mm, self.n_cp, self.n_arcs,
                     self.arc_offset_deg, self.n_rows, self.n_cols, self.pitch_vox,
                     self.mu_per_vox, self.sigma_vox, self.cutoff, self.trunc_vox)


@dataclasses.dataclass
class Machine:
    """Delivery limits of Eq. 2: gantry speed, its change between CPs, dose rate
    and leaf speed.  Angles in degrees, times in seconds, leaf travel in MLC
    columns (the paper gives no values; these are parameters)."""
    cp_step_deg: float      # gantry angle between adjacent CPs of an arc
    speed_min: float        # S^L (deg/s)
    speed_max: float        # S^U (deg/s)
    speed_step_max: float   # Delta S: largest change of gantry speed per CP step (deg/s)
    rate_min: float         # R^L (MU/s)
    rate_max: float         # R^U (MU/s)
    leaf_speed_cols: float  # largest leaf speed (columns/s)


@dataclasses.dataclass
class MLC:
    """Beamlet layout j = (k*n_rows + r)*n_cols + c; arcs are CP ranges."""
    K: int
    n_rows: int
    n_cols: int
    arc_first_cp: np.ndarray  # int32 [n_arcs]; arc a spans [first[a], first[a+1] or K)
    travel_cols: int = 3
    interdigitation: bool = False  # adjacent rows: L_r <= R_{r-1} and L_r <= R_{r+1}
    machine: Machine | None = None  # None: every aperture's fluence rate in [0, +inf)

    @property
    def n_arcs(self) -> int:
        return int(len(self.arc_first_cp))


@dataclasses.dataclass
class Structures:
    """Per-voxel structure label and per-structure dose parameters (Eq. 1)."""
    struct_id: np.ndarray  # uint8 [V]
    T: np.ndarray          # float32 [n_struct]
    w_over: np.ndarray     # float32 [n_struct]
    w_under: np.ndarray    # float32 [n_struct]
    names: list


@dataclasses.dataclass
class Case:
    name: str
    geom: Geometry
    mlc: MLC
    vox: np.ndarray  # int32 [nnz]
    blt: np.ndarray  # int32 [nnz]
    val: np.ndarray  # float32 [nnz]
    structs: Structures
    n_apertures: int

    @property
    def V(self) -> int:
        return self.geom.V

    @property
    def J(self) -> int:
        return self.geom.J

    @property
    def nnz(self) -> int:
        return int(self.val.shape[0])


GEOMETRIES = {
    "tiny": Geometry(8, 8, 8, 5.0, 4, 4, 4),
    "ragged": Geometry(13, 11, 9, 5.0, 5, 3, 7),
    "cfg1": Geometry(40, 40, 40, 5.0, 36, 20, 20),
    "cfg2": Geometry(128, 128, 96, 2.5, 180, 64, 64),
    "cfg3": Geometry(128, 128, 96, 2.5, 180, 64, 64, n_arcs=2, arc_offset_deg=1.0),
    # cfg2 geometry with every 4th control point (8 deg): a few-GB case for profiling
    "cfg2q": Geometry(128, 128, 96, 2.5, 45, 64, 64),
}
APERTURES = {"tiny": 3, "ragged": 4, "cfg1": 20, "cfg2": 60, "cfg3": 60, "cfg2q": 30}


@dataclasses.dataclass(frozen=True)
class PlanSpec:
    """One plan of a batch workload: geometry, aperture count, structure recipe and seed."""
    name: str
    geom: Geometry
    n_apertures: int
    structures: str
    seed: int


def _cfg5_geometry(p: int, cp_div: int = 1) -> Geometry:
    """Plan p of the 24-plan batch: sizes grow with p; CP count, leaf pairs and the
    column count (set from a target beamlet count of 154e3 * 7.5^(u^2)) cycle so
    that small and large DDCs are mixed.  About 1300 nonzeros per beamlet."""
    s = p / 23.0
    nx = 80 + 8 * round(10 * s)
    nz = 60 + 4 * round(15 * s)
    n_rows = 40 + 8 * round(5 * ((p * 7) % 24) / 23.0)
    K = [90, 120, 180, 240, 360][(p * 3) % 5]
    u = ((p * 5) % 24) / 23.0
    beamlets = 154e3 * 7.5 ** (u * u)
    n_cols = int(min(max(round(beamlets / (K * n_rows)), 16), 80))
    n_arcs = 1 if K <= 180 else 2
    n_cp = max(K // n_arcs // cp_div, 2)
    return Geometry(nx, nx, nz, 2.5, n_cp, n_rows, n_cols, n_arcs=n_arcs, arc_offset_deg=1.0)


def batch_specs(name: str) -> list:
    """Plans of a batch workload (see the module docstring)."""
    if name in ("cfg5", "cfg5q"):
        div = 1 if name == "cfg5" else 4
        geoms = [_cfg5_geometry(p, div) for p in range(24)]
        return [PlanSpec(f"{name}_{p:02d}", g, min(60 if div == 1 else 30, g.K), "prostate", p)
                for p, g in enumerate(geoms)]
    if name == "batch_small":
        return [PlanSpec("bs_0", GEOMETRIES["tiny"], 3, "tiny", 0),
                PlanSpec("bs_1", GEOMETRIES["ragged"], 4, "ragged", 0),
                PlanSpec("bs_2", Geometry(24, 20, 16, 5.0, 12, 8, 10), 6, "prostate", 2),
                PlanSpec("bs_3", GEOMETRIES["cfg1"], 12, "cfg1", 3)]
    raise KeyError(name)


def make_truncated_case(name: str, trunc_vox: float, seed: int = 0) -> "Case":
    """The named workload with its DDC truncated to trunc_vox voxels about each
    beamlet axis (same geometry, structures and MLC)."""
    geom = dataclasses.replace(GEOMETRIES[name], trunc_vox=float(trunc_vox))
    vox, blt, val = generate_coo(geom)
    return Case(f"{name}_trunc{trunc_vox:g}", geom, make_mlc(geom), vox, blt, val,
                make_structures(name, geom, seed), APERTURES[name])


def make_plan_case(spec: PlanSpec) -> "Case":
    """Generate one plan of a batch (not cached: batches can exceed host memory if kept)."""
    vox, blt, val = generate_coo(spec.geom)
    return Case(spec.name, spec.geom, make_mlc(spec.geom), vox, blt, val,
                make_structures(spec.structures, spec.geom, spec.seed), spec.n_apertures)


def generate_coo(geom: Geometry):
    """Return (vox int32, blt int32, val float32) COO arrays, beamlet-major."""
    lib = _load()
    g = geom._c()
    J = geom.J
    counts = np.zeros(J, dtype=np.int64)
    total = lib.synth_count(ctypes.byref(g), counts.ctypes.data)
    offsets = np.zeros(J + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    assert offsets[-1] == total
    vox = np.empty(total, dtype=np.int32)
    blt = np.empty(total, dtype=np.int32)
    val = np.empty(total, dtype=np.float32)
    rc = lib.synth_fill(ctypes.byref(g), offsets.ctypes.data, vox.ctypes.data,
                        blt.ctypes.data, val.ctypes.data)
    if rc != 0:
        raise RuntimeError("synthetic DDC generator: count/fill mismatch")
    return vox, blt, val


def generate_coo_cps(geom: Geometry, cps):
    """COO of the beamlets of the listed CPs only, renumbered as a K' = len(cps) geometry:
    beamlet (t, r, c) of the result has the geometry of (cps[t], r, c)."""
    lib = _load()
    g = geom._c()
    bpc = geom.n_rows * geom.n_cols
    js = (np.asarray(cps, np.int64)[:, None] * bpc + np.arange(bpc, dtype=np.int64)[None, :]).ravel()
    counts = np.zeros(len(js), dtype=np.int64)
    total = lib.synth_count_list(ctypes.byref(g), js.ctypes.data, len(js), counts.ctypes.data)
    offsets = np.zeros(len(js) + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    vox = np.empty(total, dtype=np.int32)
    blt = np.empty(total, dtype=np.int32)
    val = np.empty(total, dtype=np.float32)
    if lib.synth_fill_list(ctypes.byref(g), js.ctypes.data, len(js), offsets.ctypes.data, vox.ctypes.data,
                           blt.ctypes.data, val.ctypes.data) != 0:
        raise RuntimeError("synthetic DDC generator: count/fill mismatch")
    return vox, blt, val


def _grid_coords(geom: Geometry):
    z, y, x = np.meshgrid(np.arange(geom.nz), np.arange(geom.ny), np.arange(geom.nx), indexing="ij")
    c = np.array([(geom.nx - 1) / 2, (geom.ny - 1) / 2, (geom.nz - 1) / 2])
    return x.ravel() - c[0], y.ravel() - c[1], z.ravel() - c[2]


def make_structures(name: str, geom: Geometry, seed: int) -> Structures:
    """Seeded targets/OARs.  Priority: target (higher prescription) > OAR > tissue.

    Label 0 is normal tissue with an overdose penalty only
    (w_over = 0.05, threshold 0.6 * max prescription).  Targets get
    (w_over, w_under) = (1, 1) with T = prescription; OARs (0.3, 0) with T = limit.
    """
    rng = np.random.default_rng(seed)
    x, y, z = _grid_coords(geom)
    V = geom.V
    sid = np.zeros(V, dtype=np.uint8)
    T, wo, wu, names = [], [], [], []
    if name == "cfg2q":
        name = "cfg2"
    if name == "prostate":
        # target ellipsoid near the centre; rectum behind it (elongated along z),
        # bladder above and in front; sizes in proportion to the grid
        n = np.array([geom.nx, geom.ny, geom.nz], float)
        ct = rng.uniform(-0.03, 0.03, size=3) * n
        at = np.array([0.11, 0.09, 0.10]) * n * rng.uniform(0.9, 1.1, size=3)
        ar = np.array([0.06, 0.06, 0.20]) * n
        ab = np.array([0.14, 0.11, 0.09]) * n
        targets = [(ct, at, 1.0)]
        oars = [(ct - np.array([0.0, at[1] + ar[1] + 1.0, 0.0]), ar, 0.5),
                (ct + np.array([0.0, 0.4 * at[1], at[2] + ab[2] + 1.0]), ab, 0.5)]
    elif name in ("cfg1", "tiny", "ragged"):
        r_t = {"cfg1": 8.0, "tiny": 2.5, "ragged": 2.5}[name]
        r_o = {"cfg1": 5.0, "tiny": 1.5, "ragged": 1.5}[name]
        # continuous centre offsets: a sphere centred on a grid point is mirror
        # symmetric, which makes opposite CPs price exactly alike (exact ties)
        ct = rng.uniform(-2, 2, size=3) if name == "cfg1" else rng.uniform(-1, 1, size=3)
        targets = [(ct, np.array([r_t] * 3), 1.0)]
        oars = []
        for _ in range(2):
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            oars.append((ct + d * (r_t + r_o + (2.0 if name == "cfg1" else 0.5)), np.array([r_o] * 3), 0.5))
    else:
        targets, oars = [], []
        for rx in (1.0, 0.9, 0.8):
            targets.append((rng.uniform(-12, 12, size=3) * np.array([1, 1, 0.75]),
                            rng.uniform(6, 16, size=3), rx))
        for _ in range(6):
            oars.append((rng.uniform(-24, 24, size=3) * np.array([1, 1, 0.75]),
                         rng.uniform(4, 10, size=3), 0.5))
    max_rx = max(t[2] for t in targets)
    T.append(0.6 * max_rx); wo.append(0.05); wu.append(0.0); names.append("tissue")

    def inside(c, ax):
        return ((x - c[0]) / ax[0]) ** 2 + ((y - c[1]) / ax[1]) ** 2 + ((z - c[2]) / ax[2]) ** 2 <= 1.0

    for i, (c, ax, lim) in enumerate(oars):
        sid[inside(c, ax)] = len(T)
        T.append(lim); wo.append(0.3); wu.append(0.0); names.append(f"oar{i}")
    for i, (c, ax, rx) in sorted(enumerate(targets), key=lambda e: e[1][2]):
        sid[inside(c, ax)] = len(T)
        T.append(rx); wo.append(1.0); wu.append(1.0); names.append(f"ptv{i}")
    return Structures(sid, np.array(T, np.float32), np.array(wo, np.float32),
                      np.array(wu, np.float32), names)


def make_mlc(geom: Geometry, travel_cols: int = 3) -> MLC:
    first = np.arange(geom.n_arcs, dtype=np.int32) * geom.n_cp
    return MLC(geom.K, geom.n_rows, geom.n_cols, first, travel_cols)


_CACHE: dict = {}


def make_machine(mlc: MLC, speed_min: float = 0.5, speed_max: float = 4.0, speed_step_max: float = 0.5,
                 rate_min: float = 0.02, rate_max: float = 0.025) -> Machine:
    """A delivery machine for an MLC: CPs evenly spaced over each arc's 360
    degrees, and a leaf speed 1.25x what the MLC's travel window needs at the
    slowest gantry speed (so the travel window never asks for more than the
    leaves can do).  Defaults make both fluence bounds bind on the test plans."""
    step = 360.0 * mlc.n_arcs / mlc.K
    return Machine(step, speed_min, speed_max, speed_step_max, rate_min, rate_max,
                   1.25 * max(mlc.travel_cols, 1) * speed_min / step)


def make_case(name: str, seed: int = 0, cache: bool = True) -> Case:
    """Build a named workload (see module docstring); cached per (name, seed)."""
    key = (name, seed)
    if cache and key in _CACHE:
        return _CACHE[key]
    geom = GEOMETRIES[name]
    vox, blt, val = generate_coo(geom)
    case = Case(name, geom, make_mlc(geom), vox, blt, val,
                make_structures(name, geom, seed), APERTURES[name])
    if cache:
        _CACHE[key] = case
    return case


def random_apertures(mlc: MLC, n: int, seed: int, len_lo: int = 4, len_hi: int = 40):
    """Random apertures for the differentiation workload.

    CPs drawn with replacement; every leaf row is one open interval whose
    length is uniform on {len_lo .. min(len_hi, n_cols)} and whose start is
    uniform among the positions where it fits.  Returns (cps int32 [n],
    leaves int16 [n, n_rows, 2], y float32 [n] ~ U(0, 1)).
    """
    rng = np.random.default_rng(seed)
    cps = rng.integers(0, mlc.K, size=n).astype(np.int32)
    hi = min(len_hi, mlc.n_cols)
    lo = min(len_lo, hi)
    ln = rng.integers(lo, hi + 1, size=(n, mlc.n_rows))
    start = (rng.random(size=(n, mlc.n_rows)) * (mlc.n_cols - ln + 1)).astype(np.int64)
    leaves = np.stack([start, start + ln], axis=-1).astype(np.int16)
    y = rng.random(size=n).astype(np.float32)
    return cps, leaves, y


def random_vector(n: int, seed: int, lo: float = -1.0, hi: float = 1.0, dtype=np.float32):
    """Seeded uniform vector (used as x or g in parity tests)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=n).astype(dtype)


def shuffled_coo(vox, blt, val, seed: int):
    """The same matrix with its COO entries in a seeded random order."""
    p = np.random.default_rng(seed).permutation(len(val))
    return vox[p].copy(), blt[p].copy(), val[p].copy()
