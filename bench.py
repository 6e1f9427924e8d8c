"""Benchmark: column-generation VMAT plans on the H&N-like synthetic workload.

One step = one full cg_plan (60 apertures) on the 128x128x96-voxel, 180-CP,
64x64-beamlet DDC, every hot-path stage included (gradient, beamlet price over
the unoccupied CPs, pricing, aperture dose vectors, BB master problems, final
FP32 dose).  The DDC (CSR of D and of D^T) is resident in HBM before timing.

value = effective DDC bandwidth of the plan: the algorithmic bytes of every
D x and D^T g pass the plan makes, divided by the plan's wall time (GB/s).
The D^T g passes read only the beamlet rows inside the leaf-travel windows of
the unoccupied CPs (the prices that pricing reads), so their bytes are those
rows' bytes; plan.pp1_window_frac = those bytes over the bytes of passes over
every row of the unoccupied CPs.  ms_per_step = plan wall time.  roofline =
the beamlet-price SpMV, timed by the library's CUDA events on its launch
stream during the timed plans.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only reference that exists) on
a bounded sample of the same workload.  With torchrun, every rank plans its own
replica (plans are independent; no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DDC D·x + Dᵀ·g effective HBM GB/s; CG plan wall time at matched objective"
WORKLOAD = "cfg2"
DESCS = {
    "cfg2": ("H&N-like: 128x128x96 voxels @2.5 mm, 3 targets + 6 OARs, one arc of 180 CPs, "
             "64x64 beamlets (737,280), pencil-beam DDC FP32, 60 apertures"),
    "cfg2q": ("profiling case: the H&N-like geometry with 45 CPs at 8 deg (184,320 beamlets), 30 apertures"),
    "cfg1": ("tiny FP32 case: 40^3 voxels @5 mm, one sphere target + 2 OARs, 36 CPs, 20x20 beamlets, "
             "20 apertures (L2-resident)"),
    "cfg3": ("precision case: the H&N-like geometry with two arcs (360 CPs, second arc offset by 1 deg), "
             "64x64 beamlets (1,474,560), 60 apertures"),
}
WORKLOAD_DESC = DESCS[WORKLOAD]
# SpMV configurations as the library builds them (csrc/spmv.cu, kCfgs)
SPMV_KERNELS = {0: "spmv_tile_kernel<256,16,2>", 1: "spmv_tile_kernel<256,8,3>", 2: "spmv_tile_kernel<512,8,2>",
                3: "spmv_tile_kernel<128,16,3>", 4: "spmv_warp_row_kernel<256,2>", 5: "spmv_warp_row_kernel<256,1>",
                6: "spmv_warp_row_kernel<512,4>", 7: "spmv_warp_row_kernel<256,4>", 8: "spmv_warp_row_kernel<256,8>",
                9: "spmv_warp_row_c_kernel<256,4>", 10: "spmv_warp_row_c_kernel<256,8>",
                11: "spmv_warp_row_c_kernel<512,4>", 12: "spmv_warp_row_z_kernel<256,4>",
                13: "spmv_warp_row_z_kernel<256,8>", 14: "spmv_warp_row_z_kernel<512,4>"}
# configurations that read the 16-bit column index (built with index16)
INDEX16_CFGS = (12, 13, 14)
# DRAM traffic over algorithmic bytes of the plan's windowed D^T g launches, per (value type,
# configuration, CSR(D^T) column order): dram__bytes_read.sum + dram__bytes_write.sum over the 30
# windowed launches of the 45-CP plan (the same kernels on a quarter of the CPs), over their algorithmic
# bytes, from one ncu capture each; a configuration without such a capture reports null.
WINDOWED_TRAFFIC_RATIO = {("f32", 5, "voxel"): 0.9988, ("f32", 9, "voxel"): 1.0010, ("f32", 11, "voxel"): 1.0009,
                          ("f32", 9, "brick"): 1.0039, ("f32", 11, "brick"): 1.0038}
# The paper's own plan times (Table 2 and Table 3): other hardware, patient data and aperture
# counts, so context for the line, not a baseline of its metric.
PAPER_CONTEXT = {
    "plan_total_s": 63.96, "t_pp1_s": 10.77, "t_pp2_s": 5.05, "t_mp_s": 21.24,
    "workload": "head-and-neck case P1: 26,828 voxels, 128,516 beamlets, 608,447,419 nonzeros, 199 apertures, "
                "9,364 BB iterations",
    "hardware": "4x GTX 590 (Fermi, CUDA 4.0); PP2 and the DA vectors partly on the CPU",
    "other_cases_total_s": [31.50, 37.36, 39.77, 45.46, 23.28],
    "cpu_plan_total_s": 360.85, "cpu": "the paper's CPU version, pthreads on 4 cores / 8 threads",
}
# CPU sample: every 12th CP of the same geometry (15 CPs), 5 apertures
SAMPLE_CP_STRIDE = 12
SAMPLE_APERTURES = 5


def vox_grid(case):
    """(nx, ny, nz) of a case's voxel grid: CSR(D^T) columns in brick order."""
    g = case.geom
    return (g.nx, g.ny, g.nz)


def dataclasses_asdict(x):
    import dataclasses
    return None if x is None else dataclasses.asdict(x)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 7:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for nm, v in zip(names, p[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- distributed

def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("VMAT_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch
        import torch.distributed as dist
        if dist.get_backend() == "nccl":
            dist.barrier(device_ids=[torch.cuda.current_device()])
        else:
            dist.barrier()


def _all_reduce(x, world, op):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x, world):
    import torch.distributed as dist
    return _all_reduce(x, world, dist.ReduceOp.MAX) if world > 1 else x


def sum_over_ranks(x, world):
    import torch.distributed as dist
    return _all_reduce(x, world, dist.ReduceOp.SUM) if world > 1 else x


def whole_job_gbs(bytes_local, seconds_local, world):
    """Whole-job rate: the bytes every rank moved over the slowest rank's time."""
    return sum_over_ranks(bytes_local, world) / max_over_ranks(seconds_local, world) / 1e9


# ----------------------------------------------------------------------------- CPU oracle sample

def sample_case():
    """The CPU sample: every SAMPLE_CP_STRIDE-th CP of the workload's geometry."""
    import numpy as np
    import synth
    geom = synth.GEOMETRIES[WORKLOAD]
    bpc = geom.n_rows * geom.n_cols
    keep_cp = np.arange(0, geom.K, SAMPLE_CP_STRIDE)
    vox, blt, val = synth.generate_coo_cps(geom, keep_cp)
    structs = synth.make_structures(WORKLOAD, geom, 0)
    mlc = synth.MLC(len(keep_cp), geom.n_rows, geom.n_cols, np.array([0], np.int32), 3)
    return geom.V, len(keep_cp) * bpc, vox, blt, val, structs, mlc


def _sample_dir():
    import tempfile
    base = "/dev/shm" if os.path.isdir("/dev/shm") and os.access("/dev/shm", os.W_OK) else None
    return tempfile.mkdtemp(prefix="vmat_oracle_sample_", dir=base)


def prepare_cpu_sample(path):
    """Generate the CPU sample once and store the oracle's float64 CSR of D (and the
    plan inputs) under path, so that every oracle process maps the same arrays."""
    import numpy as np
    import oracle
    V, J, vox, blt, val, structs, mlc = sample_case()
    D = oracle.ddc_matrix(V, J, vox, blt, val)
    for nm in ("data", "indices", "indptr"):
        np.save(os.path.join(path, nm + ".npy"), getattr(D, nm))
    np.savez(os.path.join(path, "meta.npz"), V=V, J=J, nnz=len(val), K=mlc.K, n_rows=mlc.n_rows,
             n_cols=mlc.n_cols, per_blt=np.bincount(blt, minlength=J),
             n_rows_D=int(np.count_nonzero(np.bincount(vox, minlength=V))), struct_id=structs.struct_id,
             T=structs.T, w_over=structs.w_over, w_under=structs.w_under)


def _load_cpu_sample(path):
    import numpy as np
    import scipy.sparse as sp
    import synth
    m = np.load(os.path.join(path, "meta.npz"))
    ld = lambda nm: np.load(os.path.join(path, nm + ".npy"), mmap_mode="r")
    D = sp.csr_matrix((ld("data"), ld("indices"), ld("indptr")), shape=(int(m["V"]), int(m["J"])), copy=False)
    structs = synth.Structures(m["struct_id"], m["T"], m["w_over"], m["w_under"], [])
    mlc = synth.MLC(int(m["K"]), int(m["n_rows"]), int(m["n_cols"]), np.array([0], np.int32), 3)
    return D, structs, mlc, m


def _plan_bytes(plan, mlc, m):
    """Bytes of a sample plan's sparse passes in the GPU's FP32-CSR byte model: each pricing
    pass counts the beamlet rows inside the leaf-travel windows of the unoccupied CPs (the
    prices pricing reads), as the GPU's windowed pass does, plus g and the window table;
    then the final D x."""
    import numpy as np
    import oracle
    from paper_1503_01721_gb300 import roofline
    V, J = int(m["V"]), int(m["J"])
    per_blt = m["per_blt"].reshape(mlc.K, mlc.n_rows, mlc.n_cols)
    col = np.arange(mlc.n_cols)[None, :]
    n_price = len(plan.cps) + (plan.stop == "price")
    b = 0.0
    occupied = np.zeros(mlc.K, bool)
    leaves_all = np.zeros((mlc.K, mlc.n_rows, 2), np.int64)
    for t in range(n_price):
        nz = rows = 0
        for k in np.flatnonzero(~occupied):
            Lmin, _, _, Rmax = oracle.leaf_windows(mlc, occupied, leaves_all, int(k))
            inw = (col >= np.asarray(Lmin)[:, None]) & (col < np.asarray(Rmax)[:, None])
            nz += int(per_blt[k][inw].sum())
            rows += int(inw.sum())
        b += nz * roofline.csr_bytes_per_nnz("f32") + rows * 12 + 4 * V + 4 * mlc.K * mlc.n_rows
        if t < len(plan.cps):
            occupied[plan.cps[t]] = True
            leaves_all[plan.cps[t]] = plan.leaves[t]
    return b + roofline.spmv_bytes(int(m["nnz"]), int(m["n_rows_D"]), J, V)


def oracle_worker(path, steps, warmup, barrier, queue):
    """One oracle process (one thread): `warmup` + `steps` sample plans, then D^T g and
    D x passes over the sample, each phase started together with the other processes."""
    import numpy as np
    import oracle
    from paper_1503_01721_gb300 import roofline
    try:
        D, structs, mlc, m = _load_cpu_sample(path)
        V, J = int(m["V"]), int(m["J"])
        rng = np.random.default_rng(0)
        g, x = rng.standard_normal(V), rng.random(J)
        times = []
        for it in range(warmup + steps):
            barrier.wait()
            t0 = time.perf_counter()
            plan = oracle.cg_plan(D, mlc, structs, SAMPLE_APERTURES)
            if it >= warmup:
                times.append(time.perf_counter() - t0)
        pt = {}
        for nm, fn, arg in (("dt_g", oracle.beamlet_price, g), ("d_x", oracle.dose_forward, x)):
            ts = []
            for _ in range(3):
                barrier.wait()
                t0 = time.perf_counter()
                fn(D, arg)
                ts.append(time.perf_counter() - t0)
            pt[nm] = float(np.median(ts))
        nnz = int(m["nnz"])
        queue.put({"sec_per_plan": sum(times) / len(times), "plan_bytes": _plan_bytes(plan, mlc, m),
                   "dt_g_s": pt["dt_g"], "d_x_s": pt["d_x"],
                   "dt_g_bytes": roofline.spmv_bytes(nnz, J, V, J), "d_x_bytes": roofline.spmv_bytes(nnz,
                   int(m["n_rows_D"]), J, V), "nnz": nnz, "J": J, "V": V, "apertures": len(plan.cps),
                   "F": plan.F})
    except BaseException as e:  # report instead of leaving the others at the barrier
        barrier.abort()
        queue.put({"error": repr(e)})


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_oracle_procs(path, n_proc, steps, warmup):
    """n_proc single-threaded oracle processes on the same sample, in step.  Whole-job
    rates: the bytes of every process over the slowest process's time."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")  # the parent may hold a CUDA context
    barrier, queue = ctx.Barrier(n_proc), ctx.Queue()
    env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
                                               "CUDA_VISIBLE_DEVICES")}
    os.environ.update(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    try:
        procs = [ctx.Process(target=oracle_worker, args=(path, steps, warmup, barrier, queue)) for _ in range(n_proc)]
        for p in procs:
            p.start()
        res = [queue.get(timeout=1800) for _ in range(n_proc)]
        for p in procs:
            p.join(timeout=60)
    finally:
        for k, v in env_keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    bad = [r["error"] for r in res if "error" in r]
    if bad:
        raise RuntimeError("oracle process failed: " + bad[0])
    r0 = res[0]
    t_plan = max(r["sec_per_plan"] for r in res)
    t_dt, t_d = max(r["dt_g_s"] for r in res), max(r["d_x_s"] for r in res)
    return {"value": sum(r["plan_bytes"] for r in res) / t_plan / 1e9, "sec_per_plan": t_plan, "procs": n_proc,
            "dt_g_gbs": n_proc * r0["dt_g_bytes"] / t_dt / 1e9, "d_x_gbs": n_proc * r0["d_x_bytes"] / t_d / 1e9,
            "nnz": r0["nnz"], "J": r0["J"], "V": r0["V"], "apertures": r0["apertures"], "F": r0["F"]}


def cpu_baseline(steps=1, warmup=0):
    """The FP64 oracle on the CPU sample: one process per host core, and one alone."""
    import shutil
    path = _sample_dir()
    try:
        prepare_cpu_sample(path)
        n = host_cores()
        single = run_oracle_procs(path, 1, steps, warmup)
        allc = run_oracle_procs(path, n, steps, warmup) if n > 1 else single
    finally:
        shutil.rmtree(path, ignore_errors=True)
    allc["single_thread"] = {k: single[k] for k in ("value", "sec_per_plan", "dt_g_gbs", "d_x_gbs")}
    return allc


def sample_desc(res):
    return (f"FP64 oracle cg_plan, {SAMPLE_APERTURES} apertures, on every {SAMPLE_CP_STRIDE}th CP of the "
            f"{WORKLOAD} geometry ({res['J']} beamlets, {res['nnz']} nonzeros), one single-threaded process per "
            f"host core ({res['procs']}) on the same sample, whole-job bytes over the slowest process's time; "
            f"same byte model (rows inside the leaf-travel windows per pricing pass)")


def cpu_block(res):
    return {"value": round(res["value"], 4), "unit": "GB/s", "cores": res["procs"], "kind": "oracle",
            "sample": sample_desc(res), "sec_per_plan": round(res["sec_per_plan"], 3),
            "spmv_passes": {"dt_g_gbs": round(res["dt_g_gbs"], 3), "d_x_gbs": round(res["d_x_gbs"], 3)},
            "single_thread": {k: round(v, 4) for k, v in res["single_thread"].items()}}


# ----------------------------------------------------------------------------- GPU arm

def sampled_dose_error(case, cps, lv, y, dose, n_ap, n=4096, seed=5):
    """Final dose against the float64 sum over the COO's float32 entries of D (A y), at
    n sampled voxels: max |d - d_ref| / max |d_ref| over the sample."""
    import numpy as np
    m = case.mlc
    cps = np.asarray(cps)[:n_ap].astype(np.int64)
    lv = np.asarray(lv).reshape(-1, m.n_rows, 2)[:n_ap].astype(np.int64)
    y = np.asarray(y)[:n_ap].astype(np.float64)
    x = np.zeros(case.J)  # x = A y: each aperture's fluence on its beamlets
    for a, k in enumerate(cps):
        for r in range(m.n_rows):
            base = (int(k) * m.n_rows + r) * m.n_cols
            x[base + lv[a, r, 0]: base + lv[a, r, 1]] += y[a]
    voxels = np.random.default_rng(seed).choice(case.V, n, replace=False)
    flag = np.zeros(case.V, bool)
    flag[voxels] = True
    sel = np.flatnonzero(flag[case.vox])
    ref = np.bincount(case.vox[sel], weights=case.val[sel].astype(np.float64) * x[case.blt[sel]],
                      minlength=case.V)[voxels]
    err = float(np.max(np.abs(np.asarray(dose)[voxels] - ref)) / max(float(np.max(np.abs(ref))), 1e-300))
    return {"rel_linf": err, "voxels": n,
            "against": "float64 sum of D (A y) over the float32 COO entries, at seeded sampled voxels"}


def precision_form(dev, steps=3, warmup=1):
    """The precision form on the two-arc case (1.93e9 nonzeros): the same 60-aperture plan
    with the DDC stored as FP32, BF16 and FP8 E4M3 (the low-precision handles also keep
    FP32 values of CSR(D) for the end-of-plan refinement)."""
    import numpy as np
    import torch
    import synth
    from paper_1503_01721_gb300 import api
    t0 = time.time()
    case = synth.make_case("cfg3", seed=0, cache=False)
    log(f"[forms] cfg3: {case.nnz} nonzeros in {time.time() - t0:.1f}s")
    pin = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dt).pin_memory()
    coo = (pin(case.vox, torch.int32), pin(case.blt, torch.int32), pin(case.val, torch.float32))
    vox = api.VoxelParams.from_numpy(case.structs, dev)
    n_ap = case.n_apertures
    stream = torch.cuda.current_stream()
    res = {}
    for dt in ("f32", "bf16", "fp8"):
        h = api.ddc_load_coo(case.V, case.J, *coo)
        api.ddc_build(h, dt, autotune=True, refine=dt != "f32", vox_grid=vox_grid(case))
        cps = torch.empty(n_ap, dtype=torch.int32)
        lv = torch.empty(n_ap * case.mlc.n_rows * 2, dtype=torch.int16)
        y = torch.empty(n_ap, dtype=torch.float32)
        dose = torch.empty(case.V, dtype=torch.float32, device=dev)
        for _ in range(warmup):
            api.cg_plan(h, case.mlc, vox, n_ap)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sts = []
        for _ in range(steps):
            F, st = api.cg_plan(h, case.mlc, vox, n_ap, cps_out=cps, leaves_out=lv, y_out=y, dose_out=dose)
            sts.append(st)
        e1.record(stream)
        torch.cuda.synchronize()
        info = api.ddc_info(h)
        api.ddc_free(h)
        st = sts[-1]
        res[dt] = {"ms_per_plan": round(e0.elapsed_time(e1) / steps, 3), "F": F,
                   "pp1_spmv_ms": round(sum(x["pp1_spmv_ms"] for x in sts) / steps, 3),
                   "pp1_spmv_gbs": round(sum(x["pp1_spmv_bytes"] for x in sts) / sum(x["pp1_spmv_ms"] for x in sts)
                                         / 1e6, 1),
                   "t_refine_ms": round(st["t_refine_ms"], 3), "F_before_refine": st["F_before_refine"],
                   "refine_bb_iters": st["refine_bb_iters"], "cfg_Dt": int(st["pp1_spmv_cfg"]),
                   "dose_err": sampled_dose_error(case, cps.numpy(), lv.numpy(), y.numpy(), dose.cpu().numpy(),
                                                  int(st["n_apertures"]))}
    f32 = res["f32"]
    return {"workload": "cfg3 " + DESCS["cfg3"] + f", {case.nnz} nonzeros", "plans": res,
            "bf16_speedup": round(f32["ms_per_plan"] / res["bf16"]["ms_per_plan"], 3),
            "fp8_speedup": round(f32["ms_per_plan"] / res["fp8"]["ms_per_plan"], 3),
            "pp1_speedup": {d: round(f32["pp1_spmv_ms"] / res[d]["pp1_spmv_ms"], 3) for d in ("bf16", "fp8")},
            "F_rel_err": {d: (res[d]["F"] - f32["F"]) / f32["F"] for d in ("bf16", "fp8")},
            "dose_rel_err": {d: res[d]["dose_err"]["rel_linf"] for d in ("f32", "bf16", "fp8")},
            "notes": "speedups and F_rel_err against the FP32 plan on the same GPU; the BF16 / FP8 plans end "
                     "with the FP32 refinement (DA of the placed apertures and the final dose from FP32 values)"}



def run_ours(args, rank, world, local):
    import numpy as np
    import torch
    import synth
    from paper_1503_01721_gb300 import api, roofline
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    t0 = time.time()
    case = synth.make_case(args.workload, seed=rank, cache=False)
    if args.interdig or args.machine:
        import dataclasses
        mlc = dataclasses.replace(case.mlc, interdigitation=bool(args.interdig))
        if args.machine:
            mlc.machine = synth.make_machine(mlc)
        case = dataclasses.replace(case, mlc=mlc)
    log(f"[rank {rank}] generated {case.nnz} nonzeros in {time.time() - t0:.1f}s")
    pin = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dt).pin_memory()
    vox_h, blt_h, val_h = pin(case.vox, torch.int32), pin(case.blt, torch.int32), pin(case.val, torch.float32)
    vox = api.VoxelParams.from_numpy(case.structs, dev)
    n_ap = case.n_apertures

    # resident DDC
    h = api.ddc_load_coo(case.V, case.J, vox_h, blt_h, val_h)
    grid = vox_grid(case) if args.vox_order == "brick" else None
    api.ddc_build(h, args.dtype, tile_cfg=args.tile_cfg, autotune=args.tile_cfg < 0, index16=args.index16,
                  vox_grid=grid)
    info = api.ddc_info(h)
    log(f"[rank {rank}] build {info['build_ms']:.1f} ms, active voxels {info['n_active_vox']}")

    cps = torch.empty(n_ap, dtype=torch.int32).pin_memory()
    lv = torch.empty(n_ap * case.mlc.n_rows * 2, dtype=torch.int16).pin_memory()
    y = torch.empty(n_ap, dtype=torch.float32).pin_memory()
    dose = torch.empty(case.V, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        api.cg_plan(h, case.mlc, vox, n_ap, dose_out=dose)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stats_all = []
    Fs = []
    launches0 = api.launch_count()
    for _ in range(args.steps):
        F, st = api.cg_plan(h, case.mlc, vox, n_ap, cps_out=cps, leaves_out=lv, y_out=y, dose_out=dose)
        stats_all.append(st)
        Fs.append(F)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = api.launch_count() - launches0
    ms_total = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    ms_step = max_over_ranks(ms_total / args.steps, world)
    bytes_step = sum(s["pp1_spmv_bytes"] + s["other_spmv_bytes"] for s in stats_all) / args.steps
    value = whole_job_gbs(bytes_step, ms_total / args.steps * 1e-3, world)

    # dominant kernel: the beamlet-price SpMV, from the library's events over the timed plans
    spmv_ms = sum(s["pp1_spmv_ms"] for s in stats_all)
    spmv_n = sum(s["pp1_spmv_launches"] for s in stats_all)
    spmv_bytes = sum(s["pp1_spmv_bytes"] for s in stats_all)
    peaks = roofline.measured_peaks()
    achieved = spmv_bytes / (spmv_ms * 1e-3) / 1e9
    cfg_dt = int(stats_all[-1]["pp1_spmv_cfg"])  # the windowed passes' configuration
    kname = SPMV_KERNELS.get(cfg_dt, f"spmv configuration {cfg_dt}") + \
        (" + spmv_fixup" if cfg_dt < 4 else "") + " (beamlet price D^T g over the unoccupied CPs)"
    bytes_launch = spmv_bytes / max(spmv_n, 1)
    ratio = WINDOWED_TRAFFIC_RATIO.get((args.dtype, cfg_dt, "brick" if info["vox_brick"] else "voxel"))
    roof = {"bound": "hbm", "kernel": kname,
            "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": round(achieved / peaks["hbm_gbs"], 4),
            "traffic": None if ratio is None else round(ratio * bytes_launch),
            "traffic_source": None if ratio is None else
            f"ncu dram bytes / algorithmic bytes = {ratio} for this kernel over the windowed D^T g launches of "
            "the 45-CP plan, times this launch's algorithmic bytes",
            "peak_source": peaks["source"], "frac_of_nominal": round(achieved / roofline.HBM_NOMINAL_GBS, 4),
            "nominal_peak": roofline.HBM_NOMINAL_GBS, "bytes_per_launch": round(bytes_launch),
            "avg_launch_ms": round(spmv_ms / max(spmv_n, 1), 4)}

    # the last timed plan's final dose against float64 sums over the COO at sampled voxels
    dose_err = sampled_dose_error(case, cps.numpy(), lv.numpy(), y.numpy(), dose.cpu().numpy(),
                                  int(stats_all[-1]["n_apertures"]))
    # master problem: the bytes its passes moved over the time of the MP phase
    mp_bytes = sum(s["mp_bytes"] for s in stats_all)
    mp_ms = sum(s["t_mp_ms"] for s in stats_all)
    mp_roof = {"bound": "hbm", "kernel": "mp_solve_kernel (persistent BB master problem over the live tiles)",
               "achieved": round(mp_bytes / (mp_ms * 1e-3) / 1e9, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
               "frac": round(mp_bytes / (mp_ms * 1e-3) / 1e9 / peaks["hbm_gbs"], 4),
               "bytes_per_step": round(mp_bytes / args.steps), "ms_per_step": round(mp_ms / args.steps, 3),
               "bb_iters_per_step": stats_all[-1]["bb_iters_total"],
               "timing": "library CUDA events around each plan's master-problem phase"}

    # isolated full passes: D^T g and D x over the whole matrix
    g = torch.rand(case.V, device=dev)
    x = torch.rand(case.J, device=dev)
    pi = torch.empty(case.J, device=dev)
    d = torch.empty(case.V, device=dev)
    for _ in range(3):
        api.beamlet_price(h, g, pi)
        api.dose_forward(h, x, d)
    torch.cuda.synchronize()
    reps = 21  # each pass timed on its own; the median is reported

    def median_ms(fn):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
        ev[0].record(stream)
        for i in range(reps):
            fn()
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
        return float(np.median([ev[i].elapsed_time(ev[i + 1]) for i in range(reps)]))

    t_dt = median_ms(lambda: api.beamlet_price(h, g, pi))
    t_d = median_ms(lambda: api.dose_forward(h, x, d))
    b_dt = roofline.spmv_bytes(case.nnz, case.J, case.V, case.J, args.dtype, case.J if args.dtype == "fp8" else 0)
    b_d = roofline.spmv_bytes(case.nnz, info["n_active_vox"], case.J, case.V, args.dtype,
                              case.J if args.dtype == "fp8" else 0)
    pair = {"timing": f"median of {reps} passes each", "dt_g_ms": round(t_dt, 4),
            "dt_g_gbs": round(b_dt / t_dt / 1e6, 1), "d_x_ms": round(t_d, 4),
            "d_x_gbs": round(b_d / t_d / 1e6, 1), "pair_gbs": round((b_dt + b_d) / (t_dt + t_d) / 1e6, 1),
            "pair_frac": round((b_dt + b_d) / (t_dt + t_d) / 1e6 / peaks["hbm_gbs"], 4),
            "pair_frac_of_nominal": round((b_dt + b_d) / (t_dt + t_d) / 1e6 / roofline.HBM_NOMINAL_GBS, 4)}

    # end to end through the C ABI with host buffers: H2D of the COO, build, plan, D2H of the results
    dose_h = torch.empty(case.V, dtype=torch.float32).pin_memory()
    e2e_times, e2e_parts = [], []
    for it in range(1 + args.e2e_steps):
        torch.cuda.synchronize()
        t_a = time.perf_counter()
        h2 = api.ddc_load_coo(case.V, case.J, vox_h, blt_h, val_h)
        torch.cuda.synchronize()
        t_b = time.perf_counter()
        # the SpMV configurations the autotuner chose for the resident handle (tuned once per machine)
        api.ddc_build(h2, args.dtype, tile_cfg=int(info["cfg_D"]), tile_cfg_Dt=cfg_dt,
                      index16=args.index16, vox_grid=grid)
        torch.cuda.synchronize()
        t_c = time.perf_counter()
        F2, st2 = api.cg_plan(h2, case.mlc, vox, n_ap, cps_out=cps, leaves_out=lv, y_out=y, dose_out=dose_h)
        torch.cuda.synchronize()
        t_d = time.perf_counter()
        e2e_times.append(t_d - t_a)
        e2e_parts.append((t_b - t_a, t_c - t_b, t_d - t_c))
        api.ddc_free(h2)
    timed = e2e_times[1:] or e2e_times  # the first call pays one-time set-up; time the rest
    e2e_local = sum(timed) / len(timed)
    e2e_s = max_over_ranks(e2e_local, world)
    # bytes copied per step by the whole job (every rank copies its own inputs and results)
    h2d = int(sum_over_ranks(12 * case.nnz, world))
    d2h = int(sum_over_ranks(cps.numel() * 4 + lv.numel() * 2 + y.numel() * 4 + dose_h.numel() * 4, world))
    e2e = {"value": round(whole_job_gbs(bytes_step, e2e_local, world), 1), "unit": "GB/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_s * 1e3, 2),
           "parts_ms": dict(zip(("coo_upload", "ddc_build", "cg_plan_and_readback"),
                                (round(1e3 * sum(p[i] for p in e2e_parts[1:] or e2e_parts) /
                                       len(e2e_parts[1:] or e2e_parts), 2) for i in range(3)))),
           "includes": "COO host->device, ddc_build (with the SpMV configurations tuned once on this GPU), "
                       "cg_plan, results device->host"}

    out = None
    forms = None
    if rank == 0 and world == 1 and args.forms != "none":
        api.ddc_free(h)  # room for the forms' matrices
        h = None
        forms = {}
        try:
            forms["precision"] = precision_form(dev)
        except Exception as e:  # the headline line stands without it
            forms["precision"] = {"error": repr(e)[:400]}
        if args.forms == "full":
            try:
                b = batch_measure("cfg5", "bf16", 1, 1)
                forms["batching"] = {k: b[k] for k in ("workload", "n_plans", "nnz", "dtype", "batched",
                                                       "one_by_one", "speedup", "F_rel_diff_max")}
            except Exception as e:
                forms["batching"] = {"error": repr(e)[:400]}
    if rank == 0:
        cpu = cpu_baseline(1, 0) if world == 1 and not args.no_cpu else None
        st = stats_all[-1]
        out = {
            "metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.dtype == "f32" else args.dtype, "data": "synthetic",
            "config": {"workload": f"{args.workload} {DESCS[args.workload]}", "V": case.V, "J": case.J, "nnz": case.nnz,
                       "n_active_vox": info["n_active_vox"], "n_apertures": n_ap, "storage": args.dtype,
                       "dt_column_order": "4x4x2 voxel bricks" if info["vox_brick"] else "voxel",
                       "interdigitation": bool(args.interdig),
                       "machine": dataclasses_asdict(case.mlc.machine),
                       "l2": "inputs larger than L2 (CSR D + D^T %.1f GB)" % ((info["bytes_D"] + info["bytes_Dt"]) / 1e9),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roof,
            "cpu_baseline": None if cpu is None else cpu_block(cpu),
            "e2e": e2e, "clocks": clk, "gpu_launches": int(launches),
            "plan": {"F": Fs[-1], "F_spread": max(Fs) - min(Fs), "apertures": st["n_apertures"],
                     "stop": st["stop"], "bb_iters": st["bb_iters_total"],
                     "pp1_window_frac": round(st["pp1_spmv_bytes"] / max(st["pp1_full_bytes"], 1.0), 4),
                     "phases_ms": {k: round(st[k], 3) for k in
                                   ("t_pp1_ms", "t_pp2_ms", "t_da_ms", "t_mp_ms", "t_final_ms", "t_total_ms")},
                     "build_ms": round(info["build_ms"], 1)},
            "spmv_pair": pair,
            "mp_roofline": mp_roof,
            "paper_context": PAPER_CONTEXT,
            "forms": forms,
        }
        out["plan"]["dose_err"] = dose_err
    if h is not None:
        api.ddc_free(h)
    return out


def run_spmv_only(args):
    """Profiling driver: build the workload's DDC, then 3 x (D^T g, D x)."""
    import numpy as np
    import torch
    import synth
    from paper_1503_01721_gb300 import api
    import __graft_entry__

    from paper_1503_01721_gb300 import roofline

    __graft_entry__.build()
    case = synth.make_case(args.workload, seed=0, cache=False)
    d = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)
    coo = (d(case.vox, torch.int32), d(case.blt, torch.int32), d(case.val, torch.float32))
    grid = vox_grid(case) if args.vox_order == "brick" else None
    g = torch.rand(case.V, device="cuda")
    x = torch.rand(case.J, device="cuda")
    pi = torch.empty(case.J, device="cuda")
    dd = torch.empty(case.V, device="cuda")
    out = {"mode": "spmv", "vox_order": args.vox_order, "workload": args.workload, "nnz": case.nnz, "dtype": args.dtype, "configs": {}}
    from paper_1503_01721_gb300 import _lib
    for cfg in (range(api.spmv_config_count()) if args.sweep else [args.tile_cfg]):
        z = cfg in INDEX16_CFGS
        try:
            ddc = api.Ddc(case.V, case.J, *coo, dtype=args.dtype, tile_cfg=cfg, index16=z or args.index16,
                          vox_grid=grid)
        except _lib.VmatError:
            if not z:
                raise
            try:  # CSR(D) without a 16-bit index: time D^T g alone
                ddc = api.Ddc(case.V, case.J, *coo, dtype=args.dtype, tile_cfg=cfg, index16=True, build_D=False,
                              vox_grid=grid)
            except _lib.VmatError as e:
                out["configs"][cfg] = {"unavailable": str(e)}
                continue
        info = ddc.info()
        has_d = bool(info["built_D"])
        for _ in range(3):
            api.beamlet_price(ddc.h, g, pi)
            if has_d:
                api.dose_forward(ddc.h, x, dd)
        torch.cuda.synchronize()
        if args.sweep:
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record()
            for _ in range(10):
                api.beamlet_price(ddc.h, g, pi)
            ev[1].record()
            for _ in range(10 if has_d else 0):
                api.dose_forward(ddc.h, x, dd)
            ev[2].record()
            torch.cuda.synchronize()
            sc = case.J if args.dtype == "fp8" else 0
            # chunk counts from the index sizes (2 bytes per nonzero, 4 per chunk, 8 per row pointer)
            chunks = lambda b16, rows: (b16 - 2 * case.nnz - 8 * (rows + 1)) // 4
            if z:
                b_t = roofline.spmv_bytes_index16(case.nnz, chunks(info["bytes16_Dt"], case.J), case.J, case.V,
                                                  case.J, args.dtype, sc)
            else:
                b_t = roofline.spmv_bytes(case.nnz, case.J, case.V, case.J, args.dtype, sc)
            t_t = ev[0].elapsed_time(ev[1]) / 10
            rec = {"dt_g_gbs": round(b_t / t_t / 1e6, 1), "dt_g_ms": round(t_t, 4), "dt_g_bytes": b_t}
            if has_d:
                if z:
                    nr = info["n_active_vox"]
                    b_d = roofline.spmv_bytes_index16(case.nnz, chunks(info["bytes16_D"], nr), nr, case.J, case.V,
                                                      args.dtype, sc)
                else:
                    b_d = roofline.spmv_bytes(case.nnz, info["n_active_vox"], case.J, case.V, args.dtype, sc)
                t_d = ev[1].elapsed_time(ev[2]) / 10
                rec.update({"d_x_gbs": round(b_d / t_d / 1e6, 1), "d_x_ms": round(t_d, 4)})
            else:
                rec["d_x"] = "CSR(D) holds no 16-bit index (a chunk spans 65,536 columns or more)"
            out["configs"][cfg] = rec
        ddc.close()
    return out


def run_mp_only(args):
    """Master-problem driver: fixed-length BB solves (stopping rules off) on DA built
    from seeded random apertures, for several aperture counts."""
    import numpy as np
    import torch
    import synth
    from paper_1503_01721_gb300 import api
    import __graft_entry__

    __graft_entry__.build()
    case = synth.make_case(args.workload, seed=0, cache=False)
    d = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)
    ddc = api.Ddc(case.V, case.J, d(case.vox, torch.int32), d(case.blt, torch.int32), d(case.val, torch.float32),
                  dtype=args.dtype, build_Dt=False)
    vox = api.VoxelParams.from_numpy(case.structs)
    out = {"mode": "mp", "workload": args.workload, "V": case.V, "sizes": {}}
    iters = 60
    opts = api.BBOptions(max_iter=iters, rel_tol5=0.0, step_tol=0.0)
    for n in (8, 30, 60):
        cps, leaves, _ = synth.random_apertures(case.mlc, n, n, 8, 40)
        DA = torch.empty(n, case.V, device="cuda")
        for k in range(n):
            api.aperture_dose(ddc.h, case.mlc, int(cps[k]), d(leaves[k], torch.int16), DA[k])
        DA.mul_(0.02)  # doses near the prescriptions
        z = torch.empty(case.V, device="cuda")
        y = torch.zeros(n, device="cuda")
        api.mp_bb_solve(DA, vox, y, z, opts=opts)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        y.zero_()
        rep = api.mp_bb_solve(DA, vox, y, z, opts=opts)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        b = rep["iters"] * (4.0 * n * case.V + 9.0 * case.V)
        out["sizes"][n] = {"iters": rep["iters"], "ms_per_iter": round(dt * 1e3 / rep["iters"], 4),
                           "gbs": round(b / dt / 1e9, 1), "DA_MB": round(4 * n * case.V / 1e6, 1)}
    ddc.close()
    return out


def run_batch(args):
    import __graft_entry__
    __graft_entry__.build()
    return batch_measure(args.workload, args.dtype, args.steps, args.warmup)


def batch_measure(workload, dtype, steps, warmup):
    """Batched plans: every plan of a batch workload resident in HBM, then timed
    runs of the whole batch (one CUDA graph per run) against the same plans run one
    after another through cg_plan.  Aggregate GB/s = the algorithmic bytes of every
    plan's D^T g and final D x passes over the wall time."""
    import numpy as np
    import torch
    import synth
    from paper_1503_01721_gb300 import api, roofline

    specs = synth.batch_specs(workload)
    plans, keep, nnz = [], [], 0
    t0 = time.time()
    for sp in specs:
        c = synth.make_plan_case(sp)
        h = api.ddc_load_coo(c.V, c.J, torch.from_numpy(c.vox), torch.from_numpy(c.blt), torch.from_numpy(c.val))
        api.ddc_build(h, dtype, vox_grid=vox_grid(c))
        vox = api.VoxelParams.from_numpy(c.structs)
        plans.append((h, c.mlc, vox, sp.n_apertures))
        keep.append(c.mlc)
        nnz += c.nnz
        del c
    log(f"[batch] {len(specs)} plans, {nnz} nonzeros resident in {time.time() - t0:.1f}s")
    batch = api.Batch(plans)
    info = batch.info()
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        batch.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        Fb, stb = batch.run()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_batch = e0.elapsed_time(e1) / steps
    bytes_run = sum(s["pp1_spmv_bytes"] + s["other_spmv_bytes"] for s in stb)
    # the same plans one after another
    for h, mlc, vox, n in plans:
        api.cg_plan(h, mlc, vox, n)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        Fs, sts = [], []
        for h, mlc, vox, n in plans:
            F, st = api.cg_plan(h, mlc, vox, n)
            Fs.append(F)
            sts.append(st)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1) / steps
    bytes_seq = sum(s["pp1_spmv_bytes"] + s["other_spmv_bytes"] for s in sts)
    rel = [abs(a - b) / max(abs(b), 1e-30) for a, b in zip(Fb, Fs)]
    peaks = roofline.measured_peaks()
    out = {"mode": "batch", "workload": workload, "n_plans": len(specs), "nnz": nnz, "dtype": dtype,
           "batched": {"ms_per_run": round(ms_batch, 3), "gbs": round(bytes_run / ms_batch / 1e6, 1),
                       "frac_of_hbm": round(bytes_run / ms_batch / 1e6 / peaks["hbm_gbs"], 4)},
           "one_by_one": {"ms_per_run": round(ms_seq, 3), "gbs": round(bytes_seq / ms_seq / 1e6, 1)},
           "speedup": round(ms_seq / ms_batch, 3), "bb_iters": sum(s["bb_iters_total"] for s in stb),
           "apertures": [s["n_apertures"] for s in stb], "F_rel_diff_max": max(rel),
           "info": {k: v for k, v in info.items()}}
    batch.close()
    for h, _, _, _ in plans:
        api.ddc_free(h)
    return out


def run_truncation(args):
    """The paper's method S1 (Section 2.4): plan on a DDC truncated to a radius about
    each beamlet axis (1.25 voxels keeps about a quarter of the entries, as the
    paper's 2.5 cm against 6 cm did), then evaluate that plan's dose on the full
    DDC, beside the plan optimised on the full DDC."""
    import numpy as np
    import torch
    import synth
    from paper_1503_01721_gb300 import api
    import __graft_entry__

    __graft_entry__.build()
    radius = 1.25
    full = synth.make_case(args.workload, seed=0, cache=False)
    tr = synth.make_truncated_case(args.workload, radius, seed=0)
    n = full.n_apertures
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)
    ddcs = {}
    for tag, c in (("full", full), ("trunc", tr)):
        ddcs[tag] = api.Ddc(c.V, c.J, dev(c.vox, torch.int32), dev(c.blt, torch.int32), dev(c.val, torch.float32),
                            dtype=args.dtype, autotune=True,
                            vox_grid=vox_grid(c) if args.vox_order == "brick" else None)
    vox = api.VoxelParams.from_numpy(full.structs)
    out = {"mode": "truncation", "workload": args.workload, "radius_vox": radius, "dtype": args.dtype,
           "nnz_full": full.nnz, "nnz_trunc": tr.nnz, "nnz_ratio": round(tr.nnz / full.nnz, 4)}
    res = {}
    for tag, c in (("full", full), ("trunc", tr)):
        cps = torch.empty(n, dtype=torch.int32)
        lv = torch.empty(n * c.mlc.n_rows * 2, dtype=torch.int16)
        y = torch.empty(n, dtype=torch.float32)
        dose = torch.empty(c.V, device="cuda")
        for _ in range(max(args.warmup, 1)):
            api.cg_plan(ddcs[tag].h, c.mlc, vox, n)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            F, st = api.cg_plan(ddcs[tag].h, c.mlc, vox, n, cps_out=cps, leaves_out=lv, y_out=y, dose_out=dose)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / args.steps
        res[tag] = (F, st, cps.clone(), lv.clone(), y.clone(), dose.clone(), ms)
    # the truncated plan's dose on the full matrix
    _, st_t, cps, lv, y, dose_model, _ = res["trunc"]
    m = st_t["n_apertures"]
    x = torch.empty(full.J, device="cuda")
    api.aperture_fluence(full.mlc, cps[:m].cuda(), lv[:m * full.mlc.n_rows * 2].cuda(), y[:m].cuda(), x)
    dose_true = torch.empty(full.V, device="cuda")
    api.dose_forward(ddcs["full"].h, x, dose_true)
    F_true = torch.empty(1, dtype=torch.float64, device="cuda")
    api.objective_grad(dose_true, vox, None, F_true)
    s = full.structs
    targets = [k for k in range(len(s.T)) if s.w_under[k] > 0]
    ptv = np.isin(s.struct_id, targets)
    T = s.T[s.struct_id]
    dm, dt, df = dose_model.cpu().numpy(), dose_true.cpu().numpy(), res["full"][5].cpu().numpy()
    out.update({
        "full_plan": {"F": res["full"][0], "ms": round(res["full"][6], 2), "bb_iters": res["full"][1]["bb_iters_total"],
                      "ptv_frac_over_110pct": round(float(np.mean(df[ptv] > 1.1 * T[ptv])), 4)},
        "trunc_plan": {"F_on_truncated": res["trunc"][0], "F_on_full": F_true.item(), "ms": round(res["trunc"][6], 2),
                       "bb_iters": st_t["bb_iters_total"],
                       "ptv_mean_dose_increase": round(float(np.mean((dt[ptv] - dm[ptv]) / T[ptv])), 4),
                       "ptv_frac_over_110pct": round(float(np.mean(dt[ptv] > 1.1 * T[ptv])), 4)},
        "speedup_trunc_over_full": round(res["full"][6] / res["trunc"][6], 3),
    })
    for d in ddcs.values():
        d.close()
    return out


def run_reference(args, rank, world):
    """The FP64 CPU oracle (the only reference that exists) on the machine's host cores: each
    step is one sample plan in every one of host_cores() single-threaded processes."""
    if rank != 0:
        return None
    import shutil
    path = _sample_dir()
    try:
        prepare_cpu_sample(path)
        res = run_oracle_procs(path, host_cores(), args.steps, args.warmup)
    finally:
        shutil.rmtree(path, ignore_errors=True)
    return {"impl": "reference", "metric": METRIC, "value": round(res["value"], 4), "unit": "GB/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(res["sec_per_plan"] * 1e3, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD} {WORKLOAD_DESC}", "sample": sample_desc(res)},
            "cpu_baseline": {"value": round(res["value"], 4), "unit": "GB/s", "cores": res["procs"],
                             "kind": "oracle", "sample": sample_desc(res)},
            "e2e": {"value": round(res["value"], 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "fp8"])
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--forms", default="full", choices=["full", "precision", "none"],
                    help="after the headline plan (one GPU): the precision form on the two-arc case and, with "
                         "full, the 24-plan BF16 batch against the same plans one by one")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(DESCS) + ["cfg5", "cfg5q", "batch_small"])
    ap.add_argument("--mode", default="plan", choices=["plan", "spmv", "mp", "batch", "truncation"],
                    help="spmv: only build and run D^T g and D x a few times (profiling driver); "
                         "mp: fixed-length master-problem solves; batch: a batch workload (cfg5, cfg5q, "
                         "batch_small) batched against one by one; truncation: the paper's truncated-matrix "
                         "plan evaluated on the full matrix")
    ap.add_argument("--sweep", action="store_true", help="spmv mode: time every SpMV configuration")
    ap.add_argument("--tile-cfg", type=int, default=-1, help="SpMV configuration (-1 = library default)")
    ap.add_argument("--vox-order", default="brick", choices=["brick", "voxel"],
                    help="column order of CSR(D^T): 4x4x2 voxel bricks (default) or the grid's voxel order")
    ap.add_argument("--interdig", action="store_true", help="plan mode: price with the interdigitation constraint")
    ap.add_argument("--index16", action="store_true",
                    help="also build the 16-bit column index (the autotuner then times configurations 12-14)")
    ap.add_argument("--machine", action="store_true",
                    help="plan mode: fluence-rate bounds from gantry-speed, dose-rate and leaf-speed limits")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours" and args.mode == "plan":
        log("note: fewer than 3 warm-up steps")
    rank, world, local = dist_setup(args.gpus)
    if args.mode == "spmv":
        out = run_spmv_only(args) if rank == 0 else None
    elif args.mode == "mp":
        out = run_mp_only(args) if rank == 0 else None
    elif args.mode == "batch":
        out = run_batch(args) if rank == 0 else None
    elif args.mode == "truncation":
        out = run_truncation(args) if rank == 0 else None
    else:
        out = run_reference(args, rank, world) if args.impl == "reference" else run_ours(args, rank, world, local)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
