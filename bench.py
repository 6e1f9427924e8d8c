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
# DRAM traffic over algorithmic bytes of the full D^T g pass on the 128x128x96 case, per (value type,
# configuration): dram__bytes_read.sum + dram__bytes_write.sum from one ncu capture of each kernel.
# The plan's passes are windowed: their ratio is WINDOWED_TRAFFIC_RATIO, measured on a windowed
# launch of the plan; a configuration without such a capture reports null.
WINDOWED_TRAFFIC_RATIO = {("f32", 11): 1.0103}
TRAFFIC_RATIO = {("f32", 4): 1.0055, ("f32", 5): 1.0063, ("f32", 6): 1.0032, ("f32", 7): 1.0036,
                 ("f32", 8): 1.0008, ("f32", 9): 1.0101, ("f32", 10): 1.0082, ("f32", 11): 1.0091,
                 ("bf16", 5): 1.0083, ("fp8", 5): 1.0082,
                 # 16-bit index, on the 45-CP case
                 ("f32", 12): 1.0044}
# CPU sample: every 12th CP of the same geometry (15 CPs), 5 apertures
SAMPLE_CP_STRIDE = 12
SAMPLE_APERTURES = 5


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


def run_oracle_steps(steps, warmup):
    """Time the FP64 oracle's column generation on the CPU sample (one thread)."""
    import numpy as np
    import oracle
    from paper_1503_01721_gb300 import roofline
    V, J, vox, blt, val, structs, mlc = sample_case()
    D = oracle.ddc_matrix(V, J, vox, blt, val)
    nnz = len(val)
    n_rows_D = int(np.count_nonzero(np.bincount(vox, minlength=V)))
    times, gbytes = [], 0.0
    for it in range(warmup + steps):
        t0 = time.perf_counter()
        plan = oracle.cg_plan(D, mlc, structs, SAMPLE_APERTURES)
        dt = time.perf_counter() - t0
        if it >= warmup:
            times.append(dt)
    # bytes of the plan's sparse passes in the GPU's FP32-CSR byte model: each pricing pass counts
    # the beamlet rows inside the leaf-travel windows of the unoccupied CPs (the prices pricing reads),
    # as the GPU's windowed pass does, plus g and the window table; then the final D x
    per_blt = np.bincount(blt, minlength=J).reshape(mlc.K, mlc.n_rows, mlc.n_cols)
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
    b += roofline.spmv_bytes(nnz, n_rows_D, J, V)
    per_step = sum(times) / len(times)
    return {"value": b / per_step / 1e9, "sec_per_plan": per_step, "nnz": nnz, "J": J, "V": V,
            "apertures": len(plan.cps), "F": plan.F}


def cpu_baseline_subprocess(steps=1, warmup=0):
    """Run the oracle sample in a fresh single-threaded process (no CUDA in it)."""
    # the timed oracle is single-threaded (scipy sparse products, BLAS pinned to one
    # thread); the untimed input generator keeps its OpenMP threads
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="",
               VMAT_ORACLE_SUBPROCESS="1")
    code = (f"import sys, json; sys.path.insert(0, {ROOT!r}); import bench; "
            f"print(json.dumps(bench.run_oracle_steps({steps}, {warmup})))")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed:\n" + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def sample_desc(res):
    return (f"FP64 oracle cg_plan, {SAMPLE_APERTURES} apertures, on every {SAMPLE_CP_STRIDE}th CP of the "
            f"{WORKLOAD} geometry ({res['J']} beamlets, {res['nnz']} nonzeros); same byte model (rows inside "
            f"the leaf-travel windows per pricing pass)")


# ----------------------------------------------------------------------------- GPU arm

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
    api.ddc_build(h, args.dtype, tile_cfg=args.tile_cfg, autotune=args.tile_cfg < 0, index16=args.index16)
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
    cfg_dt = int(info["cfg_Dt"])
    kname = SPMV_KERNELS.get(cfg_dt, f"spmv configuration {cfg_dt}") + \
        (" + spmv_fixup" if info["tile_nnz_Dt"] else "") + " (beamlet price D^T g over the unoccupied CPs)"
    bytes_launch = spmv_bytes / max(spmv_n, 1)
    ratio = WINDOWED_TRAFFIC_RATIO.get((args.dtype, cfg_dt))
    roof = {"bound": "hbm", "kernel": kname,
            "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": round(achieved / peaks["hbm_gbs"], 4),
            "traffic": None if ratio is None else round(ratio * bytes_launch),
            "traffic_source": None if ratio is None else
            f"ncu dram bytes / algorithmic bytes = {ratio} for this kernel on a windowed D^T g launch of the "
            "plan, times this launch's algorithmic bytes",
            "peak_source": peaks["source"], "frac_of_nominal": round(achieved / roofline.HBM_NOMINAL_GBS, 4),
            "nominal_peak": roofline.HBM_NOMINAL_GBS, "bytes_per_launch": round(bytes_launch),
            "avg_launch_ms": round(spmv_ms / max(spmv_n, 1), 4)}

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
        api.ddc_build(h2, args.dtype, tile_cfg=int(info["cfg_D"]), tile_cfg_Dt=int(info["cfg_Dt"]),
                      index16=args.index16)
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
    if rank == 0:
        cpu = cpu_baseline_subprocess(1, 0) if world == 1 and not args.no_cpu else None
        st = stats_all[-1]
        out = {
            "metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.dtype == "f32" else args.dtype, "data": "synthetic",
            "config": {"workload": f"{args.workload} {DESCS[args.workload]}", "V": case.V, "J": case.J, "nnz": case.nnz,
                       "n_active_vox": info["n_active_vox"], "n_apertures": n_ap, "storage": args.dtype,
                       "interdigitation": bool(args.interdig),
                       "machine": dataclasses_asdict(case.mlc.machine),
                       "l2": "inputs larger than L2 (CSR D + D^T %.1f GB)" % ((info["bytes_D"] + info["bytes_Dt"]) / 1e9),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roof,
            "cpu_baseline": None if cpu is None else {
                "value": round(cpu["value"], 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                "sample": sample_desc(cpu), "sec_per_plan": round(cpu["sec_per_plan"], 3)},
            "e2e": e2e, "clocks": clk, "gpu_launches": int(launches),
            "plan": {"F": Fs[-1], "F_spread": max(Fs) - min(Fs), "apertures": st["n_apertures"],
                     "stop": st["stop"], "bb_iters": st["bb_iters_total"],
                     "pp1_window_frac": round(st["pp1_spmv_bytes"] / max(st["pp1_full_bytes"], 1.0), 4),
                     "phases_ms": {k: round(st[k], 3) for k in
                                   ("t_pp1_ms", "t_pp2_ms", "t_da_ms", "t_mp_ms", "t_final_ms", "t_total_ms")},
                     "build_ms": round(info["build_ms"], 1)},
            "spmv_pair": pair,
        }
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
    g = torch.rand(case.V, device="cuda")
    x = torch.rand(case.J, device="cuda")
    pi = torch.empty(case.J, device="cuda")
    dd = torch.empty(case.V, device="cuda")
    out = {"mode": "spmv", "workload": args.workload, "nnz": case.nnz, "dtype": args.dtype, "configs": {}}
    from paper_1503_01721_gb300 import _lib
    for cfg in (range(api.spmv_config_count()) if args.sweep else [args.tile_cfg]):
        z = cfg in INDEX16_CFGS
        try:
            ddc = api.Ddc(case.V, case.J, *coo, dtype=args.dtype, tile_cfg=cfg, index16=z or args.index16)
        except _lib.VmatError:
            if not z:
                raise
            try:  # CSR(D) without a 16-bit index: time D^T g alone
                ddc = api.Ddc(case.V, case.J, *coo, dtype=args.dtype, tile_cfg=cfg, index16=True, build_D=False)
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
    """Batched plans: every plan of a batch workload resident in HBM, then timed
    runs of the whole batch (one CUDA graph per run) against the same plans run one
    after another through cg_plan.  Aggregate GB/s = the algorithmic bytes of every
    plan's D^T g and final D x passes over the wall time."""
    import numpy as np
    import torch
    import synth
    from paper_1503_01721_gb300 import api, roofline
    import __graft_entry__

    __graft_entry__.build()
    dtype = args.dtype
    specs = synth.batch_specs(args.workload)
    plans, keep, nnz = [], [], 0
    t0 = time.time()
    for sp in specs:
        c = synth.make_plan_case(sp)
        h = api.ddc_load_coo(c.V, c.J, torch.from_numpy(c.vox), torch.from_numpy(c.blt), torch.from_numpy(c.val))
        api.ddc_build(h, dtype)
        vox = api.VoxelParams.from_numpy(c.structs)
        plans.append((h, c.mlc, vox, sp.n_apertures))
        keep.append(c.mlc)
        nnz += c.nnz
        del c
    log(f"[batch] {len(specs)} plans, {nnz} nonzeros resident in {time.time() - t0:.1f}s")
    batch = api.Batch(plans)
    info = batch.info()
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        batch.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        Fb, stb = batch.run()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_batch = e0.elapsed_time(e1) / args.steps
    bytes_run = sum(s["pp1_spmv_bytes"] + s["other_spmv_bytes"] for s in stb)
    # the same plans one after another
    for h, mlc, vox, n in plans:
        api.cg_plan(h, mlc, vox, n)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        Fs, sts = [], []
        for h, mlc, vox, n in plans:
            F, st = api.cg_plan(h, mlc, vox, n)
            Fs.append(F)
            sts.append(st)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1) / args.steps
    bytes_seq = sum(s["pp1_spmv_bytes"] + s["other_spmv_bytes"] for s in sts)
    rel = [abs(a - b) / max(abs(b), 1e-30) for a, b in zip(Fb, Fs)]
    peaks = roofline.measured_peaks()
    out = {"mode": "batch", "workload": args.workload, "n_plans": len(specs), "nnz": nnz, "dtype": dtype,
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
                            dtype=args.dtype, autotune=True)
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
    if rank != 0:
        return None
    res = cpu_baseline_subprocess(args.steps, args.warmup)
    return {"impl": "reference", "metric": METRIC, "value": round(res["value"], 4), "unit": "GB/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(res["sec_per_plan"] * 1e3, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD} {WORKLOAD_DESC}", "sample": sample_desc(res)},
            "cpu_baseline": {"value": round(res["value"], 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": sample_desc(res)},
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
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(DESCS) + ["cfg5", "cfg5q", "batch_small"])
    ap.add_argument("--mode", default="plan", choices=["plan", "spmv", "mp", "batch", "truncation"],
                    help="spmv: only build and run D^T g and D x a few times (profiling driver); "
                         "mp: fixed-length master-problem solves; batch: a batch workload (cfg5, cfg5q, "
                         "batch_small) batched against one by one; truncation: the paper's truncated-matrix "
                         "plan evaluated on the full matrix")
    ap.add_argument("--sweep", action="store_true", help="spmv mode: time every SpMV configuration")
    ap.add_argument("--tile-cfg", type=int, default=-1, help="SpMV configuration (-1 = library default)")
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
