#!/usr/bin/env python3
"""Throughput of the AAHRT operator pair inside the FISTA sparse solve.

Default workload (the batched form): 512 CMP cubes (nt = 1001 at 4 ms, fold
200-3000 in 90-360 degree sectors of a 3 km disc, 64 curvatures x 24
azimuths) in one autotuned plan; one step = one 50-iteration FISTA solve of
every cube, each with its own step and threshold (each iteration is one
forward + adjoint pair with the residual and the shrinkage/momentum update
fused).  value = cube-pairs/s over the whole job; gathers/s is the rate of
whole cube solves.  Inputs are resident in HBM for `value` (26 GB of spectra,
far beyond L2, and L2 is flushed between timed steps); `e2e` passes pinned
host buffers to the C ABI so the host<->device copies of d and m are inside
the timed region.  The same JSON line carries, under "gather", the line of
the paper-scale single gather (nt = 1001, 2000 traces in a 3 km disc, 100
curvatures x 36 azimuths; one step = one 100-iteration FISTA solve) and, on
one GPU, under "slowness" and "shared64", the lines of the two workloads
below (the shared-geometry one with at most 5 timed steps).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload batch512|gather|slowness|table1|shared64]

--workload gather times the single gather alone.

--workload slowness times the same gather and solve on a uniform slowness
axis (100 slownesses 1/3500..1/1500 s/m, so the curvatures q = p^2 are not
uniform): the slice step is the direct sum of the DFT along q (a type-3
DFT), whose roofline is the special-function rate of the phases.

--workload shared64 times 64 gathers sharing one 8000-trace geometry: the
split-BF16 tensor-core plan of all 64, the FP32 plan of all 64, and one
single-gather FP32 plan applied to the 64 gathers in turn.

Under torchrun each rank runs an independent replica on its own GPU (the
path needs no communication); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("AAHRT fwd+adj pairs/s and FISTA gathers/s on 1 GB300, %HBM roofline, "
          "err vs FP64")
ITERS = 100
WORKLOAD = ("paper-scale gather: nt=1001 dt=4ms, 2000 traces in a 3 km disc, "
            "100 q x 36 azimuths; one step = one 100-iteration FISTA solve")
SLOW_WORKLOAD = ("paper-scale gather on a uniform slowness axis: nt=1001 dt=4ms, 2000 traces "
                 "in a 3 km disc, 100 slownesses 1/3500..1/1500 s/m (non-uniform q) x 36 "
                 "azimuths, direct-sum slice step; one step = one 100-iteration FISTA solve")
BATCH_ITERS = 50
BATCH_WORKLOAD = ("512 CMP cubes: nt=1001 dt=4ms, fold 200-3000 in 90-360 degree sectors "
                  "of a 3 km disc, 64 q x 24 azimuths, one autotuned plan; one step = one "
                  "50-iteration FISTA solve of every cube (per-cube step and threshold)")
NESTED_STEPS = 5
L2_NOTE = "inputs far larger than L2 (spectra of tens of GB), and L2 flushed (256 MB write)"
L2_NOTE_GATHER = "L2 flushed between timed steps (256 MB write)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="batch512",
                    choices=["gather", "batch512", "slowness", "table1", "shared64"])
    ap.add_argument("--oracle-single-core", default=None, help=argparse.SUPPRESS)
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_seed(base, rank):
    """Seed of rank's synthetic workload: every rank solves its own gather
    (or batch) -- independent replicas, no data exchange between ranks."""
    return base + rank


def job_rate(local_ms, units_per_rank, world, device):
    """Whole-job rate of independent replicas: the units all ranks processed
    divided by the slowest rank's time (MAX over ranks; every rank returns
    the same pair)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return units_per_rank * world / (ms / 1e3), ms


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    mhz.append(float(parts[1]))
                    mx = float(parts[2])
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not mhz:
            return None
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": mx, "samples": len(mhz),
                "reasons": sorted(reasons)}


def stage_bytes(info):
    """Algorithmic bytes per launch of each stage of the staged (unfused)
    FISTA iteration: each stage reads its input once and writes its output
    once.  Their sum is the implementation-independent bytes per iteration."""
    m, d = 4 * info.model_len, 4 * info.data_len
    x, y = 8 * info.xspec_len, 8 * info.yspec_len
    return [m + x,            # 0 stretch + FFT (model side)
            x + y,            # 1 slice forward
            y + 2 * d,        # 2 inverse FFT + unstretch, residual d - Lz fused
            d + y,            # 3 unstretch^T + FFT (data side)
            y + x,            # 4 slice adjoint
            x + 4 * m,        # 5 inverse FFT + stretch^T, FISTA update fused (m, z in/out)
            0]


def launch_bytes(info, launches, iters_total):
    """Algorithmic bytes per launch of the kernels the solve actually ran.
    When the solver fuses each time-domain half-iteration (no launches of
    stage 3), stage 2 is synthesis + residual + U^T + FFT (reads Y and d,
    writes Y) and stage 5 is synthesis + update + stretch + FFT of the new z
    (reads X, m, z, writes m, z, X) on all but the last iteration."""
    sb = stage_bytes(info)
    if launches[3] == 0 and launches[2] > 0:
        m, d = 4 * info.model_len, 4 * info.data_len
        x, y = 8 * info.xspec_len, 8 * info.yspec_len
        sb[2] = 2 * y + d
        n5 = max(launches[5], 1)
        fused5 = max(n5 - (launches[0] or 0), 0)      # one unfused update per solve
        sb[5] = int(x + 4 * m + x * fused5 / n5)
    return sb


def traffic_record(stage):
    """The committed ncu record of a stage's kernel (DRAM bytes per launch
    and, where taken, issue and FMA-pipe fractions), if the files that define
    that kernel (its source, the headers it includes and the plan code that
    sizes its launch) still hash to the ones the counters were taken on."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path)).get("kernels", {}).get(stage)
        if rec is None:
            return None
        h = hashlib.sha256()
        for f in rec["files"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        if rec.get("sha256") != h.hexdigest():
            return None
        return rec
    except Exception:
        return None


# ------------------------------------------------------------- workloads
def batch_geometry(seed):
    """The 512 cubes' geometry (no data) and the batch-wide largest squared
    offset that fixes their shared stretched-time plan."""
    import numpy as np
    from paper_2505_00387_gb300 import synthetic as syn
    geo = syn.cube_batch(seed=seed, with_data=False)
    r2max = max(float(np.max(c.hx ** 2 + c.hy ** 2)) for c in geo)
    return geo, r2max


def fold_picks(folds, n):
    """n cubes spread evenly over the fold range (quantiles of the sorted
    folds)."""
    import numpy as np
    order = np.argsort(np.asarray(folds), kind="stable")
    return [int(order[int(round(q * (len(folds) - 1)))]) for q in np.linspace(0.0, 1.0, n)]


def workload_config(kind, world=1, geo=None, g=None):
    """The config object of a bench line: the workload only (sizes, iteration
    count, L2 treatment), the same for the GPU arm and the reference arm."""
    if kind == "batch512":
        folds = [c.ntr for c in geo]
        c0 = geo[0]
        return {"workload": BATCH_WORKLOAD, "ncube": len(geo), "nt": c0.nt, "dt": c0.dt,
                "fold_min": min(folds), "fold_max": max(folds),
                "traces_total": int(sum(folds)), "nq": c0.nq, "ntheta": c0.ntheta,
                "fista_iters_per_step": BATCH_ITERS, "l2": L2_NOTE,
                "parallelism": f"replicas x{world}"}
    cfg = {"workload": SLOW_WORKLOAD if kind == "slowness" else WORKLOAD, "nt": g.nt,
           "dt": g.dt, "ntr": g.ntr, "nq": g.nq, "ntheta": g.ntheta,
           "fista_iters_per_step": ITERS, "l2": L2_NOTE_GATHER,
           "parallelism": f"replicas x{world}"}
    if kind == "slowness":
        cfg["slice_step"] = "direct sum (type-3 DFT along q)"
    return cfg


# ------------------------------------------------------------------ ours
def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_info()
    if world > 1:
        dist.init_process_group(backend="nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2505_00387_gb300 import build as B
    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        dist.barrier()
    line = measure(args.workload, args, rank, world, dev)
    if args.workload == "batch512":
        # the paper-scale single gather, measured the same way in the same run
        line["gather"] = measure("gather", args, rank, world, dev)
        if world == 1:
            # one GPU: the other two workloads of the bench in the same run, the
            # gather on the uniform slowness axis and the 64 shared-geometry
            # gathers (at most NESTED_STEPS timed steps each)
            import torch
            torch.cuda.empty_cache()
            line["slowness"] = measure("slowness", args, rank, world, dev)
            torch.cuda.empty_cache()
            line["shared64"] = measure_shared64(args, rank, min(args.steps, NESTED_STEPS))
            torch.cuda.empty_cache()
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def measure(kind, args, rank, world, dev):
    """One bench line of workload `kind` (batch512, gather or slowness) on
    this rank's GPU; only rank 0's return value is complete."""
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2505_00387_gb300 import _lib as L
    from paper_2505_00387_gb300 import synthetic as syn
    from paper_2505_00387_gb300.plan import AahrtPlan

    batch = kind == "batch512"
    slow = kind == "slowness"
    qa = None
    g = cubes = None
    if batch:
        cubes = syn.cube_batch(seed=replica_seed(3, rank))
        gp = AahrtPlan.batched(cubes, autotune=True)
        d_np = np.concatenate([c.d.astype(np.float32).ravel() for c in cubes])
        iters, pairs_per_step = BATCH_ITERS, BATCH_ITERS * len(cubes)
    else:
        g = syn.paper_gather(seed=replica_seed(1, rank))
        if slow:
            from paper_2505_00387_gb300.plan import q_axis_slowness
            qa = q_axis_slowness(syn.P_MIN, syn.P_MAX, g.nq)
        gp = AahrtPlan(**g.geom_kwargs(), q_axis=qa)
        d_np = g.d.astype(np.float32).ravel()
        iters, pairs_per_step = ITERS, ITERS
    info = gp.info
    d = torch.from_numpy(d_np).to(dev)
    m = torch.zeros(gp.model_len, device=dev)
    stream = torch.cuda.current_stream()

    # step lengths and lambda = 0.05 max|L^T d| from the device (setup, untimed)
    if batch:
        cg = np.zeros(len(cubes))
        cl = np.zeros(len(cubes))
        gp.sparse_solve(d, 0.0, 0, m, lambda_rel=0.05, power_iters=30, per_cube=True,
                        cube_gamma=cg, cube_lambda=cl, want_info=False)
        lam, gamma = 0.0, 0.0
        kw = dict(per_cube=True, cube_gamma=cg, cube_lambda=cl)
    else:
        _, si = gp.sparse_solve(d, 0.0, 0, m, lambda_rel=0.05, power_iters=30)
        lam, gamma = float(getattr(si, "lambda")), float(si.gamma)
        kw = dict(gamma=gamma)

    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev)

    def step():
        gp.sparse_solve(d, lam, iters, m, use_graph=True, want_info=False, **kw)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    per_step = []

    def timed(fn, k):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(k)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for i in range(k):
            flush.zero_()
            ev[i][0].record(stream)
            fn()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        per_step.clear()
        per_step.extend(a.elapsed_time(b) for a, b in ev)
        return sum(per_step)

    t_launch0 = gp.stage_times()[1]
    sampler = ClockSampler(local_index(dev))
    sampler.start()
    total_ms = timed(step, args.steps)
    step_median_ms = statistics.median(per_step)
    clocks = sampler.stop()
    t_launch1 = gp.stage_times()[1]
    launches = int(sum(t_launch1[:6]) - sum(t_launch0[:6]))

    value, total_ms = job_rate(total_ms, args.steps * pairs_per_step, world, dev)

    # end to end: pinned host d in, pinned host m out, through the C ABI
    d_host = torch.from_numpy(d_np).pin_memory()
    m_host = torch.zeros(gp.model_len, dtype=torch.float32).pin_memory()
    if batch:
        import ctypes
        dp = ctypes.POINTER(ctypes.c_double)
        o = L.aahrt_solve_opts(0, 0, 0, 1, 0.0, 0.0, 1, cg.ctypes.data_as(dp),
                               cl.ctypes.data_as(dp))
    else:
        o = L.aahrt_solve_opts(0, 0, 0, 1, gamma, 0.0)

    def step_e2e():
        L.aahrt_sparse_solve(gp.handle, d_host.data_ptr(), lam, iters, m_host.data_ptr(), o,
                             False, int(stream.cuda_stream))

    step_e2e()
    torch.cuda.synchronize()
    e2e_steps = args.steps if not batch else min(args.steps, 5)
    e2e_ms = timed(step_e2e, e2e_steps)
    e2e_value, _ = job_rate(e2e_ms, e2e_steps * pairs_per_step, world, dev)

    # per-stage device time over the same kind of steps (eager launches,
    # CUDA events around every stage on the launching stream)
    gp.set_profiling(True)
    for _ in range(args.steps if not batch else min(args.steps, 2)):
        flush.zero_()
        gp.sparse_solve(d, lam, iters, m, use_graph=False, want_info=False, **kw)
    torch.cuda.synchronize()
    st_ms, st_n = gp.stage_times()
    gp.set_profiling(False)

    if rank != 0:
        return None
    config = workload_config(kind, world, geo=cubes, g=g)
    plan_desc = {"nfft": info.nfft, "nbins": info.nbins, "spread_width": info.spread_width,
                 "theta_group": info.theta_group, "time_pairs": info.time_pairs}
    if batch:
        plan_desc["autotuned"] = True
    sb = launch_bytes(info, st_n, args.steps * iters)
    names = L.STAGE_NAMES
    per_launch = [st_ms[i] / st_n[i] if st_n[i] else 0.0 for i in range(L.AAHRT_NSTAGES)]
    top = max(range(6), key=lambda i: st_ms[i])
    peak, peak_kind = peaks()
    achieved = sb[top] / (per_launch[top] * 1e-3) / 1e9
    iter_ms = sum(st_ms[:6]) / sum(st_n[1:2] or [1])
    iter_bytes = sum(stage_bytes(info)[:6])
    fused = st_n[3] == 0 and st_n[2] > 0
    kernel_names = ["r2c_kernel", "slice_fwd_kernel",
                    "c2r_r2c_kernel" if fused else "c2r_kernel", "r2c_kernel",
                    "slice_adj_kernel", "c2r_r2c_kernel" if fused else "c2r_kernel"]
    if slow:
        kernel_names[1], kernel_names[4] = "direct_fwd_kernel", "direct_adj_kernel"
    suffix = "@direct" if slow else ("@batch512" if batch else "")
    rec = traffic_record(names[top] + suffix)
    line = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "pairs/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": max(args.warmup, 3),
        "ms_per_step": round(total_ms / args.steps, 4),
        "ms_per_step_median": round(step_median_ms, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": config,
        "plan": plan_desc,
        "gathers_per_s": round(value / iters, 4),
        "e2e": {"value": round(e2e_value, 3), "unit": "pairs/s",
                "h2d_bytes_per_step": 4 * gp.data_len, "d2h_bytes_per_step": 4 * gp.model_len,
                "steps": e2e_steps},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": rec.get("dram_bytes") if rec else None,
                     "kernel": kernel_names[top], "stage": names[top],
                     "bytes_per_launch": sb[top],
                     "avg_launch_ms": round(per_launch[top], 5),
                     "peak_source": peak_kind},
        "fused_half_iterations": bool(fused),
        "pair_hbm": {"count": "staged: every stage of the unfused iteration reads its "
                              "input once and writes its output once",
                     "algorithmic_bytes_per_iteration": iter_bytes,
                     "ms_per_iteration": round(iter_ms, 5),
                     "achieved_GBps": round(iter_bytes / (iter_ms * 1e-3) / 1e9, 1),
                     "frac_of_peak": round(iter_bytes / (iter_ms * 1e-3) / 1e9 / peak, 4)},
        "stages": {names[i]: {"ms_per_launch": round(per_launch[i], 5),
                              "launches": int(st_n[i]), "bytes_per_launch": sb[i],
                              "GBps": round(sb[i] / (per_launch[i] * 1e-3) / 1e9, 1)
                              if per_launch[i] else None}
                   for i in range(L.AAHRT_NSTAGES) if st_n[i]},
        "clocks": clocks,
    }
    if not slow:
        # the slice steps' own bound: the L1 / shared-memory data pipe, with
        # the issue slots and the FP32 pipe beside it (ncu, one launch of each
        # kernel on the same workload shape, while the sources still hash to
        # the captured ones)
        alu = {}
        for st in ("slice_fwd", "slice_adj"):
            r = traffic_record(st + suffix)
            if r and "issue_active" in r:
                alu[st] = {"l1_data_pipe": r.get("l1_data_pipe"),
                           "issue_active": r["issue_active"], "fma_pipe": r.get("fma_pipe"),
                           "kernel": r["kernel"]}
        if alu:
            line["slice_issue"] = alu
    if slow and top in (1, 4):
        # the direct sum is bound by the phases' sine/cosine pairs: one per
        # (bin, trace, curvature) and launch; peak = SMs x 16 special-function
        # results per clock / 2 (sine and cosine) x the maximum SM clock
        props = torch.cuda.get_device_properties(dev)
        mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
        peak_ph = props.multi_processor_count * 8 * mhz * 1e6 / 1e9
        phases = info.nbins * g.ntr * g.nq
        ach = phases / (per_launch[top] * 1e-3) / 1e9
        line["roofline"] = {"bound": "alu", "achieved": round(ach, 1),
                            "peak": round(peak_ph, 1), "unit": "Gphase/s",
                            "frac": round(ach / peak_ph, 4),
                            "traffic": rec.get("dram_bytes") if rec else None,
                            "kernel": kernel_names[top], "stage": names[top],
                            "phases_per_launch": phases,
                            "bytes_per_launch": sb[top],
                            "avg_launch_ms": round(per_launch[top], 5),
                            "peak_source": "derived: %d SMs x 8 sincos/clk x %.0f MHz" %
                                           (props.multi_processor_count, mhz)}
    if world == 1 and not args.no_cpu_baseline:
        if batch:
            line["cpu_baseline"], line["err_vs_fp64"] = cpu_baseline_batch(cubes, gp, d, dev)
            fe, mo = fista_error_batch(cubes, gp, d, dev, cg, cl)
            line["err_vs_fp64"]["fista"] = fe
            line["per_cube_fp32"] = per_cube_arm(cubes, info, cg, cl, fe, mo, dev, value)
        else:
            line["cpu_baseline"], line["err_vs_fp64"] = cpu_baseline(g, gp, d, dev, q_axis=qa,
                                                                     kind=kind)
    return line


def local_index(dev):
    return dev.index if dev.index is not None else 0


def single_core_seconds(kind, cube=None):
    """Seconds of one FP64 forward+adjoint pair on one host core (a child
    process with one OpenMP thread), or None if it fails."""
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-single-core",
           kind if cube is None else f"{kind}:{cube}"]
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
               MKL_NUM_THREADS="1")
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=600)
        return float(json.loads(r.stdout.strip().splitlines()[-1])["seconds"])
    except Exception:
        return None


def run_single_core(spec):
    """Child of single_core_seconds: time one oracle pair of the gather or of
    one cube of the batch (`batch512:<cube>`) and print the seconds."""
    import numpy as np

    import oracle
    from oracle import ops
    from paper_2505_00387_gb300 import synthetic as syn
    kind, _, cube = spec.partition(":")
    if kind == "batch512":
        geo, r2max = batch_geometry(3)
        c = syn.cube_batch(seed=3, cubes=[int(cube)])[0]
        p = oracle.make_plan(**c.geom_kwargs(), r2max=r2max)
        d = c.d
    else:
        c = syn.paper_gather(seed=1)
        p = oracle.make_plan(**c.geom_kwargs())
        d = c.d
    mr = np.random.default_rng(5).standard_normal((c.ntau, c.nq, c.ntheta))
    ops.slice_forward(p.subset_traces([0]), np.zeros((p.nbins, p.nq, p.ntheta), complex))
    t0 = time.perf_counter()
    ops.forward(p, mr)
    ops.adjoint(p, d)
    el = time.perf_counter() - t0
    print(json.dumps({"seconds": el, "threads": ops.threads()}))


def cpu_baseline(g, gp, d_dev, dev, pairs=6, q_axis=None, kind="gather"):
    """The FP64 checker timed on this host's cores on a bounded sample of the
    same workload (`pairs` forward+adjoint pairs of the full gather), and
    the GPU path's relative error against those FP64 results."""
    import numpy as np

    import oracle
    from oracle import ops

    p = oracle.make_plan(**g.geom_kwargs(), q_axis=q_axis)
    rng = np.random.default_rng(123)
    mr = rng.standard_normal((g.ntau, g.nq, g.ntheta)).astype(np.float32).astype(np.float64)
    ops.slice_forward(p.subset_traces([0]), np.zeros((p.nbins, p.nq, p.ntheta), complex))
    t0 = time.perf_counter()
    for _ in range(pairs):
        d_or = ops.forward(p, mr)
        m_or = ops.adjoint(p, g.d)
    el = time.perf_counter() - t0
    d_gpu = gp.forward(torch_from(mr, dev))
    m_gpu = gp.adjoint(d_dev)
    d_gpu = d_gpu.cpu().numpy().astype(np.float64).reshape(d_or.shape)
    m_gpu = m_gpu.cpu().numpy().astype(np.float64).reshape(m_or.shape)
    err = {"forward_rel_l2": float(np.linalg.norm(d_gpu - d_or) / np.linalg.norm(d_or)),
           "adjoint_rel_l2": float(np.linalg.norm(m_gpu - m_or) / np.linalg.norm(m_or)),
           "fista": "not run here (a 100-iteration FP64 solve takes minutes); "
                    "tests/test_gpu_parity.py::test_paper_gather_fista_100_iterations"}
    cb = {"value": round(pairs / el, 5), "unit": "pairs/s", "cores": ops.threads(),
          "kind": "oracle",
          "sample": f"{pairs} forward+adjoint pairs of the full gather, FP64, "
                    f"{el:.1f} s wall"}
    return cb, err


def torch_from(a, dev):
    import numpy as np
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32).ravel()).to(dev)


def cpu_baseline_batch(cubes, gp, d_dev, dev, nsample=8):
    """The FP64 checker on one forward+adjoint pair of each of nsample cubes
    spread over the fold range (on the batch's shared time plan), as cube
    pairs per second on all host cores and on one core, and the GPU error on
    those cubes."""
    import numpy as np
    import torch

    import oracle
    from oracle import ops

    folds = np.array([c.ntr for c in cubes])
    picks = fold_picks(folds, nsample)
    r2max = max(float(np.max(x.hx ** 2 + x.hy ** 2)) for x in cubes)
    rng = np.random.default_rng(124)
    m_all = rng.standard_normal(gp.model_len).astype(np.float32)
    d_gpu = gp.forward(torch.from_numpy(m_all).to(dev)).cpu().numpy().astype(np.float64)
    m_gpu = gp.adjoint(d_dev).cpu().numpy().astype(np.float64)
    c0 = cubes[0]
    msz = c0.ntau * c0.nq * c0.ntheta
    offs = np.concatenate([[0], np.cumsum([x.nt * x.ntr for x in cubes])])
    el, ef, ea = 0.0, [], []
    for i in picks:
        c = cubes[i]
        p = oracle.make_plan(**c.geom_kwargs(), r2max=r2max)
        mr = m_all[i * msz:(i + 1) * msz].astype(np.float64).reshape(c.ntau, c.nq, c.ntheta)
        t0 = time.perf_counter()
        d_or = ops.forward(p, mr)
        m_or = ops.adjoint(p, c.d)
        el += time.perf_counter() - t0
        dg = d_gpu[offs[i]:offs[i + 1]].reshape(d_or.shape)
        mg = m_gpu[i * msz:(i + 1) * msz].reshape(m_or.shape)
        ef.append(float(np.linalg.norm(dg - d_or) / np.linalg.norm(d_or)))
        ea.append(float(np.linalg.norm(mg - m_or) / np.linalg.norm(m_or)))
    err = {"cubes": picks, "folds": [int(folds[i]) for i in picks],
           "forward_rel_l2_max": max(ef), "adjoint_rel_l2_max": max(ea),
           "forward_rel_l2_median": float(np.median(ef)),
           "adjoint_rel_l2_median": float(np.median(ea))}
    mid = picks[len(picks) // 2]
    s1 = single_core_seconds("batch512", mid)
    cb = {"value": round(len(picks) / el, 5), "unit": "pairs/s", "cores": ops.threads(),
          "kind": "oracle",
          "sample": f"1 forward+adjoint pair of each of {len(picks)} cubes spread over the fold "
                    f"range ({int(folds[picks[0]])}-{int(folds[picks[-1]])} traces), FP64, "
                    f"{el:.1f} s wall; pairs/s per cube pair",
          "single_core": ({"value": round(1.0 / s1, 5), "unit": "pairs/s", "cores": 1,
                           "sample": f"1 pair of the median-fold cube of the sample "
                                     f"({int(folds[mid])} traces), one OpenMP thread"}
                          if s1 else None)}
    return cb, err


def fista_error_batch(cubes, gp, d_dev, dev, cg, cl):
    """Relative L2 error of the GPU's 50-iteration FISTA output against the
    FP64 checker's on the smallest-fold cube of the batch: the checker
    estimates that cube's step (30 power iterations) and threshold itself;
    the GPU solves the whole batch with those two values for that cube."""
    import numpy as np
    import torch

    import oracle
    from oracle import fista, ops

    folds = np.array([c.ntr for c in cubes])
    i = int(np.argmin(folds))
    c = cubes[i]
    r2max = max(float(np.max(x.hx ** 2 + x.hy ** 2)) for x in cubes)
    p = oracle.make_plan(**c.geom_kwargs(), r2max=r2max)
    t0 = time.perf_counter()
    lam = 0.05 * float(np.abs(ops.adjoint(p, c.d)).max())
    gamma = 0.95 / fista.power_sigma2(p, c.d, iters=30)
    mo = fista.solve(p, c.d, lam, BATCH_ITERS, gamma)
    el = time.perf_counter() - t0
    g2, l2 = cg.copy(), cl.copy()
    g2[i], l2[i] = gamma, lam
    m = torch.zeros(gp.model_len, device=dev)
    gp.sparse_solve(d_dev, 0.0, BATCH_ITERS, m, use_graph=False, want_info=False,
                    per_cube=True, cube_gamma=g2, cube_lambda=l2)
    msz = c.ntau * c.nq * c.ntheta
    mg = m[i * msz:(i + 1) * msz].cpu().numpy().astype(np.float64).reshape(mo.shape)
    return {"cube": i, "fold": int(folds[i]), "iters": BATCH_ITERS,
            "rel_l2": float(np.linalg.norm(mg - mo) / np.linalg.norm(mo)),
            "gamma": gamma, "lambda": lam, "oracle_seconds": round(el, 1)}, mo


def per_cube_arm(cubes, info, cg, cl, fe, mo, dev, batched_value, nsample=16):
    """The plain per-cube form of the same work: one single-cube FP32 plan
    per cube (the batch plan's spreading width, azimuth group and column
    pairs), each cube's 50-iteration FISTA solve run on its own, one cube
    after another; nsample cubes spread evenly over the fold range.  Returns
    its rate in cube-pairs/s beside the batched plan's, and the FISTA output
    error against the FP64 checker on the smallest-fold cube (solved with the
    checker's step and threshold, as in err_vs_fp64.fista)."""
    import numpy as np
    import torch

    from paper_2505_00387_gb300.plan import AahrtPlan

    folds = np.array([c.ntr for c in cubes])
    picks = fold_picks(folds, nsample)
    r2max = max(float(np.max(x.hx ** 2 + x.hy ** 2)) for x in cubes)
    runs = []
    for i in picks:
        c = cubes[i]
        # the batch's time plan (r2max): the same operator as the batched plan
        p = AahrtPlan(**c.geom_kwargs(), spread_width=info.spread_width,
                      theta_group=info.theta_group, time_pairs=info.time_pairs, r2max=r2max)
        d = torch.from_numpy(c.d.astype(np.float32).ravel()).to(dev)
        m = torch.zeros(p.model_len, device=dev)
        g, lam = (fe["gamma"], fe["lambda"]) if i == fe["cube"] else (float(cg[i]), float(cl[i]))
        runs.append((i, p, d, m, g, lam))

    def one_pass():
        for _, p, d, m, g, lam in runs:
            p.sparse_solve(d, lam, BATCH_ITERS, m, gamma=g, use_graph=True, want_info=False)

    one_pass()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 2
    e0.record()
    for _ in range(reps):
        one_pass()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    rate = len(runs) * BATCH_ITERS / (ms / 1e3)
    err = None
    for i, p, d, m, g, lam in runs:
        if i == fe["cube"]:
            mg = m.cpu().numpy().astype(np.float64).reshape(mo.shape)
            err = float(np.linalg.norm(mg - mo) / np.linalg.norm(mo))
    out = {"value": round(rate, 3), "unit": "pairs/s",
           "sample": f"{len(runs)} cubes spread over the fold range "
                     f"({int(folds[picks[0]])}-{int(folds[picks[-1]])} traces), one single-cube "
                     f"FP32 plan each, {BATCH_ITERS}-iteration FISTA per cube, one cube at a time",
           "ms_per_pass": round(ms, 3),
           "batched_over_per_cube": round(batched_value / rate, 3),
           "fista_rel_l2_vs_fp64": err,
           "fista_cube": fe["cube"]}
    for _, p, d, m, _, _ in runs:
        p.close()
    return out


# ------------------------------------------------------------- reference
def run_reference(args):
    """The FP64 checker on the host cores, on the same workload, config and
    metric: each step is a whole forward+adjoint pair (of one cube of the
    batch, cubes taken over the fold range, or of the gather)."""
    rank, world, local = dist_info()
    if rank != 0:
        return
    import numpy as np

    import oracle
    from oracle import ops
    from paper_2505_00387_gb300 import synthetic as syn

    kind = args.workload if args.workload in ("batch512", "gather", "slowness") else "batch512"
    rng = np.random.default_rng(123)
    if kind == "batch512":
        geo, r2max = batch_geometry(3)
        # timed steps: cubes evenly over the fold range; warm-up: a few more
        timed_ = fold_picks([c.ntr for c in geo], args.steps)
        warm = fold_picks([c.ntr for c in geo], max(args.warmup, 3))
        need = sorted(set(timed_) | set(warm))
        data = {c: x for c, x in zip(need, syn.cube_batch(seed=3, cubes=need))}
        plans = {c: oracle.make_plan(**data[c].geom_kwargs(), r2max=r2max) for c in need}

        def step(c):
            x = data[c]
            mr = rng.standard_normal((x.ntau, x.nq, x.ntheta))
            ops.forward(plans[c], mr)
            ops.adjoint(plans[c], x.d)
        seq_warm, seq = warm, timed_
        config = workload_config("batch512", 1, geo=geo)
        sample = (f"per step one forward+adjoint pair of one cube; the {args.steps} timed "
                  f"steps take {args.steps} cubes evenly over the fold range "
                  f"({geo[timed_[0]].ntr}-{geo[timed_[-1]].ntr} traces); FP64")
    else:
        g = syn.paper_gather(seed=1)
        qa = None
        if kind == "slowness":
            from oracle import pnmo
            qa = pnmo.q_axis_slowness(syn.P_MIN, syn.P_MAX, g.nq)
        p = oracle.make_plan(**g.geom_kwargs(), q_axis=qa)

        def step(_):
            mr = rng.standard_normal((g.ntau, g.nq, g.ntheta))
            ops.forward(p, mr)
            ops.adjoint(p, g.d)
        seq_warm, seq = [0] * max(args.warmup, 3), [0] * args.steps
        config = workload_config(kind, 1, g=g)
        sample = "per step one forward+adjoint pair of the full gather, FP64"

    for c in seq_warm:
        step(c)
    t0 = time.perf_counter()
    for c in seq:
        step(c)
    el = time.perf_counter() - t0
    value = len(seq) / el
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": round(value, 6),
        "unit": "pairs/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": max(args.warmup, 3),
        "ms_per_step": round(el / args.steps * 1e3, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": config,
        "cpu_baseline": {"value": round(value, 6), "unit": "pairs/s", "cores": ops.threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 6), "unit": "pairs/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# The paper's Table 1: adjoint (velocity scan) of regular Nx x Ny offset
# grids at dx = dy = 40 m, dt = 4 ms, 90 azimuths; (Nt, Nx, Ny, Np) and the
# paper's "proposed" seconds (hardware not stated in the paper).
TABLE1 = [(512, 128, 128, 128, 0.87), (512, 128, 128, 256, 1.14),
          (512, 256, 256, 128, 3.80), (512, 256, 256, 256, 3.98),
          (1024, 128, 128, 128, 1.97), (1024, 128, 128, 256, 2.78),
          (1024, 256, 256, 128, 8.57), (1024, 256, 256, 256, 8.82)]


def run_table1(args):
    """Velocity-scan time at the Table 1 shapes: the exact adjoint with both
    slice steps (the accurate spreading kernel and the paper's linear
    k-interpolation at sigma_q = 1) and the paper's own pull scan on the
    regular grid (Algorithm 2, B-coefficients)."""
    import numpy as np
    import torch

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    from paper_2505_00387_gb300 import build as B
    B.build()
    from paper_2505_00387_gb300 import synthetic as syn
    from paper_2505_00387_gb300.plan import AahrtPlan

    rows = []
    total = 0.0
    for nt, nx, ny, npq, paper_s in TABLE1:
        x = (np.arange(nx) - nx / 2 + 0.5) * 40.0
        y = (np.arange(ny) - ny / 2 + 0.5) * 40.0
        hx, hy = np.meshgrid(x, y, indexing="ij")
        hx, hy = hx.ravel(), hy.ravel()
        q0, dq = syn.q_axis(npq)
        row = {"nt": nt, "nx": nx, "ny": ny, "np": npq, "ntheta": 90, "paper_s": paper_s}
        for mode, kw in (("spread", {}), ("linear_k", dict(slice_interp="linear_k",
                                                           sigma_q=1.0))):
            gp = AahrtPlan(nt, 0.004, nt, npq, q0, dq, 90, hx, hy, **kw)
            d = torch.randn(gp.data_len, device="cuda")
            m = torch.empty(gp.model_len, device="cuda")
            for _ in range(max(args.warmup, 3)):
                gp.adjoint(d, m)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.steps):
                gp.adjoint(d, m)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            row[mode + "_ms"] = round(ms, 3)
            row["nfft"] = gp.info.nfft
            if mode == "spread":
                total += ms
                # the paper's own pull scan on the same grid (Algorithm 2)
                grid = (nx, ny, float(x[0]), 40.0, float(y[0]), 40.0)
                for _ in range(max(args.warmup, 3)):
                    gp.velocity_scan_grid(d, grid, m)
                torch.cuda.synchronize()
                e0.record()
                for _ in range(args.steps):
                    gp.velocity_scan_grid(d, grid, m)
                e1.record()
                torch.cuda.synchronize()
                row["pull_scan_ms"] = round(e0.elapsed_time(e1) / args.steps, 3)
            del gp, d, m
            torch.cuda.empty_cache()
        rows.append(row)
    line = {"metric": "AAHRT adjoint (velocity scan) time at the paper's Table 1 shapes",
            "value": round(total, 3), "unit": "ms (sum over the 8 shapes, accurate slice step)",
            "n_gpus": 1, "steps": args.steps, "warmup": max(args.warmup, 3),
            "higher_is_better": False, "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (random data on regular offset grids)",
            "config": {"workload": "Table 1: regular Nx x Ny grids, dx = dy = 40 m, "
                                   "dt = 4 ms, 90 azimuths, q over 1/3500..1/1500 s/m"},
            "shapes": rows}
    print(json.dumps(line), flush=True)


def tc_flops(hx, hy, nq, ntheta, nbins, G):
    """Tensor-core flops one forward and one adjoint slice launch execute
    (bf16 hi/lo splits: three products; padded tiles): forward row tiles of
    128 traces per slice, 32-curvature K chunks, N = 4 Gp; adjoint chunks of
    32 traces of slices j and j-1, M tiles of 128 curvatures, N = 2 Gp."""
    import numpy as np
    th = np.mod(np.arctan2(hy, hx), np.pi)
    j = np.floor(th / (np.pi / ntheta)).astype(np.int64)
    j[j >= ntheta] -= ntheta
    n = np.bincount(np.clip(j, 0, ntheta - 1), minlength=ntheta)
    gp = (G + 7) // 8 * 8
    kstep = 3 * 2 * 16                       # three split products, 2 flops, K = 16
    fwd = sum(-(-int(c) // 128) for c in n) * (-(-nq // 32)) * 4 * kstep * 128 * 4 * gp
    nmt = 2 if nq > 128 else 1
    adj = sum(-(-int(n[i] + n[i - 1]) // 32) for i in range(ntheta)) * nmt * 4 * kstep * 128 * 2 * gp
    return fwd * nbins, adj * nbins


def run_shared64(args):
    """--workload shared64: the shared-geometry line alone."""
    import torch

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    from paper_2505_00387_gb300 import build as B
    B.build()
    line = measure_shared64(args, rank, args.steps)
    print(json.dumps(line), flush=True)


def gpu_dot_rel(fwd, adj, m, seed):
    """FP32 dot test of a GPU operator pair, inner products accumulated in
    FP64: m given, d = L m plus as much independent noise (so <L m, d> is about
    |L m|^2, not a near-zero random projection), and
    |<L m, d> - <m, L^T d>| / |<L m, d>|."""
    import torch

    def dot64(a, b, chunk=1 << 26):
        a, b = a.reshape(-1), b.reshape(-1)
        return sum(float(torch.dot(a[i:i + chunk].double(), b[i:i + chunk].double()))
                   for i in range(0, a.numel(), chunk))

    lm = fwd(m)
    gen = torch.Generator(device=m.device).manual_seed(seed)
    d = torch.randn(lm.shape, device=m.device, generator=gen)
    d.mul_((dot64(lm, lm) / lm.numel()) ** 0.5).add_(lm)
    lhs = dot64(lm, d)
    del lm
    rhs = dot64(m, adj(d))
    return abs(lhs - rhs) / abs(lhs)


def measure_shared64(args, rank, steps):
    """Forward + adjoint of 64 gathers sharing one geometry (8000 traces in a
    4 km disc, nt = 2048 at 2 ms, 200 q x 72 azimuths), three ways: the
    split-BF16 tensor-core contraction of all 64 in one plan, the FP32
    spreading path of all 64 in one plan, and one single-gather FP32 plan
    applied to the 64 gathers in turn (the plain per-gather form).  Errors of
    each against the FP64 checker on sampled traces (forward) and azimuth
    slices (adjoint) of two gathers, and each form's FP32 dot test."""
    import numpy as np
    import torch

    from paper_2505_00387_gb300 import _lib as L
    from paper_2505_00387_gb300 import synthetic as syn
    from paper_2505_00387_gb300.plan import AahrtPlan

    geo, _ = syn.shared_batch(seed=replica_seed(4, rank), gathers=[])
    G = 64
    shape_m = (geo.ntau, geo.nq, geo.ntheta)
    flush = torch.empty(256 * 1024 * 1024 // 4, device="cuda")

    # sampled checks: two gathers' data, random models, 16 traces, 2 slices
    rng = np.random.default_rng(83)
    sample_g = [5, 50]
    traces = np.sort(rng.choice(geo.ntr, 16, replace=False))
    slices = [3, 40]
    ms = {i: rng.standard_normal(shape_m).astype(np.float32) for i in sample_g}
    _, dl = syn.shared_batch(seed=replica_seed(4, rank), gathers=sample_g)
    ds = {i: x.astype(np.float32) for i, x in zip(sample_g, dl)}
    check = rank == 0 and not args.no_cpu_baseline
    ref = {}
    full = None                 # the FP64 checker's whole pair of gather fg
    fg = sample_g[0]
    cpu = None
    if check:
        import oracle
        from oracle import ops
        op = oracle.make_plan(**geo.geom_kwargs())
        # one whole forward+adjoint pair of one gather: the CPU baseline, and
        # the reference of every arm's error on that whole gather
        t0 = time.perf_counter()
        full = (ops.forward(op, ms[fg].astype(np.float64)),
                ops.adjoint(op, ds[fg].astype(np.float64)))
        el = time.perf_counter() - t0
        cpu = {"value": round(1.0 / el, 5), "unit": "gather-pairs/s", "cores": ops.threads(),
               "kind": "oracle",
               "sample": f"1 forward+adjoint pair of one of the {G} gathers (all "
                         f"{geo.ntr} traces, {geo.nq} q x {geo.ntheta} azimuths), FP64, "
                         f"{el:.1f} s wall"}
        ref[fg] = (full[0][:, traces], full[1][:, :, slices])
        for i in sample_g[1:]:
            ref[i] = (ops.forward_traces(op, ms[i].astype(np.float64), traces),
                      ops.adjoint_slices(op, ds[i].astype(np.float64), slices))

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    def timed_steps(pair):
        for _ in range(max(args.warmup, 3)):
            pair()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for e0, e1 in ev:
            flush.zero_()
            e0.record()
            pair()
            e1.record()
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / steps

    res = {}
    for prec in ("split_bf16", "fp32"):
        gp = AahrtPlan(**geo.geom_kwargs(), ngather=G, precision=prec)
        tc = prec == "split_bf16"
        gen = torch.Generator(device="cuda").manual_seed(4)
        m = torch.randn(gp.model_len, device="cuda", generator=gen)
        d = torch.randn(gp.data_len, device="cuda", generator=gen)
        mo = torch.empty_like(m)
        do = torch.empty_like(d)

        def pair():
            gp.forward(m, do)
            gp.adjoint(d, mo)
        ms_pair = timed_steps(pair)
        gp.set_profiling(True)
        for _ in range(steps):
            pair()
        torch.cuda.synchronize()
        t, n = gp.stage_times()
        gp.set_profiling(False)
        if tc:
            gp.status()
        err = None
        if check:
            # the sampled gathers' inputs in this plan's layout
            mv = m.view(shape_m + (G,)) if tc else m.view((G,) + shape_m)
            dv = d.view((geo.nt, geo.ntr, G)) if tc else d.view((G, geo.nt, geo.ntr))
            for i in sample_g:
                mt = torch.from_numpy(ms[i]).cuda()
                dt_ = torch.from_numpy(ds[i]).cuda()
                if tc:
                    mv[..., i] = mt
                    dv[..., i] = dt_
                else:
                    mv[i] = mt
                    dv[i] = dt_
            pair()
            if tc:
                gp.status()
            err = {}
            for i in sample_g:
                if tc:
                    dgi = do.view(geo.nt, geo.ntr, G)[:, :, i]
                    mgi = mo.view(shape_m + (G,))[..., i]
                else:
                    dgi = do.view(G, geo.nt, geo.ntr)[i]
                    mgi = mo.view((G,) + shape_m)[i]
                dgh = dgi.cpu().numpy().astype(np.float64)
                mgh = mgi.cpu().numpy().astype(np.float64)
                err[i] = (rel(dgh[:, traces], ref[i][0]), rel(mgh[:, :, slices], ref[i][1]))
                if i == fg:
                    err_full = (rel(dgh, full[0]), rel(mgh, full[1]))
        res[prec] = {"ms_per_pair": round(ms_pair, 3),
                     "gather_pairs_per_s": round(G / (ms_pair / 1e3), 2),
                     "stages_ms": {L.STAGE_NAMES[i]: round(t[i] / n[i], 3)
                                   for i in range(6) if n[i]},
                     "nbins": gp.info.nbins,
                     "dot_test_rel": gpu_dot_rel(gp.forward, gp.adjoint, m, 11)}
        if tc:
            gp.status()
        if err:
            res[prec]["err_vs_fp64"] = {
                "forward_rel_l2_max": max(e[0] for e in err.values()),
                "adjoint_rel_l2_max": max(e[1] for e in err.values()),
                "whole_gather": {"gather": fg, "forward_rel_l2": err_full[0],
                                 "adjoint_rel_l2": err_full[1]}}
        del gp, m, d, mo, do
        torch.cuda.empty_cache()

    # the plain per-gather form: one FP32 single-gather plan, 64 gathers in turn
    g1 = AahrtPlan(**geo.geom_kwargs())
    gen = torch.Generator(device="cuda").manual_seed(4)
    m1 = torch.randn((G, g1.model_len), device="cuda", generator=gen)
    d1 = torch.randn((G, g1.data_len), device="cuda", generator=gen)
    mo1 = torch.empty_like(m1)
    do1 = torch.empty_like(d1)

    def pair1():
        for i in range(G):
            g1.forward(m1[i], do1[i])
            g1.adjoint(d1[i], mo1[i])
    ms1 = timed_steps(pair1)
    err1 = None
    if check:
        err1 = {}
        for i in sample_g:
            dg = g1.forward(torch.from_numpy(ms[i].ravel()).cuda()).cpu().numpy()
            mg = g1.adjoint(torch.from_numpy(ds[i].ravel()).cuda()).cpu().numpy()
            dgh = dg.reshape(geo.nt, geo.ntr).astype(np.float64)
            mgh = mg.reshape(shape_m).astype(np.float64)
            err1[i] = (rel(dgh[:, traces], ref[i][0]), rel(mgh[:, :, slices], ref[i][1]))
            if i == fg:
                err1_full = (rel(dgh, full[0]), rel(mgh, full[1]))
    res["fp32_per_gather"] = {"ms_per_pair": round(ms1, 3),
                              "gather_pairs_per_s": round(G / (ms1 / 1e3), 2),
                              "dot_test_rel": gpu_dot_rel(g1.forward, g1.adjoint, m1[0], 11),
                              "form": "one single-gather FP32 plan, forward + adjoint of the 64 "
                                      "gathers one after another"}
    if err1:
        res["fp32_per_gather"]["err_vs_fp64"] = {
            "forward_rel_l2_max": max(e[0] for e in err1.values()),
            "adjoint_rel_l2_max": max(e[1] for e in err1.values()),
            "whole_gather": {"gather": fg, "forward_rel_l2": err1_full[0],
                             "adjoint_rel_l2": err1_full[1]}}
    del g1, m1, d1, mo1, do1
    torch.cuda.empty_cache()

    tc = res["split_bf16"]
    ff, fa = tc_flops(geo.hx, geo.hy, geo.nq, geo.ntheta, tc["nbins"], G)
    try:
        pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak, src = float(pk["bf16_tflops"]), "measured (burst)"
    except Exception:
        peak, src = 1900.0, "fallback"
    t_f, t_a = tc["stages_ms"]["slice_fwd"], tc["stages_ms"]["slice_adj"]
    top, fl, tt = ("slice_adj", fa, t_a) if t_a >= t_f else ("slice_fwd", ff, t_f)
    ach = fl / (tt * 1e-3) / 1e12
    # DRAM bytes per launch from the committed ncu record of the same kernel
    # (a 256-bin case of this geometry scaled to these bins), while its
    # sources still hash to the captured ones
    trec = traffic_record(top + "@shared64")
    line = {"metric": "shared-geometry gathers: forward+adjoint pairs/s, split-BF16 tensor cores "
                      "vs FP32 spreading (batched and per gather)",
            "value": tc["gather_pairs_per_s"], "unit": "gather-pairs/s", "n_gpus": 1,
            "steps": steps, "warmup": max(args.warmup, 3),
            "ms_per_step": tc["ms_per_pair"], "higher_is_better": True, "vs_baseline": None,
            "dtype": "bf16x3 (split) / f32 accumulate", "data": "synthetic (seeded random m, d)",
            "config": {"workload": "64 gathers on one geometry: 8000 traces in a 4 km disc, "
                                   "nt=2048 dt=2ms, 200 q x 72 azimuths; one step = forward + "
                                   "adjoint of all gathers",
                       "l2": "spectra (tens of GB) far beyond L2, and flushed"},
            "roofline": {"bound": "tensor", "achieved": round(ach, 1), "peak": peak,
                         "unit": "TFLOP/s", "frac": round(ach / peak, 4),
                         "traffic": trec.get("dram_bytes") if trec else None,
                         "tensor_pipe": trec.get("tensor_pipe") if trec else None,
                         "kernel": top + "_tc_kernel", "flops_per_launch": fl,
                         "flops": "executed MMA flops: three bf16 products, padded tiles",
                         "avg_launch_ms": tt, "peak_source": src},
            "split_bf16": tc, "fp32": res["fp32"], "fp32_per_gather": res["fp32_per_gather"],
            "speedup_vs_fp32": round(res["fp32"]["ms_per_pair"] / tc["ms_per_pair"], 3),
            "speedup_vs_fp32_per_gather": round(res["fp32_per_gather"]["ms_per_pair"] /
                                                tc["ms_per_pair"], 3),
            "err_sample": {"gathers": sample_g, "traces": len(traces), "slices": slices,
                           "whole_gather": fg}}
    if cpu:
        line["cpu_baseline"] = cpu
    return line


if __name__ == "__main__":
    a = parse()
    if a.oracle_single_core:
        run_single_core(a.oracle_single_core)
    elif a.impl == "reference":
        run_reference(a)
    elif a.workload == "table1":
        run_table1(a)
    elif a.workload == "shared64":
        run_shared64(a)
    else:
        run_ours(a)
