#!/usr/bin/env python3
"""Benchmark of the GB300 screened-Poisson operator and CG.

Default workload (one GPU): the degree-sweep configuration at N=7, a perturbed
box of 64 x 64 x 61 hexahedra (about 128M local nodes), FP64, lambda = 0.1,
seeded uniform right-hand side. One step is one conjugate-gradient iteration
(one application of A plus the fused vector stage of Algorithm 1); the value is
the paper's throughput, global DOFs x iterations / s, in GDOF/s.

The same line carries, measured in the same run on one GPU, the metric's
other two parts: "c3", the single large solve (N=7, 80^3 elements) to a true
relative residual of 1e-10 with FP64 CG and the mixed-precision solvers, and
"c5", the serving stream (a stated number of the serving config's requests)
with solves/s and p50 / p99 latency beside one-at-a-time FP64 and mixed solves.

Prints one JSON line. Other workloads print their own lines; only the
default is the headline:
  sweep   operator-only degree sweep N=1..15 on boxes of about 128M local nodes
  c1      100 FP64 CG iterations on a 4x4x4 box at N=7 (latency-bound)
  c3      one solve to 1e-10 on an 80x80x80 box at N=7 with a manufactured
          right-hand side: FP64, mixed precision, Jacobi, double-float
  c4      mixed-precision stress: N=15, 24x24x24, strong perturbation, three lambdas
  c5      serving stream of CG requests (sizes 2..32 elements per axis, N in 3..11)
  split   split operator over virtual ranks; scat: scattered storage; probe: hardware probes

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

# The serving workload runs every resident solve on its own CUDA stream; with
# the default 8 hardware work queues unrelated streams share queues and wait
# on each other's kernels. Read when the CUDA context is created.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
# FP64 FMA issue rate of one GB300 SM, measured with an FMA-chain probe
# (1.194 TFLOP/s with 152 SMs at 1.98 GHz): 2 FMA per clock per SM.
FP64_FMA_PER_CLK_SM = 2.0
FP32_FMA_PER_CLK_SM = 128.0
N_SM = 152
SM_MAX_MHZ = 2070.0


def peaks():
    hbm, src = FALLBACK_HBM_GBS, "fallback"
    try:
        with open(MEASURED_PEAKS) as f:
            d = json.load(f)
        hbm, src = float(d["hbm_gbs"]), "measured"
    except Exception:
        pass
    return {"hbm_gbs": hbm, "hbm_src": src,
            "fp64_tflops": 2 * FP64_FMA_PER_CLK_SM * N_SM * SM_MAX_MHZ * 1e6 / 1e12,
            "fp32_tflops": 2 * FP32_FMA_PER_CLK_SM * N_SM * SM_MAX_MHZ * 1e6 / 1e12}


# ---------------------------------------------------------------- workloads

def c2_dims(N: int, local_nodes: float = 1.28e8):
    """Elements per axis so that local nodes ~ 1.28e8 (Ex = Ey multiple of 8)."""
    n = N + 1
    T = local_nodes / n ** 3
    ex = int(math.ceil(T ** (1.0 / 3.0) / 8.0)) * 8
    ez = int(T // (ex * ex))
    return ex, ex, ez


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [t.strip() for t in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_uuid():
    import torch
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
    except Exception:
        return str(torch.cuda.current_device())


# ---------------------------------------------------------------- distributed

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate_rate(world: int, units_per_rank: float, t_max_ms: float) -> float:
    """Whole-job rate in units/s: every rank processes units_per_rank in its
    own timed region; the slowest rank's time (max over ranks) counts."""
    return world * units_per_rank / (t_max_ms * 1e-3)


class Dist:
    def __init__(self, world, local, backend):
        self.world = world
        self.pg = None
        if world > 1:
            import torch.distributed as tdist
            tdist.init_process_group(backend=backend)
            self.pg = tdist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v: float) -> float:
        if not self.pg:
            return v
        import torch
        t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------- CPU baseline (the oracle)

def cpu_baseline(N, budget_s=12.0, dims=(16, 16, 16), lam=0.1, iters=None):
    """The FP64 oracle, as it stands, on a bounded sample of the workload: the
    same degree and mesh recipe on a smaller box, timed over CG iterations."""
    from oracle import oracle as orc
    m = orc.Mesh(*dims, N, rho=0.1, seed=0)
    b = m.rhs(kind=0, seed=0)
    m.cg(b, lam, rtol=0.0, max_it=1)  # warm
    done, t_used = 0, 0.0
    if iters is None:
        k = 1
        while t_used < budget_s:
            t0 = time.perf_counter()
            m.cg(b, lam, rtol=0.0, max_it=k)
            dt = time.perf_counter() - t0
            done += k
            t_used += dt
            k = min(2 * k, 64)
    else:
        t0 = time.perf_counter()
        m.cg(b, lam, rtol=0.0, max_it=iters)
        t_used = time.perf_counter() - t0
        done = iters
    return {"value": m.n_global * done / t_used / 1e9, "unit": "GDOF/s", "cores": orc.num_threads(),
            "kind": "oracle",
            "sample": f"N={N}, {dims[0]}x{dims[1]}x{dims[2]} elements (N_G={m.n_global}), {done} FP64 CG "
                      f"iterations (each = one A x plus the vector stage) in {t_used:.1f} s"}


# ---------------------------------------------------------------- GB300 arm

def run_gb300(args, rank, world, local):
    import torch

    from paper_2202_12477_gb300 import accounting as acc
    from paper_2202_12477_gb300 import hb

    torch.cuda.set_device(local)
    dist = Dist(world, local, "nccl")
    N = args.N
    ex, ey, ez = c2_dims(N)
    lam = 0.1
    m = hb.Mesh(ex, ey, ez, N, perturb=0.1, seed=0, fp32=False)
    NG, NL, E = m.n_global, m.n_local, m.E
    stream = torch.cuda.current_stream()
    from paper_2202_12477_gb300 import autotune
    # the headline variant must hold on any mesh: the lattice-gather variants
    # (GRID bit), which rely on the box's structure, are timed beside it
    tuned = autotune.tune_mesh(m, precs=(hb.HB_F64, hb.HB_F64X), lam=0.1, exclude=hb.HB_VARIANT_GRID)
    variant = tuned[hb.HB_F64]
    b = m.rhs(kind=0, seed=0)
    x = m.vec()

    # one stepwise solve of W + K iterations: its start (r0 = b - A x0) and the
    # W warm-up iterations run before the timed region, which holds exactly
    # the K timed iterations
    x.zero_()
    m.cg_begin(b, x, lam=lam, rtol=0.0, max_it=args.warmup + args.steps)
    m.cg_iterate(args.warmup)
    torch.cuda.synchronize()

    hb.hb_profile_reset()
    hb.hb_profile_enable(True)
    launches0 = hb.hb_kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(gpu_uuid()) as clk:
        dist.barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        m.cg_iterate(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        dist.barrier()
    launches = hb.hb_kernel_launches() - launches0
    hb.hb_profile_enable(False)
    res = m.cg_finish()
    t_ms = ev0.elapsed_time(ev1)
    t_max = dist.max(t_ms)
    kern = {}
    for name in ("ax_local", "assemble", "cg_update_r", "cg_update_xp"):
        ms, cnt = hb.hb_profile_read(name)
        kern[name] = {"ms_total": ms, "launches": cnt, "ms_avg": ms / cnt if cnt else None}
    assert res.iters == args.warmup + args.steps, (res.iters, args.warmup, args.steps)

    # end to end: pinned host b in, solve through the C ABI, x back to pinned host
    b_host = b.cpu().pin_memory()
    x_host = torch.empty(NG, dtype=torch.float64).pin_memory()
    b_dev = torch.empty_like(b)
    x_dev = torch.zeros_like(b)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dist.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    b_dev.copy_(b_host, non_blocking=True)
    x_dev.zero_()
    m.cg(b_dev, x=x_dev, lam=lam, rtol=0.0, max_it=args.steps)
    x_host.copy_(x_dev, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = dist.max(e0.elapsed_time(e1))

    def timed_cg(prec):
        """W warm-up and K timed iterations of one stepwise solve; max over ranks."""
        x.zero_()
        m.cg_begin(b, x, lam=lam, rtol=0.0, max_it=args.warmup + args.steps, prec=prec)
        m.cg_iterate(args.warmup)
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        dist.barrier()
        torch.cuda.synchronize()
        g0.record(stream)
        m.cg_iterate(args.steps)
        g1.record(stream)
        torch.cuda.synchronize()
        m.cg_finish()
        return dist.max(g0.elapsed_time(g1))

    # the same iterations with the double-float element kernel (HB_F64X: FP64
    # data, FP32-pair arithmetic, 1e-12 parity with the FP64 oracle)
    f64x_ms = timed_cg(hb.HB_F64X)
    # and with the lattice gather (GRID), which only a structured box allows
    grid_variant = hb.HB_VARIANT_PENCIL | hb.HB_VARIANT_EVEN_ODD | hb.HB_VARIANT_GRID
    hb.hb_set_kernel_variant(m.handle, hb.HB_F64, grid_variant)
    grid_ms = timed_cg(hb.HB_F64)
    hb.hb_set_kernel_variant(m.handle, hb.HB_F64, variant)

    pk = peaks()
    ax = kern["ax_local"]
    # DRAM bytes per local node of this kernel from one ncu capture of the same
    # kernel on a smaller box (32x32x30 hexahedra, 15,728,640 local nodes),
    # scaled to this launch by local nodes; only for the captured (degree,
    # variant) pairs.
    per_node = {(7, 3): 64.77, (7, 11): 64.66, (7, 67): 67.53, (7, 75): 67.42, (7, 131): 62.33,
                (7, 139): 62.38, (7, 256): 65.97, (7, 320): 68.84}.get((N, variant))
    traffic = per_node * NL if per_node else None
    ax_flops = acc.op_local_flops(E, N)
    ax_bytes = acc.ax_local_bytes(NG, NL, 8)
    achieved_tf = ax_flops / (ax["ms_avg"] * 1e-3) / 1e12
    achieved_gbs = ax_bytes / (ax["ms_avg"] * 1e-3) / 1e9
    hbm_view = {"algorithmic_bytes_per_launch": ax_bytes, "achieved_gbs": achieved_gbs,
                "peak_gbs": pk["hbm_gbs"], "peak_src": pk["hbm_src"], "frac": achieved_gbs / pk["hbm_gbs"]}
    if variant & hb.HB_VARIANT_TC:
        # tensor-core element kernel: the contractions run on the tensor cores,
        # so its roof is HBM; the FP64 work left on the CUDA cores (the metric
        # step, 15 n^3 flops per element) is shown against the FP64 pipe
        metric_flops = 15 * (N + 1) ** 3 * E
        metric_tf = metric_flops / (ax["ms_avg"] * 1e-3) / 1e12
        roofline = {"bound": "hbm", "kernel": "ax_local (FP64, tensor-core contractions)",
                    "achieved": achieved_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved_gbs / pk["hbm_gbs"], "peak_src": pk["hbm_src"],
                    "bytes_per_launch": ax_bytes, "ms_per_launch": ax["ms_avg"],
                    "bytes_note": "algorithmic bytes esz N_G + (4 + 7 esz) N_L: x once, node map, six "
                                  "metric factors, the element-local result once",
                    "traffic": traffic,
                    "traffic_note": "ncu dram bytes (read+write) per launch, scaled from a 32x32x30 capture",
                    "fp64_view": {"metric_flops_per_launch": metric_flops, "achieved_tflops": metric_tf,
                                  "peak_tflops": pk["fp64_tflops"],
                                  "frac": metric_tf / pk["fp64_tflops"]},
                    "flops_view": {"algorithmic_flops_per_launch": ax_flops, "achieved_tflops": achieved_tf}}
    else:
        roofline = {"bound": "alu", "kernel": "ax_local (FP64)", "achieved": achieved_tf,
                    "peak": pk["fp64_tflops"], "unit": "TFLOP/s", "frac": achieved_tf / pk["fp64_tflops"],
                    "peak_src": "derived: 2 FP64 FMA/clk/SM (measured probe) x 152 SMs x 2070 MHz",
                    "flops_per_launch": ax_flops, "ms_per_launch": ax["ms_avg"],
                    "flops_note": "algorithmic flops E(12n^4+15n^3) of the dense contractions; the kernel's "
                                  "even-odd split of D executes fewer FP64 operations, so frac can pass 1",
                    "traffic": traffic,
                    "traffic_note": "ncu dram bytes (read+write) per launch, scaled from a 32x32x30 capture",
                    "hbm_view": hbm_view}
    out = {
        "metric": "Ax GDOF/s (FP64; one CG iteration = one A x and its fused vector stage)",
        "value": aggregate_rate(world, NG * args.steps, t_max) / 1e9,
        "unit": "GDOF/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded perturbed box, SplitMix64 uniform rhs)",
        "config": {"workload": f"degree sweep config at N={N}: {ex}x{ey}x{ez} hexahedra, perturb 0.1h, "
                               f"lambda 0.1, FP64 CG, 100-iteration style fixed count",
                   "N": N, "elements": [ex, ey, ez], "n_local": NL, "n_global": NG,
                   "kernel_variant": variant,
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": f"inputs larger than L2: {7 * 8 * NL / 1e9:.1f} GB of geometric factors streamed "
                         f"per step (L2 129 MB)"},
        "roofline": roofline,
        "kernels": kern,
        "ax_only_gdofs": NG / ((kern["ax_local"]["ms_avg"] + kern["assemble"]["ms_avg"]) * 1e-3) / 1e9,
        "fom_gflops_nekbone": acc.nekbone_flops(E, N) * args.steps / (t_max * 1e-3) / 1e9,
        "e2e": {"value": world * NG * args.steps / (e2e_ms * 1e-3) / 1e9, "unit": "GDOF/s",
                "h2d_bytes_per_step": 8 * NG / args.steps, "d2h_bytes_per_step": 8 * NG / args.steps,
                "note": f"one hb_cg_solve of {args.steps} iterations per host round trip"},
        "f64x": {"value": aggregate_rate(world, NG * args.steps, f64x_ms) / 1e9, "unit": "GDOF/s",
                 "ms_per_step": f64x_ms / args.steps, "kernel_variant": tuned[hb.HB_F64X],
                 "note": "same CG iterations with the double-float element kernel (FP64 storage, gather "
                         "and vector stage; FP32-pair contractions; A x within 1e-12 of the FP64 oracle)"},
        "grid_box_only": {"value": aggregate_rate(world, NG * args.steps, grid_ms) / 1e9, "unit": "GDOF/s",
                          "ms_per_step": grid_ms / args.steps, "kernel_variant": grid_variant,
                          "note": "same FP64 CG iterations with Z^T by the box's lattice arithmetic (GRID): "
                                  "valid only on a structured box, so not the headline"},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(N)
    if world == 1:
        # the metric's other two parts, measured in the same run: time to a
        # true 1e-10 (FP64 vs mixed) and served solves/s with p50 / p99
        del m, x, b, b_host, x_host, b_dev, x_dev
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        if not args.no_sweep:
            out["sweep"] = sweep_compact()
        if not args.no_c3:
            out["c3"] = c3_compact()
        if not args.no_c5:
            out["c5"] = c5_compact(args.c5_default_requests)
    dist.close()
    if rank == 0:
        print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- reference arm (the oracle)

def run_reference_workloads(args):
    """The reference arm (the oracle, as it stands, on the host cores) on the
    other workloads: the 4x4x4 box at N=7 (A x median of 5, 100 CG
    iterations), the degree-sweep meshes for N in 3, 7, 11, 15 (A x once, 3 CG
    iterations, per iteration), and the 80x80x80 box at N=7 (per-iteration
    time, with the time to 1e-10 extrapolated from the iteration count the GPU
    solvers needed, labelled as such)."""
    from oracle import oracle as orc
    out = {"impl": "reference", "workload": "oracle timings on the host cores", "cores": orc.num_threads(),
           "results": []}

    def one(label, dims, N, ax_reps, iters, lam=0.1, kind=0):
        t0 = time.perf_counter()
        m = orc.Mesh(*dims, N, rho=0.1, seed=0)
        t_create = time.perf_counter() - t0
        x = np.random.default_rng(0).standard_normal(m.n_global)
        ts = []
        for _ in range(ax_reps):
            t0 = time.perf_counter()
            m.apply_A(x, lam)
            ts.append(time.perf_counter() - t0)
        b = m.rhs(kind=kind, seed=0, lam=0.0) if kind else m.rhs(kind=0, seed=0)
        t0 = time.perf_counter()
        m.cg(b, lam, rtol=0.0, max_it=iters)
        t_cg = time.perf_counter() - t0
        rec = {"config": label, "N": N, "elements": list(dims), "n_global": m.n_global, "setup_s": t_create,
               "ax_ms_median": float(np.median(ts)) * 1e3, "ax_gdofs": m.n_global / float(np.median(ts)) / 1e9,
               "cg_iterations": iters, "cg_ms_per_iteration": t_cg * 1e3 / iters,
               "cg_gdofs": m.n_global * iters / t_cg / 1e9}
        m.close()
        out["results"].append(rec)
        print(json.dumps(rec), flush=True)
        return rec

    one("4x4x4 box, N=7", (4, 4, 4), 7, 5, 100)
    for N in (3, 7, 11, 15):
        one("degree sweep", c2_dims(N), N, 1, 3)
    r3 = one("80x80x80 box, N=7, manufactured rhs (per iteration)", (80, 80, 80), 7, 1, 1, lam=0.0, kind=1)
    # iteration counts of the GPU solvers to 1e-10 on this mesh (FP64 CG 3710)
    r3["time_to_1e-10_s_extrapolated"] = r3["cg_ms_per_iteration"] * 3710 / 1e3
    r3["extrapolation"] = "per-iteration time x 3710 FP64 CG iterations (the GPU FP64 solver's count)"
    print(json.dumps(out), flush=True)


def run_reference(args, rank, world, local):
    if rank != 0:
        return
    if args.workload != "c2":
        run_reference_workloads(args)
        return
    from oracle import oracle as orc
    N = args.N
    ex, ey, ez = c2_dims(N)
    dims = (16, 16, 16)
    m = orc.Mesh(*dims, N, rho=0.1, seed=0)
    b = m.rhs(kind=0, seed=0)
    if args.warmup:
        m.cg(b, 0.1, rtol=0.0, max_it=args.warmup)
    t0 = time.perf_counter()
    m.cg(b, 0.1, rtol=0.0, max_it=args.steps)
    dt = time.perf_counter() - t0
    v = m.n_global * args.steps / dt / 1e9
    out = {
        "impl": "reference",
        "metric": "Ax GDOF/s (FP64; one CG iteration = one A x and its fused vector stage)",
        "value": v, "unit": "GDOF/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded perturbed box, SplitMix64 uniform rhs)",
        "config": {"workload": f"degree sweep config at N={N}: {ex}x{ey}x{ez} hexahedra (bounded sample "
                               f"{dims[0]}x{dims[1]}x{dims[2]} on the host cores)", "N": N},
        "cpu_baseline": {"value": v, "unit": "GDOF/s", "cores": orc.num_threads(), "kind": "oracle",
                         "sample": f"N={N}, {dims[0]}x{dims[1]}x{dims[2]} elements (N_G={m.n_global}), "
                                   f"{args.steps} FP64 CG iterations"},
        "e2e": {"value": v, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- operator sweep

def run_sweep(args, rank, world, local):
    """Operator-only degree sweep (mean of 50 back-to-back launches, as the paper's Sec. 4.1)."""
    import torch

    from paper_2202_12477_gb300 import accounting as acc
    from paper_2202_12477_gb300 import hb, inputs

    torch.cuda.set_device(local)
    pk = peaks()
    Ns = [int(v) for v in args.degrees.split(",")] if args.degrees else list(range(1, 16))
    variants = [int(v) for v in args.variants.split(",")] if args.variants else [None]
    for N in Ns:
        for prec in args.precisions.split(","):
            dims = c2_dims(N, args.local_nodes)
            m = hb.Mesh(*dims, N, perturb=0.1, seed=0, fp32=(prec == "f32"))
            hbprec = {"f64": hb.HB_F64, "f32": hb.HB_F32, "f64x": hb.HB_F64X}[prec]
            varprec = hbprec  # each precision keeps its own kernel variant
            dt = torch.float32 if prec == "f32" else torch.float64
            x = torch.from_numpy(inputs.random_vector(m.n_global, 1)).to("cuda", dt)
            y = torch.empty_like(x)
            for var in variants:
                if var is not None:
                    hb.hb_set_kernel_variant(m.handle, varprec, var)
                var = hb.hb_get_kernel_variant(m.handle, varprec)
                for _ in range(3):
                    m.apply_A(x, y, lam=0.1, prec=hbprec)
                torch.cuda.synchronize()
                hb.hb_profile_reset()
                hb.hb_profile_enable(True)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                reps = args.reps
                with ClockSampler(gpu_uuid()) as clk:
                    e0.record()
                    for _ in range(reps):
                        m.apply_A(x, y, lam=0.1, prec=hbprec)
                    e1.record()
                    torch.cuda.synchronize()
                hb.hb_profile_enable(False)
                t = e0.elapsed_time(e1) / reps
                axm, axn = hb.hb_profile_read("ax_local")
                asm, asn = hb.hb_profile_read("assemble")
                esz = 4 if prec == "f32" else 8
                fl = acc.op_flops(m.E, N)
                rec = {"workload": "operator sweep", "N": N, "prec": prec, "variant": var, "elements": list(dims),
                       "n_local": m.n_local, "n_global": m.n_global, "ms": t,
                       "ax_local_ms": axm / axn, "assemble_ms": asm / asn,
                       "gdofs": m.n_global / (t * 1e-3) / 1e9, "gflops_paper": fl / (t * 1e-3) / 1e9,
                       "eff_gbs_method_min": acc.ax_min_bytes(m.n_global, m.n_local, esz) / (t * 1e-3) / 1e9,
                       "ax_local_gbs": acc.ax_local_bytes(m.n_global, m.n_local, esz) / (axm / axn * 1e-3) / 1e9,
                       "assemble_gbs": acc.assemble_bytes(m.n_global, m.info.nnz, esz) / (asm / asn * 1e-3) / 1e9,
                       "hbm_peak_gbs": pk["hbm_gbs"], "clocks": clk.summary()}
                rec["hbm_frac_method_min"] = rec["eff_gbs_method_min"] / pk["hbm_gbs"]
                rec["alu_frac"] = (acc.op_local_flops(m.E, N) / (axm / axn * 1e-3) / 1e12
                                   / (pk["fp64_tflops"] if prec == "f64" else pk["fp32_tflops"]))
                if prec == "f64x":
                    # a double-float flop costs several FP32 instructions: no single ALU roof
                    rec["alu_frac"] = None
                print(json.dumps(rec), flush=True)
            m.close()
            del x, y
            torch.cuda.empty_cache()


def _solve_report(m, b, lam, prec, rtol, screen=0, max_it=200000, inner_rtol=1e-4, precond=0):
    import torch

    from paper_2202_12477_gb300 import hb
    x = m.vec()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    x, res = m.cg(b, x=x, lam=lam, rtol=rtol, max_it=max_it, prec=prec, screen=screen, inner_rtol=inner_rtol,
                  precond=precond)
    e1.record()
    torch.cuda.synchronize()
    # FP64 residual of the returned solution, recomputed with the FP64 operator
    r = b - m.apply_A(x, lam=lam, screen=screen)
    rel = float(torch.linalg.norm(r) / torch.linalg.norm(b))
    return x, {"prec": {hb.HB_F64: "f64", hb.HB_MIXED: "mixed", hb.HB_F64X: "f64x"}[prec], "precond": ["none", "jacobi"][precond],
               "time_s": e0.elapsed_time(e1) / 1e3,
               "iters": res.iters, "outer_iters": res.outer_iters, "status": hb.STATUS_NAMES[res.status],
               "rel_res_fp64": rel}


def sweep_compact(local_nodes=1.28e8, degrees=range(1, 16), reps=5):
    """The degree sweep's operator figures per N (1.28e8 local nodes, the
    degree-sweep configuration's box at each N, perturb 0.1): the FP32 element
    kernel's rate against its algorithmic bytes (the mixed solver's inner
    operator) and FP64 A x in GDOF/s, each with the mesh's default kernel
    variant (no autotuning); CUDA events over `reps` applications after 2."""
    import torch

    from paper_2202_12477_gb300 import accounting as acc
    from paper_2202_12477_gb300 import hb, inputs
    pk = peaks()
    out = {"workload": f"degree sweep, {local_nodes:.3g} local nodes per mesh, default kernel variants, "
                       f"{reps} applications after 2", "f32_element_tbs": {}, "f32_element_hbm_frac": {},
           "f64_ax_gdofs": {},
           "note": "default variants: the pencil kernels (the FP64 headline's tensor-core kernel is the autotuner's "
                   "choice at N=7, timed in the headline itself)"}
    for N in degrees:
        dims = c2_dims(N, local_nodes)
        m = hb.Mesh(*dims, N, perturb=0.1, seed=0, fp32=True)
        for prec in (hb.HB_F32, hb.HB_F64):
            dt = torch.float32 if prec == hb.HB_F32 else torch.float64
            x = torch.from_numpy(inputs.random_vector(m.n_global, 1)).to("cuda", dt)
            y = torch.empty_like(x)
            for _ in range(2):
                m.apply_A(x, y, lam=0.1, prec=prec)
            torch.cuda.synchronize()
            hb.hb_profile_reset()
            hb.hb_profile_enable(True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                m.apply_A(x, y, lam=0.1, prec=prec)
            e1.record()
            torch.cuda.synchronize()
            hb.hb_profile_enable(False)
            if prec == hb.HB_F32:
                axm, axn = hb.hb_profile_read("ax_local")
                tbs = acc.ax_local_bytes(m.n_global, m.n_local, 4) / (axm / axn * 1e-3) / 1e12
                out["f32_element_tbs"][N] = round(tbs, 3)
                out["f32_element_hbm_frac"][N] = round(tbs * 1e3 / pk["hbm_gbs"], 3)
            else:
                out["f64_ax_gdofs"][N] = round(m.n_global / (e0.elapsed_time(e1) / reps * 1e-3) / 1e9, 3)
            del x, y
        m.close()
        torch.cuda.empty_cache()
    return out


def c3_compact(E1=80, N=7):
    """The single large solve (N=7, 80^3 elements, manufactured rhs, lambda 0)
    to a true relative residual of 1e-10: plain FP64 CG, the FP32-inner / FP64
    defect-correction solver, and the same with the Jacobi preconditioner on
    its inner CG. Each time is one hb_cg_solve; rel_res_fp64 is recomputed
    here with the FP64 operator."""
    import torch

    from paper_2202_12477_gb300 import autotune, hb
    m = hb.Mesh(E1, E1, E1, N, perturb=0.1, seed=0, fp32=True)
    chosen = autotune.tune_mesh(m, lam=0.0, exclude=hb.HB_VARIANT_GRID)
    b = m.rhs(kind=1, lam=0.0)
    out = {"workload": f"single large solve N={N}, {E1}^3 elements, perturb 0.1h, manufactured rhs, lambda 0, "
                       f"true relative residual 1e-10",
           "n_global": m.n_global, "kernel_variants": {"f64": chosen[hb.HB_F64], "f32": chosen[hb.HB_F32]}}
    x64, r = _solve_report(m, b, 0.0, hb.HB_F64, 1e-10)
    out["fp64"] = r
    xm, r = _solve_report(m, b, 0.0, hb.HB_MIXED, 1e-10)
    out["mixed"] = r
    _, r = _solve_report(m, b, 0.0, hb.HB_MIXED, 1e-10, precond=1)
    out["mixed_jacobi"] = r
    out["mixed_vs_fp64_rel_err"] = float(torch.linalg.norm(xm - x64) / torch.linalg.norm(x64))
    out["speedup_mixed_over_fp64"] = out["fp64"]["time_s"] / out["mixed"]["time_s"]
    out["speedup_mixed_jacobi_over_fp64"] = out["fp64"]["time_s"] / out["mixed_jacobi"]["time_s"]
    del x64, xm, b
    m.close()
    return out


def run_c3(args, rank, world, local):
    """Single large solve: N=7, 80^3 elements, manufactured rhs, FP64 CG vs
    FP32-inner / FP64 defect correction, both to relative residual 1e-10."""
    import torch

    from paper_2202_12477_gb300 import autotune, hb
    torch.cuda.set_device(local)
    N, E1 = args.N if args.N != 7 else 7, args.c3_elems
    m = hb.Mesh(E1, E1, E1, N, perturb=0.1, seed=0, fp32=True)
    chosen = autotune.tune_mesh(m, lam=0.0)
    b = m.rhs(kind=1, lam=0.0)
    out = {"workload": f"single large solve N={N}, {E1}^3 elements, perturb 0.1h, manufactured rhs "
                       f"(u = sin sin sin), lambda 0, rtol 1e-10", "n_global": m.n_global, "n_local": m.n_local,
           "kernel_variants": {"f64": chosen[hb.HB_F64], "f32": chosen[hb.HB_F32]}, "results": []}
    xs = {}
    for prec in (hb.HB_F64, hb.HB_MIXED):
        x, rec = _solve_report(m, b, 0.0, prec, 1e-10)
        xs[prec] = x
        out["results"].append(rec)
    for prec in (hb.HB_F64, hb.HB_MIXED):  # with the Jacobi preconditioner
        _, rec = _solve_report(m, b, 0.0, prec, 1e-10, precond=1)
        out["results"].append(rec)
    # FP64 CG with the double-float element kernel
    x, rec = _solve_report(m, b, 0.0, hb.HB_F64X, 1e-10)
    out["results"].append(rec)
    out["f64x_vs_fp64_rel_err"] = float(torch.linalg.norm(x - xs[hb.HB_F64]) / torch.linalg.norm(xs[hb.HB_F64]))
    d = xs[hb.HB_MIXED] - xs[hb.HB_F64]
    out["mixed_vs_fp64_rel_err"] = float(torch.linalg.norm(d) / torch.linalg.norm(xs[hb.HB_F64]))
    out["speedup_mixed_over_fp64"] = out["results"][0]["time_s"] / out["results"][1]["time_s"]
    if args.c3_inner:
        # the inner tolerance of the mixed solver (its one free parameter), with
        # and without the Jacobi preconditioner on the inner CG
        sweep = []
        for tol in [float(v) for v in args.c3_inner.split(",")]:
            for pc in (0, 1):
                _, rec = _solve_report(m, b, 0.0, hb.HB_MIXED, 1e-10, inner_rtol=tol, precond=pc)
                rec["inner_rtol"] = tol
                sweep.append(rec)
        out["mixed_inner_sweep"] = sweep
        best = min(sweep, key=lambda r: r["time_s"] if r["rel_res_fp64"] <= 1e-10 else 1e30)
        out["mixed_best"] = best
        out["speedup_best_mixed_over_fp64"] = out["results"][0]["time_s"] / best["time_s"]
    print(json.dumps(out), flush=True)


def run_c4(args, rank, world, local):
    """Mixed-precision stress: N=15, 24^3 elements, vertex perturbation 0.3h,
    lambda in {0, 1e-3, 10}; FP32 operator / inner CG with FP64 residual, dots
    and update against plain FP64 CG; error of the mixed solution against the
    FP64 solution per lambda."""
    import torch

    from paper_2202_12477_gb300 import autotune, hb
    torch.cuda.set_device(local)
    E1 = args.c4_elems
    # 0.3h perturbations can invert an element; the library refuses such a mesh
    # (HB_ERR_GEOMETRY). Every refused seed is reported and the first valid one used.
    # If every seed tried at 0.3h inverts an element, the perturbation is stepped
    # down (seed 0) until the mesh is valid; all refusals are reported.
    refused, m, rho = [], None, 0.3
    tries = [(0.3, s) for s in range(5)] + [(r, 0) for r in (0.28, 0.26, 0.25, 0.24, 0.22, 0.2, 0.15, 0.1)]
    for rho, seed in tries:
        try:
            m = hb.Mesh(E1, E1, E1, 15, perturb=rho, seed=seed, fp32=True)
            break
        except hb.HBError as err:
            if err.status != hb.HB_ERR_GEOMETRY:
                raise
            refused.append({"perturb": rho, "seed": seed, "error": str(err)})
    if m is None:
        print(json.dumps({"workload": "mixed-precision stress", "refused": refused}), flush=True)
        return
    autotune.tune_mesh(m)
    b = m.rhs(kind=0, seed=0)
    out = {"workload": f"mixed-precision stress N=15, {E1}^3 elements, perturb {rho}h (0.3h asked), uniform rhs, "
                       f"rtol 1e-10",
           "n_global": m.n_global, "perturb_used": rho, "mesh_seed": seed, "refused": refused,
           "min_detJ": m.info.min_detJ,
           "per_lambda": []}
    for lam in (0.0, 1e-3, 10.0):
        x64, r64 = _solve_report(m, b, lam, hb.HB_F64, 1e-10)
        xm, rm = _solve_report(m, b, lam, hb.HB_MIXED, 1e-10)
        err = float(torch.linalg.norm(xm - x64) / torch.linalg.norm(x64))
        out["per_lambda"].append({"lambda": lam, "fp64": r64, "mixed": rm, "mixed_vs_fp64_rel_err": err,
                                  "speedup": r64["time_s"] / rm["time_s"]})
    print(json.dumps(out), flush=True)


def _c5_requests(n, emin, emax, seed=0):
    """Seeded request stream: Ek uniform in emin..emax, N in {3,5,7,9,11},
    rtol in {1e-8, 1e-10}, perturbation 0.1h, uniform rhs, lambda 0.1."""
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        out.append(dict(ex=int(rng.integers(emin, emax + 1)), N=int(rng.choice([3, 5, 7, 9, 11])),
                        rtol=float(rng.choice([1e-8, 1e-10])), seed=int(i), rhs_seed=int(i)))
    for r in out:
        r["ey"] = r["ez"] = r["ex"]
    return out


def _serve_run(reqs, arrivals, budget, slots, k):
    """Submits reqs at the given arrival times (s from start), waits for all;
    returns per-request latencies (ms), statuses and the makespan."""
    from paper_2202_12477_gb300 import hb
    srv = hb.Server(budget, max_slots=slots, iters_per_launch=k)
    t0 = time.perf_counter()
    tickets, lat, status = [], {}, {}
    i = 0
    while len(lat) < len(reqs):
        now = time.perf_counter() - t0
        while i < len(reqs) and arrivals[i] <= now:
            r = reqs[i]
            tickets.append(srv.submit(ex=r["ex"], ey=r["ey"], ez=r["ez"], N=r["N"], perturb=0.1, seed=r["seed"],
                                      rhs_seed=r["rhs_seed"], lam=0.1, rtol=r["rtol"]))
            i += 1
        for t in tickets:
            if t in lat:
                continue
            p = srv.poll(t)
            if p is not None:
                lat[t] = p[0].time_ms
                status[t] = p[0].status
                if p[0].status != hb.HB_OK:
                    _FAIL_MSG.setdefault(hb.STATUS_NAMES.get(p[0].status, str(p[0].status)),
                                         getattr(srv, "last_failure", ""))
        time.sleep(0.0005)
    makespan = time.perf_counter() - t0
    st = srv.stats()
    rounds = st.rounds
    srv.close()
    return [lat[t] for t in tickets], [status[t] for t in tickets], makespan, rounds


_FAIL_MSG = {}  # first failure message seen per status name


def _not_ok(statuses):
    """Counts of the statuses other than HB_OK, by name, with the first
    message each one came with."""
    from paper_2202_12477_gb300 import hb
    out = {}
    for st in statuses:
        if st != hb.HB_OK:
            name = hb.STATUS_NAMES.get(st, str(st))
            out.setdefault(name, {"count": 0, "message": _FAIL_MSG.get(name, "")})
            out[name]["count"] += 1
    return out


def c5_compact(n_requests, emax=32, budget_gb=160.0, slots=32, k=16):
    """The serving stream on n_requests requests (Ek uniform 2..emax, N in
    3..11 odd, rtol 1e-8 / 1e-10, mixed precision): capacity with every
    request submitted at once, then Poisson arrivals at 0.5, 0.8 and 1.0 x that
    capacity (solves/s, p50, p99 latency from submit to completion), the same
    requests served one at a time, and solved one at a time with hb_cg_solve
    in FP64 and in mixed precision."""
    import numpy as np
    import torch

    from paper_2202_12477_gb300 import hb
    reqs = _c5_requests(n_requests, 2, emax)
    budget = int(budget_gb * (1 << 30))
    out = {"workload": f"serving stream: {len(reqs)} of the 2,000 requests of the serving config (Ek uniform "
                       f"2..{emax}, N in 3..11 odd, rtol 1e-8 / 1e-10), mixed precision, {slots} slots, {k} inner "
                       f"iterations per launch, budget {budget_gb} GB"}
    lat, sts, mk, rounds = _serve_run(reqs, [0.0] * len(reqs), budget, slots, k)
    cap = len(reqs) / mk
    out["capacity_solves_per_s"] = cap
    out["all_at_once"] = {"solves_per_s": cap, "p50_ms": float(np.percentile(lat, 50)),
                          "p99_ms": float(np.percentile(lat, 99)), "ok": int(sum(s == hb.HB_OK for s in sts)),
                          "not_ok": _not_ok(sts)}
    rng = np.random.Generator(np.random.PCG64(1))
    for f in (0.5, 0.8, 1.0):
        arr = np.cumsum(rng.exponential(1.0 / (f * cap), size=len(reqs)))
        arr -= arr[0]
        lat, sts, mk, rounds = _serve_run(reqs, list(arr), budget, slots, k)
        out[f"load_{f:.1f}"] = {"solves_per_s": len(reqs) / mk, "p50_ms": float(np.percentile(lat, 50)),
                                "p99_ms": float(np.percentile(lat, 99)),
                                "ok": int(sum(s == hb.HB_OK for s in sts)), "not_ok": _not_ok(sts)}
    # the same requests through the server one at a time (submit, wait, next):
    # the serving path's own latency, without other requests sharing the GPU
    srv = hb.Server(budget, max_slots=slots, iters_per_launch=k)
    lat = []
    for r in reqs:
        t = srv.submit(ex=r["ex"], ey=r["ey"], ez=r["ez"], N=r["N"], perturb=0.1, seed=r["seed"],
                       rhs_seed=r["rhs_seed"], lam=0.1, rtol=r["rtol"])
        res, _ = srv.wait(t, interval=0.0001)
        lat.append(res.time_ms)
    srv.close()
    out["served_alone"] = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99))}
    for prec, name in ((hb.HB_F64, "sequential_fp64"), (hb.HB_MIXED, "sequential_mixed")):
        t0 = time.perf_counter()
        lat = []
        for r in reqs:
            ts = time.perf_counter()
            m = hb.Mesh(r["ex"], r["ey"], r["ez"], r["N"], perturb=0.1, seed=r["seed"], fp32=True)
            b = m.rhs(kind=0, seed=r["rhs_seed"])
            m.cg(b, lam=0.1, rtol=r["rtol"], max_it=200000, prec=prec)
            torch.cuda.synchronize()
            lat.append((time.perf_counter() - ts) * 1e3)
            m.close()
        mk = time.perf_counter() - t0
        out[name] = {"solves_per_s": len(reqs) / mk, "p50_ms": float(np.percentile(lat, 50)),
                     "p99_ms": float(np.percentile(lat, 99))}
    out["served_over_sequential_fp64"] = cap / out["sequential_fp64"]["solves_per_s"]
    out["served_over_sequential_mixed"] = cap / out["sequential_mixed"]["solves_per_s"]
    return out


def run_c5(args, rank, world, local):
    """Serving stream with Poisson arrivals at fractions of the measured
    capacity; mixed precision; p50/p99 latency and solves/s, beside solving
    the same requests one at a time with hb_cg_solve in FP64 and in mixed."""
    import numpy as np
    import torch

    from paper_2202_12477_gb300 import hb
    torch.cuda.set_device(local)
    reqs = _c5_requests(args.c5_requests, 2, args.c5_emax)
    budget = int(args.c5_budget_gb * (1 << 30))
    out = {"workload": f"serving stream: {len(reqs)} requests, Ek uniform 2..{args.c5_emax}, N in 3..11 odd, "
                       f"rtol 1e-8 / 1e-10, mixed precision, {args.c5_slots} slots, {args.c5_k} inner "
                       f"iterations per launch, budget {args.c5_budget_gb} GB",
           "runs": []}
    # capacity: everything submitted at once
    lat, sts, mk, rounds = _serve_run(reqs, [0.0] * len(reqs), budget, args.c5_slots, args.c5_k)
    cap = len(reqs) / mk
    out["capacity_solves_per_s"] = cap
    out["runs"].append({"offered": "all at t=0", "solves_per_s": cap, "p50_ms": float(np.percentile(lat, 50)),
                        "p99_ms": float(np.percentile(lat, 99)), "rounds": rounds,
                        "ok": int(sum(1 for s in sts if s == hb.HB_OK)),
                            "not_ok": _not_ok(sts)})
    rng = np.random.Generator(np.random.PCG64(1))
    for f in (0.5, 0.8, 1.0):
        rate = f * cap
        arr = np.cumsum(rng.exponential(1.0 / rate, size=len(reqs)))
        arr -= arr[0]
        lat, sts, mk, rounds = _serve_run(reqs, list(arr), budget, args.c5_slots, args.c5_k)
        out["runs"].append({"offered": f"{f:.1f} x capacity (Poisson)", "solves_per_s": len(reqs) / mk,
                            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                            "rounds": rounds, "ok": int(sum(1 for s in sts if s == hb.HB_OK)),
                            "not_ok": _not_ok(sts)})
    # one at a time through hb_cg_solve, FP64 and mixed
    for prec, name in ((hb.HB_F64, "sequential_fp64"), (hb.HB_MIXED, "sequential_mixed")):
        t0 = time.perf_counter()
        lat = []
        for r in reqs:
            ts = time.perf_counter()
            m = hb.Mesh(r["ex"], r["ey"], r["ez"], r["N"], perturb=0.1, seed=r["seed"], fp32=True)
            b = m.rhs(kind=0, seed=r["rhs_seed"])
            m.cg(b, lam=0.1, rtol=r["rtol"], max_it=200000, prec=prec)
            torch.cuda.synchronize()
            lat.append((time.perf_counter() - ts) * 1e3)
            m.close()
        mk = time.perf_counter() - t0
        out[name] = {"solves_per_s": len(reqs) / mk, "p50_ms": float(np.percentile(lat, 50)),
                     "p99_ms": float(np.percentile(lat, 99))}
    print(json.dumps(out), flush=True)


def run_split(args, rank, world, local):
    """Split operator with the halo / gather exchanges overlapped (Sec. 3.3),
    ranks emulated on one GPU: per rank grid, mean of `reps` back-to-back
    applications of the partitioned A against the one-mesh A (same pencil
    kernel, variant 3), the halo exchange alone, and the sum of the per-kernel
    device times over all ranks (above the wall time when ranks overlap)."""
    import time

    import torch

    from paper_2202_12477_gb300 import hb, inputs
    torch.cuda.set_device(local)
    N = args.N
    dims = c2_dims(N, args.local_nodes)
    m = hb.Mesh(*dims, N, perturb=0.1, seed=0, fp32=False)
    hb.hb_set_kernel_variant(m.handle, hb.HB_F64, 3)
    x_lex = inputs.random_vector(m.n_global, 1)
    reps = args.reps

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    xd = torch.from_numpy(x_lex).cuda()
    yd = torch.empty_like(xd)
    ms_fused = timed(lambda: m.apply_A(xd, yd, lam=0.1))
    grids = [tuple(int(v) for v in g.split("x")) for g in args.split_grids.split(",")]
    for grid in grids:
        t0 = time.time()
        part = hb.Part(m, *grid, seed=0)
        t_build = time.time() - t0
        xp = torch.from_numpy(x_lex[part.perm]).cuda()
        yp = torch.empty_like(xp)
        ms_split = timed(lambda: part.apply_A(xp, yp, lam=0.1))
        ms_exch = timed(lambda: part.halo_exchange(xp))
        # per-kernel device times over all ranks (one pass, events on each rank's stream)
        torch.cuda.synchronize()
        hb.hb_profile_reset()
        hb.hb_profile_enable(True)
        part.apply_A(xp, yp, lam=0.1)
        torch.cuda.synchronize()
        hb.hb_profile_enable(False)
        kern = {}
        for name in ("ax_local", "part_pack", "part_halo_gather", "part_local_gather", "part_final"):
            t, c = hb.hb_profile_read(name)
            kern[name] = {"ms": t, "launches": c}
        err = float(torch.max(torch.abs(yp - yd[torch.from_numpy(part.perm.astype('int64')).cuda()]))
                    / torch.max(torch.abs(yd)))
        print(json.dumps({"workload": "split operator, virtual ranks on one GPU", "N": N, "elements": list(dims),
                          "n_global": m.n_global, "ranks": list(grid), "n_shared": part.info.n_shared,
                          "exchange_values": part.info.exchange_values, "build_s": t_build,
                          "ms_fused": ms_fused, "ms_split": ms_split, "split_over_fused": ms_split / ms_fused,
                          "ms_halo_exchange_alone": ms_exch, "kernels_one_apply": kern,
                          "kernel_sum_ms": sum(v["ms"] for v in kern.values()),
                          "max_rel_diff_vs_fused": err, "reps": reps}), flush=True)
        part.close()
        del xp, yp
        torch.cuda.empty_cache()


def run_scat(args, rank, world, local):
    """Assembled against scattered (NekBone) storage: FP64 CG time per
    iteration over `steps` fixed iterations on the degree-sweep mesh (same
    pencil element kernel, variant 3), with each scheme's algorithmic bytes
    per iteration (Sec. 3.1's claim that assembled storage moves fewer)."""
    import torch

    from paper_2202_12477_gb300 import accounting as acc
    from paper_2202_12477_gb300 import hb
    torch.cuda.set_device(local)
    pk = peaks()
    Ns = [int(v) for v in args.degrees.split(",")] if args.degrees else [args.N]
    K = max(args.steps, 10)
    for N in Ns:
        dims = c2_dims(N, args.local_nodes)
        m = hb.Mesh(*dims, N, perturb=0.1, seed=0, fp32=False)
        hb.hb_set_kernel_variant(m.handle, hb.HB_F64, 3)
        sc = hb.Scat(m)
        b = m.rhs(kind=0, seed=0)
        bL = sc.scatter(b)
        out = {"workload": "assembled vs scattered storage, FP64 CG", "N": N, "elements": list(dims),
               "n_global": m.n_global, "n_local": m.n_local, "iterations": K}
        for name, solve in (("assembled", lambda: m.cg(b, lam=0.1, rtol=0.0, max_it=K)),
                            ("scattered", lambda: sc.cg(bL, lam=0.1, rtol=0.0, max_it=K))):
            solve()  # warm-up (graph capture on the assembled path)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _, res = solve()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / K
            nb = (acc.assembled_cg_min_bytes(m.n_global, m.n_local) if name == "assembled"
                  else acc.scattered_cg_min_bytes(m.n_local))
            out[name] = {"ms_per_iter": ms, "gdofs": m.n_global / (ms * 1e-3) / 1e9, "iters": res.iters,
                         "rel_res": res.rel_res, "min_bytes_per_iter": nb,
                         "bytes_time_at_hbm_peak_ms": nb / (pk["hbm_gbs"] * 1e9) * 1e3}
        out["scattered_over_assembled_time"] = out["scattered"]["ms_per_iter"] / out["assembled"]["ms_per_iter"]
        out["scattered_over_assembled_bytes"] = (out["scattered"]["min_bytes_per_iter"]
                                                 / out["assembled"]["min_bytes_per_iter"])
        out["residual_rel_diff"] = abs(out["scattered"]["rel_res"] - out["assembled"]["rel_res"]) / max(
            out["assembled"]["rel_res"], 1e-300)
        print(json.dumps(out), flush=True)
        sc.close()
        m.close()
        torch.cuda.empty_cache()


def run_c1(args, rank, world, local):
    """Small latency-bound solve: 4^3 elements, N=7, perturb 0.1h, lambda 0.1,
    uniform rhs, exactly 100 FP64 CG iterations: the fused solver (all
    iterations in one cooperative kernel, the library's choice for meshes this
    small) and, beside it, the launched kernels replayed as CUDA graphs."""
    import torch

    from paper_2202_12477_gb300 import hb
    torch.cuda.set_device(local)
    m = hb.Mesh(4, 4, 4, 7, perturb=0.1, seed=0, fp32=True)
    from paper_2202_12477_gb300 import autotune
    variant = autotune.tune_mesh(m, precs=(hb.HB_F64,), lam=0.1, reps=20)[hb.HB_F64]
    b = m.rhs(kind=0, seed=0)
    x = m.vec()
    for _ in range(max(args.warmup, 3)):
        m.cg(b, x=x.zero_(), lam=0.1, rtol=0.0, max_it=100)
    torch.cuda.synchronize()
    reps = 20

    def timed():
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            x.zero_()
            _, r = m.cg(b, x=x, lam=0.1, rtol=0.0, max_it=100)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, r

    t, res = timed()  # default: fused
    hb.lib().hb_set_cg_fused(m.handle, 1)
    m.cg(b, x=x.zero_(), lam=0.1, rtol=0.0, max_it=100)
    t_l, res_l = timed()
    hb.lib().hb_set_cg_fused(m.handle, 0)
    out = {"workload": "4x4x4 hexahedra, N=7, perturb 0.1h, lambda 0.1, uniform rhs, 100 fixed FP64 CG iterations",
           "n_global": m.n_global, "n_local": m.n_local, "ms_per_solve": t, "us_per_iteration": t * 10.0,
           "gdofs": m.n_global * 100 / (t * 1e-3) / 1e9, "rel_res": res.rel_res, "iters": res.iters,
           "solver": "fused (one cooperative kernel)",
           "launched": {"us_per_iteration": t_l * 10.0, "rel_res": res_l.rel_res, "kernel_variant": variant}}
    print(json.dumps(out), flush=True)


def run_probe(args, rank, world, local):
    """Calibration probes: the 8:1 streaming kernel (Sec. 4.1) in FP64 and FP32,
    the same traffic without arithmetic, a copy, and FMA throughput."""
    import torch

    from paper_2202_12477_gb300 import hb
    torch.cuda.set_device(local)
    nb = 4 << 30
    out = {"workload": "calibration probes (4 GiB buffers, best of 5)",
           "stream81_fp64_gbs": hb.hb_probe(hb.HB_PROBE_STREAM81_FP, hb.HB_F64, nb),
           "stream81_fp32_gbs": hb.hb_probe(hb.HB_PROBE_STREAM81_FP, hb.HB_F32, nb),
           "stream81_bits64_gbs": hb.hb_probe(hb.HB_PROBE_STREAM81_BITS, hb.HB_F64, nb),
           "copy_gbs": hb.hb_probe(hb.HB_PROBE_COPY, hb.HB_F64, nb),
           "fma_fp64_gflops": hb.hb_probe(hb.HB_PROBE_FMA, hb.HB_F64, 0),
           "fma_fp32_gflops": hb.hb_probe(hb.HB_PROBE_FMA, hb.HB_F32, 0),
           "dmma_fp64_gflops": hb.hb_probe(hb.HB_PROBE_DMMA, hb.HB_F64, 0),
           "dmma_plus_fma_fp64_gflops": hb.hb_probe(hb.HB_PROBE_DMMA_FMA, hb.HB_F64, 0)}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c2", "sweep", "c1", "c3", "c4", "c5", "probe", "split", "scat"])
    ap.add_argument("--split-grids", default="1x1x1,2x1x1,2x2x2,4x4x2")
    ap.add_argument("--c5-requests", type=int, default=200)
    ap.add_argument("--c5-emax", type=int, default=32)
    ap.add_argument("--c5-slots", type=int, default=32)
    ap.add_argument("--c5-k", type=int, default=16)
    ap.add_argument("--c5-budget-gb", type=float, default=160.0)
    ap.add_argument("--c3-elems", type=int, default=80)
    ap.add_argument("--c3-inner", default="", help="comma-separated inner tolerances to sweep in the mixed solver")
    ap.add_argument("--c4-elems", type=int, default=24)
    ap.add_argument("--N", type=int, default=7)
    ap.add_argument("--degrees", default="")
    ap.add_argument("--precisions", default="f64,f32")
    ap.add_argument("--variants", default="")
    ap.add_argument("--reps", type=int, default=50)
    ap.add_argument("--local-nodes", type=float, default=1.28e8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-c3", action="store_true", help="leave the time-to-1e-10 solves out of the default line")
    ap.add_argument("--no-c5", action="store_true", help="leave the serving stream out of the default line")
    ap.add_argument("--no-sweep", action="store_true", help="leave the per-degree operator sweep out of the default line")
    ap.add_argument("--c5-default-requests", type=int, default=300,
                    help="requests of the serving stream measured in the default line")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gb300" and args.workload == "c2":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world, local)
        return
    from paper_2202_12477_gb300 import build
    build.build()
    if args.workload == "sweep":
        run_sweep(args, rank, world, local)
    elif args.workload == "c1":
        run_c1(args, rank, world, local)
    elif args.workload == "split":
        run_split(args, rank, world, local)
    elif args.workload == "scat":
        run_scat(args, rank, world, local)
    elif args.workload == "probe":
        run_probe(args, rank, world, local)
    elif args.workload == "c3":
        run_c3(args, rank, world, local)
    elif args.workload == "c4":
        run_c4(args, rank, world, local)
    elif args.workload == "c5":
        run_c5(args, rank, world, local)
    else:
        run_gb300(args, rank, world, local)


if __name__ == "__main__":
    main()
