"""Throughput of the interfacial-system hot path on GB300.

One step = build_cover + assemble_G (mixed form) + solve on the scaled
workload, the largest configuration that fits one GPU: Omega = [0,4]^2,
L = 1/2 Laplacian, 62 x 62 square lattice of 3,844 circles (3,600 floating
disks with 48(r) x 64(theta) grids, n = 3072 unknowns each), 16 knots per
circle, 1,000 paths per Monte Carlo knot, h = 1e-5: every row a1-a13 of
the hot path.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line on rank 0.  value = knots of C assembled and solved per
second over all ranks (each rank runs its own replica: the path has no
cross-rank exchange).  Extra keys: the FP64 form on the same GPU (on a
subset of the same disks), errors against the FP64 oracle on sampled rows,
the roofline of the dominant kernel and of the disk path, the oracle timed on
the host cores, legs on the variable-coefficient, batching, Eq. 46 and
averaged-row workloads, the adjoint (a14), clocks and launch counts.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "G-assembly knots/s + MC path-steps/s at stated err vs FP64 oracle, mixed vs FP64"
WORKLOAD = ("scaled: Omega=[0,4]^2, L=1/2 Lap, f=0, g=e^x sin y; 62x62 square lattice of circles r=0.8*4/62 "
            "(3844 circles, 3600 floating); 16 knots/circle, 48(r)x64(theta) disk grid (n=3072); "
            "1000 paths/knot, h=1e-5")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-oracle", action="store_true", help="skip the oracle legs (error check, cpu_baseline)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-form comparison")
    ap.add_argument("--no-grad", action="store_true", help="skip the adjoint (a14) leg")
    ap.add_argument("--no-poisson46", action="store_true",
                    help="skip the leg on the paper's Poisson test (Eq. 46, [-50,50]^2)")
    ap.add_argument("--no-averaged", action="store_true",
                    help="skip the leg with averaged multi-subdomain rows (Eq. 38-39)")
    ap.add_argument("--no-varcoef", action="store_true", help="skip the variable-coefficient workload leg")
    ap.add_argument("--no-adaptive", action="store_true", help="skip the batching (adaptive cover) leg")
    ap.add_argument("--lu-leaf", type=int, default=0,
                    help="force the pivoted recursive LU with this leaf width (0: the pivot-free tensor-core LU)")
    ap.add_argument("--lu-tmin", type=int, default=0, help="force the tensor-core threshold (with --lu-leaf)")
    ap.add_argument("--precond", choices=["none", "ras"], default="ras",
                    help="GMRES right preconditioner (RAS: Eq. 42-45, as the paper solves)")
    return ap.parse_args()


def dist_setup(n_gpus):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, ms_max):
    """Whole-job units per second: every rank processed units_per_rank (replicas, weak
    scaling) and the job took the slowest rank's time."""
    return world * units_per_rank / (ms_max / 1e3)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def flush_l2(buf):
    buf.fill_(1.0)          # 512 MB write, larger than the 129 MB L2


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
LU = {"lu_leaf_width": 0, "lu_tensor_min": 0}
SOLVE = {"precond": "ras"}


SOLVE_MS = []


def step(pdd, cfg, precision, stream):
    import torch
    cov = pdd.Cover(cfg, stream=stream)
    S = pdd.System(cov, cfg, precision, stream=stream, **LU)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    u = S.solve(rtol=1e-13, restart=64, stream=stream, precond=SOLVE["precond"])
    e1.record(stream)
    e1.synchronize()
    SOLVE_MS.append(e0.elapsed_time(e1))
    return cov, S, u


def _timed(pdd, cfg, precision, stream, flush, steps, precond=None, **kw):
    """steps timed passes (cover + assembly + solve) after one warm-up; returns (ms list, last stats, N)."""
    import torch
    times, st, N = [], None, 0
    for rep in range(steps + 1):
        flush_l2(flush)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cov = pdd.Cover(cfg, stream=stream)
        S = pdd.System(cov, cfg, precision, stream=stream, **kw)
        u = S.solve(rtol=1e-13, restart=64, stream=stream, precond=precond or SOLVE["precond"])
        e1.record(stream)
        torch.cuda.synchronize()
        if rep:
            times.append(e0.elapsed_time(e1))
        st, N = S.stats(), cov.N
        st["gmres_iters"] = S.last_solve["iters"]
        del cov, S, u
    return times, st, N


def run_ours(args, rank, world):
    import torch

    import paper_2311_08946_gb300 as pdd
    import workloads

    pdd.load()
    LU["lu_leaf_width"], LU["lu_tensor_min"] = args.lu_leaf, args.lu_tmin
    SOLVE["precond"] = args.precond
    cfg = workloads.scaled()
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(max(3, args.warmup)):
        cov, S, u = step(pdd, cfg, "mixed", stream)
        del cov, S, u
    torch.cuda.synchronize()
    times, stats, solve = [], [], []
    launches0 = pdd.launch_count()
    with ClockSampler(torch.cuda.current_device()) as clk:
        for _ in range(args.steps):
            flush_l2(flush)
            barrier(world)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            cov, S, u = step(pdd, cfg, "mixed", stream)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            stats.append(S.stats())
            solve.append(S.last_solve)
            N = cov.N
            del cov, S, u
    launches = pdd.launch_count() - launches0            # this library's kernels in the K timed steps
    timed_solve_ms = statistics.mean(SOLVE_MS[-args.steps:])
    ms = statistics.mean(times)
    ms_max = max_over_ranks(ms, world)
    value = job_throughput(N, world, ms_max)
    st = stats[-1]
    path_steps = st["path_steps"]
    mc_rate = path_steps / (statistics.mean(s["ms_paths"] for s in stats) / 1e3)

    # e2e: the public API with host-side inputs, result copied to pinned host memory
    e2e_times = []
    u_host = torch.empty(N, dtype=torch.float64, pin_memory=True)
    for _ in range(max(2, min(args.steps, 3))):
        flush_l2(flush)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cov, S, u = step(pdd, cfg, "mixed", stream)
        u_host.copy_(u, non_blocking=True)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
        del cov, S, u
    e2e_s = max_over_ranks(statistics.mean(e2e_times), world)
    h2d = 36 + 112 + 72 + 88        # domain, cover spec, operator and option structs
    e2e = {"value": job_throughput(N, world, 1e3 * e2e_s), "unit": "knots/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": N * 8}

    out = {"metric": METRIC, "value": value, "unit": "knots/s", "n_gpus": world, "steps": args.steps,
           "warmup": max(3, args.warmup), "ms_per_step": ms_max, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "precision": "mixed (FP32 pivot-free LU on tcgen05 with split-TF32 "
                      "products + FP64 refinement; FP32 path positions, FP64 weights and scores)",
                      "solve": f"FP64 GMRES(64), rtol 1e-13, precond {args.precond}", "knots": N,
                      "l2": "flushed between steps (512 MB write); wave buffers about 58 GB, 270+ GB touched per step",
                      "parallelism": f"replicas x{world}"},
           "mc_path_steps_per_s": world * mc_rate, "path_steps_per_step": path_steps,
           "stages_ms": {k: st[k] for k in ("ms_cover_rows", "ms_disks", "ms_operator", "ms_factor",
                                            "ms_refine", "ms_eval", "ms_paths", "ms_finalize", "ms_trisolve",
                                            "ms_tc_gemm", "ms_gemm_fused")},
           "refine_tol": 1e-12,
           "gmres": dict(solve[-1], precond=args.precond, ms=timed_solve_ms),
           "refine_sweeps_max": st["max_refine_sweeps"],
           "lu": ("pivot-free recursive, 64 x 64 diagonal blocks" if st["lu_leaf_width"] == 64 and not st["lu_blocked"]
                  else ("blocked" if st["lu_blocked"] else
                        f"pivoted recursive leaf={st['lu_leaf_width']} tensor_min={st['lu_tensor_min']}")) +
                 (" (pivoted fallback used)" if st["lu_pivoted_fallback"] else ""),
           "gpu_launches": int(launches), "gpu_launches_per_step": int(launches) // max(1, args.steps), "e2e": e2e,
           "clocks": clk.summary()}

    # rooflines: the dominant kernel (device time from CUDA events inside the library) and the disk path
    out["roofline"] = roofline(stats, cfg, N, timed_solve_ms)

    if not args.no_fp64 and rank == 0:
        out["fp64_form"] = fp64_form(pdd, stream, flush)
    if not args.no_oracle and rank == 0:
        out["err_vs_oracle"] = errors_vs_oracle(pdd, cfg, stream)
        out["cpu_baseline"] = cpu_baseline(cfg)
    if rank == 0 and not args.no_grad:
        out["grad"] = grad_bench(pdd, stream)
    # the extra workloads report an error in their own key rather than lose the line
    legs = [("varcoef", not args.no_varcoef, lambda: varcoef_leg(pdd, stream, flush)),
            ("adaptive", not args.no_adaptive, lambda: adaptive_leg(pdd, stream, flush)),
            ("poisson46", not args.no_poisson46, lambda: poisson46_leg(pdd, stream, flush)),
            ("averaged_rows", not args.no_averaged, lambda: averaged_leg(pdd, workloads.varcoef(), stream, flush))]
    for name, on, fn in legs:
        if rank == 0 and on:
            try:
                out[name] = fn()
            except Exception as e:                          # noqa: BLE001
                out[name] = {"error": str(e)}
    return out


# Thread-instructions per Euler-Maruyama step of k_paths<float,0,0,0>, the variant the scaled workload
# runs (f = c = 0, no control variate), from ncu: smsp__thread_inst_executed.sum / path-steps on the
# 6 x 6 lattice of the scaled workload's circles (profiles/k_paths_poisson46_mixed.md).  Refresh when
# the kernel changes.
PATHS_THREAD_INST_PER_STEP = 149.3
# FP32 FMA peak from the unit counts: 152 SMs x 128 FP32 lanes x 2 flop x the maximum SM clock
FP32_LANES_PER_SM = 128
# DRAM bytes (read + write) per useful flop of k_tc_gemm_pipe<1> from one ncu capture: the top-level
# Schur update (M = N = K = 1536) of 16 disks of the scaled workload, 795.7 MB read + 138.1 MB written
# for 1.1596e11 flop (profiles/k_tc_gemm_pipe_scaled_mixed.md).  Its operands and C grow with the
# flops of the same shape, so a full launch's traffic is taken in proportion.
GEMM_DRAM_BYTES_PER_FLOP = (795.685888e6 + 138.077440e6) / (16 * 2.0 * 1536 ** 3)


def tf32_peak(pk):
    """TF32 dense tensor peak: the measured BF16 peak x the nominal TF32/BF16 ratio (1.1 / 2.25)."""
    return pk["bf16_tflops"] * (1.1 / 2.25)


def roofline(stats, cfg, N, ms_solve):
    """Rooflines of the heaviest kernels, each from its own device time (CUDA events around its launches
    inside the library, on the stream they run on); the dominant one is the line's roofline, the others
    go under "others"; "disk_path" is the whole floating-disk stage (a6-a9) against the TF32 peak."""
    pk, src = peaks()
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    st = stats[-1]
    mean = lambda k: statistics.mean(s[k] for s in stats)
    n, nrhs = cfg["n_r"] * cfg["n_theta"], cfg["n_knots"] + 1
    issue = 152 * 4 * 32 * sm_mhz * 1e6
    fp32_peak = 152 * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    tf32 = tf32_peak(pk)
    out = {"stage_ms": {"paths": mean("ms_paths"), "factor": mean("ms_factor"), "refine": mean("ms_refine"),
                        "finalize": mean("ms_finalize"), "operator": mean("ms_operator"), "eval": mean("ms_eval"),
                        "solve": ms_solve}}
    # a7: split-TF32 GEMMs of the pivot-free LU on tcgen05 (useful 2MNK flop; three TF32 products each).
    # The long-K updates stream pre-split tiles (k_tc_gemm_pipe, tensor-bound); the K = 64 updates split
    # their operands in the kernel (k_tc_gemm_fused, bound by HBM: A, B and C move once per launch).
    ms_fz = mean("ms_gemm_fused")
    ms_pp = mean("ms_tc_gemm") - ms_fz
    flop_pp = st["tc_gemm_flop"] - st["gemm_fused_flop"]
    n_pp = max(1, st.get("gemm_pipe_launches", 1))
    gem = {"kernel": "k_tc_gemm_pipe (a7 Schur and TRSM updates with K > 64, pre-split tiles)", "bound": "tensor",
           "ms": ms_pp, "unit": "TFLOP/s", "launches": n_pp,
           "achieved": flop_pp / (ms_pp / 1e3) / 1e12 if ms_pp > 0 else None,
           "peak": tf32 / 3.0,
           "peak_source": f"TF32 dense = {src} bf16_tflops x 1.1/2.25 (nominal ratio) = {tf32:.1f}, / 3 products "
                          "per useful flop (split TF32)",
           "traffic": GEMM_DRAM_BYTES_PER_FLOP * flop_pp / n_pp,
           "traffic_note": "bytes per launch: the measured bytes per flop of one captured launch x this step's "
                           "mean flops per launch"}
    fz = {"kernel": "k_tc_gemm_fused (a7 K = 64 updates: leaf panels, leaf TRSMs, thinnest Schur/TRSM)",
          "bound": "hbm", "ms": ms_fz, "unit": "GB/s",
          "achieved": st["gemm_fused_bytes"] / (ms_fz / 1e3) / 1e9 if ms_fz > 0 else None,
          "peak": pk["hbm_gbs"], "peak_source": f"{src} hbm_gbs (copy)", "traffic": None,
          "tflops": st["gemm_fused_flop"] / (ms_fz / 1e3) / 1e12 if ms_fz > 0 else None,
          "note": "algorithmic bytes = A and B read once, C written (read and written when subtracting)"}
    # a8: right-looking triangular solves, FP32 FMA (2 n^2 (n_k+1) flop per disk and sweep)
    tri_flop = st["disk_solves"] * 2.0 * n * n * nrhs
    tri = {"kernel": "k_lu_solve_rl (a8)", "bound": "hbm", "ms": mean("ms_trisolve"), "unit": "GB/s",
           "achieved": st["disk_solves"] * 4.0 * n * n / (mean("ms_trisolve") / 1e3) / 1e9
           if mean("ms_trisolve") else None, "peak": pk["hbm_gbs"],
           "peak_source": f"{src} hbm_gbs (copy)", "traffic": None,
           "fp32_tflops": tri_flop / (mean("ms_trisolve") / 1e3) / 1e12 if mean("ms_trisolve") else None,
           "fp32_peak_tflops": fp32_peak,
           "note": "algorithmic bytes = the FP32 factors read once per disk and sweep (4 n^2)"}
    # a11: the path kernel, bound by instruction issue (and the INT32 high-multiply pipe of Philox)
    pth = {"kernel": "k_paths<float> (a11)", "bound": "alu", "ms": mean("ms_paths"),
           "achieved": st["path_steps"] / (mean("ms_paths") / 1e3) / 1e9, "unit": "Gpath-steps/s",
           "traffic": None, "peak": issue / PATHS_THREAD_INST_PER_STEP / 1e9,
           "peak_source": (f"152 SMs x 4 schedulers x 32 lanes x {sm_mhz:.0f} MHz / "
                           f"{PATHS_THREAD_INST_PER_STEP:.0f} thread-instructions per step (ncu, this "
                           "kernel variant on a 6 x 6 lattice of the workload's circles)")}
    ks = [gem, fz, tri, pth]
    for k in ks:
        k["frac"] = (k["achieved"] / k["peak"]) if (k.get("achieved") and k.get("peak")) else None
    ks.sort(key=lambda k: -(k["ms"] or 0.0))
    out.update(ks[0])
    out["others"] = ks[1:]
    # the disk path (a6-a9): 2/3 n^3 (LU) + 2 n^2 (n_k + 1) per sweep (solves) per disk, over its stage time
    sweeps = st["disk_solves"] / max(1, st["floating_disks"])
    per_disk = 2.0 / 3.0 * n ** 3 + 2.0 * n * n * nrhs * sweeps
    disk_ms = mean("ms_disks")
    out["disk_path"] = {"flop_per_disk": per_disk, "disks": st["floating_disks"], "sweeps_per_disk": sweeps,
                        "ms": disk_ms, "achieved_tflops": st["floating_disks"] * per_disk / (disk_ms / 1e3) / 1e12,
                        "tf32_peak_tflops": tf32,
                        "frac_of_tf32": st["floating_disks"] * per_disk / (disk_ms / 1e3) / 1e12 / tf32,
                        "frac_of_tf32_over_3": st["floating_disks"] * per_disk / (disk_ms / 1e3) / 1e12 / (tf32 / 3)}
    return out


def _scaled_subset(k=12):
    """The scaled workload's circles, grids and data on [0, 12 s]^2 (12 x 12 lattice: 100 floating disks of
    the same n = 3072): the sample on which the FP64 form is timed beside the mixed form."""
    import workloads
    cfg = workloads.scaled()
    s = cfg["cover"]["spacing"]
    cfg["cover"] = dict(cfg["cover"], nx=k, ny=k)
    cfg["domain"] = {"kind": "square", "p": [0.0, 0.0, k * s, k * s]}
    return cfg


def fp64_form(pdd, stream, flush):
    """The plain FP64 form (FP64 blocked LU with partial pivoting, FP64 paths) against the mixed form on the
    same GPU and the same disks (a subset of the workload: the FP64 form of all 3,600 disks takes ~70 s),
    with the mixed-vs-FP64 differences of every floating row, of r and of u."""
    import numpy as np
    cfg = _scaled_subset()
    res = {"sample": "12 x 12 lattice of the scaled workload's circles (100 floating disks, n = 3072)"}
    for prec in ("mixed", "fp64"):
        t, st, N = _timed(pdd, cfg, prec, stream, flush, 2)
        res[prec] = {"ms_per_step": statistics.mean(t), "knots_per_s": N / (statistics.mean(t) / 1e3),
                     "ms_disks": st["ms_disks"], "ms_factor": st["ms_factor"], "ms_refine": st["ms_refine"],
                     "ms_paths": st["ms_paths"], "disks": st["floating_disks"],
                     "ms_disks_per_disk": st["ms_disks"] / max(1, st["floating_disks"])}
    res["disk_stage_speedup_mixed_over_fp64"] = res["fp64"]["ms_disks"] / res["mixed"]["ms_disks"]
    # differences on the same cover: mixed disks (FP64 paths, identical streams) vs the FP64 form
    cov = pdd.Cover(cfg, stream=stream)
    S64 = pdd.System(cov, cfg, "fp64", stream=stream)
    Sm = pdd.System(cov, cfg, "mixed", stream=stream, path_precision="fp64")
    u64 = S64.solve(rtol=1e-14, stream=stream).cpu().numpy()
    um = Sm.solve(rtol=1e-14, stream=stream).cpu().numpy()
    a = {k: v.cpu().numpy() for k, v in cov.arrays().items()}
    g64, gm = S64.csr(), Sm.csr()
    v64, vm = g64["val"].cpu().numpy(), gm["val"].cpu().numpy()
    b64, bm = g64["b"].cpu().numpy(), gm["b"].cpu().numpy()
    worst = 0.0
    for i in range(cov.N):
        m = a["row_sub"][i]
        if m >= 0 and a["floating"][m]:
            p0, p1 = a["rowptr"][i], a["rowptr"][i + 1]
            worst = max(worst, float(np.abs(v64[p0:p1] - vm[p0:p1]).max() / np.abs(v64[p0:p1]).max()))
    res["mixed_vs_fp64_floating_rows_max_rel"] = worst
    res["mixed_vs_fp64_b_max_rel"] = float(np.abs(b64 - bm).max() / np.abs(b64).max())
    res["mixed_vs_fp64_u_max_rel"] = float(np.abs(u64 - um).max() / np.abs(u64).max())
    return res


def varcoef_leg(pdd, stream, flush, steps=3):
    """The variable-coefficient workload (hex lattice of 1,003 circles, 32 x 32 disk grids, 10^4 paths per
    Monte Carlo knot): the same step, mixed form."""
    import workloads
    cfg = workloads.varcoef()
    t, st, N = _timed(pdd, cfg, "mixed", stream, flush, steps)
    ms = statistics.mean(t)
    return {"workload": "varcoef: Omega=[0,2]^2, L=1/2 Lap+(sin x,cos y).grad, c=-(1+x^2+y^2), "
                        "u*=sin(pi x)cos(pi y); hex lattice R=0.05 spacing 0.07 (1003 circles); 32 knots/circle, "
                        "32x32 disk grid; 1e4 paths/knot, h=1e-5",
            "value": N / (ms / 1e3), "unit": "knots/s", "ms_per_step": ms, "steps": steps,
            "mc_path_steps_per_s": st["path_steps"] / (st["ms_paths"] / 1e3),
            "stages_ms": {k: st[k] for k in ("ms_disks", "ms_factor", "ms_refine", "ms_paths", "ms_finalize",
                                             "ms_tc_gemm", "ms_trisolve")},
            "gmres_iters": st["gmres_iters"]}


def adaptive_leg(pdd, stream, flush, steps=2):
    """The batching workload: unit disk, ~10^4 circles of log-normal radii with grids from 16 x 16 to 64 x 64
    grouped by shape, adaptive path counts (pilot 10^3, up to 10^5 per Monte Carlo knot)."""
    import workloads
    cfg = workloads.adaptive()
    # plain GMRES: the 64-knot circles' RAS subsets exceed the 128-knot limit of the FP32 inverses
    t, st, N = _timed(pdd, cfg, "mixed", stream, flush, steps, precond="none")
    ms = statistics.mean(t)
    return {"workload": "adaptive: unit disk, c(x) from 64 Gaussian RBFs (clipped <= 0); adaptive cover of "
                        "log-normal radii in [0.02, 0.1] (grids 16^2..64^2 by radius); 10^3-10^5 paths/knot by "
                        "per-row standard error (target 2e-3), h=1e-5",
            "value": N / (ms / 1e3), "unit": "knots/s", "ms_per_step": ms, "steps": steps, "knots": N,
            "disks": st["floating_disks"], "mc_rows": st["mc_rows"], "paths_total": st["paths_total"],
            "extended_rows": st["extended_rows"],
            "mc_path_steps_per_s": st["path_steps"] / (st["ms_paths"] / 1e3) if st["ms_paths"] else None,
            "stages_ms": {k: st[k] for k in ("ms_disks", "ms_factor", "ms_refine", "ms_paths", "ms_finalize")},
            "gmres_iters": st["gmres_iters"], "precond": "none"}


# The [-50,50]^2 column of the paper's Table 1 (Sec. 4): 1152 A64FX cores, 96 MPI processes,
# METIS + MUMPS RAS, Gobet-Menozzi paths with pathwise variance reduction.
TABLE1_50 = {"subdomains": 100, "N": 3636, "sparsity": 0.02066, "rho_C_minus_I": 0.9558,
             "max_offdiag_C": 0.0445, "kappa2_C": 84.0, "rms_error": 3.72e-5, "gmres_iters": 19,
             "total_s": 76.0, "solve_s": 1.55}


def poisson46_leg(pdd, stream, flush, steps=3):
    """The paper's Poisson test (Eq. 46) on [-50,50]^2 at its Sec. 4 parameters (5,000 paths per
    Monte Carlo knot, h = 0.015, boundary shift, 44 knots, 22 x 44 disk nodes, c^2 = 1.5):
    throughput of the same step, and the statistics of Table 1 computed from the GPU's C, r and u
    (rho(C - I), max off-diagonal C_ij, kappa_2(C) on the host in FP64)."""
    import numpy as np
    import scipy.sparse as sp
    import torch

    import workloads
    cfg = workloads.poisson46()
    for _ in range(2):
        cov, S, u = step(pdd, cfg, "mixed", stream)
        del cov, S, u
    times = []
    for _ in range(steps):
        flush_l2(flush)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cov, S, u = step(pdd, cfg, "mixed", stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.mean(times)
    st = S.stats()
    a = {k: v.cpu().numpy() for k, v in cov.arrays().items()}
    g = {k: v.cpu().numpy() for k, v in S.csr().items()}
    un = u.cpu().numpy()
    N = cov.N
    C = sp.csr_matrix((g["val"], a["col"], a["rowptr"]), shape=(N, N))
    kx, ky = a["kx"], a["ky"]
    # u46 of Eq. 46 at the knots (the exact solution, evaluated here for the error statistics)
    s_ = np.sqrt(1.0 + kx * kx / 100.0 + ky * ky / 50.0)
    w_ = np.sin(3.0 * kx / 25.0 + ky / 20.0) + np.sin(kx / 20.0 - 3.0 * ky / 25.0)
    uex = 3.0 + np.sin(s_) / 3.0 + np.tanh(w_) / 3.0
    err = un - uex
    Cd = C.toarray()
    sv = np.linalg.svd(Cd, compute_uv=False)
    ev = np.linalg.eigvals(Cd - np.eye(N))
    off = Cd - np.diag(np.diag(Cd))
    res = {"workload": "poisson46: Omega=[-50,50]^2, Lap u = F with u = Eq. 46; 10x10 square lattice "
                       "of radius-9 circles (pitch 10); 44 knots/circle, 22x44 disk grid; 5000 paths/knot, "
                       "h=0.015, boundary shift; c^2=1.5",
           "value": N / (ms / 1e3), "unit": "knots/s", "ms_per_step": ms, "steps": steps,
           "mc_path_steps_per_s": st["path_steps"] / (st["ms_paths"] / 1e3),
           "path_steps_per_step": st["path_steps"],
           "stages_ms": {k: st[k] for k in ("ms_disks", "ms_factor", "ms_refine", "ms_paths", "ms_finalize")},
           "gmres": dict(S.last_solve, precond=SOLVE["precond"]),
           "subdomains": cov.M, "N": N, "sparsity": C.nnz / float(N) ** 2,
           "rho_C_minus_I": float(np.abs(ev).max()), "max_offdiag_C": float(off.max()),
           "kappa2_C": float(sv[0] / sv[-1]),
           "rms_error": float(np.sqrt(np.mean(err * err))), "max_error": float(np.abs(err).max()),
           "table1_column_50": TABLE1_50}
    del cov, S, u
    return res


def averaged_leg(pdd, cfg, stream, flush, steps=3):
    """The same workload with averaged multi-subdomain rows (Eq. 38-39): every knot's row sums the
    subdomains that hold it.  Plain GMRES (the RAS subsets assume one subdomain per row)."""
    import torch
    acfg = dict(cfg, cover=dict(cfg["cover"], rows="averaged"))

    def one():
        cov = pdd.Cover(acfg, stream=stream)
        S = pdd.System(cov, acfg, "mixed", stream=stream, **LU)
        u = S.solve(rtol=1e-13, restart=64, stream=stream, precond="none")
        return cov, S, u

    for _ in range(2):
        cov, S, u = one()
        del cov, S, u
    times = []
    for _ in range(steps):
        flush_l2(flush)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cov, S, u = one()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.mean(times)
    st = S.stats()
    a = cov.arrays()
    npairs = int(a["pi_ptr"][-1].item())
    nint = int((a["pi_ptr"][1:] > a["pi_ptr"][:-1]).sum().item())
    res = {"value": cov.N / (ms / 1e3), "unit": "knots/s", "ms_per_step": ms, "steps": steps,
           "nnz": cov.nnz, "subdomains_per_interior_row": npairs / max(1, nint),
           "mc_entries": st["mc_rows"], "floating_entries": st["floating_rows"],
           "mc_path_steps_per_s": st["path_steps"] / (st["ms_paths"] / 1e3),
           "stages_ms": {k: st[k] for k in ("ms_disks", "ms_factor", "ms_refine", "ms_eval", "ms_paths",
                                            "ms_finalize")},
           "gmres": dict(S.last_solve, precond="none")}
    del cov, S, u
    return res


def errors_vs_oracle(pdd, cfg, stream, n_disks=2, n_mc=3):
    """Per-stage errors against the FP64 oracle on sampled rows of the workload: the cover (bit-exact),
    floating rows of C and their r (Householder QR oracle) in the mixed form, and Monte Carlo moments,
    C entries and r on identical Philox streams (FP64 paths, mixed disks)."""
    import numpy as np

    from oracle import cover as ocover
    from oracle import problem, spectral
    from oracle import system as osystem

    t0 = time.time()
    cov = pdd.Cover(cfg, stream=stream)
    out = {}
    oc = ocover.full_cover(cfg)
    a = {k: v.cpu().numpy() for k, v in cov.arrays().items()}
    out["cover_bit_exact"] = bool(all(np.array_equal(a[k].astype(np.int64), getattr(oc, k).astype(np.int64))
                                      for k in ("knot_ptr", "kowner", "row_sub", "rowptr", "col")))
    op = problem.Operator(cfg["op"], oc.domain)
    rng = np.random.default_rng(0)
    disks = [m for m in range(oc.M) if oc.floating[m] and oc.sub_rows(m).size]
    S = pdd.System(cov, cfg, "mixed", stream=stream, path_precision="fp64")
    g = {k: v.cpu().numpy() for k, v in S.csr().items()}
    worst_c, worst_b = 0.0, 0.0
    for m in rng.choice(disks, n_disks, replace=False):
        for i, (cols, v, bi) in spectral.floating_rows(oc, op, int(m)).items():
            pos = oc.rowptr[i] + np.searchsorted(oc.col[oc.rowptr[i]:oc.rowptr[i + 1]], cols)
            worst_c = max(worst_c, float(np.abs(g["val"][pos] - v).max() / np.abs(v).max()))
            worst_b = max(worst_b, abs(g["b"][i] - bi) / max(1.0, abs(bi)))
    out["floating_rows_C_mixed_max_rel"] = worst_c
    out["floating_rows_b_mixed_max_rel"] = worst_b
    out["floating_disks_sampled"] = n_disks
    mc = {k: v.cpu().numpy() for k, v in S.mc().items()}
    rows = mc["rows"]
    pick = rng.choice(rows.size, n_mc, replace=False)
    ref = osystem.assemble(cfg, oc, rows=[int(rows[k]) for k in pick], threads=n_mc)
    wm, wc, wb = 0.0, 0.0, 0.0
    for k in pick:
        i = int(rows[k])
        r = ref.mc_rows[i]
        wm = max(wm, float(np.abs(mc["moments"][mc["mom_ptr"][k]:mc["mom_ptr"][k + 1]] - r.moments).max() /
                           np.abs(r.moments).max()))
        pos = oc.rowptr[i] + np.searchsorted(oc.col[oc.rowptr[i]:oc.rowptr[i + 1]], r.cols)
        wc = max(wc, float(np.abs(g["val"][pos] - r.vals).max() / np.abs(r.vals).max()))
        wb = max(wb, abs(g["b"][i] - r.b) / max(1.0, abs(r.b)))
    out["mc_moments_identical_streams_max_rel"] = wm
    out["mc_C_identical_streams_max_rel"] = wc
    out["mc_b_identical_streams_max_rel"] = wb
    out["mc_rows_sampled"] = n_mc
    out["oracle_seconds"] = time.time() - t0
    return out


def cpu_baseline(cfg, budget_s=20.0):
    """The oracle as it stands, on the host cores, over a bounded sample of the workload: whole floating
    disks (Householder QR, every right-hand side, evaluation at the knots) and whole Monte Carlo rows,
    extrapolated to every disk and row of the workload."""
    import numpy as np

    from oracle import cover as ocover
    from oracle import problem, spectral
    from oracle import system as osystem

    cores = len(os.sched_getaffinity(0))
    oc = ocover.full_cover(cfg)
    op = problem.Operator(cfg["op"], oc.domain)
    disks = [m for m in range(oc.M) if oc.floating[m] and oc.sub_rows(m).size]
    mc_rows = [i for i in range(oc.N) if oc.row_sub[i] >= 0 and not oc.floating[oc.row_sub[i]]]
    rng = np.random.default_rng(1)
    t0 = time.time()
    nd = 0
    fl_rows = 0
    shapes = {}
    while (time.time() - t0 < budget_s / 2 or nd == 0) and nd < len(disks):
        m = int(disks[rng.integers(len(disks))])
        fl_rows += len(spectral.floating_rows(oc, op, m, shapes))
        nd += 1
    t_disk = (time.time() - t0) / nd
    t1 = time.time()
    picked = list(rng.choice(mc_rows, min(len(mc_rows), 2 * cores), replace=False))
    ref = osystem.assemble(cfg, oc, rows=[int(i) for i in picked], threads=cores)
    t_mc = time.time() - t1
    steps = sum(r.steps for r in ref.mc_rows.values())
    total = t_disk * len(disks) + t_mc * len(mc_rows) / len(picked)
    return {"value": oc.N / total, "unit": "knots/s", "cores": cores, "kind": "oracle",
            "sample": f"{nd} floating disks (Householder QR of n = {int(oc.n_r[disks[0]] * oc.n_theta[disks[0]])}, "
                      f"{fl_rows} rows, one after another: numpy's LAPACK uses the host's cores) + "
                      f"{len(picked)} Monte Carlo rows ({int(cfg['mc']['paths'])} paths each, {steps} path-steps, "
                      f"{cores} threads) of the workload, extrapolated to all {len(disks)} disks and "
                      f"{len(mc_rows)} Monte Carlo rows",
            "seconds_per_disk": t_disk, "mc_path_steps_per_s": steps / t_mc}


def grad_bench(pdd, stream):
    """a14 on the gradient workload: forward + adjoint, device time."""
    import numpy as np
    import torch

    import workloads
    cfg = workloads.grad(paths=1000)
    cov = pdd.Cover(cfg, stream=stream)
    S = pdd.System(cov, cfg, "fp64", stream=stream)
    u = S.solve(rtol=1e-14, stream=stream)
    a = cov.arrays()
    u_obs = torch.exp(a["kx"]) * torch.sin(a["ky"])
    dJ = 2.0 * (u - u_obs)
    S.grad(u, dJ, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g = S.grad(u, dJ, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    return {"workload": "grad: tiny geometry, 64 RBF weights of c + 16 RBF weights of f + 32 boundary Fourier "
                        "coefficients of g, "
                        "1000 paths/knot", "ms": e0.elapsed_time(e1), "n_params": int(g.numel()),
            "grad_norm": float(g.norm().item())}


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle, as it stands, on the host cores
# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return None
    import workloads
    cfg = workloads.scaled()
    if args.warmup > 0:
        cpu_baseline(cfg, budget_s=2.0)     # builds the C path simulator and warms the caches
    vals, secs = [], []
    bl = None
    for _ in range(max(1, args.steps)):
        t0 = time.time()
        bl = cpu_baseline(cfg, budget_s=max(4.0, 60.0 / max(1, args.steps)))
        secs.append(time.time() - t0)
        vals.append(bl["value"])
    value = statistics.mean(vals)
    bl["value"] = value
    return {"metric": METRIC, "value": value, "unit": "knots/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "fp64 (oracle)",
                       "step": "one bounded sample of the workload (see cpu_baseline.sample); value extrapolates "
                               "its per-disk and per-row times to the whole workload"},
            "impl": "reference", "cpu_baseline": bl,
            "e2e": {"value": value, "unit": "knots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        world = int(os.environ.get("WORLD_SIZE", "1"))
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out))
        return
    rank, world, _ = dist_setup(args.gpus)
    out = run_ours(args, rank, world)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
