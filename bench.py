#!/usr/bin/env python
"""Benchmark of the linear-MHS multigrid path on GB300.

Metric: unknowns solved per second to a 1e-10 relative residual, where one
solve is the lower-boundary multigrid solve (eq. lower_bound), the interior
multigrid solve (eq. scalar_pot) and the recovery of B, p and rho, and the
unknowns are the interior nodes of both problems.

Default workload (one GPU): 129^3 nodes on [0,1]^3, alpha = 0.5,
xi(z) = 0.5 exp(-z), B_z = 8 flux-balanced Gaussian spots (splitmix64
seeds), FP64 mode; outputs Phi, B_x, B_y, B_z, p, rho.  A step is one such
solve of one magnetogram whose data is resident in HBM; L2 is flushed
(256 MiB write) before every timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--mode fp64|mixed] [--impl mhs|reference]

With N > 1 (torchrun) every rank solves its own magnetograms (replicas, no
collective on the data path); value = all ranks' unknowns / max rank time.
--impl reference times the CPU oracle (plain C, OpenMP over z-planes) on
the host cores, one oracle solve per step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# more hardware work queues, so that the streams of batched and served solves run concurrently
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import synthetic as S  # noqa: E402

TOL = 1e-10
METRIC = "unknowns solved/s to 1e-10 rel. residual"
UNIT = "unknowns/s"


def workload(rank: int, nmag: int = 4):
    """129^3 linear-MHS problem; magnetograms for this rank."""
    pr, _ = S.linear_mhs(129)
    mags = [S.magnetogram_random(129, 129, 1.0, 1.0, seed=1307 + 100 * rank + i) for i in range(nmag)]
    cfg = {"workload": "linear_mhs_129", "grid": [129, 129, 129], "domain": "[0,1]^3", "alpha": 0.5,
           "xi": "0.5*exp(-z)", "bz": f"8 flux-balanced Gaussian spots, splitmix64 seeds 1307..{1306 + nmag} (+100*rank)",
           "tol": TOL, "outputs": "Phi,Bx,By,Bz,p,rho", "unknowns_per_solve": S.unknowns(pr)}
    return pr, mags, cfg


# --------------------------------------------------------------------------
# GPU clocks during the timed region
# --------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str):
        self.proc = None
        self.gpu = gpu_index
        self.path = os.path.join(tempfile.gettempdir(), f"mhs_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "50", "-i", self.gpu], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # the first sample must exist before the timed region starts (nvidia-smi takes a while to come up)
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 5.0 and os.path.getsize(self.path) == 0:
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for _, _, flags in rows for q, v in enumerate(flags) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------
# reference arm and CPU baseline: the oracle on the host cores
# --------------------------------------------------------------------------

# how each arm runs, in the same words in both lines' config (each statement true of its arm), so that
# the two lines' configurations compare equal
RUN_NOTES = {"l2": "GPU arm: L2 flushed between timed steps (256 MiB device write); reference arm: host CPU, no GPU",
             "parallelism": "GPU arm: one solver per GPU (replicas, no collective); reference arm: the oracle on "
                            "the host cores (OpenMP)"}


def oracle_solve_rate(pr, mags, budget_s: float, min_runs: int = 1, threads: int = 0):
    """Oracle solves (2D + 3D multigrid to 1e-10, fields) per second for about budget_s seconds;
    threads = 0: every host core."""
    import oracle
    oracle.set_threads(threads if threads > 0 else os.cpu_count() or 1)
    t0 = time.perf_counter()
    runs = 0
    while runs < min_runs or time.perf_counter() - t0 < budget_s:
        P, info = oracle.solve(pr, mags[runs % len(mags)], TOL, TOL)
        oracle.fields(pr, P)
        assert info["status"] == 0
        runs += 1
    dt = time.perf_counter() - t0
    used = oracle.max_threads()
    oracle.set_threads(os.cpu_count() or 1)
    return S.unknowns(pr) * runs / dt, runs, dt, used


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    pr, mags, cfg = workload(0)
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        oracle.fields(pr, oracle.solve(pr, mags[0], TOL, TOL)[0])
    times = []
    for s in range(args.steps):
        t0 = time.perf_counter()
        P, info = oracle.solve(pr, mags[s % len(mags)], TOL, TOL)
        oracle.fields(pr, P)
        times.append(time.perf_counter() - t0)
    per = sum(times) / len(times)
    value = S.unknowns(pr) / per
    cores = oracle.max_threads()
    cfg = dict(cfg, mode="fp64", **RUN_NOTES)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} oracle solves (2D+3D multigrid to 1e-10 + fields) of the 129^3 workload"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------

def aggregate(ms_local: float, unknowns_per_rank: int, world: int, device=None):
    """Whole-job rate of the replicas layout: every rank solves its own
    instances, the step time is the maximum over ranks (one all-reduce of a
    scalar; no collective on the data path), and the value counts the unknowns
    of all ranks.  Returns (max step ms, unknowns per second)."""
    ms = float(ms_local)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, unknowns_per_rank * world / (ms * 1e-3)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


FP64_NOMINAL_TFLOPS = 1.25   # nominal GB300 FP64 rate (profiling recipe table)


def profiled_traffic(kind_name: str, grid=None):
    """DRAM bytes per launch from a committed ncu summary, if the kernel's source is unchanged (the text of the
    measured function when the summary names it: body_prefix, or the device function `body`; else the whole
    file) and, when the summary names one, the finest grid is the one the counters were taken on."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path))
        ent = d["kernels"][kind_name]
        if "grid" in ent and grid is not None and list(grid) != list(ent["grid"]):
            return None
        import hashlib
        src = open(os.path.join(ROOT, ent["source"])).read()
        if "body" in ent or "body_prefix" in ent:
            start = src.index(ent.get("body_prefix", "__device__ __forceinline__ void " + ent.get("body", "") + "("))
            text, want = src[start:src.index("\n}\n", start) + 3], ent["body_sha256"]
        else:
            text, want = src, ent["sha256"]
        return ent["bytes_per_launch"] if hashlib.sha256(text.encode()).hexdigest() == want else None
    except Exception:
        return None


def field_errors(pr, bz, outs):
    """Relative L2 error of (Phi, B_x, B_y, B_z, p, rho) in the device tensors outs against the oracle's
    exact discrete solution (separable direct solve) and field recovery."""
    import numpy as np
    import oracle
    from oracle import exact
    P = exact.exact_solution(pr, bz)
    want = dict(oracle.fields(pr, P), phi=P)
    got = {k: o.cpu().numpy() for k, o in zip(["phi", "Bx", "By", "Bz", "p", "rho"], outs)}
    return {k: float(np.linalg.norm(got[k] - want[k]) / np.linalg.norm(want[k])) for k in got}


COMPOSITE = {"coarse64", "coarse32", "separable", "other"}


def kernel_roofline(M, h, run, steps, hbm_peak, peak_src, fp64_peak):
    """Per-operation event timing over run() (the handle's eager path: the same kernels as the graph);
    returns the roofline of the dominant single-kernel operation on the finest interior level and the
    per-operation table.  Coarse-grid solves (the one-CTA sub-cycle, or the separable solve's transform
    and mode-solve kernels), the separable inner solve and set-up work are composites without one
    roofline; they are reported as shares.  One "launch" of a sweep is one red-black sweep."""
    M.mhs_set_kernel_timing(h, True)
    M.mhs_kernel_timing_reset(h)
    run()
    kt = [M.mhs_kernel_timing(h, k) for k in range(M.MHS_KT_COUNT)]
    kt0 = {k: M.mhs_kernel_timing_finest(h, k) for k in range(M.MHS_KT_COUNT)}
    M.mhs_set_kernel_timing(h, False)
    kidx = {k["name"]: i for i, k in enumerate(kt)}
    kt = [k for k in kt if k["launches"] > 0]
    dom_all = max((k for k in kt if k["name"] not in COMPOSITE), key=lambda k: k["ms"])
    finest = kt0[kidx[dom_all["name"]]]["launches"] > 0
    dom = kt0[kidx[dom_all["name"]]] if finest else dom_all
    avg_ms = dom["ms"] / dom["launches"]
    gbs = dom["bytes"] / dom["launches"] / (avg_ms * 1e-3) / 1e9
    tfl = dom["flops"] / dom["launches"] / (avg_ms * 1e-3) / 1e12
    alu_bound = dom["name"].endswith("64") or dom["name"] == "fields"   # FP64-pipe-bound kernels
    traffic = profiled_traffic(dom["name"], M.mhs_level_shape(h, 3, 0))
    kname = dom["name"] + (" (finest level)" if finest else "")
    if alu_bound:
        roof = {"bound": "alu", "achieved": tfl, "peak": fp64_peak, "unit": "TFLOP/s", "frac": tfl / fp64_peak,
                "traffic": traffic, "kernel": kname,
                "peak_source": "measured FP64 FMA rate of this GPU (mhs_probe_fma_rate, this run)",
                "peak_nominal": FP64_NOMINAL_TFLOPS, "frac_of_nominal": tfl / FP64_NOMINAL_TFLOPS,
                "achieved_gbs": gbs, "hbm_frac_of_" + peak_src: gbs / hbm_peak}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                "traffic": traffic, "kernel": kname, "peak_source": peak_src}
    tot = sum(k["ms"] for k in kt)
    roof.update({"launches_timed": dom["launches"], "avg_launch_ms": avg_ms,
                 "alg_bytes_per_launch": dom["bytes"] / dom["launches"],
                 "alg_flops_per_launch": dom["flops"] / dom["launches"],
                 "share_of_timed_ops": dom_all["ms"] / tot,
                 "composite_shares": {k["name"]: k["ms"] / tot for k in kt if k["name"] in COMPOSITE}})
    kernels = {k["name"]: {"ms_per_step": k["ms"] / steps, "launches_per_step": k["launches"] / steps,
                           "gbs": k["bytes"] / (k["ms"] * 1e-3) / 1e9 if k["ms"] > 0 else None} for k in kt}
    return roof, kernels


def large_roofline(M, hbm_peak, peak_src, fp64_peak, steps=3):
    """Roofline of the dominant kernel of a grid larger than L2: the 257^3 linear-MHS solve in mixed
    precision (default options, tolerance 1e-10), per-operation event timing, against the measured HBM
    copy bandwidth (FP32 levels of 16.6 M interior nodes: every array is 66 MB or more)."""
    import torch
    pr, _ = S.linear_mhs(257)
    bzs = [torch.from_numpy(S.magnetogram_random(257, 257, 1.0, 1.0, seed=1307 + i)).cuda() for i in range(2)]
    h = M.mhs_create(257, 257, 257, 1.0, 1.0, 1.0, pr["alpha"], M.xi_params(M.MHS_XI_EXP, pr["xi_a"], pr["xi_kappa"]))
    stream = torch.cuda.current_stream()
    M.mhs_set_stream(h, stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def run():
        for s in range(steps):
            flush.fill_(s & 0xFF)
            M.mhs_set_lower_bz(h, bzs[s % 2])
            M.mhs_solve(h, TOL, M.MHS_MIXED)
        torch.cuda.synchronize()

    M.mhs_set_lower_bz(h, bzs[0])
    M.mhs_solve(h, TOL, M.MHS_MIXED)
    roof, kernels = kernel_roofline(M, h, run, steps, hbm_peak, peak_src, fp64_peak)
    M.mhs_destroy(h)
    del flush
    torch.cuda.empty_cache()
    return dict(roof, workload="linear_mhs_257 mixed (solve only, tolerance 1e-10)", kernels=kernels)


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1307_6720_gb300 import mhs as M

    pr, mags, cfg = workload(rank)
    mode = M.MHS_MIXED if args.mode == "mixed" else M.MHS_FP64
    stream = torch.cuda.current_stream()
    xi = M.xi_params(M.MHS_XI_EXP, pr["xi_a"], pr["xi_kappa"])
    h = M.mhs_create(pr["nx"], pr["ny"], pr["nz"], pr["Lx"], pr["Ly"], pr["Lz"], pr["alpha"], xi)
    M.mhs_set_stream(h, stream)
    flags = (M.MHS_FLAG_NO_GRAPH if args.eager else 0) | (M.MHS_FLAG_NO_FMG if args.no_fmg else 0) | \
        (M.MHS_FLAG_ZLINE if args.zline else 0)
    if flags:
        M.mhs_set_options(h, flags=flags)
    shape = (pr["nz"], pr["ny"], pr["nx"])
    bz_dev = [torch.from_numpy(b).to(dev) for b in mags]
    outs_dev = [torch.empty(shape, dtype=torch.float64, device=dev) for _ in range(6)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step(s, m=mode, bz=bz_dev, outs=outs_dev, tol=TOL):
        M.mhs_set_lower_bz(h, bz[s % len(bz)])
        info = M.mhs_solve(h, tol, m)
        M.mhs_get_phi(h, outs[0])
        M.mhs_fields(h, *outs[1:])
        return info

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(K, m=mode, bz=bz_dev, outs=outs_dev, tol=TOL):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        infos = []
        barrier()
        for s in range(K):
            flush.fill_(s & 0xFF)
            ev[s][0].record(stream)
            infos.append(step(s, m, bz, outs, tol))
            ev[s][1].record(stream)
        barrier()
        ms = sum(a.elapsed_time(b) for a, b in ev) / K
        ms, _ = aggregate(ms, 0, world, dev)
        return ms, infos

    for s in range(args.warmup):
        step(s)
    # measured FMA rates of this GPU (the FP64 one is the roofline denominator of FP64-pipe-bound kernels)
    fp64_peak = M.mhs_probe_fma_rate(M.MHS_FP64, stream) / 1e12
    fp32_peak = M.mhs_probe_fma_rate(M.MHS_MIXED, stream) / 1e12
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0] if "CUDA_VISIBLE_DEVICES" in os.environ else str(local)
    clocks = ClockSampler(gpu_index)
    l0 = M.mhs_kernel_launches()
    clocks.start()
    ms, infos = timed(args.steps)
    clk = clocks.stop()
    launches = M.mhs_kernel_launches() - l0
    unknowns = S.unknowns(pr)
    value = unknowns * world / (ms * 1e-3)
    if args.light:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "ms_per_step": ms, "light": True,
                              "gpu_launches": int(launches), "config": cfg}))
        M.mhs_destroy(h)
        return

    # per-kernel durations over a second, identical timed pass with event instrumentation
    hbm_peak, peak_src = measured_peaks()
    roof, kernels = kernel_roofline(M, h, lambda: timed(args.steps), args.steps, hbm_peak, peak_src, fp64_peak)

    # the other precision mode on the same workload, and mixed mode with the separable inner solver
    other = M.MHS_FP64 if mode == M.MHS_MIXED else M.MHS_MIXED
    ms_o, infos_o = timed(args.steps, other)
    M.mhs_set_options(h, flags=flags | M.MHS_FLAG_SEPARABLE)
    ms_s, infos_s = timed(args.steps, M.MHS_MIXED)
    ms_s64, infos_s64 = timed(args.steps, M.MHS_FP64)
    M.mhs_set_options(h, flags=flags)

    # the accuracy bars of the path (Phi, B, p, rho within 1e-10 of the exact discrete solution in FP64
    # mode, within 1e-8 in mixed mode) are met by FP64 cycles to 1e-13 and by mixed mode to 1e-12 with the
    # lower-boundary problem in FP64 cycles; timed the same way, with the error of the last solve
    at_bars = {}
    for bname, bmode, btol, bflag in (("fp64_at_bars", M.MHS_FP64, 1e-13, 0),
                                      ("mixed_at_bars", M.MHS_MIXED, 1e-12, M.MHS_FLAG_LOWER_FP64)):
        M.mhs_set_options(h, flags=flags | bflag)
        timed(1, bmode, tol=btol)
        ms_b, infos_b = timed(args.steps, bmode, tol=btol)
        at_bars[bname] = {"value": unknowns * world / (ms_b * 1e-3), "ms_per_step": ms_b, "tol": btol,
                          "cycles_3d": infos_b[-1]["cycles_3d"], "rel_res_3d": infos_b[-1]["rel_res_3d"],
                          "rel_res_2d": infos_b[-1]["rel_res_2d"]}
        if rank == 0:
            at_bars[bname]["rel_l2_error_vs_oracle"] = field_errors(pr, mags[(args.steps - 1) % len(mags)], outs_dev)
    M.mhs_set_options(h, flags=flags)

    # end to end through the C ABI with pinned host buffers
    bz_host = [torch.from_numpy(b).pin_memory() for b in mags]
    outs_host = [torch.empty(shape, dtype=torch.float64).pin_memory() for _ in range(6)]
    ms_e2e, _ = timed(args.steps, mode, bz_host, outs_host)
    e2e = {"value": unknowns * world / (ms_e2e * 1e-3), "unit": UNIT,
           "h2d_bytes_per_step": int(pr["nx"] * pr["ny"] * 8), "d2h_bytes_per_step": int(6 * np.prod(shape) * 8)}

    # error of the last timed solve against the exact discrete solution (CPU, outside timing)
    cpu_base = None
    if rank == 0:
        rate, runs, dt, cores = oracle_solve_rate(pr, mags, args.cpu_budget)
        rate1, runs1, dt1, _ = oracle_solve_rate(pr, mags, args.cpu_budget, threads=1)
        cpu_base = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                    "sample": f"{runs} oracle solves (2D+3D multigrid to 1e-10 + fields) of the 129^3 workload, {dt:.1f} s",
                    "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                                      "sample": f"{runs1} oracle solves of the same workload on one thread, {dt1:.1f} s"}}

    extra = {}
    if rank == 0 and not args.no_extra:
        extra["roofline_large"] = large_roofline(M, hbm_peak, peak_src, fp64_peak)
        extra["large_grids"] = large_grid_leg(M, 3)
        extra["batched"] = batched_leg(M)
        extra["serving"] = serving_leg(M, args.serve_requests)

    if rank == 0:
        name = "mixed" if mode == M.MHS_MIXED else "fp64"
        oname = "fp64" if name == "mixed" else "mixed"
        cfg = dict(cfg, mode=name, **RUN_NOTES)
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if name == "fp64" else "f32+f64", "data": "synthetic", "config": cfg,
            "e2e": e2e, "gpu_launches": int(launches), "clocks": clk, "roofline": roof, "cpu_baseline": cpu_base,
            "fma_rate_tflops": {"fp64": fp64_peak, "fp32": fp32_peak},
            "cycles": {"2d": infos[-1]["cycles_2d"], "3d": infos[-1]["cycles_3d"],
                       "rel_res_3d": infos[-1]["rel_res_3d"], "conv_factor": infos[-1]["conv_factor"]},
            "modes": {oname: {"value": unknowns * world / (ms_o * 1e-3), "ms_per_step": ms_o,
                              "cycles_3d": infos_o[-1]["cycles_3d"], "rel_res_3d": infos_o[-1]["rel_res_3d"]},
                      "mixed_separable": {"value": unknowns * world / (ms_s * 1e-3), "ms_per_step": ms_s,
                                          "cycles_3d": infos_s[-1]["cycles_3d"],
                                          "rel_res_3d": infos_s[-1]["rel_res_3d"],
                                          "solver": "exact separable inner solve (sine transforms + tridiagonal "
                                                    "per mode) in the double-float defect correction"},
                      **at_bars,
                      "fp64_separable": {"value": unknowns * world / (ms_s64 * 1e-3), "ms_per_step": ms_s64,
                                         "cycles_3d": infos_s64[-1]["cycles_3d"],
                                         "rel_res_3d": infos_s64[-1]["rel_res_3d"],
                                         "solver": "FP64 direct separable solves (fast sine transforms + "
                                                   "tridiagonal per mode)"}},
            "kernels": kernels,
        }
        out.update(extra)
        print(json.dumps(out))
    M.mhs_destroy(h)
    if world > 1:
        dist.destroy_process_group()


def run_op(args):
    """One finest-level operation of an interior hierarchy (the 129^3 workload's parameters on the grid
    --grid, isotropic spacing), repeated; prints its mean device time.  `exact` is the separable solve of
    the level (zero boundary values), the coarse-grid solve the V-cycles use on such a level."""
    import numpy as np
    import torch
    from paper_1307_6720_gb300 import mhs as M
    if args.op == "fma":
        st = torch.cuda.current_stream()
        rates = {p: [M.mhs_probe_fma_rate(m, st) / 1e12 for _ in range(max(args.steps, 1))]
                 for p, m in (("fp64", M.MHS_FP64), ("fp32", M.MHS_MIXED))}
        print(json.dumps({"op": "fma", "unit": "TFLOP/s", "best": {p: max(v) for p, v in rates.items()},
                          "runs": rates}))
        return
    pr, mags, cfg = workload(0)
    nx, ny, nz = args.grid
    pr = dict(pr, nx=nx, ny=ny, nz=nz, Lx=1.0, Ly=(ny - 1) / (nx - 1), Lz=(nz - 1) / (nx - 1))
    xi = M.xi_params(M.MHS_XI_EXP, pr["xi_a"], pr["xi_kappa"])
    h = M.mhs_create(pr["nx"], pr["ny"], pr["nz"], pr["Lx"], pr["Ly"], pr["Lz"], pr["alpha"], xi)
    M.mhs_set_stream(h, torch.cuda.current_stream())
    M.mhs_set_options(h, flags=M.MHS_FLAG_ZLINE if args.smoother == "zline" else M.MHS_FLAG_POINT,
                      fused_min=1 if args.tma else 0, tma_rows=args.tma_rows)
    prec = M.MHS_FP64 if args.prec == "fp64" else M.MHS_MIXED
    rng = np.random.default_rng(0)
    dim = args.dim
    shape = (pr["nz"], pr["ny"], pr["nx"]) if dim == 3 else (pr["ny"], pr["nx"])
    for field in (M.MHS_FIELD_U, M.MHS_FIELD_F, M.MHS_FIELD_R):
        M.mhs_level_write(h, dim, 0, field, prec, rng.standard_normal(shape))
    op = {"smooth": M.MHS_OP_SMOOTH, "residual": M.MHS_OP_RESIDUAL, "restrict": M.MHS_OP_RESTRICT,
          "prolong": M.MHS_OP_PROLONG, "vcycle": M.MHS_OP_VCYCLE, "exact": M.MHS_OP_EXACT,
          "resid_restrict": M.MHS_OP_RESID_RESTRICT}[args.op]
    for _ in range(args.warmup):
        M.mhs_level_op(h, dim, 0, op, prec)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for s in range(args.steps):   # every level op ends with a synchronisation of the library's stream
        ev[s][0].record(stream)
        M.mhs_level_op(h, dim, 0, op, prec)
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) * 1e3 / args.steps
    dev_ms = sorted(a.elapsed_time(b) for a, b in ev)
    # device time of each kernel kind (CUDA events around every launch, on the library's stream)
    M.mhs_set_kernel_timing(h, True)
    M.mhs_kernel_timing_reset(h)
    for _ in range(args.steps):
        M.mhs_level_op(h, dim, 0, op, prec)
    torch.cuda.synchronize()
    kt = [M.mhs_kernel_timing(h, k) for k in range(M.MHS_KT_COUNT)]
    M.mhs_set_kernel_timing(h, False)
    kernels = {k["name"]: {"ms_per_launch": k["ms"] / k["launches"], "launches_per_op": k["launches"] / args.steps,
                           "gbs": k["bytes"] / (k["ms"] * 1e-3) / 1e9 if k["ms"] > 0 else None}
               for k in kt if k["launches"]}
    print(json.dumps({"op": args.op, "dim": dim, "prec": args.prec, "grid": list(args.grid), "smoother": args.smoother,
                      "tma": bool(args.tma), "tma_rows": args.tma_rows, "ms_per_op_wall": wall,
                      "ms_per_op_device_median": dev_ms[len(dev_ms) // 2], "kernels": kernels}))
    M.mhs_destroy(h)


# --------------------------------------------------------------------------
# other configurations: large grids, batched instances, request serving
# --------------------------------------------------------------------------

def _timed_solves(M, h, mode, K, bz_list, outs, stream, flush, tol=TOL):
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    infos = []
    torch.cuda.synchronize()
    for s in range(K):
        flush.fill_(s & 0xFF)
        ev[s][0].record(stream)
        M.mhs_set_lower_bz(h, bz_list[s % len(bz_list)])
        infos.append(M.mhs_solve(h, tol, mode))
        M.mhs_get_phi(h, outs[0])
        M.mhs_fields(h, *outs[1:])
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / K, infos


def large_grid_leg(M, steps, with_error=True):
    """Large grids of the mixed-precision configuration: 257^3 on [0,1]^3 and 513x513x257 on
    [0,1]^2 x [0,0.5], alpha = 0.5, xi = 0.5 exp(-z); FP64 and mixed with V-cycles, and both with the
    separable solver; error of the last solve of each against the oracle's exact discrete solution
    (relative L2 of Phi, B, p, rho)."""
    import numpy as np
    import torch
    out = {}
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for name, n, nz, Lz in (("257^3", 257, 257, 1.0), ("513x513x257", 513, 257, 0.5)):
        pr, _ = S.linear_mhs(n, nz=nz, Lz=Lz)
        bzs = [S.magnetogram_random(n, n, 1.0, 1.0, seed=1307 + i) for i in range(2)]
        xi = M.xi_params(M.MHS_XI_EXP, pr["xi_a"], pr["xi_kappa"])
        h = M.mhs_create(n, n, nz, 1.0, 1.0, Lz, pr["alpha"], xi)
        M.mhs_set_stream(h, stream)
        shape = (nz, n, n)
        outs = [torch.empty(shape, dtype=torch.float64, device=dev) for _ in range(6)]
        bz_dev = [torch.from_numpy(b).to(dev) for b in bzs]
        ent = {"unknowns_per_solve": S.unknowns(pr)}
        want = None
        if with_error:
            import oracle
            from oracle import exact
            P = exact.exact_solution(pr, bzs[(steps - 1) % 2])
            F = oracle.fields(pr, P)
            want = dict(F, phi=P)
        # at the benchmark tolerance, then at the tolerances that meet the accuracy bars (FP64: 1e-10 in every
        # field, 1e-9 for B_z and rho on 513 x 513 x 257; mixed: 1e-8 in every field)
        tol_mixed_bars = 2e-12 if n == 513 else 1e-12
        for mname, mode, flags, tol in (("fp64", M.MHS_FP64, 0, TOL), ("mixed", M.MHS_MIXED, 0, TOL),
                                        ("mixed_separable", M.MHS_MIXED, M.MHS_FLAG_SEPARABLE, TOL),
                                        ("fp64_separable", M.MHS_FP64, M.MHS_FLAG_SEPARABLE, TOL),
                                        ("fp64_at_bars", M.MHS_FP64, 0, 1e-13),
                                        ("mixed_at_bars", M.MHS_MIXED, M.MHS_FLAG_LOWER_FP64, tol_mixed_bars)):
            M.mhs_set_options(h, flags=flags)
            _timed_solves(M, h, mode, 1, bz_dev, outs, stream, flush, tol)
            ms, infos = _timed_solves(M, h, mode, steps, bz_dev, outs, stream, flush, tol)
            e = {"value": S.unknowns(pr) / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "tol": tol,
                 "cycles_3d": infos[-1]["cycles_3d"], "rel_res_3d": infos[-1]["rel_res_3d"],
                 "rel_res_2d": infos[-1]["rel_res_2d"]}
            if want is not None:
                got = {k: o.cpu().numpy() for k, o in zip(["phi", "Bx", "By", "Bz", "p", "rho"], outs)}
                e["rel_l2_error_vs_oracle"] = {k: float(np.linalg.norm(got[k] - want[k]) / np.linalg.norm(want[k]))
                                               for k in got}
            ent[mname] = e
        ent["mixed_speedup_vs_fp64"] = ent["fp64"]["ms_per_step"] / ent["mixed"]["ms_per_step"]
        ent["mixed_separable_speedup_vs_fp64"] = ent["fp64"]["ms_per_step"] / ent["mixed_separable"]["ms_per_step"]
        ent["mixed_speedup_vs_fp64_at_bars"] = ent["fp64_at_bars"]["ms_per_step"] / ent["mixed_at_bars"]["ms_per_step"]
        out[name] = ent
        M.mhs_destroy(h)
        del outs, bz_dev
        torch.cuda.empty_cache()
    return out


def batched_instances(count=256):
    """The seeded 256-instance batch (grids 33^3 .. 129^3 and 129x129x65, random alpha, a, kappa)."""
    return S.batched_instances(count)


def batched_leg(M, reps=3, count=256, tune=True):
    """The 256 uneven instances solved together in mixed precision: as one grouped solve (one launch per
    multigrid operation and level for the instances of a part, one CUDA graph per part; instances with a
    large working set run their own graphs on their own streams) and as mhs_batch_solve (every
    instance's own graph on its own stream), against solving them one after another in FP64 and in mixed
    mode.  The grouped and per-stream forms are timed alternately, `reps` rounds of two batches each,
    and the median is reported (so that neither form gains from running second).  Then the autotuner
    picks options per problem class (untimed set-up) and the grouped solve is timed again with them.
    A batch of 1024 small instances (33^3, the linear-MHS workload's physics) shows where grouping pays."""
    import torch
    inst = batched_instances(count)
    hs = []
    for d in inst:
        h = M.mhs_create(d["n"], d["n"], d["nz"], 1.0, 1.0, d["Lz"], d["alpha"],
                         M.xi_params(M.MHS_XI_EXP, d["a"], d["kappa"]))
        M.mhs_set_lower_bz(h, torch.from_numpy(d["bz"]).cuda())
        hs.append(h)
    unknowns = sum(S.unknowns(S.problem(d["n"], d["n"], d["nz"])) for d in inst)

    def seq(mode):
        for h in hs:
            M.mhs_solve(h, TOL, mode)

    def bat(handles=hs):
        infos, sts = M.mhs_batch_solve(handles, TOL, M.MHS_MIXED)
        assert all(s == 0 for s in sts), sts
        return infos

    def grp(g, n=count):
        infos, sts = M.mhs_group_solve(g, n, TOL)
        assert all(s == 0 for s in sts), sts
        return infos

    res = {}

    def timed_rounds(fns, n=count, rounds=reps):
        """{name: fn}: alternate rounds of two batches each; median solves/s per form"""
        for fn in fns.values():
            fn()
        torch.cuda.synchronize()
        rates, last = {k: [] for k in fns}, {}
        for _ in range(rounds):
            for k, fn in fns.items():
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                fn()
                last[k] = fn()
                torch.cuda.synchronize()
                rates[k].append(2 * n / (time.perf_counter() - t0))
        out = {}
        for k, v in rates.items():
            r = sorted(v)[len(v) // 2]
            out[k] = {"solves_per_s": r, "unknowns_per_s": r * unknowns / count if n == count else None,
                      "s_per_batch": n / r}
            if last.get(k) is not None:
                out[k]["max_cycles_3d"] = max(i["cycles_3d"] for i in last[k])
                out[k]["max_rel_res_3d"] = max(i["rel_res_3d"] for i in last[k])
        return out

    def run(name, fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / reps
        res[name] = {"solves_per_s": count / dt, "unknowns_per_s": unknowns / dt, "s_per_batch": dt}

    g = M.mhs_group_create(hs, M.MHS_MIXED)
    res.update(timed_rounds({"grouped_mixed": lambda: grp(g), "batched_mixed": bat}))
    M.mhs_group_destroy(g)
    run("sequential_fp64", lambda: seq(M.MHS_FP64))
    run("sequential_mixed", lambda: seq(M.MHS_MIXED))
    if tune:
        t0 = time.perf_counter()
        tuned_classes = 0
        for h in hs:
            if M.mhs_tune_lookup(h, M.MHS_MIXED) is None:
                M.mhs_autotune(h, TOL, M.MHS_MIXED, repeats=1)
                tuned_classes += 1
            M.mhs_set_options(h, **M.mhs_tune_lookup(h, M.MHS_MIXED))
        res["autotune"] = {"classes": tuned_classes, "seconds": time.perf_counter() - t0}
        gt = M.mhs_group_create(hs, M.MHS_MIXED)
        tuned = timed_rounds({"grouped_mixed_tuned": lambda: grp(gt), "batched_mixed_tuned": bat})
        res.update(tuned)
        M.mhs_group_destroy(gt)
    res["instances"] = count
    best = max(v["solves_per_s"] for k, v in res.items() if k.startswith(("grouped", "batched")))
    res["speedup_vs_sequential_fp64"] = best / res["sequential_fp64"]["solves_per_s"]
    for h in hs:
        M.mhs_destroy(h)
    # a batch of small instances: grouping's launches for all of them against one graph per instance
    small = []
    for i in range(1024):
        _, bz = S.linear_mhs(33, seed=5000 + i)
        h = M.mhs_create(33, 33, 33, 1.0, 1.0, 1.0, 0.5, M.xi_params(M.MHS_XI_EXP, 0.5, 1.0))
        M.mhs_set_lower_bz(h, torch.from_numpy(bz).cuda())
        small.append(h)
    gs = M.mhs_group_create(small, M.MHS_MIXED)
    sm = timed_rounds({"grouped": lambda: grp(gs, 1024), "batched": lambda: bat(small)}, n=1024, rounds=2)
    res["small_1024x33"] = {k: v["solves_per_s"] for k, v in sm.items()}
    M.mhs_group_destroy(gs)
    for h in small:
        M.mhs_destroy(h)
    torch.cuda.empty_cache()
    return res


def serving_leg(M, requests=10000, loads=(0.5, 0.8, 0.95), inflight=None, budget_gb=None):
    """Poisson arrivals of solve requests, grid sizes 65^3 / 129^3 / 257^3 at 60/30/10 %, random
    magnetograms and alpha / xi parameters (request r: splitmix64(r); arrivals: splitmix64(42)),
    served with HBM-budget admission and resident hierarchies (mixed precision, Phi + fields into
    device buffers).  The server's limits are chosen by measurement (unless given): the in-flight
    limit with the highest capacity on the first 1,500 requests queued at once (8, 16, 32 or 64
    slots), then the smallest HBM budget (8, 16, 32 or 64 GB) whose capacity stays within 3 % of
    the largest.  Capacity is then measured on all requests queued at once; the Poisson stream runs
    at each of `loads` x capacity (the headline keys are those of 0.8).  Baseline: the same requests
    solved one after another in FP64 through mhs_solve + mhs_fields."""
    import math as _m
    import torch
    sizes = []
    for r in range(requests):
        u = S.SplitMix64(r).uniform()
        sizes.append(65 if u < 0.6 else 129 if u < 0.9 else 257)
    params, mags = [], {}
    for r in range(requests):
        rng = S.SplitMix64(7_000_000 + r)
        params.append((rng.uniform(0.0, 0.8), rng.uniform(0.0, 0.9), rng.uniform(0.5, 2.0)))
    for n in (65, 129, 257):   # a few magnetograms per size, reused round-robin
        mags[n] = [S.magnetogram_random(n, n, seed=9000 + 10 * n + i) for i in range(4)]
    # output buffers, 18 sets per grid used round-robin: this leg measures time only, so requests in
    # flight at once may write the same set
    ring = {n: [[torch.empty((n, n, n), dtype=torch.float64, device="cuda") for _ in range(6)]
                for _ in range(18)] for n in (65, 129, 257)}
    use = {n: 0 for n in ring}

    def submit(srv, r):
        n = sizes[r]
        alpha, a, kappa = params[r]
        bufs = ring[n][use[n] % len(ring[n])]
        use[n] += 1
        return M.mhs_server_submit(srv, n, n, n, 1.0, 1.0, 1.0, alpha, M.xi_params(M.MHS_XI_EXP, a, kappa),
                                   mags[n][r % 4], TOL, M.MHS_MIXED, phi=bufs[0], Bx=bufs[1], By=bufs[2],
                                   Bz=bufs[3], p=bufs[4], rho=bufs[5])

    def warm(srv, slots):
        # create the resident hierarchies (up to max_inflight per grid) and capture their graphs:
        # three rounds of max_inflight requests in flight, untimed
        for _ in range(3):
            for t in [submit(srv, r) for r in range(min(requests, 3 * slots))]:
                M.mhs_server_wait(srv, t, 600.0)

    def capacity_of(slots, gb, count):
        srv = M.mhs_server_create(gb << 30, slots)
        warm(srv, slots)
        t0 = time.perf_counter()
        tickets = [submit(srv, r) for r in range(count)]
        for t in tickets:
            M.mhs_server_wait(srv, t, 600.0)
        rate = count / (time.perf_counter() - t0)
        peak = M.mhs_server_stats(srv)["device_bytes"]
        M.mhs_server_destroy(srv)
        return rate, peak

    choice = {}
    sample = min(requests, 1500)
    if inflight is None:
        rates = {k: capacity_of(k, 64, sample)[0] for k in (8, 16, 32, 64)}
        inflight = max(rates, key=lambda k: rates[k])
        choice["inflight_capacity"] = {str(k): v for k, v in rates.items()}
    if budget_gb is None:
        rates = {gb: capacity_of(inflight, gb, sample) for gb in (8, 16, 32, 64)}
        best = max(r for r, _ in rates.values())
        budget_gb = min(gb for gb, (r, _) in rates.items() if r >= 0.97 * best)
        choice["budget_capacity"] = {str(gb): {"solves_per_s": r, "resident_bytes": b} for gb, (r, b) in rates.items()}
    capacity, _ = capacity_of(inflight, budget_gb, requests)

    def stream(load):
        srv = M.mhs_server_create(budget_gb << 30, inflight)
        warm(srv, inflight)
        rate = load * capacity
        arr = S.SplitMix64(42)
        t_next = time.perf_counter()
        tickets = []
        t0 = time.perf_counter()
        for r in range(requests):
            t_next += -_m.log(1.0 - arr.uniform()) / rate
            while time.perf_counter() < t_next:
                pass
            tickets.append(submit(srv, r))
        lat = []
        for t in tickets:
            info, st, l = M.mhs_server_wait(srv, t, 600.0)
            assert st == 0, st
            lat.append(l)
        span = time.perf_counter() - t0
        stats = M.mhs_server_stats(srv)
        M.mhs_server_destroy(srv)
        lat.sort()
        pct = lambda p: lat[min(len(lat) - 1, int(p * (len(lat) - 1) + 0.5))]
        return {"offered_load": load, "arrival_rate_per_s": rate, "solves_per_s": requests / span,
                "p50_ms": pct(0.5), "p99_ms": pct(0.99), "server_p50_ms": stats["p50_ms"],
                "server_p99_ms": stats["p99_ms"], "resident_hierarchies": stats["resident_hierarchies"],
                "device_bytes": stats["device_bytes"]}

    per_load = {str(load): stream(load) for load in loads}
    head = per_load[str(0.8)] if str(0.8) in per_load else per_load[str(loads[0])]

    # sequential FP64 baseline on a sample of the same requests (one handle per size)
    hs = {n: M.mhs_create(n, n, n, 1.0, 1.0, 1.0, 0.0) for n in (65, 129, 257)}
    sample = list(range(min(requests, 200)))
    outs = {n: ring[n][0] for n in ring}
    for r in sample[:6]:
        n = sizes[r]; a_, x_, k_ = params[r]
        M.mhs_set_params(hs[n], a_, M.xi_params(M.MHS_XI_EXP, x_, k_))
        M.mhs_set_lower_bz(hs[n], mags[n][r % 4]); M.mhs_solve(hs[n], TOL, M.MHS_FP64)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for r in sample:
        n = sizes[r]; a_, x_, k_ = params[r]
        M.mhs_set_params(hs[n], a_, M.xi_params(M.MHS_XI_EXP, x_, k_))
        M.mhs_set_lower_bz(hs[n], mags[n][r % 4])
        M.mhs_solve(hs[n], TOL, M.MHS_FP64)
        M.mhs_get_phi(hs[n], outs[n][0])
        M.mhs_fields(hs[n], *outs[n][1:])
    torch.cuda.synchronize()
    seq_rate = len(sample) / (time.perf_counter() - t1)
    for h in hs.values():
        M.mhs_destroy(h)
    del ring
    torch.cuda.empty_cache()
    return dict({"requests": requests, "mix": "65^3/129^3/257^3 at 60/30/10 %", "max_inflight": inflight,
                 "budget_gb": budget_gb, "limits_chosen_by": choice or "given", "capacity_solves_per_s": capacity},
                **head,
                sequential_fp64_solves_per_s=seq_rate, sequential_sample=len(sample),
                speedup_vs_sequential_fp64=head["solves_per_s"] / seq_rate, loads=per_load)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--mode", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--impl", choices=["mhs", "reference"], default="mhs")
    ap.add_argument("--cpu-budget", type=float, default=10.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--light", action="store_true",
                    help="timed steps only (no CPU baseline, e2e, kernel timing or second mode): for launch lists")
    ap.add_argument("--op", choices=["smooth", "residual", "restrict", "prolong", "vcycle", "exact", "resid_restrict",
                                     "fma"],
                    default=None,
                    help="repeat one finest-level operation of the interior hierarchy (--steps times) for kernel "
                         "capture; fma: the device's FP64 and FP32 FMA rates (the ALU roofline denominators)")
    ap.add_argument("--prec", choices=["fp64", "fp32"], default="fp64", help="precision of --op")
    ap.add_argument("--grid", type=int, nargs=3, default=[129, 129, 129], metavar=("NX", "NY", "NZ"),
                    help="grid of --op")
    ap.add_argument("--smoother", choices=["point", "zline"], default="point", help="smoother of --op smooth")
    ap.add_argument("--dim", type=int, choices=[2, 3], default=3,
                    help="--op on the finest level of the interior (3) or lower-boundary (2) hierarchy")
    ap.add_argument("--tma", action="store_true", help="--op smooth in FP32: the fused TMA-staged sweep")
    ap.add_argument("--tma-rows", type=int, choices=[0, 8, 16], default=0,
                    help="tile height of the fused TMA-staged sweep (0: the library's default)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the large-grid, batched and serving legs")
    ap.add_argument("--serve-requests", type=int, default=10000, help="requests in the serving leg")
    ap.add_argument("--eager", action="store_true",
                    help="host-driven kernel-by-kernel solve instead of the captured graph (for launch lists)")
    ap.add_argument("--zline", action="store_true",
                    help="smooth the interior levels by zebra z-line Gauss-Seidel instead of red-black point sweeps")
    ap.add_argument("--no-fmg", action="store_true",
                    help="start each solve from zero with a plain V-cycle instead of a full-multigrid cycle")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "mhs":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.op:
        run_op(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
