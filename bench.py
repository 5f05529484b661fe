#!/usr/bin/env python3
"""Benchmark of the GB300 diffusion-based coarse-graining path.

One step = the whole method (locate + ordered deposition + implicit-Euler diffusion
to T = b^2/4, 10 pseudo-steps) on the 128^3 clustered unit-cube workload
(2,000,000 spheres of d = 0.004 in 20 Gaussian clusters), once for each bandwidth
b/dx in {1, 2, 4, 8}, in the mixed path (FP32 Chebyshev inner solves with
double-float iterative refinement to ||r|| <= 1e-13 ||b|| per pseudo-step).  The
other precision modes (FP64 CG, FP32 + IEEE-FP64 refinement, BF16 + double-float
refinement) are timed on the same workload and reported beside it.

Metric: diffusion cell-updates/s (one cell-update = one application of the implicit
operator at one cell for one field), whole job over all ranks.  The same line carries
the FP64 GPU path, end-to-end throughput through the host-pointer C entry point, a
roofline entry for the dominant kernel, the oracle CPU baseline and the SM clocks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py profile-case ...   (one case alone, for ncu; see profile_case)
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1409_0001_gb300.ranks import dist_env, reduce_scalar  # noqa: E402

B_OVER_DX = (1.0, 2.0, 4.0, 8.0)
NSTEPS = 10
TOL = 1e-13
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n-side", type=int, default=128)
    ap.add_argument("--n-particles", type=int, default=2_000_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the tet, batched and channel workloads")
    ap.add_argument("--concurrency", type=int, default=2,
                    help="the four bandwidths of a step are independent problems; run this many "
                         "at a time (cg_coarse_grain_concurrent; 1 = one after another)")
    ap.add_argument("--sweep-shape", type=int, default=0,
                    help="inner-solve sweep shape for the mixed modes (include/cg.h "
                         "sweep_shape; 0 = autotuned)")
    return ap.parse_args()


def workload_name(a):
    return ("clustered_cube_%d: %d^3 unit cube, %d spheres d=0.004 in 20 Gaussian clusters "
            "(sigma 0.05, <=8 per cell), b/dx in {1,2,4,8}, %d implicit-Euler pseudo-steps, "
            "tol 1e-13" % (a.n_side, a.n_side, a.n_particles, NSTEPS))


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def source_section(path, start, end):
    """The text of a source file from the line that begins with `start` up to (not
    including) the line that begins with `end`."""
    with open(os.path.join(ROOT, path)) as f:
        text = f.read()
    i = text.index(start)
    return text[i:text.index(end, i + len(start))]


def ncu_record(kernel_entry):
    """The committed ncu capture of a kernel (roofline_traffic.json), or None when the
    kernel's source section changed since the counters were taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
            rec = json.load(f).get(kernel_entry)
        if not rec:
            return None
        sec = source_section(rec["source"], rec["section_start"], rec["section_end"])
        sha = hashlib.sha256(sec.encode()).hexdigest()
        return rec if sha == rec["section_sha256"] else None
    except (OSError, ValueError, KeyError):
        return None


def ncu_traffic(kernel_entry):
    """DRAM bytes per launch of a kernel from the committed ncu capture, or None."""
    rec = ncu_record(kernel_entry)
    return rec["dram_bytes_per_launch"] if rec else None


def nvtx(push, name):
    """Open (push) or close an NVTX range, where torch's NVTX binding is present."""
    try:
        import torch
        if push:
            torch.cuda.nvtx.range_push(name)
        else:
            torch.cuda.nvtx.range_pop()
    except (RuntimeError, AttributeError):
        pass


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ----------------------------------------------------------------------------- reference arm
def run_reference(a):
    """The oracle (plain FP64 C, single thread, as it stands) as the reference arm, on the
    same workload and metric.  Each step is a bounded sample of the benchmark's step: the
    full locate and ordered deposition of every particle, then the first implicit-Euler
    pseudo-step (same dtau as in the 10-step run) at each of b/dx = 1, 2, 4, 8.  The metric
    is a rate (cell-updates per second), so it compares directly; the whole 10-step run
    would take about ten times as long per step at a similar rate (later steps of a
    smoothing converge in fewer CG iterations, so the sample, if anything, favours the
    oracle's rate less than it)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    import workloads as W
    oracle.build()
    c = W.clustered_cube(n_side=a.n_side, n_particles=a.n_particles)

    def step():
        cell, _ = oracle.locate_structured(c.dims, c.origin, c.dx, c.pos)
        eps0, _ = oracle.deposit(cell, c.w, c.ncells, vc_uniform=(c.dx * c.dx) * c.dx)
        upd = 0
        for bdx in B_OVER_DX:
            b = bdx * c.dx
            _, iters = oracle.diffuse_structured(eps0, c.dims, c.dx, b * b / 4 / NSTEPS, 1, tol=TOL)
            upd += (iters + 1) * c.ncells      # CG iterations + one residual per step
        return upd

    for _ in range(a.warmup):
        step()
    t0 = time.perf_counter()
    total_updates = 0
    for _ in range(a.steps):
        total_updates += step()
    dt = time.perf_counter() - t0
    v = total_updates / dt
    line = {"impl": "reference", "metric": "diffusion cell-updates/s", "value": v,
            "unit": "cell-updates/s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": dt * 1e3 / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a)},
            "cpu_baseline": {"value": v, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
                             "sample": "per step: locate+deposit all %d particles, then the first of "
                                       "the 10 implicit-Euler steps at each of b/dx = 1, 2, 4, 8 "
                                       "(FP64 CG to 1e-13); a rate, so the full 10-step run "
                                       "extrapolates at about 10x the time per step" % a.n_particles,
                             "host": host_cpu()},
            "e2e": {"value": v, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ----------------------------------------------------------------------------- our arm
def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
        return
    import torch
    import torch.distributed as dist

    import paper_1409_0001_gb300 as cg
    import workloads as W
    from paper_1409_0001_gb300 import build as libbuild

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    libbuild.build()
    lib = cg.load_library()

    c = W.clustered_cube(n_side=a.n_side, n_particles=a.n_particles, seed=rank)
    # one mesh per bandwidth: concurrent problems need their own workspaces
    meshes = [cg.StructuredMesh(c.dims, c.origin, c.dx) for _ in B_OVER_DX]
    pos = torch.from_numpy(c.pos).cuda()
    w = torch.from_numpy(c.w).cuda()
    outs = [torch.empty((1, c.ncells), dtype=torch.float64, device="cuda") for _ in B_OVER_DX]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def params(bdx, precision):
        return cg.Params(bandwidth=bdx * c.dx, nsteps=NSTEPS, precision=precision, tol=TOL,
                         sweep_shape=a.sweep_shape if precision != cg.PREC_FP64 else 0)

    streams = [torch.cuda.Stream() for _ in B_OVER_DX]

    def one_step_seq(precision, reps, p_=None, w_=None):
        for i, bdx in enumerate(B_OVER_DX):
            _, r = cg.coarse_grain(meshes[i], pos if p_ is None else p_, w if w_ is None else w_,
                                   params(bdx, precision), out=outs[i], report=True)
            reps.append(r)

    def one_step(precision, reps, p_=None, w_=None):
        """The four coarse-grainings of a step, a.concurrency at a time."""
        if a.concurrency <= 1:
            return one_step_seq(precision, reps, p_, w_)
        k = len(B_OVER_DX)
        _, r = cg.coarse_grain_concurrent(
            meshes, [pos if p_ is None else p_] * k, [w if w_ is None else w_] * k,
            [params(bdx, precision) for bdx in B_OVER_DX], out=outs, streams=streams,
            max_concurrent=a.concurrency, report=True)
        reps.extend(r)

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
            torch.cuda.synchronize()

    def timed(fn, steps, label=None):
        """Per-step CUDA-event time (L2 flushed before every step, outside the events).
        With a label, each step is an NVTX range of that name (a profiler can select the
        step's kernels by it)."""
        stream = torch.cuda.current_stream()
        tot = 0.0
        for _ in range(steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            if label:
                nvtx(True, label)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            if label:
                nvtx(False, label)
            tot += e0.elapsed_time(e1)
        return tot

    def max_over_ranks(x):
        return reduce_scalar(x, "max", device="cuda")

    def sum_over_ranks(x):
        return reduce_scalar(x, "sum", device="cuda")

    MAIN = cg.PREC_FP32_DF_REFINE
    # ---------------- warm-up (the first calls autotune each mesh's sweep shape, one
    # problem at a time so that no other work disturbs the candidates' timings)
    one_step_seq(MAIN, [])
    for _ in range(a.warmup):
        one_step(MAIN, [])
    barrier()

    # ---------------- timed region (clean: no per-kernel events)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    launches_before = int(lib.cg_launch_count())
    lib.cg_launch_count_reset()
    reps = []
    barrier()
    ms = timed(lambda: one_step(MAIN, reps), a.steps, label="timed_step")
    barrier()
    launches = int(lib.cg_launch_count())
    clocks = sampler.stop()
    ms = max_over_ranks(ms)
    updates = sum_over_ranks(float(sum(r["cell_updates"] for r in reps)))
    value = updates / (ms * 1e-3)
    rounds = sum(r["refine_rounds"] for r in reps) / max(len(reps), 1)
    worst_res = max(r["final_rel_residual"] for r in reps)
    mass_err = max(abs(r["mass_out"][0] - r["mass_in"][0]) / r["mass_in"][0] for r in reps)
    ms_phase = {k: sum(r[k] for r in reps) / a.steps for k in ("ms_locate", "ms_deposit",
                                                               "ms_diffuse")}
    # calls that deposited (problems sharing one deposition report zero deposition time)
    dep_ms = [r["ms_locate"] + r["ms_deposit"] for r in reps if r["ms_locate"] + r["ms_deposit"] > 0]
    n_dep = len(dep_ms)
    dep_rate = c.n * n_dep / (sum(dep_ms) * 1e-3) if dep_ms else None

    # ---------------- per-kernel device time: the same steps again with event pairs
    cg.profile_reset()
    cg.profile_enable(True)
    prof_reps = []
    ms_prof = timed(lambda: one_step_seq(MAIN, prof_reps), a.steps)   # events need one at a time
    cg.profile_enable(False)
    kern = cg.profile_read()

    # ---------------- the other precision modes, same workload
    main_out = [o.clone() for o in outs]
    modes = {}
    mode_out = {}
    for name, prec in (("fp64_cg", cg.PREC_FP64), ("fp32_fp64refine", cg.PREC_FP32_REFINE),
                       ("bf16_dfrefine", cg.PREC_BF16_DF_REFINE)):
        one_step_seq(prec, [])                  # warm (and autotune) the mode
        one_step(prec, [])
        mreps = []
        msm = timed(lambda: one_step(prec, mreps), max(a.fp64_steps, 1)) / max(a.fp64_steps, 1)
        msm = max_over_ranks(msm)
        mode_out[name] = [o.clone() for o in outs]
        if name == "fp64_cg":
            fp64_reps = mreps
        modes[name] = {"ms_per_step": msm,
                       "cell_updates_per_s": sum(r["cell_updates"] for r in mreps)
                       / max(a.fp64_steps, 1) / (msm * 1e-3),
                       "cell_pseudo_steps_per_s": len(B_OVER_DX) * NSTEPS * c.ncells / (msm * 1e-3)}
    fp64_out = mode_out["fp64_cg"]
    try:
        fp64_gemm = measure_fp64_gemm()
    except Exception:   # noqa: BLE001 -- e.g. no room for the two 512 MB operands
        fp64_gemm = None
    modes["fp64_cg"]["roofline"] = fp64_roofline(fp64_reps, outs[0].shape[0], modes["fp64_cg"]["ms_per_step"],
                                                 max(a.fp64_steps, 1), measured_peaks()[0], measured_tflops=fp64_gemm)
    for name in modes:
        modes[name]["maxrel_vs_fp64_gpu"] = max(float((m - f).abs().max() / f.abs().max())
                                                for m, f in zip(mode_out[name], fp64_out))
    modes["fp32_dfrefine"] = {"ms_per_step": ms / a.steps,
                              "maxrel_vs_fp64_gpu": max(float((m - f).abs().max() / f.abs().max())
                                                        for m, f in zip(main_out, fp64_out))}
    outs = main_out

    # ---------------- end to end through the C ABI with host buffers: each of the step's
    # coarse-grainings copies the pinned host particles in and its field out
    # (cg_coarse_grain_host, several at a time through cg_coarse_grain_concurrent)
    main_ref = [o.cpu() for o in main_out]
    pos_h = torch.from_numpy(c.pos).pin_memory()
    w_h = torch.from_numpy(c.w).pin_memory()
    out_h = [torch.empty((1, c.ncells), dtype=torch.float64).pin_memory() for _ in B_OVER_DX]

    def e2e_step(reps_e):
        if a.concurrency > 1:
            k = len(B_OVER_DX)
            _, r = cg.coarse_grain_concurrent(meshes, [pos_h] * k, [w_h] * k,
                                              [params(bdx, MAIN) for bdx in B_OVER_DX], out=out_h,
                                              streams=streams, max_concurrent=a.concurrency,
                                              report=True)
            reps_e.extend(r)
        else:
            for i, bdx in enumerate(B_OVER_DX):
                _, r = cg.coarse_grain_host(meshes[i], pos_h, w_h, params(bdx, MAIN), out=out_h[i],
                                            report=True)
                reps_e.append(r)

    e2e_step([])
    reps_e = []
    barrier()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        e2e_step(reps_e)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e_updates = sum_over_ranks(float(sum(r["cell_updates"] for r in reps_e)))
    # the concurrent entry copies host arrays shared by several problems once
    h2d = (1 if a.concurrency > 1 else len(B_OVER_DX)) * (pos_h.numel() + w_h.numel()) * 8
    d2h = len(B_OVER_DX) * c.ncells * 8
    e2e_ok = all(bool(torch.equal(o, h)) for o, h in zip(main_ref, out_h))

    # ---------------- roofline of the dominant kernel
    peaks, peak_src = measured_peaks()
    top = max(kern.items(), key=lambda kv: kv[1]["ms"]) if kern else (None, None)
    roof = None
    if top[0] is not None:
        name, k = top
        achieved = k["bytes"] / (k["ms"] * 1e-3) / 1e9
        peak = float(peaks["hbm_gbs"])
        roof = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "traffic": ncu_traffic(name),
                "algorithmic_bytes_per_launch": k["bytes"] / k["launches"],
                "peak_source": peak_src + " hbm_gbs (STREAM-style copy)",
                "avg_launch_us": k["ms"] * 1e3 / k["launches"],
                "share_of_kernel_time": k["ms"] / sum(v["ms"] for v in kern.values()),
                "note": "at 128^3 the sweep's four FP32 arrays (33.5 MB) stay in L2 within a step, "
                        "so this fraction is an L2-resident kernel's algorithmic rate against the "
                        "HBM peak; roofline_hbm is the dominant kernel where the working set leaves "
                        "L2 (the 512x256x256 channel, where the autotuner picks two iterations per "
                        "launch: algorithmic bytes 16 B per cell for a round's first pair and its "
                        "last single iteration, 20 B for the other pairs)"}

    # ---------------------------------------------------------------- several ranks: the
    # 64-snapshot batch split over the ranks by cost (independent snapshots, no data-path
    # collective), each rank smoothing its share in one batched call
    sharded = None
    if ws > 1 and not a.no_extras:
        sharded = sharded_batch(ws, rank, max_over_ranks, sum_over_ranks, barrier)

    line = None
    ext = None
    if rank == 0 and not a.no_extras:
        try:
            ext = extras()
        except Exception as e:   # the main line is printed whatever an extra workload does
            import traceback
            traceback.print_exc()
            ext = {"error": "%s: %s" % (type(e).__name__, e)}
    if rank == 0:
        cpu = None
        if not a.no_cpu_baseline and ws == 1:
            try:
                cpu = cpu_baseline(c, outs, fp64_out)
            except Exception as e:
                import traceback
                traceback.print_exc()
                cpu = {"error": "%s: %s" % (type(e).__name__, e), "kind": "oracle"}
        ncells = c.ncells
        cps = ws * a.steps * len(B_OVER_DX) * NSTEPS * ncells / (ms * 1e-3)
        line = {
            "metric": "diffusion cell-updates/s", "value": value, "unit": "cell-updates/s",
            "n_gpus": ws, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(a),
                       "precision": "fp32 Chebyshev inner solves + double-float (fp32 hi/lo) "
                                    "refinement of the implicit-step residual",
                       "l2": "flushed before every step (256 MB write, outside the timed events)",
                       "concurrency": ("the four bandwidths as independent problems, %d at a time "
                                       "(cg_coarse_grain_concurrent, which deposits the particles "
                                       "they share once)" % a.concurrency
                                       if a.concurrency > 1 else "one bandwidth after another"),
                       "parallelism": "replicas" if ws > 1 else "single"},
            "e2e": {"value": e2e_updates / e2e_s, "unit": "cell-updates/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "entry_point": "cg_coarse_grain_host per bandwidth (pinned host buffers, copies "
                                   "inside), %s" % ("%d at a time through cg_coarse_grain_concurrent, "
                                                    "which copies the particle arrays the four share "
                                                    "in once per step and deposits them once" % a.concurrency
                                                    if a.concurrency > 1 else "one after another"),
                    "result_identical_to_device_run": e2e_ok},
            "gpu_launches": launches,
            "gpu_launches_before_timed": launches_before,
            "sweep_shape_used": sorted({r["sweep_shape_used"] for r in reps}),
            "clocks": clocks,
            "roofline": roof,
            "cpu_baseline": cpu,
            "cell_pseudo_steps_per_s": cps,
            "particles_per_s": dep_rate,
            "particles_per_s_note": "locate + ordered deposition of one field (F = 1), from the "
                                    "phase times (device events) of the calls that deposited: "
                                    "the four bandwidths deposit the same particles on meshes of "
                                    "one geometry, so the concurrent entry deposits once per step "
                                    "(%d depositions in %d calls)" % (n_dep, len(reps)),
            "roofline_hbm": (ext or {}).get("channel_512x256x256", {}).get("roofline_hbm")
                            if isinstance(ext, dict) else None,
            "ms_per_phase_per_step": ms_phase,
            "refine_rounds_per_solve": rounds,
            "worst_rel_residual": worst_res,
            "worst_rel_mass_error": mass_err,
            "modes": modes,
            "batched_64_sharded": sharded,
            "mixed_speedup_vs_fp64_gpu": modes["fp64_cg"]["ms_per_step"] / (ms / a.steps),
            "profiled_ms_per_step": ms_prof / a.steps,
            "other_workloads": ext,
            "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 4),
                            "GBps": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else None}
                        for k, v in sorted(kern.items(), key=lambda kv: -kv[1]["ms"])},
        }
        print(json.dumps(line))
    for m in meshes:
        m.close()
    if ws > 1:
        dist.destroy_process_group()


def sharded_batch(ws, rank, max_over_ranks, sum_over_ranks, barrier, reps=2):
    """The 64-snapshot batch shared out over the ranks: shard_by_cost gives each rank its
    snapshots (cost ~ cells x fields), which it deposits and smooths in one batched call on
    its GPU.  Time = the slowest rank's; the result is strong scaling of one batch."""
    import torch
    import paper_1409_0001_gb300 as cg
    import workloads as W
    from paper_1409_0001_gb300.ranks import shard_by_cost
    cases = W.batched_snapshots()
    mine = shard_by_cost([c.ncells for c in cases], ws, rank)
    sel = [cases[i] for i in mine]
    meshes = [cg.StructuredMesh(c.dims, c.origin, c.dx) for c in sel]
    bp = [torch.from_numpy(c.pos).cuda() for c in sel]
    bw = [torch.from_numpy(c.w).cuda() for c in sel]
    prm = cg.Params(nsteps=10, precision=cg.PREC_FP32_DF_REFINE)
    upd = 0
    if sel:
        cg.coarse_grain_batched(meshes, bp, bw, prm, bandwidths=[c.b for c in sel])   # tune
    barrier()
    t0 = time.perf_counter()
    for _ in range(reps):
        if sel:
            _, rep = cg.coarse_grain_batched(meshes, bp, bw, prm, bandwidths=[c.b for c in sel],
                                             report=True)
            upd += rep["cell_updates"]
    torch.cuda.synchronize()
    dt = max_over_ranks(time.perf_counter() - t0)
    barrier()
    total = sum_over_ranks(float(upd))
    for m in meshes:
        m.close()
    return {"ranks": ws, "snapshots_on_rank0": len(mine) if rank == 0 else None,
            "ms_per_batch": dt * 1e3 / reps, "cell_updates_per_s": total / dt,
            "scaling": "strong", "partition": "shard_by_cost over cells (longest first)"}


def _timed_call(fn, reps=2, warm=1):
    """Device time (CUDA events on the current stream) of fn(), the mean of reps timed
    calls after warm untimed ones; returns (ms, the last call's result)."""
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(warm):
        fn()
    tot = 0.0
    out = None
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    return tot / reps, out


# ----------------------------------------------------------------------------- FP64 references
def _omp_oracle():
    """The oracle's multi-core build (oracle/omp.py), or None where it does not compile."""
    try:
        from oracle import omp
        return omp if omp.available() else None
    except Exception:   # noqa: BLE001 -- no OpenMP compiler: the single-thread oracle serves
        return None


def oracle_structured(c, b, nsteps, scheme=0, pos=None, w=None):
    """FP64 oracle of the whole method on a uniform mesh (locate, ordered deposition,
    nsteps implicit steps to T = b^2/4 by CG to 1e-14): the multi-core build when it is
    available (the same deposition bits, diffusion within 1e-12 of the single-thread
    oracle), else the single-thread oracle.  Returns (eps(T) [nf, ncells], kind)."""
    import oracle
    pos = c.pos if pos is None else pos
    w = c.w if w is None else w
    omp = _omp_oracle()
    vcu = (c.dx * c.dx) * c.dx
    if omp is not None:
        cell, nout = omp.locate_structured(c.dims, c.origin, c.dx, pos)
        eps0 = omp.deposit(cell, w, c.ncells, vc_uniform=vcu)
        u, _ = omp.diffuse_structured(eps0, c.dims, c.dx, b * b / 4, nsteps, scheme=scheme, tol=1e-14)
        return u, "oracle, multi-core build (%d threads)" % omp.threads()
    cell, nout = oracle.locate_structured(c.dims, c.origin, c.dx, pos)
    eps0, _ = oracle.deposit(cell, w, c.ncells, vc_uniform=vcu)
    u, _ = oracle.diffuse_structured(eps0, c.dims, c.dx, b * b / 4, nsteps, scheme=scheme, tol=1e-14)
    return u, "oracle, single thread"


def maxrel_np(u, ref):
    """max over fields of max_k |u - ref| / max_k |ref| (the parity metric)."""
    u, ref = np.atleast_2d(np.asarray(u)), np.atleast_2d(np.asarray(ref))
    return float(max(np.max(np.abs(u[f] - ref[f])) / max(np.max(np.abs(ref[f])), 1e-300)
                     for f in range(ref.shape[0])))


def dct_closed_form(u0, dims, dx, T, nsteps):
    """Exact solution of nsteps implicit-Euler steps of the zero-flux 7-point system on a
    uniform mesh: the separable orthonormal DCT-II diagonalises it (eigenvalue
    -(4/dx^2) sin^2(pi j / (2N)) per axis)."""
    import scipy.fft
    nx, ny, nz = dims
    uh = scipy.fft.dctn(np.asarray(u0).reshape(nz, ny, nx), type=2, norm="ortho",
                        workers=os.cpu_count() or 1)
    dt = T / nsteps
    s = [(4.0 * dt / dx ** 2) * np.sin(np.pi * np.arange(n) / (2.0 * n)) ** 2 for n in (nx, ny, nz)]
    a = s[2][:, None, None] + s[1][None, :, None] + s[0][None, None, :]
    uh *= (1.0 / (1.0 + a)) ** nsteps
    return scipy.fft.idctn(uh, type=2, norm="ortho", workers=os.cpu_count() or 1).ravel()


def deposit_rate(n, nf, rep):
    """Particles deposited per second: the locate and deposition phases of a call."""
    ms = rep["ms_locate"] + rep["ms_deposit"]
    return {"particles_per_s": n / (ms * 1e-3) if ms > 0 else None, "fields": nf,
            "ms_locate_plus_deposit": ms}


def kernel_roofline(kern, peaks, peak_src, traffic_key=None):
    """Roofline of the dominant kernel of a profiled call (per-kernel CUDA event pairs)."""
    if not kern:
        return None
    name, k = max(kern.items(), key=lambda kv: kv[1]["ms"])
    achieved = k["bytes"] / (k["ms"] * 1e-3) / 1e9
    peak = float(peaks["hbm_gbs"])
    rec = ncu_record(traffic_key or name)
    out = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak, "traffic": rec["dram_bytes_per_launch"] if rec else None,
           "algorithmic_bytes_per_launch": k["bytes"] / k["launches"],
           "peak_source": peak_src + " hbm_gbs (STREAM-style copy)",
           "avg_launch_us": k["ms"] * 1e3 / k["launches"], "launches": k["launches"],
           "share_of_kernel_time": k["ms"] / sum(v["ms"] for v in kern.values())}
    if rec and "algorithmic_bytes_of_captured_launch" in rec:
        # the capture is one launch of a group whose launches move different byte counts
        out["traffic_launch_algorithmic_bytes"] = rec["algorithmic_bytes_of_captured_launch"]
    return out


def extras():
    """The other configurations of the method, each measured the same way (whole method
    per call, CUDA events, the mean of timed calls after a warm-up call), each mixed mode
    against the FP64 GPU path and every mode against the FP64 oracle."""
    import torch
    import paper_1409_0001_gb300 as cg
    import workloads as W
    import oracle

    def maxrel(a, b):
        return float((a - b).abs().max() / b.abs().max())

    def cpu(t):
        return t.cpu().numpy()

    peaks, peak_src = measured_peaks()
    res = {}
    # config 1: the plain FP64 method on the 32^3 unit cube, 10,000 spheres, b = 3 dx
    c1 = W.uniform_cube()
    mesh = cg.StructuredMesh(c1.dims, c1.origin, c1.dx)
    dp, dw = torch.from_numpy(c1.pos).cuda(), torch.from_numpy(c1.w).cuda()
    _, ref1, _, _ = oracle.coarse_grain_structured(c1.dims, c1.origin, c1.dx, c1.pos, c1.w, c1.b,
                                                   c1.nsteps)
    out = {}
    for name, prec in (("fp64_cg", cg.PREC_FP64), ("fp32_dfrefine", cg.PREC_FP32_DF_REFINE)):
        ms, (u, rep) = _timed_call(lambda: cg.coarse_grain(mesh, dp, dw, cg.Params(
            bandwidth=c1.b, nsteps=c1.nsteps, precision=prec), report=True), reps=5)
        out[name] = (ms, cpu(u), rep)
    res["uniform_32"] = {
        "workload": "32^3 unit cube, 10,000 spheres d=0.01 at U[0,1]^3, b=3dx, 10 IE steps, plain FP64 "
                    "method (and the mixed path beside it)",
        "modes": {k: {"ms": v[0], "cell_updates_per_s": v[2]["cell_updates"] / (v[0] * 1e-3),
                      "maxrel_vs_oracle": maxrel_np(v[1], ref1), **deposit_rate(c1.n, 1, v[2])}
                  for k, v in out.items()},
        "oracle": "oracle, single thread"}
    mesh.close()
    del dp, dw
    # config 3 (unstructured): 100^3 hexes -> 6,000,000 jittered Kuhn tets, 5,000,000
    # layered spheres
    xyz, tets = W.kuhn_tet_mesh(100)
    mesh = cg.TetMesh(xyz, tets)
    pos, w, _ = W.layered_cube()
    dp, dw = torch.from_numpy(pos).cuda(), torch.from_numpy(w).cuda()
    out = {}
    for name, prec in (("fp32_fp64refine", cg.PREC_FP32_REFINE), ("fp64_pcg", cg.PREC_FP64)):
        ms, (u, rep) = _timed_call(lambda: cg.coarse_grain(mesh, dp, dw, cg.Params(
            bandwidth=0.03, nsteps=10, precision=prec), report=True))
        out[name] = (ms, u.clone(), rep)
    vc, _, rp, col, val = oracle.tet_build(xyz, tets)
    omp = _omp_oracle()
    if omp is not None:
        cell, _ = omp.locate_tet_bucketed(xyz, tets, pos)
        eps0 = omp.deposit(cell, w, len(vc), vc=vc)
        ref3, _ = omp.diffuse_csr(eps0, vc, rp, col, val, 0.03 ** 2 / 4, 10, tol=1e-14)
        kind3 = "oracle, multi-core build (%d threads)" % omp.threads()
    else:
        cell, _ = oracle.locate_tet_bucketed(xyz, tets, pos)
        eps0, _ = oracle.deposit(cell, w, len(vc), vc=vc)
        ref3, _ = oracle.diffuse_csr(eps0, vc, rp, col, val, 0.03 ** 2 / 4, 10, tol=1e-14)
        kind3 = "oracle, single thread"
    res["tet_layered_6M"] = {
        "workload": "100^3 hexes -> 6,000,000 jittered Kuhn tets (two-point-flux FV), 5,000,000 "
                    "spheres d=0.003 with a dense bottom layer, b=0.03, 10 IE steps",
        "modes": {k: {"ms": v[0], "cell_updates_per_s": v[2]["cell_updates"] / (v[0] * 1e-3),
                      "cell_pseudo_steps_per_s": 10 * 6e6 / (v[0] * 1e-3),
                      "maxrel_vs_oracle": maxrel_np(cpu(v[1]), ref3), **deposit_rate(5e6, 1, v[2])}
                  for k, v in out.items()},
        "ms_per_phase": {k: out["fp32_fp64refine"][2][k] for k in ("ms_locate", "ms_deposit", "ms_diffuse")},
        "mixed_speedup_vs_fp64_gpu": out["fp64_pcg"][0] / out["fp32_fp64refine"][0],
        "mixed_vs_fp64_maxrel": maxrel(out["fp32_fp64refine"][1], out["fp64_pcg"][1]),
        "oracle": kind3}
    mesh.close()
    del dp, dw, out, ref3, eps0
    # config 4 (batched): 64 snapshots, 32^3..96^3, 10^4..10^6 particles, 5 fields
    cases = W.batched_snapshots()
    meshes = [cg.StructuredMesh(c.dims, c.origin, c.dx) for c in cases]
    bp = [torch.from_numpy(c.pos).cuda() for c in cases]
    bw = [torch.from_numpy(c.w).cuda() for c in cases]
    bands = [c.b for c in cases]
    ms_b, (ub, rep_b) = _timed_call(lambda: cg.coarse_grain_batched(
        meshes, bp, bw, cg.Params(nsteps=10, precision=cg.PREC_FP32_DF_REFINE),
        bandwidths=bands, report=True), reps=3)
    ub = [u.clone() for u in ub]
    # the persistent launch alone, for comparison
    ms_p, (up_, rep_p) = _timed_call(lambda: cg.coarse_grain_batched(
        meshes, bp, bw, cg.Params(nsteps=10, precision=cg.PREC_FP32_DF_REFINE, sweep_shape=16),
        bandwidths=bands, report=True), reps=2)

    def loop64():
        outs, upd = [], 0
        for m, p_, w_, b in zip(meshes, bp, bw, bands):
            u, r = cg.coarse_grain(m, p_, w_, cg.Params(bandwidth=b, nsteps=10,
                                                         precision=cg.PREC_FP64), report=True)
            outs.append(u)
            upd += r["cell_updates"]
        return outs, upd
    ms_f, (uf, upd_f) = _timed_call(loop64, reps=1)
    prm = [cg.Params(bandwidth=b, nsteps=10, precision=cg.PREC_FP32_DF_REFINE) for b in bands]
    for m, p_, w_, q in zip(meshes, bp, bw, prm):
        cg.coarse_grain(m, p_, w_, q)
    cstreams = [torch.cuda.Stream() for _ in cases]
    ms_c, (uc, reps_c) = _timed_call(lambda: cg.coarse_grain_concurrent(
        meshes, bp, bw, prm, streams=cstreams, max_concurrent=4, report=True))
    sample = (0, 17, 42, 63)
    err_b, err_f = 0.0, 0.0
    kind4 = None
    for s_ in sample:
        ref4, kind4 = oracle_structured(cases[s_], cases[s_].b, 10)
        err_b = max(err_b, maxrel_np(cpu(ub[s_]), ref4))
        err_f = max(err_f, maxrel_np(cpu(uf[s_]), ref4))
    ncell = sum(c.ncells for c in cases)
    res["batched_64"] = {
        "workload": "64 snapshots, cube sides U{32..96} (%d cells), round(10^U(4,6)) particles "
                    "(%d), 5 fields, b=3dx, 10 IE steps" % (ncell, sum(c.n for c in cases)),
        "ms": ms_b, "cell_updates_per_s": rep_b["cell_updates"] / (ms_b * 1e-3),
        "cell_pseudo_steps_per_s": 5 * 10 * ncell / (ms_b * 1e-3),
        **deposit_rate(sum(c.n for c in cases), 5, rep_b),
        "ms_per_phase": {k: rep_b[k] for k in ("ms_locate", "ms_deposit", "ms_diffuse")},
        "schedule": rep_b["sweep_shape_used"],
        "schedule_note": "z planes per work item; 500 + z = one launch per phase, else the "
                         "persistent cooperative launch",
        "persistent_launch": {"ms": ms_p, "schedule": rep_p["sweep_shape_used"],
                              "bit_identical": all(bool(torch.equal(a, b)) for a, b in zip(ub, up_))},
        "maxrel_vs_oracle_sampled": err_b, "fp64_loop_maxrel_vs_oracle_sampled": err_f,
        "oracle_sample": "snapshots %s, every field; %s" % (list(sample), kind4),
        "fp64_cg_loop_ms": ms_f, "fp64_cg_loop_cell_updates_per_s": upd_f / (ms_f * 1e-3),
        "speedup_vs_fp64_gpu_loop": ms_f / ms_b,
        "maxrel_vs_fp64_gpu": max(maxrel(a, b) for a, b in zip(ub, uf)),
        "concurrent_single_mesh_calls": {
            "ms": ms_c, "max_concurrent": 4,
            "cell_updates_per_s": sum(r["cell_updates"] for r in reps_c) / (ms_c * 1e-3),
            "maxrel_vs_fp64_gpu": max(maxrel(a, b) for a, b in zip(uc, uf))}}
    for m in meshes:
        m.close()
    del bp, bw, ub, uf, uc, up_
    # config 5: channel 512x256x256 over 4x2x2, 50,000,000 spheres, b = 4 dx, 40 IE steps
    ch = W.channel()
    mesh = cg.StructuredMesh(ch.dims, ch.origin, ch.dx)
    dp, dw = torch.from_numpy(ch.pos).cuda(), torch.from_numpy(ch.w).cuda()
    out = {}
    for name, prec, reps in (("bf16_dfrefine", cg.PREC_BF16_DF_REFINE, 2),
                             ("fp32_dfrefine", cg.PREC_FP32_DF_REFINE, 2),
                             ("fp64_cg", cg.PREC_FP64, 1)):
        ms, (u, rep) = _timed_call(lambda: cg.coarse_grain(mesh, dp, dw, cg.Params(
            bandwidth=ch.b, nsteps=ch.nsteps, precision=prec), report=True), reps=reps)
        out[name] = (ms, u.clone(), rep)
    # the dominant kernel of the FP32 path where its working set (4 x 134 MB) leaves L2
    cg.profile_reset()
    cg.profile_enable(True)
    cg.coarse_grain(mesh, dp, dw, cg.Params(bandwidth=ch.b, nsteps=ch.nsteps,
                                            precision=cg.PREC_FP32_DF_REFINE))
    cg.profile_enable(False)
    kern5 = cg.profile_read()
    top5 = max(kern5, key=lambda k: kern5[k]["ms"]) if kern5 else ""
    roof5 = kernel_roofline(kern5, peaks, peak_src, traffic_key=top5 + "_channel512")
    ref5, kind5 = oracle_structured(ch, ch.b, ch.nsteps)
    cell5, _ = oracle.locate_structured(ch.dims, ch.origin, ch.dx, ch.pos)
    eps5, _ = oracle.deposit(cell5, ch.w, ch.ncells, vc_uniform=(ch.dx * ch.dx) * ch.dx)
    cf5 = dct_closed_form(eps5[0], ch.dims, ch.dx, ch.b ** 2 / 4, ch.nsteps)
    del cell5, eps5
    # the explicit reading of the same case: 40 explicit Euler steps (dtau/dx^2 = 0.1)
    ex = {}
    for name, prec, k in (("explicit_df", cg.PREC_FP32_DF_REFINE, 0), ("explicit_fp64", cg.PREC_FP64, 0),
                          ("explicit_fp32_k1", 0, 1), ("explicit_fp32_blocked_k2", 0, 2),
                          ("explicit_fp32_blocked_k3", 0, 3), ("explicit_fp32_blocked_k4", 0, 4)):
        ms, (u, rep) = _timed_call(lambda: cg.coarse_grain(mesh, dp, dw, cg.Params(
            bandwidth=ch.b, nsteps=ch.nsteps, scheme=2, precision=prec, fused_k=k), report=True))
        ex[name] = (ms, u.clone(), rep)
    e0 = cg.deposit(mesh, dp, dw)
    fp32_diffusion = {}
    for k in (1, 2, 3, 4):
        u = e0.clone()
        ms, _ = _timed_call(lambda: cg.diffuse(mesh, u, cg.Params(
            bandwidth=ch.b, nsteps=ch.nsteps, scheme=2, fused_k=k)), reps=3)
        fp32_diffusion["k%d" % k] = {
            "ms": ms, "cell_steps_per_s": ch.nsteps * ch.ncells / (ms * 1e-3),
            "algorithmic_GBps": (ch.ncells * 8 * -(-ch.nsteps // k)) / (ms * 1e-3) / 1e9}
    del e0
    res["channel_512x256x256_explicit"] = {
        "workload": "the channel case with 40 explicit Euler steps (dtau/dx^2 = 0.1)",
        "modes": {k: {"ms": v[0], "cell_updates_per_s": v[2]["cell_updates"] / (v[0] * 1e-3),
                      "maxrel_vs_fp64_gpu": maxrel(v[1], ex["explicit_fp64"][1])}
                  for k, v in ex.items()},
        "fp32_diffusion_only": fp32_diffusion,
        "df_vs_fp64_maxrel": maxrel(ex["explicit_df"][1], ex["explicit_fp64"][1]),
        "explicit_vs_implicit_fp64_maxrel": maxrel(ex["explicit_fp64"][1], out["fp64_cg"][1])}
    del ex
    res["channel_512x256x256"] = {
        "workload": "512x256x256 over 4x2x2, 50,000,000 spheres d=0.004, density 1+0.5 sin(2 pi x), "
                    "b=4dx, 40 IE steps",
        "modes": {k: {"ms": v[0], "cell_updates_per_s": v[2]["cell_updates"] / (v[0] * 1e-3),
                      "cell_pseudo_steps_per_s": 40 * ch.ncells / (v[0] * 1e-3),
                      "maxrel_vs_fp64_gpu": maxrel(v[1], out["fp64_cg"][1]),
                      "maxrel_vs_oracle": maxrel_np(cpu(v[1]), ref5),
                      "maxrel_vs_dct_closed_form": maxrel_np(cpu(v[1])[0], cf5),
                      **deposit_rate(ch.n, 1, v[2])}
                  for k, v in out.items()},
        "oracle": kind5 + "; the DCT-II closed form of the discrete system beside it",
        "oracle_vs_closed_form_maxrel": maxrel_np(ref5[0], cf5),
        "roofline_hbm": roof5,
        "kernels_fp32_dfrefine": {k: {"launches": v["launches"], "ms": round(v["ms"], 4),
                                      "GBps": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else None}
                                  for k, v in sorted(kern5.items(), key=lambda kv: -kv[1]["ms"])}}
    mesh.close()
    del out, ref5, cf5
    # the same channel periodic in x (Section 3.1) with the particles' momentum as three
    # more fields, then the solid velocity (diffused momentum / diffused solid fraction)
    dw4 = torch.from_numpy(np.vstack([ch.w, ch.w * W.channel_velocities(ch.pos)])).cuda()
    mesh = cg.StructuredMesh(ch.dims, ch.origin, ch.dx, periodic=(True, False, False))
    per = {}
    for name, prec, reps in (("fp32_dfrefine", cg.PREC_FP32_DF_REFINE, 2), ("fp64_cg", cg.PREC_FP64, 1)):
        ms, (u, rep) = _timed_call(lambda: cg.coarse_grain(mesh, dp, dw4, cg.Params(
            bandwidth=ch.b, nsteps=ch.nsteps, precision=prec), report=True), reps=reps)
        per[name] = (ms, u.clone(), rep)
    um = per["fp32_dfrefine"][1]
    ms_us, us = _timed_call(lambda: cg.solid_velocity(mesh, um[0], um[1:], eps_min=1e-6), reps=3)
    res["channel_periodic_x_solid_velocity"] = {
        "workload": "the channel case periodic in x, 4 fields (V_p and V_p u, u = 1 + 0.5 sin(2 pi x) "
                    "streamwise + N(0, 0.1)), b=4dx, 40 IE steps, then U_s = diffused momentum / "
                    "diffused solid fraction",
        "modes": {k: {"ms": v[0], "cell_updates_per_s": v[2]["cell_updates"] / (v[0] * 1e-3),
                      "maxrel_vs_fp64_gpu": maxrel(v[1], per["fp64_cg"][1]),
                      "sweep_shape_used": v[2]["sweep_shape_used"]} for k, v in per.items()},
        "solid_velocity_ms": ms_us, "solid_velocity_cells_per_s": ch.ncells / (ms_us * 1e-3),
        "solid_velocity_GBps": ch.ncells * (4 + 3) * 8 / (ms_us * 1e-3) / 1e9,
        "mean_streamwise_velocity": float(us[0].mean())}
    mesh.close()
    del dp, dw, dw4, per, um, us
    # Crank-Nicolson (the paper's scheme, Section 5.1) on the 128^3 clustered case, b = 4 dx
    c = W.clustered_cube()
    mesh = cg.StructuredMesh(c.dims, c.origin, c.dx)
    dp, dw = torch.from_numpy(c.pos).cuda(), torch.from_numpy(c.w).cuda()
    cn = {}
    for name, prec in (("fp32_dfrefine", cg.PREC_FP32_DF_REFINE), ("fp64_cg", cg.PREC_FP64)):
        ms, (u, rep) = _timed_call(lambda: cg.coarse_grain(mesh, dp, dw, cg.Params(
            bandwidth=4 * c.dx, nsteps=10, scheme=1, precision=prec), report=True))
        cn[name] = (ms, u.clone(), rep)
    refcn, kindcn = oracle_structured(c, 4 * c.dx, 10, scheme=1)
    res["clustered_128_crank_nicolson"] = {
        "workload": "the 128^3 clustered case, b = 4 dx, 10 Crank-Nicolson steps",
        "modes": {k: {"ms": v[0], "cell_updates_per_s": v[2]["cell_updates"] / (v[0] * 1e-3),
                      "maxrel_vs_fp64_gpu": maxrel(v[1], cn["fp64_cg"][1]),
                      "maxrel_vs_oracle": maxrel_np(cpu(v[1]), refcn)} for k, v in cn.items()},
        "oracle": kindcn}
    mesh.close()
    del dp, dw, cn
    # stretched 128^3 mesh with a cell diffusion constant (0 in one block, 4 in another)
    xf, yf, zf, D, pos, w = W.stretched_box()
    mesh = cg.HexMesh(xf, yf, zf, D)
    dp, dw = torch.from_numpy(pos).cuda(), torch.from_numpy(w).cuda()
    eps0 = cg.deposit(mesh, dp, dw)
    frozen = torch.from_numpy(D == 0.0).cuda()
    hx = {}
    for name, prec in (("fp32_fp64refine", cg.PREC_FP32_REFINE), ("fp64_pcg", cg.PREC_FP64)):
        ms, (u, rep) = _timed_call(lambda: cg.coarse_grain(mesh, dp, dw, cg.Params(
            bandwidth=2.0 / 128, nsteps=10, precision=prec), report=True))
        hx[name] = (ms, u.clone(), rep)
    res["stretched_hex_128"] = {
        "workload": "128^3 stretched mesh (z faces geometric, ratio 1.02), D = 1 with a D = 0 block "
                    "and a D = 4 block, 5,000,000 layered spheres with 4 fields, b = 2/128, 10 IE steps",
        "modes": {k: {"ms": v[0], "cell_updates_per_s": v[2]["cell_updates"] / (v[0] * 1e-3),
                      "maxrel_vs_fp64_gpu": maxrel(v[1], hx["fp64_pcg"][1])} for k, v in hx.items()},
        "frozen_cells_bit_identical_to_pcm": all(
            bool(torch.equal(v[1][:, frozen], eps0[:, frozen])) for v in hx.values())}
    mesh.close()
    return res


# FP64 operations of the FP64 conjugate-gradient path per cell (a fused multiply-add
# counts two): an iteration's first pass forms p = r + beta p (2), the six-neighbour sum
# (5), A p = dg p - ce s (3) and p.Ap (2); its second pass the sum and A p again (8),
# x += alpha p, r -= alpha Ap and r.r (6): 26.  A step's initial residual c L x with
# r.r and b.b: 12.  Bytes per cell and iteration: 24 (pass 1) + 40 (pass 2).
FP64_FLOPS_PER_ITER, FP64_FLOPS_PER_INIT, FP64_BYTES_PER_ITER = 26, 12, 64
FP64_NOMINAL_TFLOPS = 1.25


def measure_fp64_gemm(n=8192, reps=3):
    """FP64 throughput this GPU reaches in cuBLAS's DGEMM (torch float64 matmul, n^3,
    best of reps after a warm-up): a measured FP64 ceiling to set the FP64 path against,
    beside the nominal figure."""
    import torch
    a = torch.rand((n, n), dtype=torch.float64, device="cuda")
    b = torch.rand((n, n), dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = None
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        t = e0.elapsed_time(e1)
        best = t if best is None else min(best, t)
    del a, b
    torch.cuda.empty_cache()
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def fp64_roofline(reps, nf, ms_per_step, steps, peaks, measured_tflops=None):
    """The FP64 path against GB300's FP64 units and against HBM, from the library's
    operation counts (iters includes one initial residual per step and field)."""
    flops = 0.0
    by = 0.0
    for r in reps:
        n = r["cell_updates"] / max(r["iters"], 1)
        inits = NSTEPS * nf
        cg_it = r["iters"] - inits
        flops += n * (FP64_FLOPS_PER_ITER * cg_it + FP64_FLOPS_PER_INIT * inits)
        by += n * (FP64_BYTES_PER_ITER * cg_it + 24 * inits)
    sec = ms_per_step * 1e-3 * steps
    tf = flops / sec / 1e12
    gbs = by / sec / 1e9
    peak = measured_tflops if measured_tflops else FP64_NOMINAL_TFLOPS
    return {"bound": "fp64", "achieved": tf, "peak": peak, "unit": "TFLOP/s",
            "frac": tf / peak,
            "peak_source": ("measured on this GPU: cuBLAS DGEMM 8192^3 through torch float64 matmul"
                            if measured_tflops else "nominal GB300 FP64 (no measured FP64 peak)"),
            "nominal_tflops": FP64_NOMINAL_TFLOPS, "frac_of_nominal": tf / FP64_NOMINAL_TFLOPS,
            "hbm_achieved_gbs": gbs, "hbm_frac": gbs / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None,
            "flops_per_cell_iteration": FP64_FLOPS_PER_ITER, "bytes_per_cell_iteration": FP64_BYTES_PER_ITER}


def cpu_baseline(c, outs, fp64_out):
    """The oracle as it stands, single-threaded on this host: locate + deposit of all
    particles and the full 10-step implicit-Euler diffusion at b/dx = 2, with the
    max-relative error of the GPU results there.  Beside it the oracle's multi-core build
    (OpenMP, every host core) on the same sample, and on the whole step (all four
    bandwidths), whose results give the GPU errors at every bandwidth."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    cell, _ = oracle.locate_structured(c.dims, c.origin, c.dx, c.pos)
    eps0, _ = oracle.deposit(cell, c.w, c.ncells, vc_uniform=(c.dx * c.dx) * c.dx)
    t1 = time.perf_counter()
    b = 2.0 * c.dx
    ref, iters = oracle.diffuse_structured(eps0, c.dims, c.dx, b * b / 4, NSTEPS, tol=TOL)
    dt = time.perf_counter() - t0
    updates = (iters + NSTEPS) * c.ncells
    i = B_OVER_DX.index(2.0)
    mixed = outs[i].cpu().numpy()[0]
    f64 = fp64_out[i].cpu().numpy()[0]
    scale = np.max(np.abs(ref))
    res = {"value": updates / dt, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
           "sample": "locate+deposit all %d particles and 10 implicit-Euler steps at b/dx=2 "
                     "(FP64 CG to 1e-13), %.1f s" % (c.n, dt),
           "particles_per_s": c.n / (t1 - t0),
           "diffusion_cell_updates_per_s": updates / (dt - (t1 - t0)),
           "host": host_cpu(),
           "mixed_maxrel_vs_oracle": float(np.max(np.abs(mixed - ref)) / scale),
           "fp64_maxrel_vs_oracle": float(np.max(np.abs(f64 - ref)) / scale)}
    omp = _omp_oracle()
    if omp is None:
        res["multicore"] = {"unavailable": "the oracle's OpenMP build does not compile here"}
        return res
    # the same sample on every core
    t0 = time.perf_counter()
    cell2, _ = omp.locate_structured(c.dims, c.origin, c.dx, c.pos)
    e2 = omp.deposit(cell2, c.w, c.ncells, vc_uniform=(c.dx * c.dx) * c.dx)
    t1 = time.perf_counter()
    ref2, iters2 = omp.diffuse_structured(e2, c.dims, c.dx, b * b / 4, NSTEPS, tol=TOL)
    dt2 = time.perf_counter() - t0
    upd2 = (iters2 + NSTEPS) * c.ncells
    # the whole step: every bandwidth, 10 steps, CG to 1e-14
    errs = {}
    t2 = time.perf_counter()
    upd_all = 0
    for j, bdx in enumerate(B_OVER_DX):
        bj = bdx * c.dx
        rj, itj = omp.diffuse_structured(e2, c.dims, c.dx, bj * bj / 4, NSTEPS, tol=1e-14)
        upd_all += (itj + NSTEPS) * c.ncells
        errs["b/dx=%g" % bdx] = {"mixed": maxrel_np(outs[j].cpu().numpy(), rj),
                                 "fp64_cg": maxrel_np(fp64_out[j].cpu().numpy(), rj)}
    dt_all = time.perf_counter() - t2 + (t1 - t0)
    res["multicore"] = {
        "value": upd2 / dt2, "unit": "cell-updates/s", "cores": omp.threads(),
        "kind": "oracle, multi-core build (OpenMP, fixed-order chunked dot products)",
        "sample": "the same as the single-thread leg, %.2f s" % dt2,
        "particles_per_s": c.n / (t1 - t0),
        "deposition_bit_identical_to_single_thread": bool(np.array_equal(
            e2.view(np.int64), eps0.view(np.int64))),
        "maxrel_vs_single_thread": maxrel_np(ref2, ref),
        "whole_step": {"seconds": dt_all, "cell_updates_per_s": upd_all / dt_all,
                       "what": "locate+deposit and 10 implicit-Euler steps at each of b/dx = 1, 2, 4, 8"}}
    res["gpu_maxrel_vs_oracle_per_bandwidth"] = errs
    return res


def host_cpu():
    """The host's logical CPU count and model name (/proc/cpuinfo, else lscpu)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.strip().lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return {"nproc": os.cpu_count(), "model": model, "machine": platform.machine()}


# ----------------------------------------------------------------------------- profiling cases
def profile_case(argv=None):
    """One smoothing (or deposition, locate, batched) case on its own, for a profiler
    (ncu) or a quick timing:

        python bench.py profile-case --n 256 --precision 3 --reps 2

    A seeded random field on an n^3 (or --dims) hex mesh of unit-cube spacing is
    smoothed --reps times with the chosen precision mode (include/cg.h), b = --b-over-dx
    cells, --nsteps implicit-Euler steps (with --explicit-k K: --nsteps explicit steps in
    FP32, K steps per launch; with --tet --locate N: the point location of N particles).
    Prints the wall time of each call."""
    ap = argparse.ArgumentParser(prog="bench.py profile-case")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--dims", type=int, nargs=3, default=None)
    ap.add_argument("--precision", type=int, default=3)
    ap.add_argument("--b-over-dx", type=float, default=2.0)
    ap.add_argument("--nsteps", type=int, default=10)
    ap.add_argument("--nfields", type=int, default=1)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--tet", action="store_true", help="Kuhn tet mesh of n^3 hexes instead")
    ap.add_argument("--shape", type=int, default=0, help="sweep_shape (0 = autotuned)")
    ap.add_argument("--explicit-k", type=int, default=0,
                    help="explicit Euler instead: fused_k steps per launch (FP32, temporal "
                         "blocking), --nsteps steps at dtau/dx^2 = 0.1")
    ap.add_argument("--batched", type=int, default=0,
                    help="the first N snapshots of the 64-snapshot batch (cube sides 32..96, "
                         "5 fields, b = 3 dx) through one batched call instead")
    ap.add_argument("--deposit", action="store_true",
                    help="ordered deposition of the clustered n^3 workload (2,000,000 spheres "
                         "at n = 128) instead of a diffusion")
    ap.add_argument("--locate", type=int, default=0,
                    help="with --tet: point location of N particles of the layered workload "
                         "(a dense bottom layer) on the Kuhn tet mesh instead of a diffusion")
    a = ap.parse_args(argv)

    import numpy as np
    import torch

    import paper_1409_0001_gb300 as cg
    from paper_1409_0001_gb300 import build
    import workloads as W

    build.build()
    if a.batched:
        cases = W.batched_snapshots()[:a.batched]
        meshes = [cg.StructuredMesh(c.dims, c.origin, c.dx) for c in cases]
        pos = [torch.from_numpy(c.pos).cuda() for c in cases]
        w = [torch.from_numpy(c.w).cuda() for c in cases]
        for r in range(a.reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, rep = cg.coarse_grain_batched(meshes, pos, w, cg.Params(nsteps=a.nsteps, precision=a.precision,
                                                                       sweep_shape=a.shape),
                                             bandwidths=[c.b for c in cases], report=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            print("rep %d: %.3f ms, %d cell-updates, %.3e cell-updates/s, schedule %d"
                  % (r, dt * 1e3, rep["cell_updates"], rep["cell_updates"] / dt,
                     rep["sweep_shape_used"]))
        return
    if a.deposit:
        c = W.clustered_cube(n_side=a.n, n_particles=2_000_000 * (a.n // 128) ** 3 or 2_000_000)
        mesh = cg.StructuredMesh(c.dims, c.origin, c.dx)
        pos, w = torch.from_numpy(c.pos).cuda(), torch.from_numpy(c.w).cuda()
        for r in range(a.reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, rep = cg.deposit(mesh, pos, w, cg.Params(), report=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            print("rep %d: %.3f ms (locate %.3f, deposit %.3f), %.3e particles/s"
                  % (r, dt * 1e3, rep["ms_locate"], rep["ms_deposit"], c.n / dt))
        mesh.close()
        return
    dims = tuple(a.dims) if a.dims else (a.n, a.n, a.n)
    dx = 1.0 / dims[0]
    if a.tet:
        xyz, tets = W.kuhn_tet_mesh(a.n)
        mesh = cg.TetMesh(xyz, tets)
        if a.locate:
            pos = torch.from_numpy(W.layered_cube(n_particles=a.locate)[0]).cuda()
            for r in range(a.reps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, nout = cg.locate(mesh, pos)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                print("rep %d: %.3f ms, %d outside, %.3e particles/s" % (r, dt * 1e3, nout, a.locate / dt))
            mesh.close()
            return
    else:
        mesh = cg.StructuredMesh(dims, (0.0, 0.0, 0.0), dx)
    rng = np.random.default_rng(0)
    u0 = torch.from_numpy(rng.random((a.nfields, mesh.ncells))).cuda()
    if a.explicit_k:
        p = cg.Params(T=0.1 * dx * dx * a.nsteps, nsteps=a.nsteps, scheme=2, fused_k=a.explicit_k)
    else:
        p = cg.Params(bandwidth=a.b_over_dx * dx, nsteps=a.nsteps, precision=a.precision,
                      sweep_shape=a.shape)
    for r in range(a.reps):
        u = u0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, rep = cg.diffuse(mesh, u, p, report=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        print("rep %d: %.3f ms, %d cell-updates, %.3e cell-updates/s, residual %.2e"
              % (r, dt * 1e3, rep["cell_updates"], rep["cell_updates"] / dt,
                 rep["final_rel_residual"]))
    mesh.close()



if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "profile-case":
        profile_case(sys.argv[2:])
    else:
        main()
