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


def ncu_traffic(kernel_entry):
    """DRAM bytes per launch of a kernel from the committed ncu capture, or None when the
    kernel's source section changed since the counters were taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
            rec = json.load(f).get(kernel_entry)
        if not rec:
            return None
        sec = source_section(rec["source"], rec["section_start"], rec["section_end"])
        sha = hashlib.sha256(sec.encode()).hexdigest()
        return rec["dram_bytes_per_launch"] if sha == rec["section_sha256"] else None
    except (OSError, ValueError, KeyError):
        return None


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
    """The oracle (plain FP64 C, single thread) as the reference arm: each step is a
    bounded sample of the workload -- the full deposition of every particle and the
    first 2 of the 10 implicit-Euler pseudo-steps at b/dx = 2 (same dtau)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    import workloads as W
    oracle.build()
    c = W.clustered_cube(n_side=a.n_side, n_particles=a.n_particles)
    b = 2.0 * c.dx
    T_full = b * b / 4.0
    k_sample = 2

    def step():
        cell, _ = oracle.locate_structured(c.dims, c.origin, c.dx, c.pos)
        eps0, _ = oracle.deposit(cell, c.w, c.ncells, vc_uniform=(c.dx * c.dx) * c.dx)
        _, iters = oracle.diffuse_structured(eps0, c.dims, c.dx, T_full * k_sample / NSTEPS,
                                             k_sample, tol=TOL)
        return iters

    for _ in range(a.warmup):
        step()
    t0 = time.perf_counter()
    total_updates = 0
    for _ in range(a.steps):
        iters = step()
        total_updates += (iters + k_sample) * c.ncells   # CG iterations + one residual per step
    dt = time.perf_counter() - t0
    v = total_updates / dt
    line = {"impl": "reference", "metric": "diffusion cell-updates/s", "value": v,
            "unit": "cell-updates/s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": dt * 1e3 / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a)},
            "cpu_baseline": {"value": v, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
                             "sample": "per step: locate+deposit all %d particles, 2 of 10 "
                                       "implicit-Euler steps at b/dx=2, FP64 CG to 1e-13"
                                       % a.n_particles, "host": host_cpu()},
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
    modes["fp64_cg"]["roofline"] = fp64_roofline(fp64_reps, outs[0].shape[0], modes["fp64_cg"]["ms_per_step"],
                                                 max(a.fp64_steps, 1), measured_peaks()[0])
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
                "share_of_kernel_time": k["ms"] / sum(v["ms"] for v in kern.values())}

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
                                       "(cg_coarse_grain_concurrent)" % a.concurrency
                                       if a.concurrency > 1 else "one bandwidth after another"),
                       "parallelism": "replicas" if ws > 1 else "single"},
            "e2e": {"value": e2e_updates / e2e_s, "unit": "cell-updates/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "entry_point": "cg_coarse_grain_host per bandwidth (pinned host buffers, copies "
                                   "inside), %s" % ("%d at a time through cg_coarse_grain_concurrent, "
                                                    "which copies the particle arrays the four share "
                                                    "in once per step" % a.concurrency
                                                    if a.concurrency > 1 else "one after another"),
                    "result_identical_to_device_run": e2e_ok},
            "gpu_launches": launches,
            "gpu_launches_before_timed": launches_before,
            "sweep_shape_used": sorted({r["sweep_shape_used"] for r in reps}),
            "clocks": clocks,
            "roofline": roof,
            "cpu_baseline": cpu,
            "cell_pseudo_steps_per_s": cps,
            "particles_per_s": ws * a.steps * len(B_OVER_DX) * c.n / (ms * 1e-3),
            "ms_per_phase_per_step": ms_phase,
            "refine_rounds_per_solve": rounds,
            "worst_rel_residual": worst_res,
            "worst_rel_mass_error": mass_err,
            "modes": modes,
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


def _timed_call(fn, reps=2, warm=1):
    """Device time (CUDA events on the current stream) of fn(), best of reps."""
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(warm):
        fn()
    best = None
    out = None
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        t = e0.elapsed_time(e1)
        best = t if best is None else min(best, t)
    return best, out


def extras():
    """The other workloads of the method, each measured the same way (whole method per
    call, CUDA events, best of 2 after a warm-up call), mixed vs FP64 GPU."""
    import torch
    import paper_1409_0001_gb300 as cg
    import workloads as W

    def maxrel(a, b):
        return float((a - b).abs().max() / b.abs().max())

    res = {}
    # unstructured: 100^3 hexes -> 6,000,000 jittered Kuhn tets, 5,000,000 layered spheres
    xyz, tets = W.kuhn_tet_mesh(100)
    mesh = cg.TetMesh(xyz, tets)
    pos, w, _ = W.layered_cube()
    dp, dw = torch.from_numpy(pos).cuda(), torch.from_numpy(w).cuda()
    out = {}
    for name, prec in (("fp32_fp64refine", cg.PREC_FP32_REFINE), ("fp64_pcg", cg.PREC_FP64)):
        ms, (u, rep) = _timed_call(lambda: cg.coarse_grain(mesh, dp, dw, cg.Params(
            bandwidth=0.03, nsteps=10, precision=prec), report=True))
        out[name] = (ms, u.clone(), rep)
    res["tet_layered_6M"] = {
        "workload": "100^3 hexes -> 6,000,000 jittered Kuhn tets (two-point-flux FV), 5,000,000 "
                    "spheres d=0.003 with a dense bottom layer, b=0.03, 10 IE steps",
        "modes": {k: {"ms": v[0], "cell_updates_per_s": v[2]["cell_updates"] / (v[0] * 1e-3),
                      "cell_pseudo_steps_per_s": 10 * 6e6 / (v[0] * 1e-3)} for k, v in out.items()},
        "particles_per_s": 5e6 / (out["fp32_fp64refine"][0] * 1e-3),
        "ms_per_phase": {k: out["fp32_fp64refine"][2][k] for k in ("ms_locate", "ms_deposit", "ms_diffuse")},
        "mixed_speedup_vs_fp64_gpu": out["fp64_pcg"][0] / out["fp32_fp64refine"][0],
        "mixed_vs_fp64_maxrel": maxrel(out["fp32_fp64refine"][1], out["fp64_pcg"][1])}
    mesh.close()
    del dp, dw
    # batched: 64 snapshots, 32^3..96^3, 10^4..10^6 particles, 5 fields, one persistent launch
    cases = W.batched_snapshots()
    meshes = [cg.StructuredMesh(c.dims, c.origin, c.dx) for c in cases]
    bp = [torch.from_numpy(c.pos).cuda() for c in cases]
    bw = [torch.from_numpy(c.w).cuda() for c in cases]
    bands = [c.b for c in cases]
    ms_b, (ub, rep_b) = _timed_call(lambda: cg.coarse_grain_batched(
        meshes, bp, bw, cg.Params(nsteps=10, precision=cg.PREC_FP32_DF_REFINE),
        bandwidths=bands, report=True))
    ub = [u.clone() for u in ub]

    def loop64():
        outs, upd = [], 0
        for m, p_, w_, b in zip(meshes, bp, bw, bands):
            u, r = cg.coarse_grain(m, p_, w_, cg.Params(bandwidth=b, nsteps=10,
                                                         precision=cg.PREC_FP64), report=True)
            outs.append(u)
            upd += r["cell_updates"]
        return outs, upd
    ms_f, (uf, upd_f) = _timed_call(loop64, reps=1)
    # the same snapshots as independent single-mesh calls, four at a time (each mesh
    # autotuned first by one call on its own)
    prm = [cg.Params(bandwidth=b, nsteps=10, precision=cg.PREC_FP32_DF_REFINE) for b in bands]
    for m, p_, w_, q in zip(meshes, bp, bw, prm):
        cg.coarse_grain(m, p_, w_, q)
    cstreams = [torch.cuda.Stream() for _ in cases]
    ms_c, (uc, reps_c) = _timed_call(lambda: cg.coarse_grain_concurrent(
        meshes, bp, bw, prm, streams=cstreams, max_concurrent=4, report=True))
    ncell = sum(c.ncells for c in cases)
    res["batched_64"] = {
        "workload": "64 snapshots, cube sides U{32..96} (%d cells), round(10^U(4,6)) particles "
                    "(%d), 5 fields, b=3dx, 10 IE steps" % (ncell, sum(c.n for c in cases)),
        "ms": ms_b, "cell_updates_per_s": rep_b["cell_updates"] / (ms_b * 1e-3),
        "cell_pseudo_steps_per_s": 5 * 10 * ncell / (ms_b * 1e-3),
        "particles_per_s": sum(c.n for c in cases) / (ms_b * 1e-3),
        "ms_per_phase": {k: rep_b[k] for k in ("ms_locate", "ms_deposit", "ms_diffuse")},
        "z_planes_per_item": rep_b["sweep_shape_used"],
        "fp64_cg_loop_ms": ms_f, "fp64_cg_loop_cell_updates_per_s": upd_f / (ms_f * 1e-3),
        "speedup_vs_fp64_gpu_loop": ms_f / ms_b,
        "maxrel_vs_fp64_gpu": max(maxrel(a, b) for a, b in zip(ub, uf)),
        "concurrent_single_mesh_calls": {
            "ms": ms_c, "max_concurrent": 4,
            "cell_updates_per_s": sum(r["cell_updates"] for r in reps_c) / (ms_c * 1e-3),
            "maxrel_vs_fp64_gpu": max(maxrel(a, b) for a, b in zip(uc, uf))}}
    for m in meshes:
        m.close()
    del bp, bw, ub, uf, uc
    # channel: 512x256x256 over 4x2x2, 50,000,000 spheres, b = 4 dx, 40 IE steps
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
    # the explicit reading of the same case: 40 explicit Euler steps (dtau/dx^2 = 0.1)
    ex = {}
    for name, prec, k in (("explicit_df", cg.PREC_FP32_DF_REFINE, 0), ("explicit_fp64", cg.PREC_FP64, 0),
                          ("explicit_fp32_k1", 0, 1), ("explicit_fp32_blocked_k2", 0, 2),
                          ("explicit_fp32_blocked_k3", 0, 3), ("explicit_fp32_blocked_k4", 0, 4)):
        ms, (u, rep) = _timed_call(lambda: cg.coarse_grain(mesh, dp, dw, cg.Params(
            bandwidth=ch.b, nsteps=ch.nsteps, scheme=2, precision=prec, fused_k=k), report=True))
        ex[name] = (ms, u.clone(), rep)
    # the diffusion phase alone for the FP32 modes: cell-steps per second and the
    # algorithmic bytes of one launch (read and write one FP32 value per cell) per time
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
                      "maxrel_vs_fp64_gpu": maxrel(v[1], out["fp64_cg"][1])}
                  for k, v in out.items()},
        "particles_per_s": ch.n / (out["bf16_dfrefine"][0] * 1e-3)}
    mesh.close()
    del out
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
    res["clustered_128_crank_nicolson"] = {
        "workload": "the 128^3 clustered case, b = 4 dx, 10 Crank-Nicolson steps",
        "modes": {k: {"ms": v[0], "cell_updates_per_s": v[2]["cell_updates"] / (v[0] * 1e-3),
                      "maxrel_vs_fp64_gpu": maxrel(v[1], cn["fp64_cg"][1])} for k, v in cn.items()}}
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


def fp64_roofline(reps, nf, ms_per_step, steps, peaks):
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
    return {"bound": "fp64", "achieved": tf, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
            "frac": tf / FP64_NOMINAL_TFLOPS, "peak_source": "nominal GB300 FP64 (no measured FP64 peak)",
            "hbm_achieved_gbs": gbs, "hbm_frac": gbs / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None,
            "flops_per_cell_iteration": FP64_FLOPS_PER_ITER, "bytes_per_cell_iteration": FP64_BYTES_PER_ITER}


def cpu_baseline(c, outs, fp64_out):
    """The oracle as it stands, single-threaded on this host: locate + deposit of all
    particles and the full 10-step implicit-Euler diffusion at b/dx = 2.  Also gives
    the max-relative error of the GPU results for that bandwidth."""
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
    return {"value": updates / dt, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
            "sample": "locate+deposit all %d particles and 10 implicit-Euler steps at b/dx=2 "
                      "(FP64 CG to 1e-13), %.1f s" % (c.n, dt),
            "particles_per_s": c.n / (t1 - t0),
            "diffusion_cell_updates_per_s": updates / (dt - (t1 - t0)),
            "host": host_cpu(),
            "mixed_maxrel_vs_oracle": float(np.max(np.abs(mixed - ref)) / scale),
            "fp64_maxrel_vs_oracle": float(np.max(np.abs(f64 - ref)) / scale)}


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
