"""Host-side pieces of bench.py (no GPU): the traffic record of the roofline's dominant
kernel matches the kernel's current source (else the benchmark would report no traffic),
the FP64 path's operation accounting, and the host description."""
import hashlib
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def test_traffic_record_matches_current_source():
    b = load_bench()
    with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
        recs = json.load(f)
    assert recs
    for name, rec in recs.items():
        sec = b.source_section(rec["source"], rec["section_start"], rec["section_end"])
        assert len(sec) > 1000, name            # the section is the kernel's code, not a stub
        assert hashlib.sha256(sec.encode()).hexdigest() == rec["section_sha256"], (
            "%s: the kernel changed since its DRAM traffic was captured; re-capture it" % name)
        assert b.ncu_traffic(name) == rec["dram_bytes_per_launch"] > 0
        assert rec["dram_bytes_per_launch"] == rec["dram_bytes_read"] + rec["dram_bytes_write"]
        assert "--clock-control none" in rec["command"]


def test_fp64_roofline_accounting():
    """Two problems of n cells, one field, 10 steps: iters counts one initial residual per
    step plus the CG iterations; FLOPs = 26 per cell and CG iteration + 12 per cell and
    initial residual, bytes 64 and 24."""
    b = load_bench()
    n, cg_it = 1000, 37
    reps = [{"iters": cg_it + b.NSTEPS, "cell_updates": (cg_it + b.NSTEPS) * n}] * 2
    r = b.fp64_roofline(reps, 1, ms_per_step=2.0, steps=3, peaks={"hbm_gbs": 1000.0})
    flops = 2 * n * (26 * cg_it + 12 * b.NSTEPS)
    by = 2 * n * (64 * cg_it + 24 * b.NSTEPS)
    sec = 2.0e-3 * 3
    assert abs(r["achieved"] - flops / sec / 1e12) <= 1e-12 * r["achieved"]
    assert abs(r["hbm_achieved_gbs"] - by / sec / 1e9) <= 1e-12 * r["hbm_achieved_gbs"]
    assert r["frac"] == r["achieved"] / b.FP64_NOMINAL_TFLOPS
    assert r["hbm_frac"] == r["hbm_achieved_gbs"] / 1000.0


def test_host_cpu_description():
    b = load_bench()
    h = b.host_cpu()
    assert h["nproc"] == os.cpu_count() and h["nproc"] >= 1
    assert isinstance(h["machine"], str) and h["machine"]


def test_kernel_roofline_takes_the_dominant_kernel_and_its_capture():
    """The roofline is the kernel with the most event time; achieved = its algorithmic bytes
    / its time; traffic (and, for a capture of one launch of a mixed group, that launch's
    algorithmic bytes) comes from the committed record named by the traffic key."""
    b = load_bench()
    kern = {"cheb2_fp32": {"ms": 50.0, "bytes": 4.0e11, "launches": 400},
            "refine_df": {"ms": 10.0, "bytes": 5.0e10, "launches": 41}}
    peaks = {"hbm_gbs": 8000.0}
    r = b.kernel_roofline(kern, peaks, "measured", traffic_key="cheb2_fp32_channel512")
    assert r["kernel"] == "cheb2_fp32"
    assert abs(r["achieved"] - 4.0e11 / 50e-3 / 1e9) <= 1e-9 * r["achieved"]
    assert r["frac"] == r["achieved"] / 8000.0
    assert r["algorithmic_bytes_per_launch"] == 1.0e9
    assert abs(r["share_of_kernel_time"] - 50.0 / 60.0) <= 1e-15
    rec = b.ncu_record("cheb2_fp32_channel512")
    assert rec is not None
    assert r["traffic"] == rec["dram_bytes_per_launch"]
    assert r["traffic_launch_algorithmic_bytes"] == rec["algorithmic_bytes_of_captured_launch"]
    # no record under the key: no traffic, and no captured-launch bytes
    r2 = b.kernel_roofline(kern, peaks, "measured", traffic_key="no_such_capture")
    assert r2["traffic"] is None and "traffic_launch_algorithmic_bytes" not in r2
    assert b.kernel_roofline({}, peaks, "measured") is None
