"""Host-side helpers of bench.py: the algorithmic byte counts of the
roofline, and the DRAM traffic read from a committed profile summary, which
must be dropped as soon as a profiled source file changes."""
import os

import numpy as np

import bench
import mqo_inputs as mi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_algorithmic_bytes_formula():
    G = mi.pack([mi.erdos_renyi(50, 0.2, 1), mi.erdos_renyi(40, 0.1, 2)])
    B = 32
    got = bench.algorithmic_bytes_per_step(G, B, 2, 2)
    # CSR once (int32 col + row_ptr), x and V read + written, one rounding word per node
    want = G.nnz * 4 + (G.n + 1) * 4 + 2 * G.n * B * 2 + 2 * G.n * B * 2 + G.n * 4
    assert got == want
    assert bench.fb_kernel_bytes(G, 64, True) - bench.fb_kernel_bytes(G, 64, False) == G.n * 64 * 4


def test_profile_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    srcs = ("mqo_step.cu", "mqo_step.cuh", "mqo_dev.cuh")
    h = bench.source_hash(srcs)
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "x.txt").write_text(f"source_sha256: {h}\ndram_bytes_per_launch[smem]: 1.5e8\n")
    (prof / "y.txt").write_text(f"source_sha256: {'0' * 64}\ndram_bytes_per_launch[smem]: 1.5e8\n")
    # read the summaries from the temporary folder, the sources from the repository
    real_join = os.path.join

    def join(*parts):
        if len(parts) >= 2 and parts[0] == bench.ROOT and parts[1] == "profiles":
            return real_join(str(prof), *parts[2:])
        return real_join(*parts)
    monkeypatch.setattr(bench.os.path, "join", join)
    assert bench.profile_traffic("x", "smem", srcs) == 1.5e8
    assert bench.profile_traffic("y", "smem", srcs) is None      # the kernel changed since the capture
    assert bench.profile_traffic("x", "global", srcs) is None    # no figure for that variant
    assert bench.profile_traffic("missing", "smem", srcs) is None


def test_code_text_ignores_comments_and_blanks_only():
    a = 'int f(int x) {  // one\n  return x + 1; /* two */ }\nconst char* s = "// kept";\n'
    b = 'int f(int x) { return x + 1; }\nconst char* s = "// kept";'
    assert bench.code_text(a) == bench.code_text(b)
    assert bench.code_text(a) != bench.code_text(a.replace("x + 1", "x + 2"))
    assert '"// kept"' in bench.code_text(a)


def test_committed_profiles_carry_traffic_for_the_current_sources():
    """The summaries under profiles/ were captured from the current kernel
    sources (their recorded hash matches), so the bench reports their DRAM
    traffic."""
    assert bench.step_kernel_traffic("mis_batched", "bf16", "smem_wide_ell") is not None
    assert bench.step_kernel_traffic("maxcut_regular", "bf16", "global") is not None
    assert bench.step_kernel_traffic("maxcut_regular", "bf16", "staged") is not None
    assert bench.profile_traffic("fb_kernel_autograd_powerlaw_f32", "fb_seg", ("mqo_grad.cu", "mqo_dev.cuh")) \
        is not None


def test_reference_sample_is_the_oracle_on_a_bounded_sample():
    G = mi.pack([mi.erdos_renyi(60, 0.15, k) for k in range(3)])
    wl = dict(bench.WORKLOADS["mis_batched"], batch=4)
    try:
        r = bench.oracle_sample(G, wl, 1, 1, target_s=0.2, cores=2)
    finally:  # no pool threads left behind for later tests that fork
        for p in bench._POOLS.values():
            p.terminate()
            p.join()
        bench._POOLS.clear()
    assert r["kind"] == "oracle" and r["cores"] == 2 and r["value"] > 0 and r["single_core_value"] > 0
    assert np.isfinite(r["value"])


def test_step_roofline_takes_the_measured_shared_memory_peak():
    """The shared-memory roofline divides by the probe's measured bandwidth
    when the bench has one (and says so), else by the derived 128 B/clk/SM
    figure; the ELL plans name their own profile variant."""
    G = mi.pack([mi.erdos_renyi(60, 0.2, k) for k in range(2)])
    plan = {"step_kernel": "smem_wide", "ell": True, "col16": False}
    assert bench.step_variant(plan) == "smem_wide_ell"
    assert bench.step_variant({"step_kernel": "smem", "ell": False}) == "smem"
    assert bench.step_variant({"step_kernel": "staged", "ell": True}) == "staged"
    clocks = {"sm_mhz": 2000.0}
    derived = 128.0 * 152 * 2000.0 * 1e6 / 1e9
    r0 = bench.step_roofline(G, 32, 2, 2, 0.1, plan, "none", "bf16", 6000.0, "measured", clocks, 152, {})
    assert r0["peak"] == derived and r0["peak_source"] == "derived"
    r1 = bench.step_roofline(G, 32, 2, 2, 0.1, plan, "none", "bf16", 6000.0, "measured", clocks, 152,
                             {"smem_probe_gbs": 39000.0})
    assert r1["peak"] == 39000.0 and r1["peak_source"].startswith("measured") and r1["peak_derived"] == derived
    assert abs(r1["frac"] * 39000.0 - r0["frac"] * derived) < 1e-6 * derived
    # ELL index bytes: 4 per entry in the algorithmic HBM bytes
    assert r1["hbm"]["algorithmic_bytes_per_launch"] == bench.algorithmic_bytes_per_step(G, 32, 2, 2, 4)
