"""CPU checks of bench.py's own arithmetic: the algorithmic FLOP counts the
roofline divides by, and the rule that a DRAM-traffic record only counts for
the kernel sources it was taken of."""
import json
import os
import re
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    sys.path.insert(0, ROOT)
    saved = sys.argv
    sys.argv = ["bench.py"]
    import bench as b
    sys.argv = saved
    return b


def _macs(H, layer_sizes, valid_layers, pixels):
    """Multiply-accumulates counted layer by layer from (out, in) shapes."""
    per_layer = sum(o * i for o, i in layer_sizes["layer"])
    per_pixel = sum(o * i for o, i in layer_sizes["pixel"])
    return per_layer * valid_layers + per_pixel * pixels


@pytest.mark.parametrize("H,pooling,pe,rk", [(128, "max_mean", 0, 1), (128, "sum", 0, 1), (64, "max_mean", 4, 1),
                                             (128, "max_mean", 0, 3), (64, "sum", 2, 3)])
def test_algorithmic_flops_match_the_folded_layer_shapes(bench, H, pooling, pe, rk):
    """2 x the MACs of the folded network (the latent enters as per-scene
    biases), phi on the valid layers only, rho only for [max ; mean], R1 with
    k^2 H inputs for a k x k kernel, R2 with 3 outputs."""
    e = 1 + 2 * pe
    sizes = {"layer": [(H, 12 * e), (H, H)],
             "pixel": ([] if pooling == "sum" else [(H, 2 * H)]) + [(H, 14 * e + H), (H, H), (H, rk * rk * H), (3, H)]}
    counts = np.random.default_rng(0).integers(0, 9, size=(7, 5)).astype(np.uint8)
    want = 2.0 * _macs(H, sizes, int(counts.sum()), counts.size)
    assert bench.algorithmic_flops(H, counts, pooling, pe, rk) == want


def test_headline_flops_per_frame(bench):
    """The benchmark frame's 72.2 GFLOP (doubled widths, Poisson(3) counts)."""
    from gen import synth
    f = synth.make_frame(512, 512, 8, counts="poisson3", seed=0)
    g = bench.algorithmic_flops(128, f.counts) / 1e9
    assert 71.5 < g < 73.0, g


def test_traffic_record_only_counts_for_its_kernel_sources(bench, tmp_path):
    rec = {"kernel_sha256": bench.kernel_digest(), "dram_bytes_per_launch": 123}
    p = tmp_path / "t.json"
    p.write_text(json.dumps(rec))
    assert bench.profiled_traffic(str(p)) == 123
    rec["kernel_sha256"] = "0" * 64
    p.write_text(json.dumps(rec))
    assert bench.profiled_traffic(str(p)) is None
    assert bench.profiled_traffic(str(tmp_path / "absent.json")) is None


def test_committed_traffic_records_name_their_command_and_workload(bench):
    for name in ("fused_bf16_512x512_K8", "fused_bf16_sum_512x512_K8", "fused_bf16_pe4_512x512_K8",
                 "fused_bf16_h64_512x512_K8", "fused_compact_h64_512x512_K8",
                 "fused_bf16_pe4_h128_512x512_K8"):
        with open(os.path.join(ROOT, "profiles", name + ".traffic.json")) as f:
            rec = json.load(f)
        assert rec["dram_bytes_per_launch"] == rec["dram_bytes_read"] + rec["dram_bytes_write"]
        assert rec["command"].startswith("ncu ") and "--clock-control none" in rec["command"]
        assert "bench.py" in rec["command"] and rec["workload"].startswith("512x512")


def test_each_leg_takes_the_capture_of_its_own_kernel(bench):
    """(fp8, r_kernel, pe, base widths, sum pooling) -> the record taken of
    that fused kernel, or none."""
    assert bench.traffic_record(False, 1, 0, False, False) == bench.PROFILE_TRAFFIC
    assert bench.traffic_record(False, 1, 0, False, True) == bench.PROFILE_TRAFFIC_SUM
    assert bench.traffic_record(False, 1, 0, True, False) == bench.PROFILE_TRAFFIC_H64
    assert bench.traffic_record(False, 1, 4, True, False) == bench.PROFILE_TRAFFIC_PE
    assert bench.traffic_record(False, 1, 4, False, False) == bench.PROFILE_TRAFFIC_PE128
    for args in [(True, 1, 0, False, False), (False, 3, 0, False, False), (False, 1, 2, True, False),
                 (False, 1, 4, True, True), (False, 1, 0, True, True), (False, 1, 4, False, True),
                 (False, 1, 2, False, False)]:
        assert bench.traffic_record(*args) is None, args


@pytest.mark.parametrize("root,attr", [("fused_bf16.cu", "KERNEL_SOURCES"),
                                       ("fused_compact.cu", "COMPACT_SOURCES")])
def test_kernel_digest_covers_every_source_of_the_captured_kernels(bench, root, attr):
    """The traffic records are keyed by a hash of the fused kernel's and the
    plan kernel's sources: every repository file they include, transitively,
    is hashed, except the public C header (declarations and enum values the
    kernels never branch on at compile time)."""
    csrc = os.path.join(ROOT, "paper_2405_19056_gb300", "csrc")
    seen, todo = set(), [root, "plan.cu"]
    while todo:
        name = todo.pop()
        if name in seen:
            continue
        seen.add(name)
        with open(os.path.join(csrc, name)) as f:
            for inc in re.findall(r'^#include "([^"]+)"', f.read(), flags=re.M):
                if not inc.endswith("include/glassnet.h"):
                    todo.append(inc)
    assert seen == set(getattr(bench, attr))


def test_layer_rows_of_both_schedules(bench):
    """Executed / valid (pixel, layer) rows.  Every pixel with K layers: both
    schedules run exactly the valid rows.  One pixel with 8 layers in a
    512-pixel window of empty pixels: the sorted tile runs 8 slots of 128
    rows, the compacted block one 128-row tile."""
    full = np.full((16, 64), 5, dtype=np.uint8)
    assert bench.layer_rows(full, "sorted") == (5 * 1024, 5 * 1024)
    assert bench.layer_rows(full, "compact") == (5 * 1024, 5 * 1024)
    one = np.zeros((8, 64), dtype=np.uint8)
    one[3, 7] = 8
    assert bench.layer_rows(one, "sorted") == (8 * 128, 8)
    assert bench.layer_rows(one, "compact") == (128, 8)
    # a ragged frame: 300 pixels of count 1 -> blocks of 256 and 44 pixels
    rag = np.ones((1, 300), dtype=np.uint8)
    assert bench.layer_rows(rag, "compact") == (128 * 2 + 128, 300)
    assert bench.layer_rows(rag, "sorted") == (128 * 3, 300)


def test_serving_stream_follows_the_stated_workload(bench):
    """The serving stream: Poisson arrivals at the given rate, sizes 256 /
    512 / 1024 squared w.p. 0.5 / 0.35 / 0.15, K in 1..8, 32 scenes; the
    same seed gives the same stream."""
    res, Ks, arrive, scenes = bench.serving_stream(800, 20000, seed=0)
    res2, _, arrive2, _ = bench.serving_stream(800, 20000, seed=0)
    assert np.array_equal(res, res2) and np.array_equal(arrive, arrive2)
    frac = [np.mean(res == r) for r in (256, 512, 1024)]
    assert np.allclose(frac, (0.5, 0.35, 0.15), atol=0.015)
    assert Ks.min() == 1 and Ks.max() == 8
    assert scenes.min() == 0 and scenes.max() == 31
    gaps = np.diff(np.concatenate([[0.0], arrive]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 1.0 / 800) < 0.03 / 800  # mean inter-arrival 1/rate
    assert abs(np.std(gaps) / gaps.mean() - 1.0) < 0.05  # exponential: CV = 1


def test_selected_legs(bench):
    class A:
        legs, no_extras = None, False
    a = A()
    assert bench.selected_legs(a) == set(bench.EXTRA_LEGS)
    a.no_extras = True
    assert bench.selected_legs(a) == set()
    a.legs = "streaming, fp8"
    assert bench.selected_legs(a) == {"streaming", "fp8"}
    a.legs = "nope"
    with pytest.raises(SystemExit):
        bench.selected_legs(a)


def test_clock_summary_uses_timed_samples_and_names_reasons(bench):
    """Samples inside the timed region are used when there are at least 3;
    otherwise the same-load samples right after it are added and said so;
    throttle reasons come from the NVML bit mask."""
    c = bench.ClockSampler(0)
    c.source = "test"
    c.t_begin, c.t_end = 10.0, 11.0
    c.samples = [(10.1, 2070.0, 2070.0, 0), (10.5, 2050.0, 2070.0, 0x4), (10.9, 2060.0, 2070.0, 0),
                 (11.5, 1000.0, 2070.0, 0x40)]
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2060.0 and s["reasons"] == ["sw_power_cap"]
    c.samples = [(10.5, 2070.0, 2070.0, 0), (11.2, 1900.0, 2070.0, 0x8), (11.3, 1950.0, 2070.0, 0)]
    c._t_ext = (11.0, 12.0)
    s = c.summary()
    assert s["samples"] == 3 and s["samples_in_timed_region"] == 1
    assert s["reasons"] == ["hw_slowdown"] and "note" in s
    c.samples = []
    s = c.summary()
    assert s["sm_mhz"] is None and s["why"]
