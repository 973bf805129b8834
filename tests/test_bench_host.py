"""Host logic of bench.py checked without a GPU: the headline workload's sizes, and the
algorithmic-byte model and launch count of the one-RHS section (sizes from the host-only
plan, the same set-up code as the GPU handle) against the committed ncu summaries that its
roofline line reads."""
import os
import re
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _plan_info(name):
    import bench
    from paper_2210_04892_gb300 import bi
    try:
        bi.load()
    except (ImportError, OSError) as e:  # pragma: no cover - library not built here
        pytest.skip(f"library not loadable: {e}")
    v, t, _ = bench.workload_mesh(name)
    p = bi.Plan(v, t, bench.K0, digits=3)
    info = p.info()
    p.close()
    return bench, info


@pytest.fixture(scope="module")
def bench_info():
    import bench
    return _plan_info(bench.SECONDARY["name"])


@pytest.mark.slow
def test_headline_workload_sizes():
    import bench
    bench, info = _plan_info(bench.HEADLINE["name"])
    assert info["n_unknowns"] == 3484860 and info["levels"] == 9
    assert str(info["n_unknowns"]) in bench.WORKLOAD.replace(",", "")
    assert bench.HEADLINE["nrhs"] == 8


def test_secondary_workload_sizes(bench_info):
    bench, info = bench_info
    assert info["n_unknowns"] == 61440 and info["levels"] == 5
    assert str(info["n_unknowns"]) in bench.SECONDARY["desc"].replace(",", "")


def test_stage_roofline_picks_the_slower_bound(bench_info):
    """A stage is ALU-bound when its flops at the FP32 peak take longer than its bytes at the
    HBM peak; the fraction is that ideal time over the measured one."""
    bench, info = bench_info
    sb, sf = bench.stage_bytes(info, 64), bench.stage_flops(info, 64)
    stages = {k: 1.0 for k in sb}
    sr = bench.stage_roofline(info, 64, stages, 6000.0)
    for k in sb:
        t_hbm = sb[k] / 6e12
        t_alu = sf[k] / (bench.ALU_FP32_TFLOPS * 1e12)
        assert sr[k]["bound"] == ("alu" if t_alu > t_hbm else "hbm")
        assert abs(sr[k]["frac"] - max(t_hbm, t_alu) / 1e-3) < 1e-12
    # one right-hand side: the near product is bandwidth-bound (2 flop/B), 64 make it ALU-bound
    assert bench.stage_roofline(info, 1, stages, 6000.0)["near"]["bound"] == "hbm"
    assert sr["near"]["bound"] == "alu"


def test_fused_gather_and_scatter_fold_into_their_stages(bench_info):
    """When the gather of x and the scatter of y time as empty (fused into the near and the
    receive kernels), their bytes count in those stages and they get no fraction of their own."""
    bench, info = bench_info
    sb = bench.stage_bytes(info, 8)
    stages = {k: 1.0 for k in sb}
    stages["gather"] = stages["scatter"] = 0.0
    sr = bench.stage_roofline(info, 8, stages, 6000.0)
    assert "gather" not in sr and "scatter" not in sr
    assert sr["near"]["bytes"] == sb["near"] + sb["gather"]
    assert sr["receive"]["bytes"] == sb["receive"] + info["n_unknowns"] * 8 * 8


def test_measured_traffic_matches_the_byte_model(bench_info):
    """Every HBM-bound kernel of the roofline has a committed per-launch DRAM figure that fits
    the algorithmic bytes of its stage: at most 5% above (the kernels re-read nothing), and
    below only by the leaf outgoing/incoming patterns, which may stay in L2 between
    kernels.  That also ties the summary to this workload."""
    bench, info = bench_info
    traffic = bench.measured_traffic()
    model = bench.stage_bytes(info, 1)
    lf = info["leaf_level"]
    leaf_patterns = info["boxes"][lf] * info["K"][lf] * 2 * 8
    assert set(traffic) == {"near", "receive", "aggregate"}
    for stage, (kernel, nbytes) in traffic.items():
        assert kernel.startswith("k_")
        assert model[stage] - leaf_patterns - 0.01 * model[stage] <= nbytes <= 1.05 * model[stage], \
            (stage, nbytes, model[stage])


def test_launch_count_matches_the_launch_summary(bench_info):
    """Kernels per single-RHS product on the 5-level tree: near, aggregation, one translation
    per level 2..4, interpolation and anterpolation per level pair, receive."""
    bench, info = bench_info
    n = bench.launches_per_step(info)
    assert n == 1 + 1 + 3 + 2 + 2 + 1
    text = open(os.path.join(ROOT, "profiles", "launches_matvec_sphere_r2_61440.md")).read()
    assert re.search(r"\(%d product kernels each" % n, text)
    rows = re.findall(r"^\| (k_\w+)<[^|]*\| (\d+) \| [\d.]+ \| [\d.]+ \| [\d.]+% \|$", text, re.M)
    launches = sum(int(c) for _, c in rows)
    products = max(int(c) for _, c in rows if _ == "k_near_stream")
    assert abs(launches / products - n) < 0.1 * n


@pytest.mark.slow
def test_headline_launch_count_matches_the_launch_summary():
    """Kernels per product of the headline workload (9 levels, 8 RHS): the gather of x, near,
    aggregation, 7 translations, 6 interpolation and 6 anterpolation steps, receive (23), plus
    one more launch for each level pass tuned to a two-pass form.  The committed launch list of
    one product holds 27 launches, of which the two-pass forms are the theta/phi pairs (`_p2`);
    the count built from those tuned forms matches it."""
    import bench
    bench, info = _plan_info(bench.HEADLINE["name"])
    text = open(os.path.join(ROOT, "profiles", "launches_matvec_sphere_r20_3484860.md")).read()
    order = re.findall(r"^\| \d+ \| (k_\w+)<", text, re.M)
    assert len(order) == 27
    n_int = order.count("k_interp_theta_p2")
    n_ant = order.count("k_anterp_theta_p2")
    assert order.count("k_interp_phi_p2") == n_int and order.count("k_anterp_phi_p2") == n_ant
    tuned = "\n".join(["translate level %d E 16: 2 pairs/thread (1 us)" % l for l in range(2, 9)] +
                      ["interpolate level %d E 16: two-pass, entry pairs (1 us)" % (2 + i) for i in range(n_int)] +
                      ["interpolate level %d E 16: rows per CTA, chunk 16 (1 us)" % (2 + n_int + i)
                       for i in range(6 - n_int)] +
                      ["anterpolate level %d E 16: two-pass, entry pairs (1 us)" % (2 + i) for i in range(n_ant)] +
                      ["anterpolate level %d E 16: per child, chunk 8 (1 us)" % (2 + n_ant + i) for i in range(6 - n_ant)] +
                      ["interpolate level 2 E 128: two-pass (1 us)"])     # another column count: not counted
    assert bench.launches_per_step(info, 8) == 23
    assert bench.launches_per_step(info, 8, tuned) == len(order)


def test_peaks_are_the_measured_file_when_present(bench_info):
    bench, _ = bench_info
    peak, kind = bench.peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        import json
        assert kind == "measured" and peak == float(json.load(open(path))["hbm_gbs"])
    else:
        assert kind == "fallback" and peak == 6800.0


@pytest.mark.slow
def test_headline_traffic_matches_the_byte_model():
    """The committed one-product DRAM capture of the headline workload has one `traffic:` line
    per stage, each within 0.95-1.5 of the stage's algorithmic bytes at 8 RHS (the gather of x
    counted in the near stage, the scatter of y in the receive): the product re-reads little
    from HBM, and the summary belongs to this workload.  The upper end leaves room for the
    intermediates that the two-pass forms of the coarse level passes write and read back, and
    for the outgoing leaf patterns of the aggregation, which pass through L2 to DRAM."""
    import bench
    bench, info = _plan_info(bench.HEADLINE["name"])
    traffic = bench.measured_traffic("dram_matvec_sphere_r20_3484860.md")
    sb = bench.stage_bytes(info, 8)
    sb["near"] += sb["gather"]
    sb["receive"] += info["n_unknowns"] * 8 * 8
    assert set(traffic) == {"near", "aggregate", "interpolate", "translate", "anterpolate", "receive"}
    for stage, (kernel, nbytes) in traffic.items():
        assert kernel.startswith("k_")
        assert 0.95 * sb[stage] <= nbytes <= 1.5 * sb[stage], (stage, nbytes, sb[stage])
