"""Host arithmetic of bench.py that turns library counters into the reported rooflines (CPU only)."""
import bench


def test_kernel_revision_follows_the_name():
    v = "lrs 0.4 (sm_103a) chi0-tc r1 dyson-gj r4"
    assert bench.kernel_revision(v, "chi0-tc") == "r1"
    assert bench.kernel_revision(v, "dyson-gj") == "r4"
    assert bench.kernel_revision(v, "absent") is None
    assert bench.kernel_revision("lrs dyson-gj", "dyson-gj") is None   # no tag after the name


def test_tensor_core_update_is_reported_against_hbm():
    """16 algorithmic bytes per updated element; the library counts 2 kb = 64 flop per element."""
    elems, launches, ms = 3.2e6, 81, 3.0
    st = {"w_main_launches": launches, "ms_w_main": ms, "flop_w_main": 64.0 * elems * launches,
          "dyson_update_tc": True}
    r = bench.dyson_roofline(st, "single-site-3520", "r4", hbm_gbs=6684.1)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["algorithmic_bytes_per_launch"] - 16.0 * elems) < 1e-6 * elems
    assert abs(r["achieved"] - 16.0 * elems * launches / (ms * 1e-3) / 1e9) < 1e-9 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / 6684.1) < 1e-12
    assert abs(r["fp64_equivalent_tflops"] - 64.0 * elems * launches / (ms * 1e-3) / 1e12) < 1e-9
    assert r["traffic"] == bench.DYSON_TRAFFIC[("single-site-3520", "r4")]
    assert abs(r["avg_launch_us"] - 1e3 * ms / launches) < 1e-12


def test_fp64_update_is_reported_against_the_fma_rate():
    st = {"w_main_launches": 10, "ms_w_main": 2.0, "flop_w_main": 2.0e9, "dyson_update_tc": False}
    r = bench.dyson_roofline(st, "other-workload", "r9", hbm_gbs=6684.1)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - 1.0) < 1e-12              # 2e9 flop in 2 ms
    assert abs(r["peak"] - 152 * 4 * 2.07e9 / 1e12) < 1e-12
    assert r["traffic"] is None                          # no counters for an unmeasured revision
    assert bench.dyson_roofline({"w_main_launches": 0}) is None


def test_peaks_have_every_denominator():
    peaks = bench.load_peaks()
    for key in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained", "source"):
        assert key in peaks
    assert peaks["hbm_gbs"] > 1000 and peaks["bf16_tflops_sustained"] > 100
