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


def test_both_arms_name_the_same_config():
    import argparse
    from paper_2005_07834_gb300 import synth
    args = argparse.Namespace(projection="exact")
    wl = synth.single_site_260()
    a = bench.workload_config("single-site-260", wl, args)
    assert a == bench.workload_config("single-site-260", wl, args)
    assert "precision" not in a and a["npts"] == 260 and a["K"] == 256


def test_oracle_leg_reports_errors_of_each_path():
    """The cpu_baseline leg's accuracy report, fed the oracle's own chi0 (perturbed by a known
    relative amount) as a library result: errors of that size come back, and the Dyson check of an
    exact W is at rounding level."""
    import numpy as np
    from oracle import chi0 as ochi0, coulomb as ocoul, dyson as odys
    from paper_2005_07834_gb300 import synth
    from tests.oracle_problem import OracleProblem
    wl = synth.single_site_260()
    pr = OracleProblem(wl)
    chi = ochi0.chi0_green(*pr.args(), pr.t, pr.W)
    v = ocoul.coulomb_multipole(pr.site.pts, pr.site.lmax)
    bad = chi * (1.0 + 1e-6)
    res = {"mixed": (bad, odys.screened_interaction(v, bad, pr.site.wts), v),
           "fp64": (chi, odys.screened_interaction(v, chi, pr.site.wts), v)}
    cpu, acc = bench.oracle_single_site_leg(wl, res)
    assert cpu["value"] > 0 and cpu["cores"] >= 1
    assert abs(acc["mixed"]["chi0_rows"]["fro"] - 1e-6) < 1e-9
    assert acc["fp64"]["chi0_rows"]["fro"] < 1e-13
    for name in ("mixed", "fp64"):
        assert acc[name]["dyson_w"]["fro"] < 1e-13 and acc[name]["v"]["fro"] < 1e-14
    assert abs(acc["mixed_vs_fp64_gpu"]["chi0"]["fro"] - 1e-6) < 1e-9


def test_sampled_oracle_leg_on_library_like_results():
    """The sampled checks of large sites, fed the oracle's own orbitals, chi0 and W (chi0 perturbed by
    a known relative amount): the projection and Dyson checks are at rounding level, the chi0 rows
    report the perturbation."""
    import numpy as np
    from oracle import chi0 as ochi0, coulomb as ocoul, dyson as odys
    from paper_2005_07834_gb300 import synth
    from tests.oracle_problem import OracleProblem
    wl = synth.single_site_260()
    pr = OracleProblem(wl)
    chi = ochi0.chi0_green(*pr.args(), pr.t, pr.W) * (1.0 + 2e-6)
    v = ocoul.coulomb_multipole(pr.site.pts, pr.site.lmax)
    w = odys.screened_interaction(v, chi, pr.site.wts)
    psi = pr.psi.reshape(pr.site.npts, -1)
    cpu, acc = bench.oracle_sampled_sites_leg(wl, {0: (chi, w, v, psi)}, rows=8, points=16)
    a = acc["0"]
    assert a["psi_sampled_points"]["fro"] < 1e-13
    assert abs(a["chi0_rows_from_library_psi"]["fro"] - 2e-6) < 1e-9
    assert a["dyson_w"]["fro"] < 1e-13 and a["v"]["fro"] < 1e-14
    assert cpu["value"] > 0


def test_blocked_update_is_reported_against_the_tensor_peak():
    """128-wide pivot blocks: the library reports 2 kb flop per rewritten element with kb = 128; the
    bench counts 36 slice products per K element issued and reports against the bf16 peak."""
    elems, launches, ms = 3.2e6, 20, 1.0
    st = {"w_main_launches": launches, "ms_w_main": ms, "flop_w_main": 2.0 * 128 * elems * launches,
          "w_main_elements": elems * launches, "dyson_update_tc": True}
    r = bench.dyson_roofline(st, "x", "r5", hbm_gbs=6700.0, bf16_tflops=1900.0)
    assert r["bound"] == "tensor" and r["pivot_block"] == 128
    assert abs(r["achieved"] - 36 * 2.0 * 128 * elems * launches / (ms * 1e-3) / 1e12) < 1e-6
    assert abs(r["hbm_gbs_algorithmic"] - 16.0 * elems * launches / (ms * 1e-3) / 1e9) < 1e-6


def test_site_subset_of_a_multi_site_workload():
    """--sites keeps the named sites of a multi-site workload (profiling runs) and the bench line's
    config says so."""
    import argparse
    import bench
    wl = bench.make_workload("batched-64-sites", 0, [2, 5])
    full = bench.make_workload("batched-64-sites")
    assert len(wl.sites) == 2
    assert wl.sites[0].npts == full.sites[2].npts and wl.sites[1].npts == full.sites[5].npts
    args = argparse.Namespace(projection="exact", sites=[2, 5])
    cfg = bench.workload_config("batched-64-sites", wl, args)
    assert cfg["sites"] == 2 and cfg["site_subset"] == [2, 5]


def test_bench_line_is_strict_json():
    """A non-finite float anywhere in the line (a failed sub-measurement) is printed as null."""
    import json
    import bench
    line = {"value": 1.0, "a": {"b": [float("nan"), 2.0, float("inf")]}, "c": None}
    out = json.loads(json.dumps(bench.strict_json(line), allow_nan=False))
    assert out == {"value": 1.0, "a": {"b": [None, 2.0, None]}, "c": None}


def test_config1_against_both_kernels():
    """The bench's report of the 260-point plain build against the pair-sum oracle: fed the
    oracle's own kappa_N build it reads zero against kappa_N and the quadrature error (about
    4e-8 at 12 frequencies) against kappa_exact."""
    import bench
    from oracle import chi0 as ochi0, coulomb as ocoul, dyson as odys, projection as oproj, quadrature as oquad
    from paper_2005_07834_gb300 import synth
    wl = synth.single_site_260()
    o, s = wl.orbitals, wl.sites[0]
    psi = oproj.project_direct(o.cell, o.kpts, o.gvec, o.coeff, s.center, s.pts)
    po, pu, eo, eu, wo, wu = oproj.split_occupied(psi, o.energies, o.nocc, o.kweights)
    mu = oquad.chemical_potential_midgap(o.energies, o.nocc)
    t, W = oquad.frequency_grid(wl.nfreq, oquad.zeta_rule(o.energies, mu))
    v = ocoul.coulomb_multipole(s.pts, s.lmax)
    c = ochi0.chi0_pairs(po, pu, eo, eu, wo, wu, mu, t, W)
    out = bench.config1_vs_kappa((c, odys.screened_interaction(v, c, s.wts), v))
    assert out["vs_kappa_N"]["chi0"]["fro"] < 1e-14 and out["vs_kappa_N"]["w"]["fro"] < 1e-14
    assert 1e-9 < out["vs_kappa_exact"]["chi0"]["fro"] < 1e-6


def test_multisite_update_traffic_from_bytes_per_element():
    """For the 64-site workload the update's DRAM traffic is the measured bytes per rewritten
    element of the largest site's capture times the average launch's elements."""
    import bench
    per = bench.DYSON_TRAFFIC_PER_ELEMENT[("batched-64-sites", "r6")]
    st = {"w_main_launches": 4, "ms_w_main": 0.4, "flop_w_main": 2.0 * 32 * 8.0e6,
          "w_main_elements": 8.0e6, "dyson_update_tc": True}
    r = bench.dyson_roofline(st, "batched-64-sites", "r6", 6758.5, 1871.0)
    assert abs(r["traffic"] - per * 2.0e6) < 1.0 and "traffic_source" in r
    assert 13.0 < per < 14.0
    assert bench.dyson_roofline(st, "batched-64-sites", "r5", 6758.5, 1871.0)["traffic"] is None
