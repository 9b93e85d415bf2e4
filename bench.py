"""Throughput of site chi0 + W builds on GB300 (one JSON line on stdout).

A step is one pass of the whole hot path over one site with the orbitals
resident in HBM: projection of the Bloch coefficients onto the site grid,
frequency denominators, the Green's-function contraction for chi0 with its
FP64 frequency accumulation, the Coulomb operator and the Dyson solve for W
(lm basis: symmetric positive definite form inverted by blocked Gauss-Jordan
exchange steps, float64-accurate products on the tensor cores in the mixed
precisions).  `value` is site builds per second over all ranks; `e2e`
measures the same through the C-ABI with page-locked host buffers
(host->device copy of the coefficients and device->host copy of W inside the
timed region).

After the timed region (default 3520-point site):
  plain_fp64          the same build on the plain FP64 path, and the mixed path's
                      chi0, W and W - v errors against it;
  backward            the adjoint of L = q^T W q on this site (device buffers,
                      tensor roofline) and on the 260-point differentiation case;
  workloads           the 64-site workload (graph replay, rooflines, mixed vs
                      plain FP64 on a seeded sample of sites, oracle on the two
                      smallest sites);
  cpu_baseline        the FP64 oracle on the host cores on a bounded sample of the
                      build, whose outputs (chi0 rows, dense LU on each path's chi0)
                      give accuracy_vs_oracle.

--impl reference times the FP64 CPU oracle on the host cores instead (rank 0
only), each step a bounded sample of the same workload; its `ms_per_step` is
the sample's wall time and `value` the throughput scaled from it.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# FP64 FMA: 2 per SM per clock (1.25 TFLOP/s nominal / (152 SMs x 2.07 GHz) = 3.97 flop/clk/SM).
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12

# dram__bytes_read.sum + dram__bytes_write.sum of one chi0 launch, from one ncu capture
# (profiles/ncu_chi0_single-site-3520_bf16x3.md), valid only for the kernel revision named.
CHI0_TRAFFIC = {("single-site-3520", "bf16x3", "r1"): 23.26e9, ("single-site-3520", "bf16x3", "r2"): 20.77e9,
                ("single-site-3520", "bf16x3", "r3"): 31.05e9}


def strict_json(x):
    """The bench line as strict JSON: non-finite floats (a failed sub-measurement) become null."""
    import math
    if isinstance(x, float):
        return x if math.isfinite(x) else None
    if isinstance(x, dict):
        return {k: strict_json(v) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [strict_json(v) for v in x]
    return x


def kernel_revision(version, name):
    """Revision tag that follows `name` in the library version string (ncu counters are only
    reused while the kernel they were taken on is unchanged)."""
    tok = version.split()
    return tok[tok.index(name) + 1] if name in tok[:-1] else None

WORKLOADS = {
    "single-site-3520": "single_site_3520",
    "single-site-260": "single_site_260",
    "batched-64-sites": "batched_64_sites",
    "large-cell-16-sites": "large_cell_16_sites",
    "gamma-site-3520": "gamma_site_3520",
}
MULTI_SITE = {"batched-64-sites", "large-cell-16-sites"}


# (workload, dyson-gj revision) -> ncu DRAM bytes (read + write) per launch of the update kernel
DYSON_TRAFFIC = {("single-site-3520", "r1"): 27.2e6, ("single-site-3520", "r2"): 28.5e6,
                 ("single-site-3520", "r4"): 28.52e6, ("single-site-3520", "r5"): 28.52e6,
                 ("single-site-3520", "r6"): 28.51e6, ("single-site-3520", "r8"): 28.54e6}
# Multi-site workloads (launches of many sizes): DRAM bytes per rewritten element of one ncu capture
# on the workload's largest site (r = 6768, block 100: 187.27 MB read + 119.26 MB written for
# 22,475,160 elements), applied to the average launch; valid only for the revision named.
DYSON_TRAFFIC_PER_ELEMENT = {("batched-64-sites", "r6"): (187.27e6 + 119.26e6) / 22475160,
                             ("batched-64-sites", "r8"): (187.30e6 + 118.30e6) / 22475160}


def dyson_roofline(st, workload=None, version=None, hbm_gbs=None, bf16_tflops=None):
    """The SPD inverse's trailing updates.  On the FP64 pipe (FP64 context) they are bound by the
    FP64 FMA rate.  On the tensor cores their float64 work is one subtraction per element and their
    algorithmic traffic one read and one write of each updated element (16 bytes; the library
    reports the elements rewritten).  With 32-wide pivot blocks (28 slice products over K = 32 per
    element) that traffic bounds the update, so it is reported against the HBM copy bandwidth;
    with 128-wide blocks (36 slice products over K = 128 per element, the float64-accurate GEMM)
    the issued tensor work does, so it is reported against the bf16 peak.  The FP64-equivalent rate
    is given beside either."""
    if not st.get("w_main_launches"):
        return None
    ms = st["ms_w_main"]
    tc = st.get("dyson_update_tc", False)
    fp64_eq = st["flop_w_main"] / (ms * 1e-3) / 1e12
    elems = st.get("w_main_elements") or st["flop_w_main"] / (2.0 * 32)
    kb = st["flop_w_main"] / (2.0 * elems)
    traffic = DYSON_TRAFFIC.get((workload, version))
    per_elem = DYSON_TRAFFIC_PER_ELEMENT.get((workload, version))
    if traffic is None and per_elem is not None:
        traffic = per_elem * elems / st["w_main_launches"]
    common = {"launches": st["w_main_launches"], "avg_launch_us": 1e3 * ms / st["w_main_launches"],
              "pivot_block": round(kb), "traffic": traffic}
    if per_elem is not None and (workload, version) not in DYSON_TRAFFIC:
        common["traffic_source"] = ("ncu DRAM bytes per rewritten element on the workload's largest site "
                                    f"({per_elem:.2f} B), times the average launch's elements")
    algo_bytes = 16.0 * elems
    if tc and kb > 64 and bf16_tflops:
        issued = 36 * 2.0 * kb * elems
        r = {"bound": "tensor",
             "kernel": "oz_gemm_kernel (rank-128 trailing update, float64-accurate bf16 slices on tcgen05)",
             "achieved": issued / (ms * 1e-3) / 1e12, "peak": bf16_tflops, "unit": "TFLOP/s",
             "peak_source": "bf16 burst, measured (36 slice products per K element issued)",
             "hbm_gbs_algorithmic": algo_bytes / (ms * 1e-3) / 1e9,
             "algorithmic_bytes_per_launch": algo_bytes / st["w_main_launches"],
             "fp64_equivalent_tflops": fp64_eq, "fp64_equivalent_vs_fp64_fma_peak": fp64_eq / FP64_PEAK_TFLOPS,
             **common}
    elif tc and hbm_gbs:
        r = {"bound": "hbm",
             "kernel": "oz_update_kernel (SPD-inverse trailing update, float64-accurate bf16 slices on tcgen05)",
             "achieved": algo_bytes / (ms * 1e-3) / 1e9, "peak": hbm_gbs, "unit": "GB/s",
             "peak_source": "HBM copy bandwidth, measured",
             "algorithmic_bytes_per_launch": algo_bytes / st["w_main_launches"],
             "fp64_equivalent_tflops": fp64_eq, "fp64_equivalent_vs_fp64_fma_peak": fp64_eq / FP64_PEAK_TFLOPS,
             **common}
    else:
        r = {"bound": "alu", "kernel": "gj_update_kernel (SPD-inverse trailing update, FP64 FMA)",
             "achieved": fp64_eq, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
             "peak_source": "FP64 FMA rate: 152 SMs x 2 DFMA/clk x 2.07 GHz", **common}
    r["frac"] = r["achieved"] / r["peak"]
    return r


def proj_mode(lrs, args):
    return lrs.LRS_PROJ_FFT_LAGRANGE3 if args.projection == "fft" else lrs.LRS_PROJ_EXACT


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["source"] = "measured"
        return d
    d = dict(PEAKS_FALLBACK)
    d["source"] = "fallback"
    return d


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

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
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def make_workload(name, nfreq=0, sites=None):
    """The named synthetic workload; nfreq > 0 replaces its frequency count and `sites` (indices)
    keeps a subset of a multi-site workload's sites (smaller profiler captures)."""
    import dataclasses
    from paper_2005_07834_gb300 import synth
    wl = getattr(synth, WORKLOADS[name])()
    if nfreq:
        wl = dataclasses.replace(wl, nfreq=nfreq)
    if sites:
        wl = dataclasses.replace(wl, sites=[wl.sites[i] for i in sites])
    return wl


# ----------------------------------------------------------------------------- shared descriptions

DTYPE = {"fp64": "f64",
         "bf16x3": "bf16x3 chi0/adjoint + fp16x3 projection, f32 accumulate, f64 denominators/frequency sum/Dyson",
         "fp16x3": "fp16x3, f32 accumulate, f64 denominators/frequency sum/Dyson"}
DYSON_SAMPLE_SITES = 4      # sites of the 64-site workload rebuilt by the plain FP64 path for the error report
ORACLE_ROWS = 48            # chi0 rows the oracle evaluates on the single-site workloads


def workload_config(name, wl, args):
    """The `config` object of both arms: names the workload and its sizes (no precision: `dtype`
    and `precision` say how each arm computes)."""
    o = wl.orbitals
    K = o.nk * o.nbands
    if name in MULTI_SITE:
        sizes = [s.npts for s in wl.sites]
        cfg = {"workload": name, "sites": len(sizes), "npts_min": min(sizes), "npts_max": max(sizes),
               "npts_sum": sum(sizes), "K": K, "nfreq": wl.nfreq, "ng": o.ng, "projection": args.projection,
               "graph": "one CUDA graph replay per step", "l2": "inputs larger than L2"}
        if getattr(args, "sites", None):
            cfg["site_subset"] = list(args.sites)   # a profiling run, not the named workload
        return cfg
    s = wl.sites[0]
    return {"workload": name, "npts": s.npts, "K": K, "nfreq": wl.nfreq, "ng": o.ng, "replicas_per_gpu": 1,
            "projection": args.projection, "real_orbitals": name.startswith("gamma"),
            "l2": "inputs larger than L2 (coefficients %d MB, orbitals %d MB)" % (
                o.coeff.nbytes >> 20, (s.npts * K * 16) >> 20)}


def errors(a, ref):
    """Relative Frobenius and element-wise (max |d| / max |ref|) error."""
    d = a - ref
    return {"fro": float(np.linalg.norm(d) / np.linalg.norm(ref)), "max": float(np.max(np.abs(d)) / np.max(np.abs(ref)))}


def matrix_errors(chi, w, v, chi_ref, w_ref):
    return {"chi0": errors(chi, chi_ref), "w": errors(w, w_ref), "w_minus_v": errors(w - v, w_ref - v)}


# ----------------------------------------------------------------------------- CPU legs (FP64 oracle)

def oracle_reference_sample(wl):
    """One step of the reference arm: the FP64 oracle on one site, on a bounded sample of the
    build - projection of the first k-point (its orbitals stand in for the other k-points'), the
    Green's-function chi0 on the first frequency over all rows, and the full dense Dyson LU on that
    chi0 (each frequency term is negative semidefinite, so the solve is a representative one).
    Returns the measured seconds and the seconds of one whole build scaled from them
    (projection x nk, chi0 x nfreq, LU x 1)."""
    from oracle import chi0 as ochi0, coulomb as ocoul, dyson as odys, projection as oproj, quadrature as oquad
    o, s = wl.orbitals, wl.sites[0]
    t0 = time.perf_counter()
    psi_k = oproj.project_direct(o.cell, o.kpts[:1], o.gvec, o.coeff[:1], s.center, s.pts)
    t_proj = time.perf_counter() - t0
    psi = np.concatenate([psi_k] * o.nk, axis=1)
    po, pu, eo, eu, wo, wu = oproj.split_occupied(psi, o.energies, o.nocc, o.kweights)
    mu = oquad.chemical_potential_midgap(o.energies, o.nocc)
    t, W = oquad.frequency_grid(wl.nfreq, oquad.zeta_rule(o.energies, mu))
    t0 = time.perf_counter()
    chi = ochi0.chi0_green(po, pu, eo, eu, wo, wu, mu, t[:1], W[:1])
    t_chi = time.perf_counter() - t0
    t0 = time.perf_counter()
    v = ocoul.coulomb_multipole(s.pts, s.lmax)
    odys.screened_interaction(v, chi, s.wts)
    t_w = time.perf_counter() - t0
    measured = t_proj + t_chi + t_w
    scaled = t_proj * o.nk + t_chi * wl.nfreq + t_w
    return measured, scaled, {"t_project_s": t_proj, "t_chi0_s": t_chi, "t_w_s": t_w,
                              "scale_project": o.nk, "scale_chi0": wl.nfreq, "scale_w": 1}


def oracle_single_site_leg(wl, results, config1=None):
    """cpu_baseline leg of the single-site workloads: the FP64 oracle on the host cores on a bounded
    sample of one build, timed, whose outputs double as the accuracy reference:
      * orbitals on every site point for every k-point by the direct sum (Sec. VI.B method 1), timed;
      * chi0 by the Green's-function route over all rows on the first frequency, timed (x nfreq);
      * v and the dense LU of (I - v Q chi0 Q) W = v on the library's chi0, timed;
      * chi0 on ORACLE_ROWS seeded rows at every frequency (not timed): the accuracy reference.
    `results` maps a path name to (chi0, W, v) from the library; each is compared with the oracle:
    its chi0 rows element-wise and by row norms, and its W and W - v with the oracle's dense LU applied
    to that path's own chi0 (the Dyson route, the rounding of chi0 taken out).  The mixed path is
    also compared with the plain one.  `config1` is the plain FP64 build (chi0, W, v) of the
    260-point site, compared whole with the oracle at the quadrature (kappa_N) and with the exact
    frequency integral (kappa_exact: the quadrature error itself).  Returns (cpu_baseline dict,
    accuracy dict)."""
    from oracle import chi0 as ochi0, coulomb as ocoul, dyson as odys, projection as oproj, quadrature as oquad
    o, s = wl.orbitals, wl.sites[0]
    rows = np.sort(np.random.default_rng(3).choice(s.npts, ORACLE_ROWS, replace=False))
    t0 = time.perf_counter()
    psi = oproj.project_direct(o.cell, o.kpts, o.gvec, o.coeff, s.center, s.pts)
    t_proj = time.perf_counter() - t0
    po, pu, eo, eu, wo, wu = oproj.split_occupied(psi, o.energies, o.nocc, o.kweights)
    mu = oquad.chemical_potential_midgap(o.energies, o.nocc)
    t, W = oquad.frequency_grid(wl.nfreq, oquad.zeta_rule(o.energies, mu))
    t0 = time.perf_counter()
    ochi0.chi0_green(po, pu, eo, eu, wo, wu, mu, t[:1], W[:1])
    t_chi1 = time.perf_counter() - t0
    first = next(iter(results))
    t0 = time.perf_counter()
    v = ocoul.coulomb_multipole(s.pts, s.lmax)
    w_first = odys.screened_interaction(v, results[first][0], s.wts)
    t_w = time.perf_counter() - t0
    t_build = t_proj + t_chi1 * wl.nfreq + t_w
    chi_rows = ochi0.chi0_green(po, pu, eo, eu, wo, wu, mu, t, W, rows=rows)
    acc = {"reference": "FP64 oracle on the host cores: orbitals by the direct sum on every point, chi0 on "
                        f"{len(rows)} seeded rows (Green's-function route), W by a dense LU on each path's own chi0",
           "rows": int(len(rows))}
    for name, (chi, w, v_lib) in results.items():
        w_lu = w_first if name == first else odys.screened_interaction(v, chi, s.wts)
        acc[name] = {"chi0_rows": errors(chi[rows], chi_rows),
                     "chi0_rows_max_row_fro": float(np.max(np.linalg.norm(chi[rows] - chi_rows, axis=1)
                                                           / np.linalg.norm(chi_rows, axis=1))),
                     "v": errors(v_lib, v), "dyson_w": errors(w, w_lu), "dyson_w_minus_v": errors(w - v, w_lu - v)}
    if "mixed" in results and "fp64" in results:
        cm, wm, _ = results["mixed"]
        cp, wp, _ = results["fp64"]
        acc["mixed_vs_fp64_gpu"] = {"chi0": errors(cm, cp), "w": errors(wm, wp), "w_minus_v": errors(wm - v, wp - v)}
    if config1 is not None:
        acc["plain_fp64_260_points"] = config1_vs_kappa(config1)
    cpu = {"value": 1.0 / t_build, "unit": "builds/s", "cores": os.cpu_count(), "kind": "oracle",
           "sample": f"one site: orbitals on all {s.npts} points for all {o.nk} k-points, chi0 over all rows on 1 "
                     f"of {wl.nfreq} frequencies (x {wl.nfreq}), full Dyson LU",
           "parts_s": {"t_project_s": t_proj, "t_chi0_one_frequency_s": t_chi1, "t_w_s": t_w},
           "measured_s": t_proj + t_chi1 + t_w}
    return cpu, acc


def config1_vs_kappa(built):
    """The plain FP64 build of the 260-point site against the pair-sum oracle with the quadrature
    kernel kappa_N (the method's own result) and with kappa_exact (the exact frequency integral)."""
    from oracle import chi0 as ochi0, coulomb as ocoul, dyson as odys, projection as oproj, quadrature as oquad
    from paper_2005_07834_gb300 import synth
    wl = synth.single_site_260()
    o, s = wl.orbitals, wl.sites[0]
    psi = oproj.project_direct(o.cell, o.kpts, o.gvec, o.coeff, s.center, s.pts)
    po, pu, eo, eu, wo, wu = oproj.split_occupied(psi, o.energies, o.nocc, o.kweights)
    mu = oquad.chemical_potential_midgap(o.energies, o.nocc)
    t, W = oquad.frequency_grid(wl.nfreq, oquad.zeta_rule(o.energies, mu))
    v = ocoul.coulomb_multipole(s.pts, s.lmax)
    chi, w, _ = built
    out = {"reference": "pair-sum oracle (Eq. chi1) on the whole 260-point site, 12 frequencies"}
    for name, exact in (("vs_kappa_N", False), ("vs_kappa_exact", True)):
        c = ochi0.chi0_pairs(po, pu, eo, eu, wo, wu, mu, t, W, exact=exact)
        wr = odys.screened_interaction(v, c, s.wts)
        out[name] = {"chi0": errors(chi, c), "w": errors(w, wr), "w_minus_v": errors(w - v, wr - v)}
    return out


def oracle_multisite_leg(wl, sites, lib):
    """cpu_baseline leg of the multi-site workloads: the whole FP64 oracle build (direct-sum
    orbitals, Green's-function chi0, dense LU) of the given sites, timed and scaled to every site by
    the algorithmic cost 8 N^2 K nf + 14/3 N^3; `lib` maps a site to the mixed path's (chi0, W, v)
    for the accuracy report."""
    from oracle import chi0 as ochi0, coulomb as ocoul, dyson as odys, projection as oproj, quadrature as oquad
    o = wl.orbitals
    K = o.nk * o.nbands
    mu = oquad.chemical_potential_midgap(o.energies, o.nocc)
    t, W = oquad.frequency_grid(wl.nfreq, oquad.zeta_rule(o.energies, mu))
    acc, t_all = {}, 0.0
    for i in sites:
        s = wl.sites[i]
        t0 = time.perf_counter()
        psi = oproj.project_direct(o.cell, o.kpts, o.gvec, o.coeff, s.center, s.pts)
        po, pu, eo, eu, wo, wu = oproj.split_occupied(psi, o.energies, o.nocc, o.kweights)
        chi = ochi0.chi0_green(po, pu, eo, eu, wo, wu, mu, t, W)
        v = ocoul.coulomb_multipole(s.pts, s.lmax)
        w = odys.screened_interaction(v, chi, s.wts)
        t_all += time.perf_counter() - t0
        c, g, _ = lib[i]
        acc[str(i)] = {"npts": s.npts, **matrix_errors(c, g, v, chi, w)}
    scale = sum(site_cost(s, K, wl.nfreq) for s in wl.sites) / sum(site_cost(wl.sites[i], K, wl.nfreq)
                                                                   for i in sites)
    cpu = {"value": len(wl.sites) / (t_all * scale), "unit": "site builds/s", "cores": os.cpu_count(),
           "kind": "oracle", "sample": f"sites {list(sites)} built whole by the oracle ({t_all:.2f} s), scaled to all "
                                       f"{len(wl.sites)} sites by 8 N^2 K nf + 14/3 N^3 (x{scale:.1f})"}
    return cpu, acc


def oracle_sampled_sites_leg(wl, lib, rows=16, points=64):
    """cpu_baseline leg of workloads whose sites are too large for a whole oracle build on the host
    (the 9312-point sites of the large cell: the direct-sum projection alone is 8 N N_G K ~ 4e13 flop
    per site).  Per site, timed, on the library's own intermediate results:
      * orbitals by the direct sum on `points` seeded grid points, every band and k-point, against the
        library's projection;
      * chi0 on `rows` seeded rows by the Green's-function route, every frequency, from the library's
        orbitals (isolates the mixed-precision contraction);
      * v and the dense LU of (I - v Q chi0 Q) W = v on the library's chi0 (isolates the Dyson route).
    The measured time is scaled to a whole build of every site (projection x N / points, chi0 rows x
    N / 2 rows, LU x 1, then x sites) for the cpu_baseline value."""
    from oracle import chi0 as ochi0, coulomb as ocoul, dyson as odys, projection as oproj, quadrature as oquad
    o = wl.orbitals
    mu = oquad.chemical_potential_midgap(o.energies, o.nocc)
    t, W = oquad.frequency_grid(wl.nfreq, oquad.zeta_rule(o.energies, mu))
    acc, t_scaled = {}, 0.0
    for i, (chi, w, v_lib, psi_lib) in lib.items():
        s = wl.sites[i]
        rng = np.random.default_rng(17 + i)
        pts = np.sort(rng.choice(s.npts, points, replace=False))
        rws = np.sort(rng.choice(s.npts, rows, replace=False))
        t0 = time.perf_counter()
        psi = oproj.project_direct(o.cell, o.kpts, o.gvec, o.coeff, s.center, s.pts[pts]).reshape(points, -1)
        t_p = time.perf_counter() - t0
        po, pu, eo, eu, wo, wu = oproj.split_occupied(psi_lib.reshape(s.npts, o.nk, o.nbands), o.energies, o.nocc,
                                                      o.kweights)
        t0 = time.perf_counter()
        chi_rows = ochi0.chi0_green(po, pu, eo, eu, wo, wu, mu, t, W, rows=rws)
        t_c = time.perf_counter() - t0
        t0 = time.perf_counter()
        v = ocoul.coulomb_multipole(s.pts, s.lmax)
        w_lu = odys.screened_interaction(v, chi, s.wts)
        t_w = time.perf_counter() - t0
        t_scaled += t_p * s.npts / points + t_c * s.npts / (2.0 * rows) + t_w
        acc[str(i)] = {"npts": s.npts, "psi_sampled_points": errors(psi_lib[pts], psi),
                       "chi0_rows_from_library_psi": errors(chi[rws], chi_rows), "v": errors(v_lib, v),
                       "dyson_w": errors(w, w_lu), "dyson_w_minus_v": errors(w - v, w_lu - v),
                       "oracle_s": {"project_sampled": t_p, "chi0_rows": t_c, "dense_lu": t_w}}
    scale = len(wl.sites) / len(lib)
    cpu = {"value": len(wl.sites) / (t_scaled * scale), "unit": "site builds/s", "cores": os.cpu_count(),
           "kind": "oracle", "sample": f"sites {sorted(lib)}: direct-sum orbitals on {points} points, chi0 on {rows} "
                                       "rows, dense Dyson LU; scaled to whole builds of every site"}
    return cpu, acc


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    wl = make_workload(args.workload)
    cores = os.cpu_count()
    if args.workload in MULTI_SITE:
        # the smallest site, the oracle's whole build, scaled by the algorithmic cost
        o = wl.orbitals
        K = o.nk * o.nbands
        small = min(range(len(wl.sites)), key=lambda i: wl.sites[i].npts)
        sub = type(wl)(wl.name, o, [wl.sites[small]], wl.nfreq, wl.fft_grid)
        work = site_cost(wl.sites[small], K, wl.nfreq) / sum(site_cost(s, K, wl.nfreq) for s in wl.sites)

        def one_step():
            m, scaled, parts = oracle_reference_sample(sub)
            return m, scaled / work, parts
        sample = (f"site {small} ({wl.sites[small].npts} points) of {args.workload}: projection of 1 of {o.nk} "
                  f"k-points, chi0 on 1 of {wl.nfreq} frequencies (all rows), full Dyson LU; scaled to that site "
                  "(x nk, x nfreq) and to all sites by 8 N^2 K nf + 14/3 N^3")
        unit = "site builds/s"
        per_build = len(wl.sites)
    else:
        def one_step():
            return oracle_reference_sample(wl)
        sample = (f"one site of {args.workload}: projection of 1 of {wl.orbitals.nk} k-points, chi0 "
                  f"(Green's-function route) on 1 of {wl.nfreq} frequencies over all rows, full Dyson LU; "
                  "scaled to one build (x nk, x nfreq, x 1)")
        unit = "builds/s"
        per_build = 1
    for _ in range(max(args.warmup, 0)):
        one_step()
    measured, scaled, parts = [], [], None
    for _ in range(args.steps):
        m, sc, parts = one_step()
        measured.append(m)
        scaled.append(sc)
    ms_sample = 1e3 * statistics.mean(measured)
    s_build = statistics.mean(scaled)
    value = per_build / s_build
    line = {"impl": "reference", "metric": "site chi0+W builds/s", "value": value, "unit": unit,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            # wall time of one step as run (the bounded sample); `value` comes from the scaled time
            "ms_per_step": ms_sample,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "precision": "fp64 oracle on the host cores", "data": "synthetic (seeded generator)",
            "config": workload_config(args.workload, wl, args),
            "sample_ms_per_step": ms_sample, "scaled_s_per_build": s_build,
            "scale_factor": s_build * 1e3 / ms_sample,
            "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "parts_s": parts}
    print(json.dumps(strict_json(line), allow_nan=False), flush=True)


# ----------------------------------------------------------------------------- GPU legs

def timed_on(stream, fn, warmup, steps):
    """Median device time (ms) of fn() by CUDA events on `stream`."""
    import torch
    for _ in range(warmup):
        fn()
    ms = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return float(np.median(ms))


def backward_leg(lrs, scr, stream, s, K, nf, peaks, precision, real=False):
    """Adjoint of L = q^T W q (q seeded N(0,1)) for one site, device buffers, event-timed: the
    Green's functions recomputed per frequency (8 N^2 K) and the four H psi products (16 N^2 K)."""
    import torch
    n = s.npts
    from paper_2005_07834_gb300 import synth
    q = torch.tensor(synth.loss_weights(n, seed=2), dtype=torch.float64, device="cuda")
    gw = torch.outer(q, q).contiguous()
    ge = torch.empty(K, dtype=torch.float64, device="cuda")
    gp = torch.empty((n, K), dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()
    ms = timed_on(stream, lambda: scr.backward_dev(0, gw.data_ptr(), 0, ge.data_ptr(), gp.data_ptr()), 1, 3)
    st = scr.stats()
    flop = (12.0 if real else 24.0) * n * n * K * nf
    out = {"ms": ms, "ms_library": st["ms_backward"], "flop": flop,
           "achieved_tflops": flop / (ms * 1e-3) / 1e12, "device_bytes_peak": st["device_bytes_peak"],
           "flop_model": "per frequency: G recompute 8 N^2 K + four H psi products 16 N^2 K (complex)"}
    if precision == "fp64":
        out.update({"bound": "alu", "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "peak_source": "FP64 FMA rate: 152 SMs x 2 DFMA/clk x 2.07 GHz"})
    else:
        pk = peaks["bf16_tflops_sustained"]
        out.update({"bound": "tensor", "peak": pk, "unit": "TFLOP/s",
                    "peak_source": f"bf16 sustained, {peaks['source']}",
                    "issued_frac": 3 * out["achieved_tflops"] / pk})
    out["frac"] = out["achieved_tflops"] / out["peak"]
    return out


def config4_backward(lrs, stream):
    """Differentiation workload: 260-point site, FP64 context, L = q^T W q; microseconds per
    forward build (eager and replayed from a recorded CUDA graph) and per backward (device
    buffers, event-timed medians).  Also returns the build's (chi0, W, v) for the oracle leg."""
    import torch
    from paper_2005_07834_gb300 import synth
    wl = synth.single_site_260()
    o, s = wl.orbitals, wl.sites[0]
    scr = lrs.Screening(0, "fp64", stream.cuda_stream)
    scr.load(o)
    scr.set_sites([s])
    scr.set_frequency_quadrature(wl.nfreq)

    def fwd():
        scr.project()
        scr.build_chi0()
        scr.solve_w()
    ms_f = timed_on(stream, fwd, 3, 20)
    built = (scr.get_chi0(0), scr.get_w(0), scr.get_v(0))   # for the oracle leg (kappa_N and exact)
    # the same build recorded once as a CUDA graph and replayed (this size is launch-bound)
    try:
        scr.graph_capture()
        ms_g = timed_on(stream, scr.graph_launch, 3, 20)
        scr.synchronize()
    except lrs.LrsError as ex:   # reported, not fatal to the line
        ms_g = None
        graph_error = str(ex)
    else:
        graph_error = None
    q = torch.tensor(synth.loss_weights(s.npts, seed=2), dtype=torch.float64, device="cuda")
    gw = torch.outer(q, q).contiguous()
    K = o.nk * o.nbands
    ge = torch.empty(K, dtype=torch.float64, device="cuda")
    gp = torch.empty((s.npts, K), dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()
    ms_b = timed_on(stream, lambda: scr.backward_dev(0, gw.data_ptr(), 0, ge.data_ptr(), gp.data_ptr()), 3, 20)
    scr.close()
    return {"workload": "single-site-260 (differentiation)", "precision": "fp64", "us_forward": 1e3 * ms_f,
            "us_forward_graph_replay": 1e3 * ms_g if ms_g else None,
            "builds_per_s_graph_replay": 1e3 / ms_g if ms_g else None,
            "graph_error": graph_error,
            "us_backward": 1e3 * ms_b, "loss": "q^T W q, q ~ N(0,1) seed 2",
            "timing": "median of 20 after 3 warm-ups, CUDA events on the context stream"}, built


def gpu_path(lrs, precision, stream, wl, sites, pmode):
    """A context with the workload's orbitals and `sites` built once (projection, chi0, W)."""
    scr = lrs.Screening(0, precision, stream.cuda_stream)
    scr.load(wl.orbitals)
    scr.set_sites(sites)
    scr.set_frequency_quadrature(wl.nfreq)
    scr.set_fft_grid(*wl.fft_grid)
    scr.project(mode=pmode)
    scr.build_chi0()
    scr.solve_w()
    scr.synchronize()
    return scr


def multisite_measure(args, lrs, wl, stream, steps, warmup, peaks, compare=True, oracle_sites=0, keep_psi=()):
    """Graph-replayed build of every site of a multi-site workload: site builds/s, both rooflines,
    the eager stage split, and (compare) the mixed path against the plain FP64 path on a seeded sample
    of sites, and (oracle_sites > 0) against the FP64 oracle on the smallest sites.  The mixed
    results of the sites in `keep_psi` (orbitals included) are returned for sampled oracle checks."""
    import torch
    o = wl.orbitals
    K = o.nk * o.nbands
    pmode = proj_mode(lrs, args)
    scr = lrs.Screening(0, args.precision, stream.cuda_stream)
    scr.load(o)
    scr.set_sites(wl.sites)
    scr.set_frequency_quadrature(wl.nfreq)
    scr.set_fft_grid(*wl.fft_grid)
    scr.set_option(lrs.LRS_OPT_GRAPH_PROJECTION, pmode)
    if args.dyson_lanes:
        scr.set_option(lrs.LRS_OPT_DYSON_LANES, args.dyson_lanes)
    if args.dyson_panel:
        scr.set_option(lrs.LRS_OPT_DYSON_PANEL, args.dyson_panel)
    tuned = None
    if args.precision != "fp64":
        scr.project(mode=pmode)
        tuned = scr.autotune()
    scr.graph_capture()
    scr.synchronize()
    for _ in range(warmup):
        scr.graph_launch()
    scr.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    torch.cuda.synchronize()
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        scr.graph_launch()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    scr.synchronize()   # raises if a device-side wait timed out during the replays
    ms = e0.elapsed_time(e1) / steps
    # stage split of one eager build (event-timed inside the library); its kernel count is the
    # count of one replay (the graph records the same launches)
    launches0 = scr.stats()["kernel_launches"]
    scr.project(mode=pmode)
    scr.build_chi0()
    scr.solve_w()
    st = scr.stats()
    launches_per_build = st["kernel_launches"] - launches0
    flop_chi0 = sum(8.0 * s.npts ** 2 * K * wl.nfreq for s in wl.sites)
    flop_all = sum(site_cost(s, K, wl.nfreq) for s in wl.sites)
    main_ms = st["ms_chi0_main"]
    pk = peaks["bf16_tflops_sustained"]
    roof = {"bound": "tensor", "achieved": flop_chi0 / (main_ms * 1e-3) / 1e12, "peak": pk, "unit": "TFLOP/s",
            "peak_source": f"bf16 sustained, {peaks['source']}",
            "issued_frac": 3 * flop_chi0 / (main_ms * 1e-3) / 1e12 / pk, "traffic": None,
            "traffic_source": "not captured for this workload",
            "kernel": "zgemm_tc_kernel<chi0> (all sites, one launch per workspace group)"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    # The update roofline comes from one more solve on a single Dyson lane: with several lanes the
    # updates of different sites overlap, and each launch's event interval then counts the time
    # it shares the SMs with another lane's update.
    lanes = args.dyson_lanes or 4
    st_w = st
    if lanes > 1:
        scr.set_option(lrs.LRS_OPT_DYSON_LANES, 1)
        scr.solve_w()
        st_w = scr.stats()
        scr.set_option(lrs.LRS_OPT_DYSON_LANES, lanes)
    st_w["dyson_update_tc"] = args.precision != "fp64"
    roof_w = dyson_roofline(st_w, args.workload, kernel_revision(lrs.lrs_version().decode(), "dyson-gj"),
                            peaks["hbm_gbs"], peaks["bf16_tflops"])
    if roof_w is not None:
        roof_w["timed_with_lanes"] = 1
        # the W stage of that solve (wall time on one lane) against the updates' share of it
        roof_w["w_stage_ms_one_lane"] = st_w["ms_w"]
        roof_w["update_ms_one_lane"] = st_w["ms_w_main"]
    dominant_w = roof_w is not None and st_w["ms_w_main"] > main_ms
    out = {"value": len(wl.sites) * 1e3 / ms, "unit": "site builds/s", "ms_per_step": ms, "steps": steps,
           "warmup": warmup, "tflops": flop_all / (ms * 1e-3) / 1e12, "autotuned": tuned,
           "dyson_lanes": lanes, "config": workload_config(args.workload, wl, args),
           "stage_ms_eager": {"project": st["ms_project"], "chi0": st["ms_chi0"], "chi0_main": main_ms,
                              "w": st["ms_w"]},
           "roofline": roof_w if dominant_w else roof,
           "roofline_chi0" if dominant_w else "roofline_dyson": roof if dominant_w else roof_w,
           "clocks": clocks, "device_bytes_peak": st["device_bytes_peak"],
           "gpu_launches": int(launches_per_build) * steps,
           "gpu_launches_note": "kernels of one eager build x replays (a replay launches the recorded kernels)"}
    mixed = {}
    for i in keep_psi:
        mixed[i] = (scr.get_chi0(i), scr.get_w(i), scr.get_v(i), scr.get_site_orbitals(i))
    if compare and args.precision != "fp64":
        rng = np.random.default_rng(5)
        order = sorted(range(len(wl.sites)), key=lambda i: wl.sites[i].npts)
        pick = sorted({order[0], order[-1], *rng.choice(order[1:-1], DYSON_SAMPLE_SITES - 2, replace=False)})
        for i in set(pick) | set(order[:oracle_sites]):
            mixed[i] = (scr.get_chi0(i), scr.get_w(i), scr.get_v(i))
        plain = gpu_path(lrs, "fp64", stream, wl, [wl.sites[i] for i in pick], pmode)
        ms_plain = timed_on(stream, lambda: (plain.build_chi0(), plain.solve_w()), 0, 1)
        cmp = {}
        for j, i in enumerate(pick):
            c, w, v = mixed[i]
            cmp[str(i)] = {"npts": wl.sites[i].npts,
                           **matrix_errors(c, w, v, plain.get_chi0(j), plain.get_w(j))}
        plain.close()
        t_mixed = st["ms_chi0"] + st["ms_w"]    # eager, all sites
        frac = sum(site_cost(wl.sites[i], K, wl.nfreq) for i in pick) / flop_all
        out["mixed_vs_fp64_plain"] = {
            "sites": cmp, "reference": "plain FP64 GPU path (chi0 on the FP64 pipe, Dyson with float64 FMAs)",
            "fp64_plain_ms_sample_chi0_w": ms_plain,
            "fp64_plain_site_builds_per_s_est": len(pick) / (ms_plain * 1e-3),
            "mixed_eager_site_builds_per_s": len(wl.sites) / (t_mixed * 1e-3),
            "note": f"plain FP64 timed on the sampled sites ({frac:.3f} of the workload's algorithmic flop)"}
    scr.close()
    return out, mixed


def run_multisite_line(args):
    """--workload batched-64-sites / large-cell-16-sites: one JSON line for the multi-site build."""
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2005_07834_gb300 import lrs
    t_gen = time.perf_counter()
    wl = make_workload(args.workload, args.nfreq, args.sites)
    t_gen = time.perf_counter() - t_gen
    o = wl.orbitals
    K = o.nk * o.nbands
    nsites_total = len(wl.sites)
    if world > 1:
        # sites are independent: each rank builds its own share (no data-path collective)
        from paper_2005_07834_gb300 import sharding
        mine = sharding.shard_sites(wl.sites, K, wl.nfreq, rank, world)
        wl = type(wl)(wl.name, o, [wl.sites[i] for i in mine], wl.nfreq, wl.fft_grid)
    stream = torch.cuda.Stream()
    peaks = load_peaks()
    if world > 1:
        torch.distributed.barrier()
    large = max(s.npts for s in wl.sites) * K > 2e7     # whole oracle or FP64 builds take minutes per site
    keep = (0, 1) if (large and rank == 0 and not args.no_cpu_baseline) else ()
    res, mixed = multisite_measure(args, lrs, wl, stream, args.steps, args.warmup, peaks,
                                   compare=(rank == 0 and not args.no_fp64_compare and not large),
                                   oracle_sites=0 if (args.no_cpu_baseline or large) else 2, keep_psi=keep)
    if large:
        res["mixed_vs_fp64_plain"] = ("not run: a plain FP64 build of one site is 8 N^2 K nf = %.0f TFLOP on the "
                                      "FP64 pipe; accuracy comes from the sampled oracle checks" % (
                                          8.0 * wl.sites[0].npts ** 2 * K * wl.nfreq / 1e12))
    backward = None
    if rank == 0 and not args.no_backward and large:
        one = lrs.Screening(0, args.precision, stream.cuda_stream)
        one.load(o)
        one.set_sites(wl.sites[:1])
        one.set_frequency_quadrature(wl.nfreq)
        one.set_fft_grid(*wl.fft_grid)
        one.project(mode=proj_mode(lrs, args))
        one.build_chi0()
        one.solve_w()
        backward = {"site": 0, **backward_leg(lrs, one, stream, wl.sites[0], K, wl.nfreq, peaks, args.precision)}
        one.close()
    ms = res["ms_per_step"]
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    if rank == 0:
        cpu, acc = None, None
        if not args.no_cpu_baseline and mixed and large:
            cpu, acc = oracle_sampled_sites_leg(wl, {i: mixed[i] for i in keep})
        elif not args.no_cpu_baseline and mixed:
            small = sorted(range(len(wl.sites)), key=lambda i: wl.sites[i].npts)[:2]
            cpu, acc = oracle_multisite_leg(wl, small, {i: mixed[i][:3] for i in small})
        line = {"metric": "site chi0+W builds/s", "value": nsites_total * 1e3 / ms, "unit": "site builds/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": DTYPE[args.precision], "precision": args.precision,
                "data": "synthetic (seeded generator; no DFT orbitals)", **{k: v for k, v in res.items()
                                                                              if k not in ("value", "ms_per_step",
                                                                                           "steps", "warmup")},
                "cpu_baseline": cpu, "accuracy_vs_oracle": acc, "e2e": None, "generation_s": t_gen,
                "backward": backward}
        print(json.dumps(strict_json(line), allow_nan=False), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def e2e_measure(lrs, torch, wl, pmode, precision, device, reps):
    """Site builds per second through the C-ABI from page-locked host buffers: every step loads the
    coefficients, energies, k-points and the site grid (host -> device), projects, builds chi0 and W
    and reads W back into host memory (device -> host).  Three contexts on three streams take the
    steps in turn, so that the next steps' host -> device copies and queued kernels overlap the
    current step's build (a caller with a stream of builds would do the same; a third build in
    flight fills the SMs that the Dyson stage's pivot chain leaves idle); the one-context figure
    without any overlap is reported beside it.  One untimed step per context first (allocations)."""
    import dataclasses
    o, s = wl.orbitals, wl.sites[0]
    h2d = o.coeff.nbytes + o.energies.nbytes + o.kpts.nbytes + o.kweights.nbytes + o.gvec.nbytes + \
        s.pts.nbytes + s.wts.nbytes
    d2h = s.npts * s.npts * 8

    def pinned(a):   # a page-locked host copy (made before the timed region)
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    o_host = dataclasses.replace(o, coeff=pinned(o.coeff), energies=pinned(o.energies), kpts=pinned(o.kpts),
                                 kweights=pinned(o.kweights), gvec=pinned(o.gvec))
    s_host = dataclasses.replace(s, pts=pinned(s.pts), wts=pinned(s.wts))
    nctx = 3
    w_host = [torch.empty((s.npts, s.npts), dtype=torch.float64, pin_memory=True).numpy() for _ in range(nctx)]
    streams = [torch.cuda.Stream() for _ in range(nctx)]
    ctxs = [lrs.Screening(device, precision, st.cuda_stream) for st in streams]

    def prepare(c):    # host -> device: coefficients, energies, k-points, site grid
        c.load(o_host)
        c.set_sites([s_host])
        c.set_frequency_quadrature(wl.nfreq)
        c.set_fft_grid(*wl.fft_grid)

    def launch(c):     # asynchronous on the context's stream
        c.project(mode=pmode)
        c.build_chi0()

    for i, c in enumerate(ctxs):   # untimed: first-use allocations
        prepare(c)
        launch(c)
        c.solve_w()
        c.get_w(0, out=w_host[i])
    torch.cuda.synchronize()
    # one context, no overlap
    t0 = time.perf_counter()
    for _ in range(reps):
        prepare(ctxs[0])
        launch(ctxs[0])
        ctxs[0].solve_w()
        ctxs[0].get_w(0, out=w_host[0])
    serial_s = (time.perf_counter() - t0) / reps
    # three contexts on three streams, one host thread: steps i + 1 and i + 2 have their inputs
    # copied and their projection, chi0 and Dyson solve queued (lrs_solve_w_async) while step i
    # runs; then step i's status is read (lrs_synchronize) and W copied back
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(min(nctx - 1, reps)):
        prepare(ctxs[i])
        launch(ctxs[i])
        ctxs[i].solve_w_async()
    for i in range(reps):
        c = ctxs[i % nctx]
        if i + nctx - 1 < reps:
            nxt = ctxs[(i + nctx - 1) % nctx]   # its previous step (i - 1) has been read back
            prepare(nxt)
            launch(nxt)
            nxt.solve_w_async()
        c.synchronize()
        c.get_w(0, out=w_host[i % nctx])
    e2e_s = (time.perf_counter() - t0) / reps
    for c in ctxs:
        c.close()
    return {"value": 1.0 / e2e_s, "unit": "builds/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "steps": reps, "contexts": nctx, "one_context_value": 1.0 / serial_s,
            "method": "page-locked host buffers; every step loads coefficients, energies, k-points and the site "
                      "grid and reads W back; three contexts on three streams take the steps in turn from one "
                      "host thread: the next two steps' inputs are copied and their projection, chi0 and Dyson "
                      "solve queued (lrs_solve_w_async) while the current step runs"}


def run_ours(args):
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2005_07834_gb300 import lrs

    wl = make_workload(args.workload, args.nfreq)
    o, s = wl.orbitals, wl.sites[0]
    stream = torch.cuda.Stream()
    scr = lrs.Screening(local, args.precision, stream.cuda_stream)
    scr.load(o)
    scr.set_sites([s])
    scr.set_frequency_quadrature(wl.nfreq)

    pmode = proj_mode(lrs, args)
    scr.set_fft_grid(*wl.fft_grid)
    if args.dyson_panel:
        scr.set_option(lrs.LRS_OPT_DYSON_PANEL, args.dyson_panel)

    def step():
        scr.project(mode=pmode)
        scr.build_chi0()
        scr.solve_w()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches0 = scr.stats()["kernel_launches"]
    sampler = ClockSampler(local)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    barrier()
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
        # per-stage device times are read after the timed region (events inside the library)
    e1.record(stream)
    barrier()
    clocks = sampler.stop()
    ms_total = e0.elapsed_time(e1)
    # stage times of the last timed step, event-timed inside the library on the same stream
    st = scr.stats()
    launches = st["kernel_launches"] - launches0
    ms = ms_total / args.steps
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    value = world * 1e3 / ms

    # end to end through the C-ABI with host buffers
    e2e = None
    if rank == 0 and not args.no_e2e:
        e2e = e2e_measure(lrs, torch, wl, pmode, args.precision, local,
                          reps=1 if args.precision == "fp64" else max(3, min(2 * args.steps, 20)))

    peaks = load_peaks()
    n, K, nf = s.npts, o.nk * o.nbands, wl.nfreq
    real = bool(scr.orbitals_are_real())
    # complex x complex products: 8 flop per multiply-add; Gamma-point real orbitals make B real (4)
    # and each frequency's product symmetric, so that its lower triangle (half) is the work
    flop_chi0 = (2.0 if real else 8.0) * n * n * K * nf
    # share of the square's 128-row tiles the kernel issues: those reaching the lower triangle
    t_rows = -(-n // 128)
    issued_share = (t_rows + 1) / (2.0 * t_rows) if real else 1.0
    main_ms = st["ms_chi0_main"]
    if args.precision == "fp64":
        roof = {"bound": "alu", "achieved": flop_chi0 / (main_ms * 1e-3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "peak_source": "FP64 FMA rate: 152 SMs x 2 DFMA/clk x 2.07 GHz"}
    else:
        pk = peaks["bf16_tflops_sustained"]
        roof = {"bound": "tensor", "achieved": flop_chi0 / (main_ms * 1e-3) / 1e12, "peak": pk,
                "unit": "TFLOP/s", "peak_source": f"bf16 sustained, {peaks['source']}",
                "issued_frac": 3 * flop_chi0 / (0.5 if real else 1.0) * issued_share / (main_ms * 1e-3) / 1e12 / pk}
        if clocks.get("sm_mhz") and peaks.get("clocks_under_load", {}).get("sm_mhz_median"):
            # the sustained peak was taken at the clock the driver saw under its GEMM loop; the burst
            # peak scaled to this run's median SM clock is the tighter denominator when they differ
            burst_here = peaks["bf16_tflops"] * clocks["sm_mhz"] / peaks.get("sm_max_mhz", 2070.0)
            roof["frac_of_burst_at_sampled_clock"] = roof["achieved"] / burst_here
    roof["frac"] = roof["achieved"] / roof["peak"]
    version = lrs.lrs_version().decode()
    rev = kernel_revision(version, "chi0-tc")
    roof["traffic"] = CHI0_TRAFFIC.get((args.workload, args.precision, rev))
    roof["traffic_source"] = (f"stored ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch of kernel "
                              f"revision chi0-tc {rev}" if roof["traffic"] else
                              "no ncu capture of this kernel revision on this workload")
    roof["kernel"] = "chi0_fp64_kernel" if args.precision == "fp64" else "zgemm_tc_kernel<chi0>"
    roof["library"] = version
    # the SPD inverse's trailing update (one launch per pivot block), timed per launch with CUDA
    # events on its stream inside the library
    st["dyson_update_tc"] = args.precision != "fp64"   # LRS_UPDATE_AUTO: tensor cores in the mixed precisions
    roof_w = dyson_roofline(st, args.workload, kernel_revision(version, "dyson-gj"), peaks["hbm_gbs"],
                            peaks["bf16_tflops"])
    dominant_w = roof_w is not None and st["ms_w_main"] > main_ms

    chi_mixed, w_mixed, v_lib = scr.get_chi0(0), scr.get_w(0), scr.get_v(0)
    # the plain FP64 path on the same workload, one step (for "mixed vs FP64 plain")
    plain, results = None, {("mixed" if args.precision != "fp64" else "fp64"): (chi_mixed, w_mixed, v_lib)}
    if rank == 0 and args.precision != "fp64" and not args.no_fp64_compare:
        scr3 = lrs.Screening(local, "fp64", stream.cuda_stream)
        scr3.load(o)
        scr3.set_sites([s])
        scr3.set_frequency_quadrature(wl.nfreq)
        scr3.set_fft_grid(*wl.fft_grid)
        torch.cuda.synchronize()
        plain_ms = timed_on(stream, lambda: (scr3.project(mode=pmode), scr3.build_chi0(), scr3.solve_w()), 0, 1)
        st3 = scr3.stats()
        chi_plain, w_plain = scr3.get_chi0(0), scr3.get_w(0)
        scr3.close()
        results["fp64"] = (chi_plain, w_plain, v_lib)
        plain = {"builds_per_s": 1e3 / plain_ms, "ms_per_step": plain_ms,
                 "stage_ms": {"project": st3["ms_project"], "chi0": st3["ms_chi0"], "w": st3["ms_w"]},
                 "mixed_vs_plain_speedup": plain_ms / ms,
                 "mixed_vs_plain": {"chi0": errors(chi_mixed, chi_plain), "w": errors(w_mixed, w_plain),
                                    "w_minus_v": errors(w_mixed - v_lib, w_plain - v_lib)}}

    backward, config1 = None, None
    if rank == 0 and not args.no_backward:
        backward = {"workload": args.workload, "precision": args.precision,
                    **backward_leg(lrs, scr, stream, s, K, nf, peaks, args.precision, real)}
        backward["differentiation_260"], config1 = config4_backward(lrs, stream)
    scr.close()

    workloads = None
    if rank == 0 and args.workloads:
        workloads = {}
        for name in args.workloads.split(","):
            sub = argparse.Namespace(**{**vars(args), "workload": name})
            wl2 = make_workload(name)
            res, mixed = multisite_measure(sub, lrs, wl2, stream, 5, 2, peaks, compare=True,
                                           oracle_sites=0 if args.no_cpu_baseline else 2)
            if not args.no_cpu_baseline and mixed:
                small = sorted(range(len(wl2.sites)), key=lambda i: wl2.sites[i].npts)[:2]
                res["cpu_baseline"], res["accuracy_vs_oracle"] = oracle_multisite_leg(wl2, small, mixed)
            workloads[name] = res

    if rank == 0:
        cpu, acc = None, None
        if not args.no_cpu_baseline:
            cpu, acc = oracle_single_site_leg(wl, results, config1)
        line = {
            "metric": "site chi0+W builds/s", "value": value, "unit": "builds/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision], "precision": args.precision,
            "data": "synthetic (seeded generator; no DFT orbitals)",
            "config": workload_config(args.workload, wl, args),
            "tflops": (flop_chi0 + 14.0 / 3.0 * n ** 3) / (ms * 1e-3) / 1e12,
            "stage_ms": {"project": st["ms_project"], "chi0": st["ms_chi0"], "chi0_main": main_ms,
                         "w": st["ms_w"]},
            "roofline": roof_w if dominant_w else roof,
            "roofline_chi0" if dominant_w else "roofline_dyson": roof if dominant_w else roof_w,
            "dyson_stage": {"ms": st["ms_w"], "flop_executed": st["flop_w_executed"],
                            "tflops_executed": st["flop_w_executed"] / (st["ms_w"] * 1e-3) / 1e12,
                            "frac_fp64_peak": st["flop_w_executed"] / (st["ms_w"] * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                            "flop_full_grid_formula": st["flop_w"]},
            "cpu_baseline": cpu, "accuracy_vs_oracle": acc, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clocks, "device_bytes_peak": st["device_bytes_peak"], "plain_fp64": plain,
            "backward": backward, "workloads": workloads,
        }
        print(json.dumps(strict_json(line), allow_nan=False), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def site_cost(s, K, nf):
    """Algorithmic flop of one site build: 8 N^2 K nf (chi0) + 14/3 N^3 (Dyson)."""
    n = s.npts
    return 8.0 * n * n * K * nf + 14.0 / 3.0 * n ** 3


def run_rows(args):
    """One JSON line per next-row operation on the 3520-point site (bf16x3 context unless
    --precision says otherwise): device time by CUDA events around the call on the
    library's stream (median of --steps after --warmup), algorithmic work, roofline."""
    import torch
    from paper_2005_07834_gb300 import lrs, synth
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    peaks = load_peaks()
    wl = synth.single_site_3520()
    o, s = wl.orbitals, wl.sites[0]
    n, K, nf = s.npts, o.nk * o.nbands, wl.nfreq

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        ms = []
        for _ in range(max(1, args.steps)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return float(np.median(ms))

    def line(row, what, ms, work, unit, bound, peak, peak_source, extra=None):
        d = {"row": row, "operation": what, "workload": "single-site-3520", "precision": args.precision,
             "ms": ms, "unit": unit, "achieved": work / (ms * 1e-3) / (1e9 if unit == "GB/s" else 1e12),
             "bound": bound, "peak": peak, "peak_source": peak_source}
        d["frac"] = d["achieved"] / peak
        d.update(extra or {})
        print(json.dumps(strict_json(d), allow_nan=False), flush=True)

    scr = lrs.Screening(0, args.precision, stream.cuda_stream)
    scr.load(o)
    scr.set_sites([s])
    scr.set_frequency_quadrature(nf)
    scr.set_fft_grid(*wl.fft_grid)
    hbm = peaks["hbm_gbs"]
    # f1: FFT + cubic Lagrange projection; HBM-bound: per k the grid is written once by the z pass,
    # read and written by the y and x passes, read by the gather (4 passes over N^3 nb complex64)
    ms = timed(lambda: scr.project(mode=lrs.LRS_PROJ_FFT_LAGRANGE3))
    n3 = int(np.prod(wl.fft_grid))
    elem = 8 if args.precision != "fp64" else 16
    byt = o.nk * (n3 * o.nbands * elem * 5 + o.ng * o.nbands * 16) + n * K * 16
    line("f1", "project FFT 48^3 + Lagrange", ms, byt, "GB/s", "hbm", hbm, "copy, measured",
         {"bytes_model": "per k: 5 grid passes N^3 nb complex + coefficients; psi written"})
    ms_exact = timed(lambda: scr.project(mode=lrs.LRS_PROJ_EXACT))
    line("a2", "project exact (tensor cores)", ms_exact, 8.0 * n * o.ng * K, "TFLOP/s", "tensor",
         peaks["bf16_tflops"], "bf16 burst, measured", {"note": "3 products issued per algorithmic product"})
    scr.build_chi0()
    s_lmax, nrad, nang = s.lmax, s.nrad, s.nang
    # f2: induced response; FP64 work = projection of chi0 onto Y_lm (2 n^2 (l+1)^2) + the solve
    for lresp in (0, s_lmax):
        l2 = (lresp + 1) ** 2
        d = nrad * l2
        ms = timed(lambda: scr.induced_potential(0, -1.0, 1.5, lresp))
        flop = 2.0 * n * n * l2 + 2.0 * l2 * d * n + 2.0 / 3.0 * d ** 3 + 2.0 * d * d * nrad
        line("f2", f"induced potential l_resp={lresp}", ms, flop, "TFLOP/s", "alu", FP64_PEAK_TFLOPS,
             "FP64 FMA rate: 152 SMs x 2 DFMA/clk x 2.07 GHz", {"note": "synchronous call incl. host copies"})
    # f3: ALDA dressing chi_eff = (I - chi0 D)^-1 chi0 (LU + n right-hand sides): 8/3 n^3
    scr.set_fxc(0, lrs.LRS_FXC_ALDA_X)
    ms_w_alda = timed(lambda: scr.solve_w())
    st = scr.stats()
    scr.set_fxc(0, lrs.LRS_FXC_NONE)
    ms_w = timed(lambda: scr.solve_w())
    line("f3", "ALDA dressing (solve_w with kernel minus RPA solve_w)", ms_w_alda - ms_w, 8.0 / 3.0 * n ** 3,
         "TFLOP/s", "alu", FP64_PEAK_TFLOPS, "FP64 FMA rate: 152 SMs x 2 DFMA/clk x 2.07 GHz",
         {"ms_solve_w_alda": ms_w_alda, "ms_solve_w_rpa": ms_w})
    # f4: augmentation, l <= 2, two partial waves per l: 2 x (projection + update) = 16 n nproj K flop
    radii = np.linalg.norm(s.pts[::nang], axis=1)
    ps = np.array([[radii ** l * np.exp(-a * radii ** 2) for a in (0.5, 1.1)] for l in range(3)])
    bump = np.where(radii < 2.0, np.sin(np.pi * radii / 2.0) ** 2, 0.0)
    ae = ps + 0.1 * bump[None, None, :]
    ms = timed(lambda: scr.augment(0, ae, ps, 2.0))
    nproj = 9 * 2
    n_in = int(np.sum(radii <= 2.0)) * nang     # points on the shells inside the augmentation radius
    # projection and update: a real weight times a complex orbital, 4 flop each, over the inside points
    line("f4", "augmentation (9 lm x 2 partial waves, r_a = 2)", ms, 8.0 * n_in * nproj * K, "TFLOP/s", "alu",
         FP64_PEAK_TFLOPS, "FP64 FMA rate: 152 SMs x 2 DFMA/clk x 2.07 GHz",
         {"points_inside": n_in, "note": "synchronous call incl. host setup of the overlaps"})
    scr.close()
    # f1': Gamma-point real orbitals: chi0 with the real-operand contraction on the lower triangle
    # (2 n^2 K nf flop: each frequency's product is symmetric)
    wg = synth.gamma_site_3520()
    sg = lrs.Screening(0, args.precision, stream.cuda_stream)
    sg.load(wg.orbitals)
    sg.set_sites(wg.sites)
    sg.set_frequency_quadrature(wg.nfreq)
    sg.project()
    ms = timed(lambda: sg.build_chi0())
    st = sg.stats()
    t_rows = -(-n // 128)
    line("f1-gamma", "chi0, Gamma-point real orbitals", st["ms_chi0_main"], 2.0 * n * n * K * wg.nfreq, "TFLOP/s",
         "tensor", peaks["bf16_tflops_sustained"], "bf16 sustained, measured",
         {"ms_build_chi0": ms, "issued_frac": 3 * 4.0 * n * n * K * wg.nfreq * (t_rows + 1) / (2.0 * t_rows)
          / (st["ms_chi0_main"] * 1e-3) / 1e12 / peaks["bf16_tflops_sustained"]})
    sg.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=["fp64", "bf16x3", "fp16x3"])
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip the one-step timing of the plain FP64 path on the same workload")
    ap.add_argument("--workload", default="single-site-3520", choices=sorted(WORKLOADS))
    ap.add_argument("--projection", default="exact", choices=["exact", "fft"],
                    help="Sec. VI.B method 1 (direct sum) or method 2 (FFT + cubic Lagrange on the workload's grid)")
    ap.add_argument("--dyson-lanes", type=int, default=0,
                    help="concurrent Dyson solves of the multi-site workloads (0: the library default)")
    ap.add_argument("--dyson-panel", type=int, default=0, choices=[0, 32, 128],
                    help="pivot-block width of the lm-basis SPD inverse (0: the library default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-backward", action="store_true",
                    help="skip the adjoint timings (this workload and the 260-point differentiation case)")
    ap.add_argument("--sites", type=lambda t: [int(x) for x in t.split(",") if x], default=None,
                    help="comma-separated site indices: build only these sites of a multi-site workload "
                         "(profiler captures; not a bench line of the named workload)")
    ap.add_argument("--nfreq", type=int, default=0,
                    help="replace the workload's frequency count (0: keep it); for small profiler captures only")
    ap.add_argument("--workloads", default="batched-64-sites",
                    help="comma-separated multi-site workloads measured after a single-site run and reported "
                         "in its `workloads` object ('' for none)")
    ap.add_argument("--rows", action="store_true",
                    help="time each next-row operation (FFT projection, induced response, ALDA, augmentation, "
                         "Gamma point) on the 3520-point site instead of the build")
    args = ap.parse_args()
    if args.rows:
        run_rows(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload in MULTI_SITE:
        run_multisite_line(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
