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

--impl reference times the FP64 CPU oracle on the host cores instead (rank 0
only), on a bounded sample of the same workload.
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
CHI0_TRAFFIC = {("single-site-3520", "bf16x3", "r1"): 23.26e9}


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
                 ("single-site-3520", "r4"): 28.52e6}


def dyson_roofline(st, workload=None, version=None, hbm_gbs=None):
    """The SPD inverse's trailing update.  On the FP64 pipe (FP64 context) it is bound by the
    FP64 FMA rate.  On the tensor cores its float64 work is one subtraction per element and its
    algorithmic traffic one read and one write of each updated element of C (16 bytes; the
    library counts 2 kb flop per updated element, kb = 32), so it is reported against the HBM
    copy bandwidth, with the FP64-equivalent rate beside it."""
    if not st.get("w_main_launches"):
        return None
    ms = st["ms_w_main"]
    tc = st.get("dyson_update_tc", False)
    fp64_eq = st["flop_w_main"] / (ms * 1e-3) / 1e12
    common = {"launches": st["w_main_launches"], "avg_launch_us": 1e3 * ms / st["w_main_launches"],
              "traffic": DYSON_TRAFFIC.get((workload, version))}
    if tc and hbm_gbs:
        algo_bytes = st["flop_w_main"] / (2.0 * 32) * 16.0
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


def make_workload(name):
    from paper_2005_07834_gb300 import synth
    return getattr(synth, WORKLOADS[name])()


# ----------------------------------------------------------------------------- reference arm

def oracle_build_sample(wl, kfrac_k=1, nfreq_sample=2):
    """Times the FP64 oracle on one site: projection on `kfrac_k` of the k-points,
    chi0 by the Green's-function route on `nfreq_sample` of the frequencies, and
    the full Dyson solve; returns the time of one whole build scaled from it."""
    from oracle import chi0 as ochi0, coulomb as ocoul, dyson as odys, projection as oproj, quadrature as oquad
    o, s = wl.orbitals, wl.sites[0]
    t0 = time.perf_counter()
    psi_k = oproj.project_direct(o.cell, o.kpts[:kfrac_k], o.gvec, o.coeff[:kfrac_k], s.center, s.pts)
    t_proj = (time.perf_counter() - t0) * o.nk / kfrac_k
    # orbitals of the remaining k-points are not timed: reuse the sampled ones
    psi = np.concatenate([psi_k] * (o.nk // kfrac_k), axis=1)
    po, pu, eo, eu, wo, wu = oproj.split_occupied(psi, o.energies, o.nocc, o.kweights)
    mu = oquad.chemical_potential_midgap(o.energies, o.nocc)
    t, W = oquad.frequency_grid(wl.nfreq, oquad.zeta_rule(o.energies, mu))
    t0 = time.perf_counter()
    chi = ochi0.chi0_green(po, pu, eo, eu, wo, wu, mu, t[:nfreq_sample], W[:nfreq_sample])
    t_chi = (time.perf_counter() - t0) * wl.nfreq / nfreq_sample
    t0 = time.perf_counter()
    v = ocoul.coulomb_multipole(s.pts, s.lmax)
    odys.screened_interaction(v, chi, s.wts)
    t_w = time.perf_counter() - t0
    return t_proj + t_chi + t_w, {"t_project_s": t_proj, "t_chi0_s": t_chi, "t_w_s": t_w}


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    wl = make_workload(args.workload)
    cores = os.cpu_count()
    sample = (f"one site of {args.workload}: projection timed on 1 of {wl.orbitals.nk} k-points, chi0 "
              f"(Green's-function route) on 2 of {wl.nfreq} frequencies, full Dyson LU; scaled to one build")
    for _ in range(args.warmup if args.warmup < 1 else 1):
        oracle_build_sample(wl)
    times = []
    parts = None
    for _ in range(args.steps):
        t, parts = oracle_build_sample(wl)
        times.append(t)
    ms = 1e3 * statistics.mean(times)
    value = 1e3 / ms
    line = {"impl": "reference", "metric": "site chi0+W builds/s", "value": value, "unit": "builds/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded generator)",
            "config": {"workload": args.workload, "precision": "fp64-oracle-cpu"},
            "cpu_baseline": {"value": value, "unit": "builds/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "builds/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "parts_s": parts}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2005_07834_gb300 import lrs

    wl = make_workload(args.workload)
    o, s = wl.orbitals, wl.sites[0]
    stream = torch.cuda.Stream()
    scr = lrs.Screening(local, args.precision, stream.cuda_stream)
    scr.load(o)
    scr.set_sites([s])
    scr.set_frequency_quadrature(wl.nfreq)

    pmode = proj_mode(lrs, args)
    scr.set_fft_grid(*wl.fft_grid)

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

    chi_main_ms, chi_ms, w_ms, proj_ms = [], [], [], []
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
        scr2 = lrs.Screening(local, args.precision, stream.cuda_stream)
        h2d = o.coeff.nbytes + o.energies.nbytes + o.kpts.nbytes + o.kweights.nbytes + o.gvec.nbytes + \
            s.pts.nbytes + s.wts.nbytes
        d2h = s.npts * s.npts * 8
        reps = 1 if args.precision == "fp64" else max(1, min(args.steps, 3))

        def pinned(a):   # a page-locked host copy (made before the timed region)
            return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        import dataclasses
        o_host = dataclasses.replace(o, coeff=pinned(o.coeff), energies=pinned(o.energies), kpts=pinned(o.kpts),
                                     kweights=pinned(o.kweights), gvec=pinned(o.gvec))
        s_host = dataclasses.replace(s, pts=pinned(s.pts), wts=pinned(s.wts))
        w_host = torch.empty((s.npts, s.npts), dtype=torch.float64, pin_memory=True).numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            scr2.load(o_host)
            scr2.set_sites([s_host])
            scr2.set_frequency_quadrature(wl.nfreq)
            scr2.set_fft_grid(*wl.fft_grid)
            scr2.project(mode=pmode)
            scr2.build_chi0()
            scr2.solve_w()
            scr2.get_w(0, out=w_host)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / reps
        scr2.close()
        e2e = {"value": 1.0 / e2e_s, "unit": "builds/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    peaks = load_peaks()
    n, K, nf = s.npts, o.nk * o.nbands, wl.nfreq
    # complex x complex products: 8 flop per multiply-add; Gamma-point real orbitals make B real (4)
    flop_chi0 = (4.0 if scr.orbitals_are_real() else 8.0) * n * n * K * nf
    main_ms = st["ms_chi0_main"]
    if args.precision == "fp64":
        roof = {"bound": "alu", "achieved": flop_chi0 / (main_ms * 1e-3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "peak_source": "FP64 FMA rate: 152 SMs x 2 DFMA/clk x 2.07 GHz"}
    else:
        pk = peaks["bf16_tflops_sustained"]
        roof = {"bound": "tensor", "achieved": flop_chi0 / (main_ms * 1e-3) / 1e12, "peak": pk,
                "unit": "TFLOP/s", "peak_source": f"bf16 sustained, {peaks['source']}",
                "issued_frac": 3 * flop_chi0 / (main_ms * 1e-3) / 1e12 / pk}
    roof["frac"] = roof["achieved"] / roof["peak"]
    version = lrs.lrs_version().decode()
    roof["traffic"] = CHI0_TRAFFIC.get((args.workload, args.precision, kernel_revision(version, "chi0-tc")))
    roof["kernel"] = "chi0_fp64_kernel" if args.precision == "fp64" else "zgemm_tc_kernel<chi0>"
    roof["library"] = version
    # FP64 Dyson: its dominant kernel is the trailing update of the SPD inverse (one launch per
    # pivot block), timed per launch with CUDA events on its stream inside the library; algorithmic
    # flop per launch = 2 kb x the lower-triangle elements it updates
    st["dyson_update_tc"] = args.precision != "fp64"   # LRS_UPDATE_AUTO: tensor cores in the mixed precisions
    roof_w = dyson_roofline(st, args.workload, kernel_revision(version, "dyson-gj"), peaks["hbm_gbs"])
    # the roofline object describes the kernel that dominates the step; the other is kept beside it
    dominant_w = roof_w is not None and st["ms_w_main"] > main_ms

    # the plain FP64 path on the same workload, one untimed-warm step (for "mixed vs FP64 plain")
    plain = None
    if rank == 0 and args.precision != "fp64" and not args.no_fp64_compare:
        scr3 = lrs.Screening(local, "fp64", stream.cuda_stream)
        scr3.load(o)
        scr3.set_sites([s])
        scr3.set_frequency_quadrature(wl.nfreq)
        torch.cuda.synchronize()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        scr3.set_fft_grid(*wl.fft_grid)
        scr3.project(mode=pmode)
        scr3.build_chi0()
        scr3.solve_w()
        p1.record(stream)
        torch.cuda.synchronize()
        st3 = scr3.stats()
        plain_ms = p0.elapsed_time(p1)
        chi_plain, w_plain = scr3.get_chi0(0), scr3.get_w(0)
        scr3.close()
        chi_mixed, w_mixed = scr.get_chi0(0), scr.get_w(0)
        plain = {"builds_per_s": 1e3 / plain_ms, "ms_per_step": plain_ms,
                 "stage_ms": {"project": st3["ms_project"], "chi0": st3["ms_chi0"], "w": st3["ms_w"]},
                 "mixed_vs_plain_speedup": plain_ms / ms,
                 "mixed_rel_err_chi0": float(np.linalg.norm(chi_mixed - chi_plain) / np.linalg.norm(chi_plain)),
                 "mixed_rel_err_w": float(np.linalg.norm(w_mixed - w_plain) / np.linalg.norm(w_plain))}

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            t_cpu, parts = oracle_build_sample(wl)
            cpu = {"value": 1.0 / t_cpu, "unit": "builds/s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"one site: projection on 1 of {o.nk} k-points, chi0 (Green's-function route) on 2 "
                             f"of {nf} frequencies, full Dyson LU; scaled to one build", "parts_s": parts}
        line = {
            "metric": "site chi0+W builds/s", "value": value, "unit": "builds/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "bf16x3": "bf16x3/f32acc/f64", "fp16x3": "fp16x3/f32acc/f64"}[args.precision],
            "data": "synthetic (seeded generator; no DFT orbitals)",
            "config": {"workload": args.workload, "npts": n, "K": K, "nfreq": nf, "ng": o.ng,
                       "precision": args.precision, "replicas_per_gpu": 1, "projection": args.projection,
                       "real_orbitals": bool(scr.orbitals_are_real()),
                       "l2": "inputs larger than L2 (coefficients %d MB, orbitals %d MB)" % (
                           o.coeff.nbytes >> 20, (n * K * 16) >> 20)},
            "tflops": (flop_chi0 + 14.0 / 3.0 * n ** 3) / (ms * 1e-3) / 1e12,
            "stage_ms": {"project": st["ms_project"], "chi0": st["ms_chi0"], "chi0_main": main_ms,
                         "w": st["ms_w"]},
            "roofline": roof_w if dominant_w else roof,
            "roofline_chi0" if dominant_w else "roofline_dyson": roof if dominant_w else roof_w,
            "dyson_stage": {"ms": st["ms_w"], "flop_executed": st["flop_w_executed"],
                            "tflops_executed": st["flop_w_executed"] / (st["ms_w"] * 1e-3) / 1e12,
                            "frac_fp64_peak": st["flop_w_executed"] / (st["ms_w"] * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                            "flop_full_grid_formula": st["flop_w"]},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clocks, "device_bytes_peak": st["device_bytes_peak"], "plain_fp64": plain,
        }
        print(json.dumps(line), flush=True)
    scr.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def site_cost(s, K, nf):
    """Algorithmic flop of one site build: 8 N^2 K nf (chi0) + 14/3 N^3 (Dyson)."""
    n = s.npts
    return 8.0 * n * n * K * nf + 14.0 / 3.0 * n ** 3


def run_ours_multisite(args):
    """All sites of the workload per step: one CUDA-graph replay of projection,
    chi0 (one persistent tensor-core launch over every site) and the Dyson solves."""
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2005_07834_gb300 import lrs

    t_gen = time.perf_counter()
    wl = make_workload(args.workload)
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
    scr = lrs.Screening(local, args.precision, stream.cuda_stream)
    scr.load(o)
    scr.set_sites(wl.sites)
    scr.set_frequency_quadrature(wl.nfreq)
    tuned = None
    pmode = proj_mode(lrs, args)
    scr.set_fft_grid(*wl.fft_grid)
    scr.set_option(lrs.LRS_OPT_GRAPH_PROJECTION, pmode)
    if args.dyson_lanes:
        scr.set_option(lrs.LRS_OPT_DYSON_LANES, args.dyson_lanes)
    if args.precision != "fp64":
        scr.project(mode=pmode)
        tuned = scr.autotune()
    scr.graph_capture()
    scr.synchronize()
    for _ in range(args.warmup):
        scr.graph_launch()
    scr.synchronize()
    sampler = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        scr.graph_launch()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    scr.synchronize()   # raises if a device-side wait timed out during the replays
    ms = e0.elapsed_time(e1) / args.steps
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    nsites = len(wl.sites)
    value = nsites_total * 1e3 / ms
    # stage split of one eager build (event-timed inside the library)
    scr.project(mode=pmode)
    scr.build_chi0()
    scr.solve_w()
    st = scr.stats()
    flop_chi0 = sum(8.0 * s.npts ** 2 * K * wl.nfreq for s in wl.sites)
    flop_all = sum(site_cost(s, K, wl.nfreq) for s in wl.sites)
    peaks = load_peaks()
    main_ms = st["ms_chi0_main"]
    pk = peaks["bf16_tflops_sustained"]
    roof = {"bound": "tensor", "achieved": flop_chi0 / (main_ms * 1e-3) / 1e12, "peak": pk, "unit": "TFLOP/s",
            "peak_source": f"bf16 sustained, {peaks['source']}",
            "issued_frac": 3 * flop_chi0 / (main_ms * 1e-3) / 1e12 / pk, "traffic": None,
            "kernel": "zgemm_tc_kernel<chi0> (all sites, one launch per workspace group)"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    st["dyson_update_tc"] = args.precision != "fp64"
    roof_w = dyson_roofline(st, args.workload, kernel_revision(lrs.lrs_version().decode(), "dyson-gj"), peaks["hbm_gbs"])
    dominant_w = roof_w is not None and st["ms_w_main"] > main_ms
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            # the oracle on the smallest site, scaled to all sites by the algorithmic cost
            small = min(range(nsites), key=lambda i: wl.sites[i].npts)
            sub = type(wl)(wl.name, o, [wl.sites[small]], wl.nfreq)
            t_cpu, parts = oracle_build_sample(sub)
            scale = flop_all / site_cost(wl.sites[small], K, wl.nfreq)
            cpu = {"value": nsites / (t_cpu * scale), "unit": "site builds/s", "cores": os.cpu_count(),
                   "kind": "oracle",
                   "sample": f"site {small} ({wl.sites[small].npts} points): projection on 1 of {o.nk} k-points, "
                             f"chi0 on 2 of {wl.nfreq} frequencies, full LU; scaled to all {nsites} sites by "
                             "8 N^2 K nf + 14/3 N^3", "parts_s": parts}
        sizes = [s.npts for s in wl.sites]
        line = {
            "metric": "site chi0+W builds/s", "value": value, "unit": "site builds/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "bf16x3": "bf16x3/f32acc/f64", "fp16x3": "fp16x3/f32acc/f64"}[args.precision],
            "data": "synthetic (seeded generator; no DFT orbitals)",
            "config": {"workload": args.workload, "sites": nsites, "npts_min": min(sizes), "npts_max": max(sizes),
                       "npts_sum": sum(sizes), "K": K, "nfreq": wl.nfreq, "ng": o.ng, "precision": args.precision,
                       "projection": args.projection,
                       "graph": "one CUDA graph replay per step", "autotuned": tuned,
                       "dyson_lanes": args.dyson_lanes or 2,
                       "l2": "inputs larger than L2"},
            "tflops": flop_all / (ms * 1e-3) / 1e12,
            "stage_ms_eager": {"project": st["ms_project"], "chi0": st["ms_chi0"], "chi0_main": main_ms,
                               "w": st["ms_w"]},
            "roofline": roof_w if dominant_w else roof,
            "roofline_chi0" if dominant_w else "roofline_dyson": roof if dominant_w else roof_w,
            "cpu_baseline": cpu, "e2e": None, "gpu_launches": None, "clocks": clocks,
            "device_bytes_peak": st["device_bytes_peak"], "generation_s": t_gen,
        }
        print(json.dumps(line), flush=True)
    scr.close()
    if world > 1:
        torch.distributed.destroy_process_group()


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
        print(json.dumps(d), flush=True)

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
    # f1': Gamma-point real orbitals: chi0 with the real-operand contraction (4 n^2 K nf flop)
    wg = synth.gamma_site_3520()
    sg = lrs.Screening(0, args.precision, stream.cuda_stream)
    sg.load(wg.orbitals)
    sg.set_sites(wg.sites)
    sg.set_frequency_quadrature(wg.nfreq)
    sg.project()
    ms = timed(lambda: sg.build_chi0())
    st = sg.stats()
    line("f1-gamma", "chi0, Gamma-point real orbitals", st["ms_chi0_main"], 4.0 * n * n * K * wg.nfreq, "TFLOP/s",
         "tensor", peaks["bf16_tflops_sustained"], "bf16 sustained, measured",
         {"ms_build_chi0": ms, "issued_frac": 3 * 4.0 * n * n * K * wg.nfreq / (st["ms_chi0_main"] * 1e-3) / 1e12
          / peaks["bf16_tflops_sustained"]})
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
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--rows", action="store_true",
                    help="time each next-row operation (FFT projection, induced response, ALDA, augmentation, "
                         "Gamma point) on the 3520-point site instead of the build")
    args = ap.parse_args()
    if args.rows:
        run_rows(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload in MULTI_SITE:
        run_ours_multisite(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
