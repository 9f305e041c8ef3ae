#!/usr/bin/env python
"""Benchmark: ms per spin-2 synthesis + analysis pair at lmax 4095.

Workload (the configuration the headline metric is quoted on): Gauss-Legendre
grid nlat = 4096, nlon = 8191 (prime ring length), lmax = mmax = 4095, spin 2,
one (E, B) pair with C_l = 1/(l+1)^2 and zero monopole/dipole, seed 2.  One
step = one synthesis (E, B -> Q, U) followed by one analysis (Q, U -> E, B)
through the C ABI, inputs resident in HBM.  Inputs (268 MB of a_lm, 537 MB
of maps) are larger than L2 (129 MB), so no flush is needed between steps.

Reported:
  value / ms_per_step  device time per pair (CUDA events, max over ranks)
  forms                both the mixed form and the plain FP64 form
  roofline             dominant Legendre kernel: the method's algorithmic flops
                       (26 per triple at spin 2) / its event-timed duration,
                       against the FMA-flop peak of the pipe it runs on; the
                       double-float issue fraction beside it (issue_frac)
  e2e                  same pair through the public API from pinned host a_lm,
                       host<->device copies inside the timed region
  cpu_baseline         the FP64 CPU oracle on a bounded sample, host cores
  accuracy             GPU results against the oracle on that sample

--impl reference runs the oracle (the reference for this build) instead.
Multi-GPU: replicas only (one independent transform pair per rank).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SPIN, SEED = 2, 2
LMAX = NLAT = NLON = METRIC = CONFIG = None
SMS = 152


def set_workload(lmax, nlat=None):
    """GL nlat = lmax + 1, nlon = 2 lmax + 1; lmax 4095 is the headline configuration.
    A smaller nlat (profiling captures: the same rings, fewer of them) is not exact
    quadrature and not a headline configuration."""
    global LMAX, NLAT, NLON, METRIC, CONFIG
    LMAX, NLAT, NLON = lmax, nlat or lmax + 1, 2 * lmax + 1
    METRIC = f"ms per synth+analysis at lmax {LMAX} (spin 2, GL {NLAT}x{NLON})"
    nalm = (LMAX + 1) * (LMAX + 2) // 2
    big = 16 * 2 * nalm > 129e6 and 8 * 2 * NLAT * NLON > 129e6
    CONFIG = {"workload": f"spin-2 synthesis+analysis, Gauss-Legendre nlat={NLAT} nlon={NLON}, "
                          f"lmax=mmax={LMAX}, E/B a_lm C_l=1/(l+1)^2 seed 2",
              "lmax": LMAX, "nlat": NLAT, "nlon": NLON, "spin": SPIN, "ncomp": 1,
              "l2_policy": ("inputs larger than L2 (%.0f MB a_lm, %.0f MB maps)"
                            % (16 * 2 * nalm / 1e6, 8 * 2 * NLAT * NLON / 1e6)) if big
              else "inputs smaller than L2: not a headline configuration",
              "parallelism": "replicas"}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def flops_per_triple(spin, ncomp):
    """Algorithmic flops per (m, l, ring-pair) step: recursion + accumulation."""
    return (10 + 16 * ncomp) if spin else (3 + 4 * ncomp)


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows if len(r) > 8 for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if os.environ.get("SHT_BENCH_GLOO") is None else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ oracle ---
_SMALL_ORACLE = """
import time, numpy as np, oracle
from paper_1303_4945_gb300 import inputs
lmax = 127
th, w = oracle.gauss_nodes(lmax + 1)
rings = oracle.Rings(th, np.full(lmax + 1, 2 * lmax + 1), np.zeros(lmax + 1), w * 2 * np.pi / (2 * lmax + 1))
alm = inputs.scalar_gl_small(0, lmax)
oracle.synthesis(0, lmax, lmax, alm, rings)  # loads and warms the library
t = time.perf_counter()
maps = oracle.synthesis(0, lmax, lmax, alm, rings)
oracle.analysis(0, lmax, lmax, maps, rings)
print(1e3 * (time.perf_counter() - t))
"""


def oracle_small_full(threads=None):
    """The oracle on the small scalar workload in full (GL 128 x 255, lmax 127, one
    synthesis + analysis), in a process of its own: threads=1 pins it to one host
    core (OMP_NUM_THREADS=1), None lets it use every core (ms, measured)."""
    env = dict(os.environ)
    if threads:
        env["OMP_NUM_THREADS"] = str(threads)
    else:
        env.pop("OMP_NUM_THREADS", None)
    r = subprocess.run([sys.executable, "-c", _SMALL_ORACLE], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    return float(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else None


def oracle_single_thread_small():
    """The oracle on one host core for the small scalar workload (ms)."""
    return oracle_small_full(1)


def _warm_oracle():
    """Load the oracle library and start its thread pool outside any timed region."""
    import numpy as np

    import oracle

    th, w = oracle.gauss_nodes(9)
    r = oracle.Rings(th, np.full(9, 17), np.zeros(9), w * 2 * np.pi / 17)
    a = np.zeros(oracle.nalm(8, 8), dtype=np.complex128)
    maps = oracle.synthesis(0, 8, 8, [a], r)
    oracle.analysis(0, 8, 8, maps, r)


def oracle_sample_sizes(cores):
    """The fixed sample both arms time: 2 rings and 2 m values per host core, so
    that every core has work in both legs (the oracle runs its synthesis in
    parallel over rings and its analysis over m); rings evenly spaced from pole to
    pole, m evenly spaced from 0 to mmax (most costly first, as the loop hands
    them out)."""
    import numpy as np

    nr = min(NLAT, 2 * cores)
    nm = min(LMAX + 1, 2 * cores)
    rsel = np.unique(np.linspace(0, NLAT - 1, nr).round().astype(int))
    msel = np.unique(np.linspace(0, LMAX, nm).round().astype(int))
    return rsel, msel


def oracle_sample(gpu_out=None, others=None):
    """Time the FP64 CPU oracle on the fixed sample of oracle_sample_sizes and
    extrapolate to one full synthesis + analysis pair (ms):

        T_pair = t_syn * nlat / n_rings + t_ana * (mmax + 1) / n_m

    (every ring of the synthesis costs the same; the evenly spaced m values
    average the analysis's cost over m).  The library is loaded and its thread
    pool started before the timer.  If gpu_out is given, the sampled outputs are
    compared with it.
    """
    import numpy as np

    import oracle
    from paper_1303_4945_gb300 import inputs

    th, w = oracle.gauss_nodes(NLAT)
    rings = oracle.Rings(th, np.full(NLAT, NLON), np.zeros(NLAT), w * 2 * np.pi / NLON)
    alm = inputs.spin2_eb(SEED, LMAX)
    cores = os.cpu_count() or 1
    if gpu_out is not None:
        ana_in = gpu_out["maps"]  # a GPU synthesis output: the analyses are compared on equal input
    else:
        rng = np.random.default_rng(7)
        ana_in = [rng.standard_normal(rings.npix) for _ in range(2)]
    _warm_oracle()
    rsel, msel = oracle_sample_sizes(cores)
    t0 = time.perf_counter()
    maps = oracle.synthesis(SPIN, LMAX, LMAX, alm, rings, rings_sel=rsel)
    t1 = time.perf_counter()
    back = oracle.analysis(SPIN, LMAX, LMAX, ana_in, rings, m_sel=msel)
    t2 = time.perf_counter()
    ts, ta = t1 - t0, t2 - t1
    per_ring, per_m = 1e3 * ts / len(rsel), 1e3 * ta / len(msel)
    full_ms = per_ring * NLAT + per_m * (LMAX + 1)
    res = {"value": full_ms, "unit": "ms", "cores": cores, "kind": "oracle",
           "sample": f"synthesis of {len(rsel)} of {NLAT} rings ({ts:.2f} s) and analysis of {len(msel)} of "
                     f"{LMAX + 1} m values ({ta:.2f} s), evenly spaced, 2 of each per core, library loaded and "
                     f"threads started before the timer",
           "ms_per_ring_synthesis": per_ring, "ms_per_m_analysis": per_m,
           "extrapolation": f"T_pair = ms_per_ring_synthesis x {NLAT} + ms_per_m_analysis x {LMAX + 1}"}
    acc = None
    if gpu_out is not None:
        acc = {}
        o = rings.ofs
        idx = np.concatenate([np.arange(o[y], o[y] + NLON) for y in rsel])
        l, m = inputs.lm_arrays(LMAX, LMAX)
        sel = np.isin(m, msel)
        for form, out in [("head", gpu_out)] + list((others or {}).items()):
            for k, name in enumerate("QU"):
                d = out["maps"][k][idx] - maps[k][idx]
                acc[f"{form}_synthesis_{name}_rel_l2"] = float(np.linalg.norm(d) / np.linalg.norm(maps[k][idx]))
            if out is gpu_out:  # the oracle analysed this output's maps
                for k, name in enumerate("EB"):
                    d = out["alm"][k][sel] - back[k][sel]
                    acc[f"{form}_analysis_{name}_rel_l2"] = float(np.linalg.norm(d) / np.linalg.norm(back[k][sel]))
        acc["sample"] = f"{len(rsel)} rings, {len(msel)} m values, evenly spaced (both poles included)"
    return res, acc


def run_reference(args, world, rank):
    """--impl reference: the oracle itself, timed on host cores (rank 0 only): every
    step times the same fixed sample as the bench's cpu_baseline leg."""
    if rank != 0:
        return
    t0 = time.perf_counter()
    per_step = []
    base = None
    for i in range(args.warmup + args.steps):
        res, _ = oracle_sample()
        if i >= args.warmup:
            per_step.append(res["value"])
            base = res
    ms = statistics.median(per_step)
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": CONFIG,
            "cpu_baseline": {"value": ms, "unit": "ms", "cores": base["cores"], "kind": "oracle",
                             "sample": base["sample"] + "; median over the timed steps",
                             "ms_per_ring_synthesis": base["ms_per_ring_synthesis"],
                             "ms_per_m_analysis": base["ms_per_m_analysis"],
                             "extrapolation": base["extrapolation"],
                             "step_values_ms": per_step},
            "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------- GPU ---
def time_form(sht, torch, plan, alm_d, maps_d, out_d, steps, warmup, world, stream):
    for _ in range(warmup):
        sht.sht_execute(plan, sht.SHT_SYNTHESIS, alm_d, maps_d, 0, stream)
        sht.sht_execute(plan, sht.SHT_ANALYSIS, out_d, maps_d, 0, stream)
    torch.cuda.synchronize()
    barrier(world)
    plan.profile(True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(steps):
        sht.sht_execute(plan, sht.SHT_SYNTHESIS, alm_d, maps_d, 0, stream)
        sht.sht_execute(plan, sht.SHT_ANALYSIS, out_d, maps_d, 0, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = ev0.elapsed_time(ev1) / steps
    stages = plan.profile_read()
    plan.profile(False)
    return max_over_ranks(ms, world), stages


def paper_rule_times(sht, torch, plan, alm_d, maps_d, out_d, stream, budget_s=2.0, max_pairs=60):
    """The paper's timing rule (Sect. 5.2): repeat the pair until at least 2 s have
    accumulated and take the minimum per direction; the median beside it."""
    import statistics

    syn, ana = [], []
    while sum(syn) + sum(ana) < 1e3 * budget_s and len(syn) < max_pairs:
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        sht.sht_execute(plan, sht.SHT_SYNTHESIS, alm_d, maps_d, 0, stream)
        ev[1].record(stream)
        sht.sht_execute(plan, sht.SHT_ANALYSIS, out_d, maps_d, 0, stream)
        ev[2].record(stream)
        ev[2].synchronize()
        syn.append(ev[0].elapsed_time(ev[1]))
        ana.append(ev[1].elapsed_time(ev[2]))
    return {"pairs": len(syn), "synthesis_ms_min": min(syn), "synthesis_ms_median": statistics.median(syn),
            "analysis_ms_min": min(ana), "analysis_ms_median": statistics.median(ana)}


# FP32-pipe operations (FADD, FMUL and FFMA count one each: the pipe issues one
# of them per lane per clock) of the double-float arithmetic per (m, l,
# ring-pair) step, counted from the kernel source: a compensated multiply-add
# is 12 (exact product 4, two-sum 6, low-word adds 2), the product A cos(theta)
# with a three-float cos(theta) 5, a normalised two-term dot product 19, a
# three-term one 31.
#   spin s: two recursions (5 + 2 x 31) + 8 ncomp multiply-adds = 67 + 96 ncomp
#   spin 0: one recursion (5 + 19)       + 2 ncomp multiply-adds = 24 + 24 ncomp
def f32_ops_per_triple(spin, ncomp):
    return (67 + 96 * ncomp) if spin else (24 + 24 * ncomp)


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# dominant kernels, from the ncu captures summarised under profiles/, with the
# SHA-256 of the kernel's source file and device headers when they were taken:
# a changed source makes the figure stale and the bench reports null.
MEASURED_TRAFFIC = {
    # one launch at the headline size (spin 2, GL 4096 x 8191, lmax 4095), single-pass
    # dram__bytes_read.sum + dram__bytes_write.sum (the pair's traffic capture under profiles/);
    # sha256 over the kernel file and its headers (_kernel_digest)
    "mixed:legendre_analysis:tc": {"bytes": 4001973504 + 2131988992,
                                   "sha256": "8992b7456376424874dc34ab13698b6e8fdf662921ba8387a1bf6a9a3598a047"},
    "mixed:legendre_synthesis": {"bytes": 822240512 + 333381376,
                                 "sha256": "27f6f176d8deecc2e9d79217b9e50f084adec901dcffa36f46880253b4aae717"},
}


KERNEL_HEADERS = {"legendre_fp64.cu": ("sht_device.cuh",),
                  "legendre_mixed.cu": ("df.cuh", "sht_device.cuh", "mixed_common.cuh", "sht_internal.h"),
                  "legendre_tc.cu": ("df.cuh", "sht_device.cuh", "mixed_common.cuh", "tcgen05.cuh"),
                  "legendre_tc_ana.cu": ("df.cuh", "sht_device.cuh", "mixed_common.cuh", "tcgen05.cuh", "sht_internal.h")}


def _kernel_digest(kernel_file):
    """SHA-256 over the kernel's source file and the headers it includes (for the
    analysis kernel also the one holding its work-list constants)."""
    import hashlib
    h = hashlib.sha256()
    for name in (kernel_file,) + KERNEL_HEADERS.get(kernel_file, ()):
        with open(os.path.join(ROOT, "paper_1303_4945_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _traffic(kernel_file, key):
    rec = MEASURED_TRAFFIC.get(key)
    if not rec:
        return None
    return rec["bytes"] if rec["sha256"] == _kernel_digest(kernel_file) else None


def launches_per_step(spin, form, fp64_items=False):
    """Kernels one synthesis + analysis launches: Legendre, FFT each way, the tile
    reduction, the a_lm conversion (spin, or the mixed form), and for a mixed plan
    with FP64 items near the poles their two Legendre kernels (plus the P/M
    conversion they read when the spin is not 0)."""
    n = 5 + (1 if (spin != 0 or form == "mixed") else 0)
    if form == "mixed" and fp64_items:
        n += 2 + (1 if spin != 0 else 0)
    return n


def roofline_for(stages, plan, spin, precision, peaks, steps, ncomp=1):
    """Dominant Legendre kernel against the pipe it runs on, in the method's own work.

    achieved = algorithmic flops of the method per launch (flops_per_triple x the
    plan's exact triple count; an FMA counts 2) / the kernel's CUDA-event time.
    peak = the FMA-counted flop rate of the pipe the kernel runs on: the FP64 pipe
    for the FP64 form, the FP32 pipe for the mixed form (whose double-float
    arithmetic issues several FP32 operations per method flop).  The peak is the
    rate this box's own microbenchmark measured (sht_measure_pipe_peaks: FMA
    chains, 2 flops each) when it ran, else the figure derived from unit counts
    and the clock.  frac = achieved / peak.

    Beside it, for the mixed form: issue_frac, the FP32-pipe operations the
    double-float algorithm issues per triple (f32_ops_per_triple, FADD / FMUL /
    FFMA one each) over the pipe's issue rate -- how busy the emulation keeps the
    pipe, not the method's work -- and fp64_equivalent_tflops, the method's rate
    against which the FP64 pipe (fp64_pipe_tflops) compares.
    """
    # per transform: the stage's launches summed, divided by the timed steps
    syn_ms, _ = stages["legendre_synthesis"]
    ana_ms, _ = stages["legendre_analysis"]
    name, t_ms = ("legendre_synthesis", syn_ms) if syn_ms >= ana_ms else ("legendre_analysis", ana_ms)
    per_launch_ms = t_ms / max(steps, 1)
    triples = plan.triples(0)
    clock = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    flops = triples * flops_per_triple(spin, ncomp)
    sec = per_launch_ms * 1e-3
    achieved = flops / sec / 1e12
    measured = peaks.get("pipes_measured")  # this box's own microbenchmark (sht_measure_pipe_peaks)
    if precision == "fp64":
        kfile = "legendre_fp64.cu"
        derived = SMS * 2 * 2 * clock / 1e12  # 2 DFMA lanes per SM per clock, 2 flops each
        peak = measured["fp64_fma_tflops"] if measured else derived
        out = {"bound": "alu", "kernel": name, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
               "peak_source": ("FP64 pipe, measured on this GPU by sht_measure_pipe_peaks (FMA = 2 flops)"
                               if measured else
                               "FP64 pipe derived: 152 SMs x 2 DFMA lanes/clk x 2 flops x sm_max clock"),
               "peak_derived": derived}
    else:
        tc_syn = name == "legendre_synthesis" and bool(getattr(plan, "tensor_cores", False))
        tc_ana = name == "legendre_analysis" and bool(getattr(plan, "tensor_core_analysis", False))
        tc = tc_syn or tc_ana
        kfile = "legendre_tc.cu" if tc_syn else ("legendre_tc_ana.cu" if tc_ana else "legendre_mixed.cu")
        derived = SMS * 128 * 2 * clock / 1e12  # 128 FFMA lanes per SM per clock, 2 flops each
        peak = 2 * measured["fp32_fma_tops"] if measured else derived
        ops = triples * f32_ops_per_triple(spin, ncomp)
        issue_peak = measured["fp32_fma_tops"] if measured else derived / 2
        fp64_pipe = measured["fp64_fma_tflops"] if measured else SMS * 4 * clock / 1e12
        out = {"bound": "alu", "kernel": name, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
               "peak_source": ("FP32 pipe FMA-flop rate, 2 x the FFMA rate measured on this GPU by "
                               "sht_measure_pipe_peaks" if measured else
                               "FP32 pipe derived: 152 SMs x 128 FFMA lanes/clk x 2 flops x sm_max clock"),
               "peak_derived": derived,
               "issue_frac": None if tc else ops / sec / 1e12 / issue_peak,
               "issue_frac_note": ("the contraction runs on the tensor cores: the double-float operation count "
                                   "does not apply" if tc else
                                   "double-float FP32-pipe operations issued per second over the FP32 issue rate "
                                   "(emulation work included; not the method's work)"),
               "tensor_cores": tc,
               "fp32_ops_per_triple": None if tc else f32_ops_per_triple(spin, ncomp),
               "fp64_equivalent_tflops": achieved, "fp64_pipe_tflops": fp64_pipe}
    out["frac"] = achieved / peak
    out["flops_per_triple"] = flops_per_triple(spin, ncomp)
    key = ("fp64:" if precision == "fp64" else "mixed:") + name + (":tc" if precision != "fp64" and tc_ana else "")
    out["traffic"] = _traffic(kfile, key)
    out.update({"ms_per_launch": per_launch_ms, "triples_per_launch": triples,
                "algorithmic_flops_per_launch": flops})
    if precision != "fp64":
        # the mixed kernels skip each pair's steps before its join block (terms below the
        # negligible bound, as the polar cut skips whole pairs): the same work counted on
        # the steps that remain, so the skip is not read as throughput
        tj = plan.triples_joined()
        out["triples_after_join"] = tj
        out["frac_after_join"] = tj * flops_per_triple(spin, ncomp) / sec / 1e12 / peak
    return out


def stage_rooflines(stages, plan, spin, precision, peaks, steps, ncomp=1):
    """Both Legendre stages in the method's work (flops_per_triple x triples per
    launch / the stage's CUDA-event time) against the FMA-flop peak of the pipe the
    form runs on (measured on this GPU when available)."""
    measured = peaks.get("pipes_measured")
    clock = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    if precision == "fp64":
        peak = measured["fp64_fma_tflops"] if measured else SMS * 4 * clock / 1e12
    else:
        peak = 2 * measured["fp32_fma_tops"] if measured else SMS * 256 * clock / 1e12
    flops = plan.triples(0) * flops_per_triple(spin, ncomp)
    flops_j = (plan.triples_joined() if precision != "fp64" else plan.triples(0)) * flops_per_triple(spin, ncomp)
    out = {}
    for st in ("legendre_synthesis", "legendre_analysis"):
        ms = stages[st][0] / max(steps, 1)
        if ms > 0:
            out[st] = {"ms_per_launch": ms, "achieved_tflops": flops / (ms * 1e-3) / 1e12,
                       "frac": flops / (ms * 1e-3) / 1e12 / peak, "peak_tflops": peak,
                       "frac_after_join": flops_j / (ms * 1e-3) / 1e12 / peak}
    return out


def _line(metric, ms, args, world, config, dtype, extra):
    line = {"metric": metric, "value": ms / world, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": config, "roofline": None}
    line.update(extra)
    return line


def _events_ms(torch, stream, fn, steps, warmup, world):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    barrier(world)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    return max_over_ranks(e0.elapsed_time(e1) / steps, world)


def run_batch_workload(args, world, rank, local):
    """64 scalar Gauss-Legendre problems, lmax log-uniform in [64, 2048] (nlat = lmax+1,
    nlon = 2 lmax+1, seed 3) plus 8 maps at lmax 2047: one batched synthesis + analysis,
    replayed from a CUDA graph, against the same transforms as 65 per-plan calls."""
    import torch

    torch.cuda.set_device(local)
    from paper_1303_4945_gb300 import build as libbuild

    libbuild.build()
    from paper_1303_4945_gb300 import inputs, sht

    stream = torch.cuda.current_stream()
    rng, lmaxes = inputs.batched_lmax(seed=3)
    specs = [(int(l), 1) for l in lmaxes] + [(2047, 8)]
    alms = [[inputs.gaussian_alm(rng, l, l) for _ in range(n)] for l, n in specs]
    geoms = [sht.sht_geom_gauss(l + 1, 2 * l + 1) for l, _ in specs]
    forms = {}
    sampler = ClockSampler(local)
    for name, prec in (("fp64", sht.SHT_FP64), ("mixed", sht.SHT_MIXED)):
        plans = [sht.sht_plan_create(g, sht.sht_alm_create(l, l), 0, n, prec) for g, (l, n) in zip(geoms, specs)]
        for pl in plans:
            pl.autotune(stream)
        a_d = [[torch.from_numpy(x).cuda() for x in al] for al in alms]
        m_d = [[torch.empty(g.npix, dtype=torch.float64, device="cuda") for _ in al] for g, al in zip(geoms, alms)]
        o_d = [[torch.empty_like(x) for x in al] for al in a_d]
        batch = sht.sht_batch_create(plans)

        def direct():
            sht.sht_batch_execute(batch, sht.SHT_SYNTHESIS, a_d, m_d, 0, stream)
            sht.sht_batch_execute(batch, sht.SHT_ANALYSIS, o_d, m_d, 0, stream)

        direct()
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            cs = torch.cuda.current_stream()
            sht.sht_batch_execute(batch, sht.SHT_SYNTHESIS, a_d, m_d, 0, cs)
            sht.sht_batch_execute(batch, sht.SHT_ANALYSIS, o_d, m_d, 0, cs)

        def per_plan():
            for pl, a, m, o in zip(plans, a_d, m_d, o_d):
                sht.sht_execute(pl, sht.SHT_SYNTHESIS, a, m, 0, stream)
                sht.sht_execute(pl, sht.SHT_ANALYSIS, o, m, 0, stream)

        if name == "mixed":
            sampler.start()
        ms_graph = _events_ms(torch, stream, graph.replay, args.steps, args.warmup, world)
        if name == "mixed":
            clocks = sampler.stop()
        ms_batch = _events_ms(torch, stream, direct, args.steps, args.warmup, world)
        ms_plans = _events_ms(torch, stream, per_plan, args.steps, args.warmup, world)
        err = max(float(torch.linalg.norm(o[0] - a[0]) / torch.linalg.norm(a[0])) for a, o in zip(a_d, o_d))
        # our kernels per batched pair: Legendre synthesis and analysis per group (ncomp class x
        # tiling), one FFT launch each way, the tile reduction per plan, the a_lm conversion per
        # plan in the mixed form
        groups = len({(n, pl.tiling()[0]) for (l, n), pl in zip(specs, plans)})
        launches = 2 * groups + 2 + len(plans) + (len(plans) if prec == sht.SHT_MIXED else 0)
        forms[name] = {"ms_graph_batch": ms_graph, "ms_batch": ms_batch, "ms_per_plan_calls": ms_plans,
                       "gpu_launches_per_step": launches,
                       "triples": sum(pl.triples(0) for pl in plans), "max_round_trip_rel_l2": err,
                       "tilings": sorted({pl.tiling()[0] for pl in plans})}
        del graph, batch, plans
    config = {"workload": "64 scalar GL problems, lmax log-uniform in [64, 2048] (seed 3), nlat = lmax+1, "
                          "nlon = 2 lmax+1, plus ncomp 8 at lmax 2047; one batched synthesis + analysis "
                          "replayed from a CUDA graph", "parallelism": "replicas"}
    line = _line("ms per batched synth+analysis of 65 uneven problems", forms["mixed"]["ms_graph_batch"], args,
                 world, config, "f32x2", {"form": "mixed", "forms": forms, "clocks": clocks,
                                          "gpu_launches": forms["mixed"]["gpu_launches_per_step"] * args.steps})
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_grad_workload(args, world, rank, local):
    """L = ||synthesis(a_lm) - d||^2 at lmax 8191 on Gauss-Legendre 8192 x 16383 (a_lm with
    C_l = 1/(l+1)^2 from rng(4), then d ~ N(0,1)): forward synthesis + backward through the
    adjoint-synthesis kernel under torch.autograd, per step."""
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    from paper_1303_4945_gb300 import build as libbuild

    libbuild.build()
    from paper_1303_4945_gb300 import autograd, inputs, sht

    stream = torch.cuda.current_stream()
    lmax = 8191
    geom = sht.sht_geom_gauss(lmax + 1, 2 * lmax + 1)
    lay = sht.sht_alm_create(lmax, lmax)
    rng = np.random.default_rng(4)
    a = torch.from_numpy(inputs.gaussian_alm(rng, lmax, lmax, cl=inputs.cl_inverse_square)).cuda().reshape(1, -1)
    d = torch.from_numpy(rng.standard_normal(geom.npix)).cuda().reshape(1, -1)
    forms, grads = {}, {}
    sampler = ClockSampler(local)
    for name, prec in (("fp64", sht.SHT_FP64), ("mixed", sht.SHT_MIXED)):
        plan = sht.sht_plan_create(geom, lay, 0, 1, prec)
        plan.autotune(stream)
        x = a.clone().requires_grad_(True)

        def step():
            x.grad = None
            ((autograd.synthesis(plan, x) - d) ** 2).sum().backward()

        if name == "mixed":
            sampler.start()
        ms = _events_ms(torch, stream, step, args.steps, args.warmup, world)
        if name == "mixed":
            clocks = sampler.stop()
        grads[name] = x.grad.detach().clone()
        lo = plan.fp64_columns if prec == sht.SHT_MIXED else 0
        # synthesis: (conversion) Legendre (+FP64 columns) FFT; adjoint: FFT Legendre (+FP64 columns) reduction
        launches = (2 + (prec == sht.SHT_MIXED) + (lo > 0)) + (3 + (lo > 0))
        forms[name] = {"ms_per_step": ms, "triples": plan.triples(0), "fp64_columns": lo,
                       "gpu_launches_per_step": launches}
        del plan
        torch.cuda.empty_cache()
    forms["mixed"]["grad_vs_fp64_rel_l2"] = float(torch.linalg.norm(grads["mixed"] - grads["fp64"])
                                                  / torch.linalg.norm(grads["fp64"]))
    config = {"workload": "loss ||synthesis(a_lm) - d||^2 and its gradient through the adjoint-synthesis "
                          "kernel, GL nlat=8192 nlon=16383, lmax=mmax=8191, spin 0, seeds rng(4)",
              "parallelism": "replicas"}
    line = _line("ms per loss+gradient at lmax 8191 (GL 8192x16383)", forms["mixed"]["ms_per_step"], args, world,
                 config, "f32x2", {"form": "mixed", "forms": forms, "clocks": clocks,
                                   "gpu_launches": forms["mixed"]["gpu_launches_per_step"] * args.steps})
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_healpix_workload(args, world, rank, local):
    """HEALPix Nside 512, lmax 1535, spin 0, a_lm with C_l = 1/(l+1)^2 from rng(1): p = S a
    once (the data), then per step the weighted analysis with 3 Jacobi refinement
    iterations: a_0 = A p, a_{k+1} = a_k + A (p - S a_k) (4 analyses, 3 syntheses; the
    residual is one torch subtraction, the accumulation the ADD_OUTPUT flag)."""
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    from paper_1303_4945_gb300 import build as libbuild

    libbuild.build()
    from paper_1303_4945_gb300 import inputs, sht

    stream = torch.cuda.current_stream()
    lmax, nside = 1535, 512
    geom = sht.sht_geom_healpix(nside)
    lay = sht.sht_alm_create(lmax, lmax)
    a = torch.from_numpy(inputs.gaussian_alm(np.random.default_rng(1), lmax, lmax,
                                             cl=inputs.cl_inverse_square)).cuda()
    l, _ = inputs.lm_arrays(lmax, lmax)
    low = torch.from_numpy(l < 512).cuda()
    forms, results = {}, {}
    sampler = ClockSampler(local)
    for name, prec in (("fp64", sht.SHT_FP64), ("mixed", sht.SHT_MIXED)):
        plan = sht.sht_plan_create(geom, lay, 0, 1, prec)
        plan.autotune(stream)
        p = torch.empty(geom.npix, dtype=torch.float64, device="cuda")
        sht.sht_execute(plan, sht.SHT_SYNTHESIS, [a], [p], 0, stream)
        ak = torch.zeros_like(a)
        r = torch.empty_like(p)

        def step():
            sht.sht_execute(plan, sht.SHT_ANALYSIS, [ak], [p], 0, stream)
            for _ in range(3):
                sht.sht_execute(plan, sht.SHT_SYNTHESIS, [ak], [r], 0, stream)
                torch.sub(p, r, out=r)
                sht.sht_execute(plan, sht.SHT_ANALYSIS, [ak], [r], sht.SHT_ADD_OUTPUT, stream)

        if name == "mixed":
            sampler.start()
        ms = _events_ms(torch, stream, step, args.steps, args.warmup, world)
        if name == "mixed":
            clocks = sampler.stop()
        results[name] = ak.clone()
        syn_l = 2 + (prec == sht.SHT_MIXED)  # (conversion) Legendre, FFT; no FP64 items below lmax 2000
        forms[name] = {"ms_per_step": ms, "triples": plan.triples(0),
                       "rel_l2_vs_truth": float(torch.linalg.norm(ak - a) / torch.linalg.norm(a)),
                       "rel_l2_vs_truth_l_below_512": float(torch.linalg.norm((ak - a)[low])
                                                            / torch.linalg.norm(a[low])),
                       "gpu_launches_per_step": 3 * syn_l + 4 * 3}
        del plan
        torch.cuda.empty_cache()
    forms["mixed"]["vs_fp64_rel_l2"] = float(torch.linalg.norm(results["mixed"] - results["fp64"])
                                             / torch.linalg.norm(a))
    config = {"workload": "weighted analysis with 3 Jacobi iterations (4 analyses, 3 syntheses) of a "
                          "HEALPix Nside 512 map, lmax=mmax=1535, spin 0, a_lm C_l=1/(l+1)^2 rng(1)",
              "parallelism": "replicas"}
    line = _line("ms per Jacobi-refined analysis at lmax 1535 (HEALPix Nside 512)", forms["mixed"]["ms_per_step"],
                 args, world, config, "f32x2",
                 {"form": "mixed", "forms": forms, "clocks": clocks,
                  "gpu_launches": forms["mixed"]["gpu_launches_per_step"] * args.steps})
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_maps8_workload(args, world, rank, local):
    """Eight scalar maps through one plan (ncomp 8): synthesis + analysis at lmax 4095 on
    Gauss-Legendre 4096 x 8191, a_lm with C_l = 1/(l+1)^2 from rng(6); the FP64 form,
    the mixed form with the double-float contraction, and the mixed form with the
    synthesis contraction on the tensor cores (the multi-map case where the product
    has 32 columns)."""
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    from paper_1303_4945_gb300 import build as libbuild

    libbuild.build()
    from paper_1303_4945_gb300 import inputs, sht

    peaks = _peaks()
    peaks["pipes_measured"] = sht.sht_measure_pipe_peaks(local)
    stream = torch.cuda.current_stream()
    lmax, ncomp = 4095, 8
    geom = sht.sht_geom_gauss(lmax + 1, 2 * lmax + 1)
    lay = sht.sht_alm_create(lmax, lmax)
    rng = np.random.default_rng(6)
    alm_d = [torch.from_numpy(inputs.gaussian_alm(rng, lmax, lmax, cl=inputs.cl_inverse_square)).cuda()
             for _ in range(ncomp)]
    maps_d = [torch.empty(geom.npix, dtype=torch.float64, device="cuda") for _ in range(ncomp)]
    out_d = [torch.empty_like(a) for a in alm_d]
    forms, outs = {}, {}
    sampler = ClockSampler(local)
    clocks = None
    for name, prec, tc in (("fp64", sht.SHT_FP64, False), ("mixed_df", sht.SHT_MIXED, False),
                           ("mixed", sht.SHT_MIXED, True)):
        plan = sht.sht_plan_create(geom, lay, 0, ncomp, prec)
        if prec == sht.SHT_MIXED:
            plan.tensor_cores = tc
        plan.autotune(stream)
        if name == "mixed":
            sampler.start()
        ms, stages = time_form(sht, torch, plan, alm_d, maps_d, out_d, args.steps, args.warmup, world, stream)
        if name == "mixed":
            clocks = sampler.stop()
        kind = "fp64" if prec == sht.SHT_FP64 else "mixed"
        forms[name] = {"ms_per_step": ms, "stages_ms_per_step": {k: v[0] / args.steps for k, v in stages.items()},
                       "stage_rooflines": stage_rooflines(stages, plan, 0, kind, peaks, args.steps, ncomp),
                       "triples": plan.triples(0), "device_status": plan.device_status()}
        outs[name] = ([m.cpu().numpy() for m in maps_d], [a.cpu().numpy() for a in out_d])
        del plan
        torch.cuda.empty_cache()
    for name in ("mixed", "mixed_df"):
        forms[name]["vs_fp64_rel_l2"] = {
            "maps": max(float(np.linalg.norm(a - b) / np.linalg.norm(b)) for a, b in zip(outs[name][0], outs["fp64"][0])),
            "alm": max(float(np.linalg.norm(a - b) / np.linalg.norm(b)) for a, b in zip(outs[name][1], outs["fp64"][1]))}
    config = {"workload": "8 scalar maps in one plan (ncomp 8): synthesis + analysis, Gauss-Legendre nlat=4096 "
                          "nlon=8191, lmax=mmax=4095, a_lm C_l=1/(l+1)^2 rng(6)", "parallelism": "replicas"}
    line = _line("ms per synth+analysis of 8 maps at lmax 4095 (GL 4096x8191)", forms["mixed"]["ms_per_step"],
                 args, world, config, "f32x2", {"form": "mixed", "forms": forms, "clocks": clocks,
                                                "gpu_launches": 6 * args.steps})
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_decomposed(args, world, rank, local):
    """The headline pair as ONE transform distributed over the N ranks (Sect. 4.2):
    round-robin m and ring pairs per rank, the Legendre stage and ring FFTs through
    sht_execute_legendre / sht_execute_rings, one all-to-all of the phase array per
    direction (NCCL between GPUs; nothing to exchange at N = 1).  value = ms per
    synthesis + analysis of the whole problem (strong scaling)."""
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    from paper_1303_4945_gb300 import build as libbuild

    libbuild.build()
    from paper_1303_4945_gb300 import distributed as D
    from paper_1303_4945_gb300 import inputs, sht

    stream = torch.cuda.current_stream()
    geom = sht.sht_geom_gauss(NLAT, NLON)
    r = geom.rings()
    part = D.Partition.round_robin(LMAX, r["theta"], world)
    stages = D.LibraryStages(sht, geom, LMAX, LMAX, SPIN, 1, sht.SHT_MIXED, part, rank, stream)
    stages.plan_m.autotune(stream)  # the task's analysis kernel and tiling, as the headline's
    alm = inputs.spin2_eb(SEED, LMAX)
    alm_loc = [torch.from_numpy(D.alm_pack(a, LMAX, LMAX, part.m[rank])).cuda() for a in alm]

    def exchange(send, send_splits, recv_splits):
        return D.torch_exchange(send, send_splits, recv_splits) if world > 1 else send

    def step():
        maps = D.synthesis(part, rank, stages, exchange, alm_loc)
        return D.analysis(part, rank, stages, exchange, maps)

    ms = _events_ms(torch, stream, step, args.steps, args.warmup, world)
    back = step()
    torch.cuda.synchronize()
    err = max(float(np.linalg.norm(b.cpu().numpy() - D.alm_pack(a, LMAX, LMAX, part.m[rank]))
                    / np.linalg.norm(D.alm_pack(a, LMAX, LMAX, part.m[rank]))) for a, b in zip(alm, back))
    err = max_over_ranks(err, world)
    config = dict(CONFIG, parallelism=f"m/ring decomposition over {world} GPU(s), one all-to-all per direction")
    line = _line(METRIC + " [distributed decomposition]", ms, args, world, config, "f32x2",
                 {"form": "mixed", "scaling": "strong", "round_trip_rel_l2": err,
                  "phase_array_bytes_exchanged_per_pair": 2 * 16 * 2 * (LMAX + 1) * NLAT * (world - 1) / max(world, 1),
                  "gpu_launches": None})
    line["value"] = ms  # the whole problem's time: strong scaling
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_pair_workload(args, world, rank, local):
    """Profiling captures: the headline transform pair with the default mixed plan at
    --lmax (GL (lmax+1) x (2 lmax+1), spin 2, the bench's a_lm seed, analysis
    autotuned as the bench does: 3 untimed launches per candidate, the three
    double-float tilings and then the tensor-core analysis), one untimed pair and
    then --steps pairs, nothing else; prints the CUDA-event time per pair."""
    import torch

    torch.cuda.set_device(local)
    from paper_1303_4945_gb300 import build as libbuild

    libbuild.build()
    from paper_1303_4945_gb300 import inputs, sht

    stream = torch.cuda.current_stream()
    geom = sht.sht_geom_gauss(NLAT, NLON)
    plan = sht.sht_plan_create(geom, sht.sht_alm_create(LMAX, LMAX), SPIN, 1, sht.SHT_MIXED)
    plan.autotune(stream)  # the analysis tiling the bench's headline form would run
    a = [torch.from_numpy(x).cuda() for x in inputs.spin2_eb(SEED, LMAX)]
    m = [torch.empty(geom.npix, dtype=torch.float64, device="cuda") for _ in range(2)]
    b = [torch.empty_like(x) for x in a]

    def step():
        sht.sht_execute(plan, sht.SHT_SYNTHESIS, a, m, 0, stream)
        sht.sht_execute(plan, sht.SHT_ANALYSIS, b, m, 0, stream)

    ms = _events_ms(torch, stream, step, args.steps, 1, world)
    if rank == 0:
        print(json.dumps({"workload": "pair", "lmax": LMAX, "tensor_cores": plan.tensor_cores,
                          "tensor_core_analysis": plan.tensor_core_analysis, "ms_per_pair": ms,
                          "analysis_pairs_per_thread": plan.tiling()[0],
                          "device_status": plan.device_status()}), flush=True)


def run_variants_workload(args, world, rank, local):
    """The transforms beyond the headline pair, each in both forms: derivative
    synthesis at lmax 4095 (GL 4096 x 8191, Sect. 4.3), a spin-2 pair on the
    reduced Gauss-Legendre grid at lmax 4095 (Sect. 4.4.2), a scalar pair on the
    Clenshaw-Curtis grid (2049 x 4096) and one in real-harmonic storage (GL 2048 x
    4095) at lmax 2047 (Sect. 4.4, 4.5), and a spin-37 pair at lmax 2047 (Sect.
    4.1).  Each is timed with CUDA events; the line's value sums the mixed times."""
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    from paper_1303_4945_gb300 import build as libbuild

    libbuild.build()
    from paper_1303_4945_gb300 import inputs, sht

    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(5)
    cl = inputs.cl_inverse_square
    items = [
        ("deriv_synthesis_lmax4095", 4095, 1, lambda: sht.sht_geom_gauss(4096, 8191), "deriv", 0),
        ("reduced_gl_spin2_pair_lmax4095", 4095, 2, lambda: sht.sht_geom_reduced_gauss(4096, 4095, 2), "pair", 0),
        ("clenshaw_curtis_pair_lmax2047", 2047, 0, lambda: sht.sht_geom_ecp(sht.SHT_ECP_CC, 2049, 4096), "pair", 0),
        ("real_harmonics_pair_lmax2047", 2047, 0, lambda: sht.sht_geom_gauss(2048, 4095), "pair",
         sht.SHT_REAL_HARMONICS),
        ("spin37_pair_lmax2047", 2047, 37, lambda: sht.sht_geom_gauss(2048, 4095), "pair", 0),
    ]
    results, total, launches = {}, 0.0, 0
    sampler = ClockSampler(local)
    sampler.start()
    for name, lmax, spin, make, kind, flags in items:
        geom = make()
        lay = sht.sht_alm_create(lmax, lmax)
        narr = 1 if (spin == 0 or kind == "deriv") else 2
        alm = [torch.from_numpy(inputs.gaussian_alm(rng, lmax, lmax, cl=cl, lmin=0 if kind == "deriv" else spin)).cuda()
               for _ in range(narr)]
        nmaps = 2 if spin else 1
        rec = {"npix": geom.npix}
        outs = {}
        for form, prec in (("fp64", sht.SHT_FP64), ("mixed", sht.SHT_MIXED)):
            plan = sht.sht_plan_create(geom, lay, spin, 1, prec)
            plan.autotune(stream)
            maps = [torch.empty(geom.npix, dtype=torch.float64, device="cuda") for _ in range(nmaps)]
            back = [torch.empty_like(a) for a in alm]

            def step():
                if kind == "deriv":
                    sht.sht_execute(plan, sht.SHT_DERIV_SYNTHESIS, alm, maps, flags, stream)
                else:
                    sht.sht_execute(plan, sht.SHT_SYNTHESIS, alm, maps, flags, stream)
                    sht.sht_execute(plan, sht.SHT_ANALYSIS, back, maps, flags, stream)

            ms = _events_ms(torch, stream, step, args.steps, args.warmup, world)
            plan.profile(True)
            step()
            counts = plan.profile_read()
            plan.profile(False)
            n_launch = int(sum(c for _, c in counts.values()))
            rec[form] = {"ms": ms, "launches": n_launch}
            outs[form] = [x.cpu().numpy() for x in maps] + ([] if kind == "deriv" else [x.cpu().numpy() for x in back])
            if form == "mixed":
                total += ms
                launches += n_launch
            del plan
            torch.cuda.empty_cache()
        rec["mixed_vs_fp64_rel_l2"] = max(float(np.linalg.norm(a - b) / np.linalg.norm(b))
                                          for a, b in zip(outs["mixed"], outs["fp64"]))
        results[name] = rec
    clocks = sampler.stop()
    config = {"workload": "derivative synthesis (lmax 4095, GL 4096x8191), spin-2 pair on the reduced GL grid "
                          "(lmax 4095), scalar pairs on Clenshaw-Curtis 2049x4096 and in real-harmonic storage "
                          "(GL 2048x4095) at lmax 2047, spin-37 pair (lmax 2047); a_lm C_l=1/(l+1)^2 rng(5)",
              "parallelism": "replicas"}
    line = _line("ms per pass over the derivative / grid-variant / high-spin transforms", total, args, world, config,
                 "f32x2", {"form": "mixed", "items": results, "clocks": clocks, "gpu_launches": launches * args.steps})
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--lmax", type=int, default=4095, help="smaller sizes for profiling captures")
    ap.add_argument("--nlat", type=int, default=None,
                    help="fewer rings of the same length for profiling captures (default lmax + 1)")
    ap.add_argument("--decomposed", action="store_true",
                    help="spin2 workload as one transform distributed over the ranks (Sect. 4.2 m / ring "
                         "decomposition, NCCL all-to-all) instead of independent replicas")
    ap.add_argument("--workload", default="spin2", choices=["spin2", "batch", "grad", "healpix", "variants", "maps8", "pair"],
                    help="spin2: the headline (spin-2 lmax 4095 pair); batch: 64 uneven scalar problems + "
                         "8 maps at lmax 2047 in one batch; grad: loss + gradient at lmax 8191; healpix: "
                         "Jacobi-refined analysis on HEALPix Nside 512, lmax 1535; variants: derivative "
                         "synthesis, grid variants, real harmonics, spin 37; maps8: 8 scalar maps at lmax 4095 "
                         "with the tensor-core synthesis; pair: one untimed pair, then --steps pairs of the "
                         "default mixed plan at --lmax, for profiling captures")
    args = ap.parse_args()
    set_workload(args.lmax, args.nlat)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.decomposed:
        run_decomposed(args, world, rank, local)
        return
    if args.workload != "spin2":
        runners = {"batch": run_batch_workload, "grad": run_grad_workload, "healpix": run_healpix_workload,
                   "variants": run_variants_workload, "maps8": run_maps8_workload, "pair": run_pair_workload}
        runners[args.workload](args, world, rank, local)
        return
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    from paper_1303_4945_gb300 import build as libbuild

    libbuild.build()
    from paper_1303_4945_gb300 import inputs, sht

    peaks = _peaks()
    peaks["pipes_measured"] = sht.sht_measure_pipe_peaks(local)
    geom = sht.sht_geom_gauss(NLAT, NLON)
    lay = sht.sht_alm_create(LMAX, LMAX)
    # form name -> (precision, synthesis contraction on the tensor cores)
    forms = {"fp64": (sht.SHT_FP64, False)}
    try:
        sht.sht_plan_create(sht.sht_geom_gauss(8, 15), sht.sht_alm_create(7, 7), 2, 1, sht.SHT_MIXED)
        forms["mixed"] = (sht.SHT_MIXED, True)      # the library's default: tensor-core synthesis
        forms["mixed_df"] = (sht.SHT_MIXED, False)  # the same with the double-float contraction
    except sht.ShtError:
        pass
    alm_h = inputs.spin2_eb(SEED, LMAX)
    stream = torch.cuda.current_stream()
    alm_d = [torch.from_numpy(a).cuda() for a in alm_h]
    maps_d = [torch.empty(geom.npix, dtype=torch.float64, device="cuda") for _ in range(2)]
    out_d = [torch.empty_like(a) for a in alm_d]

    results = {}
    outputs = {}
    sampler = ClockSampler(local)
    data_bytes = sum(a.nbytes for a in alm_h) + 8 * 2 * geom.npix  # a_lm and maps of one pair
    clocks = None
    for name, (prec, tc) in forms.items():
        t0 = time.perf_counter()
        plan = sht.sht_plan_create(geom, lay, SPIN, 1, prec)
        if prec == sht.SHT_MIXED:
            plan.tensor_cores = tc
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        tune = plan.autotune(stream)  # analysis tiling, chosen by timing (outside the timed region)
        t2 = time.perf_counter()
        if name == "mixed" or (name == "fp64" and "mixed" not in forms):
            sampler.start()
        ms, stages = time_form(sht, torch, plan, alm_d, maps_d, out_d, args.steps, args.warmup, world, stream)
        if name == "mixed" or (name == "fp64" and "mixed" not in forms):
            clocks = sampler.stop()
        form_kind = "fp64" if prec == sht.SHT_FP64 else "mixed"
        results[name] = {"ms_per_step": ms, "stages_ms_per_step": {k: v[0] / args.steps for k, v in stages.items()},
                         "roofline": roofline_for(stages, plan, SPIN, form_kind, peaks, args.steps),
                         "stage_rooflines": stage_rooflines(stages, plan, SPIN, form_kind, peaks, args.steps),
                         "synthesis_contraction": "tensor cores (tcgen05, exact bf16 digit split)" if tc
                         else ("FP64" if prec == sht.SHT_FP64 else "double-float FP32"),
                         "triples": plan.triples(0), "workspace_bytes": plan.workspace(),
                         "setup": {"plan_create_ms": 1e3 * (t1 - t0), "autotune_ms": 1e3 * (t2 - t1),
                                   "workspace_over_data": plan.workspace() / data_bytes},
                         "fp64_columns": plan.fp64_columns if prec == sht.SHT_MIXED else 0,
                         "analysis_contraction": ("tensor cores (tcgen05, exact bf16 digit split)"
                                                  if prec == sht.SHT_MIXED and plan.tensor_core_analysis
                                                  else ("FP64" if prec == sht.SHT_FP64 else "double-float FP32")),
                         "tiling": {"analysis_pairs_per_thread": plan.tiling()[0],
                                    "tensor_core_analysis": prec == sht.SHT_MIXED and plan.tensor_core_analysis,
                                    "autotune_ms_per_candidate": {str(k): v for k, v in tune.items()}}}
        outputs[name] = {"maps": [m.cpu().numpy() for m in maps_d], "alm": [a.cpu().numpy() for a in out_d]}
        if world == 1:
            results[name]["paper_rule"] = paper_rule_times(sht, torch, plan, alm_d, maps_d, out_d, stream)
        if name == "mixed":  # the same plan with the FP64 ring-FFT engine (not the headline)
            plan.fft_precision = sht.SHT_FP64
            ms64, st64 = time_form(sht, torch, plan, alm_d, maps_d, out_d, args.steps, args.warmup, world, stream)
            results[name]["with_fp64_fft"] = {
                "ms_per_step": ms64,
                "fft_ms_per_step": {k: st64[k][0] / args.steps for k in ("fft_synthesis", "fft_analysis")}}
        del plan
    head = "mixed" if "mixed" in forms else "fp64"
    # mixed forms vs FP64 on the full output
    def rl2(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))
    for name in ("mixed", "mixed_df"):
        if name in forms:
            results[name]["vs_fp64_rel_l2"] = {
                "Q": rl2(outputs[name]["maps"][0], outputs["fp64"]["maps"][0]),
                "U": rl2(outputs[name]["maps"][1], outputs["fp64"]["maps"][1]),
                "E": rl2(outputs[name]["alm"][0], outputs["fp64"]["alm"][0]),
                "B": rl2(outputs[name]["alm"][1], outputs["fp64"]["alm"][1])}

    # end to end through the public API from pinned host memory: every step copies
    # its a_lm in and its result out.  As a serving loop would, the copies run on
    # streams of their own with double-buffered device arrays, overlapping the
    # neighbouring steps' transforms; the timed region starts before the first
    # step's upload and ends after the last step's download.
    plan = sht.sht_plan_create(geom, lay, SPIN, 1, forms[head][0])
    if forms[head][0] == sht.SHT_MIXED:
        plan.tensor_cores = forms[head][1]
    if results[head]["tiling"]["tensor_core_analysis"]:  # the analysis the autotuner chose for the headline
        plan.tensor_core_analysis = True
    else:
        plan.set_tiling(results[head]["tiling"]["analysis_pairs_per_thread"])
    host_in = [torch.from_numpy(a).pin_memory() for a in alm_h]
    host_out = [[torch.empty(a.shape, dtype=torch.complex128).pin_memory() for a in alm_h] for _ in range(2)]
    in_d = [alm_d, [torch.empty_like(a) for a in alm_d]]
    res_d = [out_d, [torch.empty_like(a) for a in out_d]]
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    used = [False, False]
    t_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for it in range(args.warmup + args.steps):
        b = it % 2
        if it == args.warmup:
            torch.cuda.synchronize()
            barrier(world)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            up.wait_event(e0)
        with torch.cuda.stream(up):
            if used[b]:
                up.wait_event(ev_done[b])  # the transform two steps back has read in_d[b]
            for d, h in zip(in_d[b], host_in):
                d.copy_(h, non_blocking=True)
            ev_in[b].record(up)
        stream.wait_event(ev_in[b])
        if used[b]:
            stream.wait_event(ev_out[b])  # res_d[b] of two steps back has been downloaded
        if it >= args.warmup:
            t_ev[it - args.warmup][0].record(stream)
        sht.sht_execute(plan, sht.SHT_SYNTHESIS, in_d[b], maps_d, 0, stream)
        sht.sht_execute(plan, sht.SHT_ANALYSIS, res_d[b], maps_d, 0, stream)
        if it >= args.warmup:
            t_ev[it - args.warmup][1].record(stream)
        ev_done[b].record(stream)
        with torch.cuda.stream(down):
            down.wait_event(ev_done[b])
            for d, h in zip(res_d[b], host_out[b]):
                h.copy_(d, non_blocking=True)
            ev_out[b].record(down)
        used[b] = True
    for ev in ev_out:
        stream.wait_event(ev)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world)
    e2e_transform_ms = sum(a.elapsed_time(b) for a, b in t_ev) / args.steps  # device time of the transforms
    e2e_gaps = [t_ev[i][1].elapsed_time(t_ev[i + 1][0]) for i in range(args.steps - 1)]  # idle between them
    e2e_edges = (e0.elapsed_time(t_ev[0][0]), t_ev[-1][1].elapsed_time(e1))  # first upload, last download
    e2e_ok = all(torch.equal(h.cpu() if h.is_cuda else h, r.cpu()) for h, r in
                 zip(host_out[(args.warmup + args.steps - 1) % 2], res_d[(args.warmup + args.steps - 1) % 2]))
    nbytes = sum(a.nbytes for a in alm_h)
    del plan

    line = {"metric": METRIC, "value": results[head]["ms_per_step"] / world, "unit": "ms", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": results[head]["ms_per_step"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32x2" if head == "mixed" else "f64", "data": "synthetic", "config": CONFIG,
            "form": head, "roofline": results[head]["roofline"], "clocks": clocks,
            "e2e": {"value": e2e_ms / world, "unit": "ms", "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                    "overlap": "uploads and downloads on their own streams, double-buffered",
                    "transform_ms_per_step": e2e_transform_ms,
                    "gap_ms_between_transforms": e2e_gaps, "first_upload_last_download_ms": e2e_edges,
                    "result_copied": e2e_ok},
            "gpu_launches": launches_per_step(SPIN, head, results[head].get("fp64_columns", 0) > 0) * args.steps,
            "forms": results}
    if world == 1 and rank == 0 and not args.no_cpu_baseline:
        others = {k: v for k, v in outputs.items() if k != head}
        cb, acc = oracle_sample(gpu_out=outputs[head], others=others)
        cb["scalar_gl128_lmax127_full_ms"] = {"one_core": oracle_small_full(1), "all_cores": oracle_small_full(None),
                                              "note": "the small scalar workload (GL 128 x 255, lmax 127, one "
                                                      "synthesis + analysis) in full, measured, not extrapolated"}
        line["cpu_baseline"] = cb
        line["accuracy_vs_oracle_sample"] = acc
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
