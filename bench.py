#!/usr/bin/env python
"""Benchmark of the GB300 beam search decoder on the [[144,12,12]] BB code.

Workload (one step): decode 10^6 seeded code-capacity shots at each of
p = 0.01, 0.03, 0.05 with the beam32_340iters preset (Table I) and min-sum
scale 0.625 -- 3 x 10^6 syndromes per GPU per step, syndromes resident in
HBM.  The metric is decoded syndromes/s; BP message updates/s, the roofline
of the dominant kernel, logical error rates, an end-to-end figure through
host buffers and the CPU oracle's throughput are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 run under torch.distributed.run: every rank decodes its own
shots (weak scaling, no collective on the data path); rank 0 prints the line.
--impl reference times the CPU oracle (the test oracle, double precision) on
a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import ctypes as C
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

METRIC = "decoded syndromes/s & BP msg-updates/s (% HBM peak) vs plain path, same LER"
PS = (0.01, 0.03, 0.05)
PRESET = "beam32_340iters"
ALPHA = 0.625
WORKLOAD = "bb144_code_capacity beam32_340iters alpha=0.625 p={0.01,0.03,0.05}"
# algorithmic ALU operations per message update of min-sum (Eqs. 1-3), the
# count of the algorithm and not of any kernel: on the check side, folding
# |E_{j->i}| into the row's two smallest magnitudes (a compare-exchange: 2)
# and its sign into the row's sign parity (1), then selecting the outgoing
# magnitude (min1, or min2 on the argmin edge) with its sign (1); on the
# error side, adding D_{i->j} into Lambda_j(t) (1) and forming the extrinsic
# E_{j->i} = Lambda_j(t) - D_{i->j} (1).  The per-row scale and the per-node
# hard decision are amortised over the edges and left out.
OPS_PER_UPDATE = 6
LANES_PER_SM = 128          # FP32/INT32 lanes per Blackwell SM
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2
# phenomenological DEM of the [[144,12,12]] code (12 noisy rounds + 1 perfect, 936 x 2592, 6912 edges)
PHEN_PS = (1e-3, 2e-3, 3e-3)
PHEN_SHOTS = 100_000
PHEN_PRESET = "beam64_640iters"
PHEN_WORKLOAD = "bb144_phenomenological_dem beam64_640iters alpha=0.625 p=q={1e-3,2e-3,3e-3}"
# unrolled weighted min-sum training: 20 iterations, checkpoints every 5, batch 4096, p = q = 2e-3
UNR_T, UNR_K, UNR_B, UNR_P, UNR_LR = 20, 5, 4096, 2e-3, 1e-2
UNR_WORKLOAD = "bb144_phenomenological_dem unrolled weighted min-sum T=20 ckpt=5 batch=4096 p=q=2e-3"
# circuit-shaped synthetic DEM: 936 x 8800, column weight 2-6, priors log-uniform [1e-5, 1e-3]
SYN_PRESETS = ("beam8_230iters", "beam32_340iters", "beam64_640iters")
SYN_SHOTS = 1_000_000
SYN_WORKLOAD = "synthetic_dem_936x8800 beam8_230iters/beam32_340iters/beam64_640iters alpha=0.625"
# XYZ decoding: [[144,12,12]] code capacity depolarizing noise, both stabilizer types in H
XYZ_PS = (0.03, 0.05, 0.07)
XYZ_SHOTS = 100_000
XYZ_PRESET = "beam64_640iters"
XYZ_WORKLOAD = "bb144_xyz_depolarizing beam64_640iters alpha=0.625 p={0.03,0.05,0.07} vs XZ decoding"
LAT_WORKLOAD = "single-syndrome latency: bb144 p=0.03 beam32_340iters; phenomenological DEM p=q=3e-3 beam32_340iters; " \
               "synthetic DEM beam32_340iters"
LAT_PER_STEP = 1000       # single-syndrome decodes per step
NR_PS = (0.03, 0.05)
NR_SHOTS = 100_000
NR_PRESETS = ("beam64_640iters", "beam64_32res_640iters")
NR_WORKLOAD = "bb144_code_capacity alpha=0.625 p={0.03,0.05}: beam64_640iters vs beam64_32res_640iters"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--shots", type=int, default=1_000_000, help="shots per p per GPU per step")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ps", default="0.01,0.03,0.05", help="physical error rates (a smaller case for profiling)")
    ap.add_argument("--workspace-gb", type=float, default=32.0, help="device workspace per decoder")
    ap.add_argument("--workload", choices=("bb144_code_capacity", "phenom_precision", "unrolled_training",
                                           "synthetic_dem", "xyz", "latency", "num_results"),
                    default="bb144_code_capacity",
                    help="phenom_precision: the phenomenological DEM with FP32, FP16 and BF16 message storage; "
                         "unrolled_training: training steps of the unrolled weighted min-sum on that DEM; "
                         "synthetic_dem: the 936 x 8800 circuit-shaped DEM with beam widths 8, 32, 64; "
                         "xyz: XYZ against XZ decoding of [[144,12,12]] under depolarizing noise; "
                         "latency: one syndrome at a time (mean and 99.9 percentile per syndrome); "
                         "num_results: beam64_640iters against beam64_32res_640iters")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default launch shapes (for profiler runs, where tuning timings "
                         "are distorted)")
    ap.add_argument("--no-side-by-side", action="store_true",
                    help="headline only: skip the phenomenological-DEM precision forms and the synthetic-DEM widths "
                         "that the default run adds to its line")
    ap.add_argument("--side-steps", type=int, default=3, help="timed steps of each side-by-side workload")
    ap.add_argument("--side-cpu-seconds", type=float, default=6.0,
                    help="target CPU time of each side-by-side workload's oracle baseline")
    ap.add_argument("--train-steps", type=int, default=300, help="unrolled_training: steps before the LER judgement")
    ap.add_argument("--judge-shots", type=int, default=1_000_000, help="unrolled_training: held-out shots")
    a = ap.parse_args()
    if a.workload == "phenom_precision":
        if a.ps == "0.01,0.03,0.05":
            a.ps = ",".join(str(x) for x in PHEN_PS)
        if a.shots == 1_000_000:
            a.shots = PHEN_SHOTS
    a.ps = tuple(float(x) for x in a.ps.split(","))
    return a


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, smax, reasons, power = [], [], set(), []
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def make_phen_workload(rank: int, shots: int, ps=PHEN_PS):
    from paper_2512_07057_gb300 import workloads as W
    out = []
    for p in ps:
        prob = W.bb_phenomenological(12, 6, 12, p, p)
        sh = W.sample_shots(prob, shots, W.shot_seed(f"bb144_phen_p{p}", rank))
        out.append((p, prob, sh))
    return out


def make_workload(rank: int, shots: int, ps=PS):
    from paper_2512_07057_gb300 import workloads as W
    out = []
    for p in ps:
        prob = W.bb144_code_capacity(p)
        sh = W.sample_shots(prob, shots, W.shot_seed(f"bb144_cc_p{p}", rank))
        out.append((p, prob, sh))
    return out


def wilson(k: int, n: int, z: float = 1.96) -> tuple[float, float]:
    """95% Wilson score interval of a binomial proportion k / n."""
    if n <= 0:
        return 0.0, 1.0
    p = k / n
    d = 1 + z * z / n
    c = (p + z * z / (2 * n)) / d
    h = z * np.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / d
    return float(max(0.0, c - h)), float(min(1.0, c + h))


def ler_of(prob, shots, obs, status):
    from paper_2512_07057_gb300 import workloads as W
    o = W.unpack_bits(obs[:, :(prob.K + 31) // 32], prob.K)
    t = W.unpack_bits(shots.obs, prob.K)
    fail = (o != t).any(1) | (status == 4)
    return float(fail.mean())


# ----------------------------------------------------------------------------
# CPU oracle (baseline line and reference arm)
# ----------------------------------------------------------------------------
def oracle_run(work, target_s: float, nthreads: int, preset: str = PRESET, n_min: int = 1000,
               calib: int = 2000) -> dict:
    """Oracle (double precision) on a bounded prefix of each p batch, sized
    from a short calibration run so the whole sample takes about target_s;
    returns the rate, the prefix size, the time and the outputs per batch."""
    import oracle
    per = []
    for p, prob, sh in work:
        g = oracle.Graph(prob, "f64")
        prm = oracle.preset(preset, ms_scale=ALPHA)
        n0 = min(calib, sh.B)
        t0 = time.perf_counter()
        g.decode_batch(sh.syndromes[:n0], prm, nthreads=nthreads)
        per.append((g, prm, sh, (time.perf_counter() - t0) / n0))
    # equal shot counts per p (the workload mixes the three p equally)
    sec_per_mix = sum(x[3] for x in per)
    n = int(max(n_min, min(work[0][2].B, target_s / max(sec_per_mix, 1e-9))))
    outs = []
    t0 = time.perf_counter()
    for g, prm, sh, _ in per:
        outs.append(g.decode_batch(sh.syndromes[:n], prm, nthreads=nthreads))
    dt = time.perf_counter() - t0
    return dict(rate=len(work) * n / dt, n=n, dt=dt, outputs=outs, params=per[0][1])


def oracle_rate(work, target_s: float, nthreads: int, preset: str = PRESET):
    r = oracle_run(work, target_s, nthreads, preset)
    return r["rate"], r["n"], r["dt"]


def cpu_baseline_of(work, target_s: float, preset: str, single_s: float = 4.0) -> tuple[dict, dict]:
    """The cpu_baseline object: the double-precision oracle on all host
    threads and, beside it, on one thread (the paper times one core), each on
    a bounded prefix of every batch; also returns the all-thread run."""
    nth = cores()
    r = oracle_run(work, target_s, nth, preset)
    r1 = oracle_run(work, single_s, 1, preset, n_min=50, calib=200)
    k = len(work)
    obj = {"value": r["rate"], "unit": "syndromes/s", "cores": nth, "kind": "oracle",
           "sample": f"first {r['n']} shots of each of the {k} batches, double-precision oracle, "
                     f"{r['dt']:.1f} s on {nth} host threads",
           "single_core": {"value": r1["rate"], "unit": "syndromes/s", "cores": 1,
                           "sample": f"first {r1['n']} shots of each of the {k} batches, {r1['dt']:.1f} s "
                                     f"on one host thread"}}
    return obj, r


def cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference_unrolled(args):
    """Reference arm of the unrolled workload: the double-precision autograd
    reference, forward + backward, on a bounded sample of each step's batch."""
    import torch

    from oracle import unrolled as U
    from paper_2512_07057_gb300 import workloads as W
    prob = W.bb_phenomenological(12, 6, 12, UNR_P, UNR_P)
    tab = U.Tables(prob)
    n = 16
    w0 = np.full((UNR_T, prob.n_edges), ALPHA)
    data = []
    for i in range(args.warmup + args.steps):
        sh = W.sample_shots(prob, n, W.shot_seed("unrolled_reference", i), keep_errors=True)
        data.append((W.unpack_bits(sh.syndromes, prob.M), W.unpack_bits(sh.errors, prob.N)))
    for i in range(args.warmup):
        U.unrolled_grad(tab, *data[i], w0)
    t0 = time.perf_counter()
    for i in range(args.steps):
        U.unrolled_grad(tab, *data[args.warmup + i], w0)
    dt = time.perf_counter() - t0
    value = n * args.steps / dt
    nth = torch.get_num_threads()
    sample = f"{n} of the {UNR_B} shots of each step's batch, float64 autograd reference, {nth} threads"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "training syndromes/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": UNR_WORKLOAD, "shots_per_step": n, "l2": "n/a (host)"},
            "cpu_baseline": {"value": value, "unit": "training syndromes/s", "cores": nth, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "training syndromes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_synthetic(args):
    """Reference arm of the synthetic-DEM workload: the double-precision oracle
    with the three presets on a bounded prefix of the same shots."""
    import oracle
    from paper_2512_07057_gb300 import workloads as W
    prob = W.synthetic_dem()
    sh = W.sample_shots(prob, min(args.shots, 100_000), W.shot_seed("synthetic_dem", 0))
    nth = cores()
    g = oracle.Graph(prob, "f64")
    prms = [oracle.preset(p, ms_scale=ALPHA) for p in SYN_PRESETS]
    _, n, _ = oracle_rate([(SYN_PRESETS[1], prob, sh)], 3.0, nth, SYN_PRESETS[1])
    for _ in range(args.warmup):
        for prm in prms:
            g.decode_batch(sh.syndromes[:max(100, n // 10)], prm, nthreads=nth)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for prm in prms:
            g.decode_batch(sh.syndromes[:n], prm, nthreads=nth)
    dt = time.perf_counter() - t0
    value = len(prms) * n * args.steps / dt
    sample = f"first {n} of the seeded shots per width per step, double-precision oracle, {nth} threads"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "syndromes/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": SYN_WORKLOAD, "shots_per_width_per_step": n, "l2": "n/a (host)"},
            "cpu_baseline": {"value": value, "unit": "syndromes/s", "cores": nth, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "syndromes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_latency(args):
    """Reference arm of the latency workload: the double-precision oracle
    decoding one syndrome at a time on one host thread."""
    import oracle
    from paper_2512_07057_gb300 import workloads as W
    cases = [("bb144_cc_p0.03", W.bb144_code_capacity(0.03)),
             ("phenom_p0.003", W.bb_phenomenological(12, 6, 12, 3e-3, 3e-3)),
             ("synthetic_dem", W.synthetic_dem())]
    n = min(args.steps * 200, 2000)
    res, means = {}, []
    for name, prob in cases:
        sh = W.sample_shots(prob, n, W.shot_seed(f"latency_{name}", 0))
        g = oracle.Graph(prob, "f64")
        prm = oracle.preset("beam32_340iters", ms_scale=ALPHA)
        lat = np.zeros(n)
        for i in range(n):
            t0 = time.perf_counter()
            g.decode_batch(sh.syndromes[i:i + 1], prm, nthreads=1)
            lat[i] = time.perf_counter() - t0
        res[name] = {"mean_us": float(lat.mean() * 1e6), "p99.9_us": float(np.quantile(lat, 0.999) * 1e6),
                     "syndromes": n}
        means.append(lat.mean())
    mean_us = float(np.mean(means) * 1e6)
    line = {"impl": "reference", "metric": METRIC, "value": 1e6 / mean_us, "unit": "syndromes/s (one at a time)",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_us * 1e-3 * 200,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": LAT_WORKLOAD, "l2": "n/a (host)"}, "latency": res,
            "cpu_baseline": {"value": 1e6 / mean_us, "unit": "syndromes/s (one at a time)", "cores": 1,
                             "kind": "oracle", "sample": f"{n} single-syndrome decodes per case, one thread"},
            "e2e": {"value": 1e6 / mean_us, "unit": "syndromes/s (one at a time)", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference(args, rank: int):
    if rank != 0:
        return
    if args.workload == "unrolled_training":
        run_reference_unrolled(args)
        return
    if args.workload == "synthetic_dem":
        run_reference_synthetic(args)
        return
    if args.workload == "latency":
        run_reference_latency(args)
        return
    phen = args.workload == "phenom_precision"
    if args.workload == "num_results":
        work = make_workload(0, min(args.shots, 20_000), NR_PS)
        preset, wl_name = NR_PRESETS[1], NR_WORKLOAD
    elif args.workload == "xyz":
        from paper_2512_07057_gb300 import workloads as W
        work = []
        for p in XYZ_PS:
            prob = W.bb_xyz_code_capacity(12, 6, p)
            work.append((p, prob, W.sample_shots(prob, 20_000, W.shot_seed(f"bb144_xyz_p{p}", 0))))
        preset, wl_name = XYZ_PRESET, XYZ_WORKLOAD
    else:
        work = (make_phen_workload if phen else make_workload)(0, min(args.shots, 200_000), args.ps)
        preset, wl_name = (PHEN_PRESET, PHEN_WORKLOAD) if phen else (PRESET, WORKLOAD)
    nth = cores()
    import oracle
    gs = [(oracle.Graph(prob, "f64"), sh) for _, prob, sh in work]
    prm = oracle.preset(preset, ms_scale=ALPHA)
    # one step: a bounded equal-size prefix of each p batch
    rate, n, _ = oracle_rate(work, 8.0, nth, preset)
    for _ in range(args.warmup):
        for g, sh in gs:
            g.decode_batch(sh.syndromes[:max(1000, n // 10)], prm, nthreads=nth)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for g, sh in gs:
            g.decode_batch(sh.syndromes[:n], prm, nthreads=nth)
    dt = time.perf_counter() - t0
    value = len(work) * n * args.steps / dt
    sample = f"first {n} of {work[0][2].B} seeded shots of each p per step, double-precision oracle, {nth} threads"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "syndromes/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl_name, "shots_per_p_per_step": n, "l2": "n/a (host)"},
            "cpu_baseline": {"value": value, "unit": "syndromes/s", "cores": nth, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "syndromes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


KIND_NAMES = {0: "k_seed", 1: "k_round", 2: "k_select", 8: "k_bs_check", 9: "k_bs_var", 10: "k_bs_retire",
              11: "k_screen"}


def kernel_ms(pr, steps: int) -> dict:
    """Event-timed milliseconds per step of each decoding kernel kind that ran."""
    ms = pr["kinds"]["ms"]
    return {n: float(ms[k]) / steps for k, n in KIND_NAMES.items() if k < len(ms) and (k < 3 or ms[k] > 0)}


def alu_roofline(prof, E: int, dev: int, traffic_case: str, shots: int = 0, msg_bytes: int = 4, M: int = 0):
    """Roofline of the dominant BP kernel from per-kernel event times.

    Per-candidate kernels (k_seed, k_round) keep their state on chip: their
    roof is the lane-operation rate of the chip at its maximum SM clock, and
    a launch does OPS_PER_UPDATE x (the full BP iterations it executed x E +
    the message updates of first-iteration screens, counted on the device)
    algorithmic operations.  The batched seed BP's passes (k_bs_check,
    k_bs_var) stream the messages of many shots through device memory: their
    roof is the measured HBM copy bandwidth, and a launch moves, per slot
    iteration, msg_bytes x E (check pass: the messages read; error-node
    pass: read and written, twice that) plus 8 x M bytes of detector records
    (written by the check pass, read by the error-node pass)."""
    import torch
    kinds_ms = np.sum([pr["kinds"]["ms"] for pr in prof], axis=0)
    kinds_ln = np.sum([pr["kinds"]["launches"] for pr in prof], axis=0)
    exec_iters = np.sum([pr["exec_iters"] for pr in prof], axis=0).astype(np.float64)
    # message updates of seed runs that ended in their first-iteration screen
    # (the columns next to flipped detectors; counted apart from full iterations)
    screen = float(sum(pr.get("screen_updates", 0) for pr in prof))
    pk, pk_kind = peaks()
    sm_mhz_max = float(pk.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak_tops = sms * LANES_PER_SM * sm_mhz_max * 1e6 / 1e12
    hbm_peak = float(pk.get("hbm_gbs", 6800.0))
    batch_it = exec_iters[2] if len(exec_iters) > 2 else 0.0
    # candidate kernels: kind, name, message updates of all their launches
    cands = [(0, "k_seed", (exec_iters[0] - batch_it) * E), (1, "k_round", exec_iters[1] * E),
             (8, "k_bs_check", batch_it * E), (9, "k_bs_var", batch_it * E), (11, "k_screen", screen)]
    dom_kind, name, updates = max(cands, key=lambda c: kinds_ms[c[0]])
    launches = max(1, int(kinds_ln[dom_kind]))
    ms_launch = float(kinds_ms[dom_kind]) / launches
    upd_launch = updates / launches
    ops_tops = OPS_PER_UPDATE * upd_launch / (ms_launch * 1e-3) / 1e12
    share = float(kinds_ms[dom_kind] / max(kinds_ms[[0, 1, 2, 8, 9, 10, 11]].sum(), 1e-9))
    common = {"kernel": name, "msg_updates_per_launch": upd_launch, "launch_ms": ms_launch, "kernel_share": share,
              "ops_per_msg_update": OPS_PER_UPDATE,
              "measured_in": "second timed region: same steps, each kernel launched alone between CUDA events "
                             "on the decode stream"}
    if name.startswith("k_bs_"):
        slot_iters_launch = batch_it / launches
        per_slot = (2 if name == "k_bs_var" else 1) * msg_bytes * E + 8 * M
        achieved = per_slot * slot_iters_launch / (ms_launch * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak, "traffic": None,
                    "peak_source": f"measured copy bandwidth ({pk_kind})",
                    "algorithmic_bytes_per_slot_iteration": per_slot,
                    "slot_iterations_per_launch": slot_iters_launch,
                    "alu_view": {"achieved_tops": ops_tops, "peak_tops": alu_peak_tops,
                                 "frac": ops_tops / alu_peak_tops}, **common}
    else:
        roofline = {"bound": "alu", "achieved": ops_tops, "peak": alu_peak_tops, "unit": "Tops/s",
                    "frac": ops_tops / alu_peak_tops, "traffic": None,
                    "peak_source": f"{sms} SMs x {LANES_PER_SM} lanes x {sm_mhz_max:.0f} MHz (sm_max_mhz {pk_kind})",
                    "msg_updates_counted": "full BP iterations x E (k_seed, k_round) or the edges the "
                                           "first-iteration screens formed (k_screen)", **common}
    # DRAM bytes per unit of work from an ncu capture of a smaller case
    # (profiles/), scaled to this run's average launch; null once the kernel
    # sources differ from the ones that were captured
    tr = _traffic_record(name, E, msg_bytes)
    if tr is not None:
        per, unit = tr
        if unit == "shot" and shots > 0:
            # the seed stage (screen and seed BP) moves its bytes per shot
            roofline["traffic"] = per * shots / launches
            roofline["traffic_source"] = f"ncu dram__bytes_read.sum + dram__bytes_write.sum of the seed stage on " \
                                         f"a {traffic_case}, per shot, scaled by the shots of a launch"
        elif unit == "candidate_iteration":
            roofline["traffic"] = per * (updates / max(E, 1) / launches)
            roofline["traffic_source"] = f"ncu dram__bytes_read.sum + dram__bytes_write.sum on a {traffic_case}, " \
                                         "scaled by candidate-iterations"
    # measured DRAM throughput and L2 hit rate of one launch (ncu), against the measured copy bandwidth
    mr = _memory_record(name, E, msg_bytes)
    if mr is not None:
        roofline["dram_gbs"] = mr["dram_gbs"]
        roofline["l2_hit"] = mr["l2_hit"]
        roofline["dram_frac_of_peak"] = mr["dram_gbs"] / hbm_peak
        roofline["dram_measured"] = {k: mr[k] for k in ("dram_bytes_captured", "duration_us_captured", "case",
                                                       "record")}
    else:
        roofline["dram_gbs"] = roofline["l2_hit"] = roofline["dram_frac_of_peak"] = None
    return roofline, exec_iters


NO_AUTOTUNE = False


def autotune(dec, synd, sample: int = 65536) -> dict:
    """Launch-shape autotuning on a prefix of the decoder's own batch (outside the timed regions)."""
    if NO_AUTOTUNE:
        gw, wpb = dec.shape
        return {"group_warps": gw, "warps_per_block": wpb, "autotuned": False}
    rep = dec.autotune(synd[:min(sample, synd.shape[0])].contiguous())
    gw, wpb = dec.shape
    return {"group_warps": gw, "warps_per_block": wpb, "sample_shots": int(min(sample, synd.shape[0])),
            "timed": [[a, b, round(ms, 4)] for a, b, ms in rep]}


def timed_region(decs, step, flush, stream, dev, steps, world, rank, profiled: bool, sample_clocks: bool):
    """`steps` calls of step() between barrier + synchronize; L2 flushed before
    each step outside the step events.  Returns (ms per step list, wall s,
    clocks, per-decoder profile reads)."""
    import torch
    import torch.distributed as dist
    for d in decs:
        d.profile(profiled)
        d.profile_read()                  # reset the device counters
        d.profile_read_kinds()
    sampler = ClockSampler(dev) if (rank == 0 and sample_clocks) else None
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    if sampler:
        sampler.start()
        time.sleep(0.3)
    t0 = time.perf_counter()
    for k in range(steps):
        flush.fill_(float(k))
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    clk = sampler.stop() if sampler else None
    prof = []
    for d in decs:
        pr = d.profile_read()             # kinds 0-2 (reset by this read), iterations, launches
        kinds = d.profile_read_kinds()    # the other kinds
        kinds["ms"][:3] = pr["ms"]
        kinds["launches"][:3] = pr["launches"]
        pr["kinds"] = kinds
        prof.append(pr)
    for d in decs:
        d.profile(False)
    return [s.elapsed_time(e) for s, e in zip(starts, ends)], wall, clk, prof


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def run_ours(args, rank: int, world: int, local_rank: int):
    import torch
    import torch.distributed as dist

    from __graft_entry__ import build
    from paper_2512_07057_gb300 import decoder as D

    torch.cuda.set_device(local_rank)
    dev = local_rank
    if rank == 0:
        build()
    if world > 1:
        dist.barrier()
        build()
    work = make_workload(rank, args.shots, args.ps)
    decs, synd, outs, tuned = [], [], [], {}
    for p, prob, sh in work:
        params = D.make_params(PRESET, ms_scale=ALPHA, workspace_bytes=int(args.workspace_gb * (1 << 30)))
        d = D.BeamSearchDecoder(prob, params, device=dev)
        decs.append(d)
        synd.append(D.to_torch_words(sh.syndromes, dev))
        outs.append(d.alloc_outputs(sh.B))
        tuned[str(p)] = autotune(d, synd[-1])
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=f"cuda:{dev}")
    stream = torch.cuda.current_stream(dev)

    def step():
        for d, s, o in zip(decs, synd, outs):
            d.decode(s, o, stream=stream)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize(dev)

    tr_args = (decs, step, flush, stream, dev, args.steps, world, rank)
    # region 1 (headline): each chunk runs as one CUDA graph
    ms_steps, t_wall, clocks, prof_graph = timed_region(*tr_args, profiled=False, sample_clocks=True)
    ms_total = float(sum(ms_steps))
    # region 2 (roofline): the same steps with every kernel bracketed by events
    ms_steps_p, _, _, prof = timed_region(*tr_args, profiled=True, sample_clocks=False)
    shots_per_step = sum(sh.B for _, _, sh in work)
    if world > 1:
        t = torch.tensor([ms_total], dtype=torch.float64, device=f"cuda:{dev}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total_max = float(t.item())
    else:
        ms_total_max = ms_total

    # ---- outputs of the last step: LER, algorithmic iterations
    E = work[0][1].n_edges
    per_p = {}
    alg_iters_step = 0
    for (p, prob, sh), o in zip(work, outs):
        obs = D.from_torch_words(o.obs_flips)
        st = D.from_torch_words(o.status)
        it = D.from_torch_words(o.iters).astype(np.int64)
        alg_iters_step += int(it.sum())
        per_p[str(p)] = {"ler": ler_of(prob, sh, obs, st), "seed_converged": float((st == 1).mean()),
                         "beam_converged": float((st == 2).mean()), "failed": float((st == 4).mean()),
                         "mean_alg_iters": float(it.mean())}
    for (p, _, _), pr in zip(work, prof):
        per_p[str(p)]["kernel_ms_per_step"] = kernel_ms(pr, args.steps)
    roofline, exec_iters = alu_roofline(prof, E, dev, "16000-shot case")
    pk, _ = peaks()
    hbm_peak = float(pk.get("hbm_gbs", 6800.0))
    steps_total_s = ms_total_max * 1e-3
    value = world * shots_per_step * args.steps / steps_total_s
    msg_alg = alg_iters_step * E * world / (steps_total_s / args.steps)
    msg_exec = float(exec_iters.sum()) * E * world / steps_total_s
    # a streaming model for context: 14.7 B per update if every iteration moved its state through HBM
    # (context only: the state of this code stays on chip; the measured figure is the roofline's dram_gbs)
    stream_bytes = 2 * 4 * E + 2 * (2 * 4 + 4) * 72 + 8 * 144
    line = {
        "metric": METRIC, "value": value, "unit": "syndromes/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "code": "[[144,12,12]] BB, H_X 72x144, 432 edges",
                   "shots_per_p_per_gpu": args.shots, "syndromes_per_step_per_gpu": shots_per_step,
                   "l2": "flushed before every timed step (256 MiB write outside the step events)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU", "launch_shapes": tuned},
        "exec_bp_iters_per_step": {"seed": float(exec_iters[0]) / args.steps, "round": float(exec_iters[1]) / args.steps},
        "msg_updates_per_s": {"algorithmic": msg_alg, "executed": msg_exec,
                              "executed_per_algorithmic": float(exec_iters.sum() / args.steps / max(alg_iters_step, 1)),
                              "streaming_model_bytes_per_update": stream_bytes / E},
        "hbm": {"dram_gbs": roofline["dram_gbs"], "pct_of_peak": (100 * roofline["dram_frac_of_peak"]
                                                                 if roofline["dram_frac_of_peak"] is not None
                                                                 else None),
                "l2_hit": roofline["l2_hit"], "peak_gbs": hbm_peak, "kernel": roofline["kernel"],
                "source": "ncu on one launch of the dominant kernel (profiles/); null when its sources changed"},
        "roofline": roofline,
        "gpu_launches": int(sum(pr["kernel_launches"] for pr in prof_graph)),
        "profiled_ms_per_step": float(sum(ms_steps_p)) / args.steps,
        "per_p": per_p,
        "clocks": clocks,
        "wall_s_timed": t_wall,
    }
    if rank == 0 and not args.no_e2e:
        line["e2e"] = e2e_host(decs, work, args, dev)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"], _ = cpu_baseline_of(work, args.cpu_seconds, PRESET)
    for d in decs:
        d.close()
    if world == 1 and not args.no_side_by_side:
        line["side_by_side"] = side_by_side(args, dev)
    if rank == 0:
        print(json.dumps(line), flush=True)


def side_by_side(args, dev) -> dict:
    """The metric's comparison in the same run: the phenomenological DEM with
    the plain FP32 path beside FP16 and BF16 message storage (10^5 shots at
    each p = q), and the synthetic 936 x 8800 DEM at beam widths 8, 32 and 64
    (10^6 shots), each with its own roofline, LER and CPU oracle baseline;
    fewer timed steps than the headline (same timing rules)."""
    from paper_2512_07057_gb300 import workloads as W
    t0 = time.perf_counter()
    steps, warm = args.side_steps, max(3, min(args.warmup, 3))
    cpu_s = None if args.no_cpu_baseline else args.side_cpu_seconds
    phen = precision_forms(make_phen_workload(0, PHEN_SHOTS), dev, steps, warm, 1, 0, args.workspace_gb, cpu_s)
    phen.pop("e2e", None)
    phen.update(workload=PHEN_WORKLOAD, steps=steps, warmup=warm,
                fp16_vs_plain_fp32=phen["forms"]["fp16"]["value"] / phen["forms"]["fp32"]["value"],
                bf16_vs_plain_fp32=phen["forms"]["bf16"]["value"] / phen["forms"]["fp32"]["value"])
    prob = W.synthetic_dem()
    sh = W.sample_shots(prob, SYN_SHOTS, W.shot_seed("synthetic_dem", 0))
    syn = synthetic_widths(prob, sh, dev, steps, warm, 1, 0, args.workspace_gb, cpu_s)
    syn.update(workload=SYN_WORKLOAD, steps=steps, warmup=warm)
    return {"phenomenological_dem": phen, "synthetic_dem": syn, "wall_s": time.perf_counter() - t0}


def precision_forms(work, dev, steps: int, warmup: int, world: int, rank: int, workspace_gb: float,
                    cpu_seconds: float | None, e2e_args=None) -> dict:
    """The phenomenological DEM decoded with FP32 (the plain path), FP16 and
    BF16 message storage, each timed on the same syndromes: per form the
    throughput, its roofline, LER and re-run shares per p.  With cpu_seconds,
    the double-precision oracle on a bounded prefix gives the cpu_baseline
    (shared by the three forms) and, per form, the decisions that differ from
    it under the parity rule (a near tie of the double-precision run at or
    before the first divergent decision excuses a difference)."""
    import torch
    import torch.distributed as dist

    from paper_2512_07057_gb300 import binding as B
    from paper_2512_07057_gb300 import decoder as D
    synd = [D.to_torch_words(sh.syndromes, dev) for _, _, sh in work]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=f"cuda:{dev}")
    stream = torch.cuda.current_stream(dev)
    E = work[0][1].n_edges
    shots_per_step = sum(sh.B for _, _, sh in work)
    forms, host_out, e2e, tuned = {}, {}, None, {}
    for name, prec in (("fp32", B.BSD_FP32), ("fp16", B.BSD_FP16), ("bf16", B.BSD_BF16)):
        decs, outs = [], []
        for p, prob, sh in work:
            params = D.make_params(PHEN_PRESET, ms_scale=ALPHA, msg_precision=prec,
                                   workspace_bytes=int(workspace_gb * (1 << 30)))
            decs.append(D.BeamSearchDecoder(prob, params, device=dev))
            outs.append(decs[-1].alloc_outputs(sh.B))
            tuned.setdefault(name, {})[str(p)] = autotune(decs[-1], synd[len(decs) - 1])

        def step():
            for d, s, o in zip(decs, synd, outs):
                d.decode(s, o, stream=stream)

        for _ in range(warmup):
            flush.fill_(1.0)
            step()
        torch.cuda.synchronize(dev)
        tr_args = (decs, step, flush, stream, dev, steps, world, rank)
        ms_steps, _, clocks, prof_graph = timed_region(*tr_args, profiled=False, sample_clocks=True)
        _, _, _, prof = timed_region(*tr_args, profiled=True, sample_clocks=False)
        ms_total = float(sum(ms_steps))
        if world > 1:
            t = torch.tensor([ms_total], dtype=torch.float64, device=f"cuda:{dev}")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms_total = float(t.item())
        roofline, exec_iters = alu_roofline(prof, E, dev, "small case of the same DEM",
                                            shots=shots_per_step * steps,
                                            msg_bytes=4 if prec == B.BSD_FP32 else 2, M=work[0][1].M)
        per_p = {}
        for (p, prob, sh), o in zip(work, outs):
            st = D.from_torch_words(o.status)
            it = D.from_torch_words(o.iters).astype(np.int64)
            per_p[str(p)] = {"ler": ler_of(prob, sh, D.from_torch_words(o.obs_flips), st & 7),
                             "seed_converged": float(((st & 7) == 1).mean()),
                             "beam_converged": float(((st & 7) == 2).mean()),
                             "failed": float(((st & 7) == 4).mean()),
                             "near_tie_flagged": float(((st & B.BSD_STATUS_NEAR_TIE) > 0).mean()),
                             "fp32_rerun": float(((st & B.BSD_STATUS_FP32_RERUN) > 0).mean()),
                             "mean_alg_iters": float(it.mean())}
            host_out[(name, p)] = (D.from_torch_words(o.corrections).copy(), st.copy())
        steps_s = ms_total * 1e-3
        forms[name] = {"value": world * shots_per_step * steps / steps_s, "unit": "syndromes/s",
                       "ms_per_step": ms_total / steps, "msg_bytes": 4 if prec == B.BSD_FP32 else 2,
                       "exec_bp_iters_per_step": {"seed": float(exec_iters[0]) / steps,
                                                  "round": float(exec_iters[1]) / steps,
                                                  "seed_batched": float(exec_iters[2]) / steps},
                       "roofline": roofline, "gpu_launches": int(sum(pr["kernel_launches"] for pr in prof_graph)),
                       "clocks": clocks, "per_p": per_p}
        if name == "fp16" and e2e_args is not None:
            e2e = e2e_host(decs, work, e2e_args, dev)
        for d in decs:
            d.close()
    res = {"forms": forms, "launch_shapes": tuned, "e2e": e2e}
    if cpu_seconds:
        import oracle
        base, run = cpu_baseline_of(work, cpu_seconds, PHEN_PRESET)
        res["cpu_baseline"] = base
        # the same prefix decoded by the double-precision oracle: decisions of
        # each form that differ, and how many a near tie before the first
        # divergent decision explains (threshold 1e-6 and the 1e-4 guard band)
        n = run["n"]
        agree = {}
        for (p, prob, sh), r in zip(work, run["outputs"]):
            g64, g32 = oracle.Graph(prob, "f64"), oracle.Graph(prob, "f32")
            s_bits = None
            for name in forms:
                corr, st = host_out[(name, p)]
                diff = np.nonzero((corr[:n] != r["corrections"]).any(1) | ((st[:n] & 7) != r["status"]))[0]
                n6 = n4 = 0
                if len(diff):
                    from paper_2512_07057_gb300 import workloads as W
                    if s_bits is None:
                        s_bits = W.unpack_bits(sh.syndromes[:n], prob.M)
                    import dataclasses
                    prm = run["params"]
                    for b in diff[:50]:
                        # the single-precision build with the form's storage (a
                        # re-run shot: single-precision messages)
                        ms = 0 if (st[b] & B.BSD_STATUS_FP32_RERUN) else {"fp32": 0, "fp16": 1, "bf16": 2}[name]
                        l64 = g64.decode_log(s_bits[b], prm)["log"]
                        l32 = g32.decode_log(s_bits[b], dataclasses.replace(prm, msg_storage=ms))["log"]
                        k = oracle.first_divergence(l64, l32)
                        n6 += int(k >= 0 and oracle.near_tie_before(l64, k, 1e-6))
                        n4 += int(k >= 0 and oracle.near_tie_before(l64, k, 1e-4))
                agree.setdefault(name, {})[str(p)] = {
                    "shots": int(n), "differ": int(len(diff)), "examined": int(min(len(diff), 50)),
                    "near_tie_before_divergence_1e-6": n6, "near_tie_before_divergence_1e-4": n4}
        res["fp64_agreement"] = agree
    return res


def run_precision(args, rank: int, world: int, local_rank: int):
    """The phenomenological DEM with FP32, FP16 and BF16 message storage side
    by side; the line's value is the FP16 form."""
    import torch
    import torch.distributed as dist

    from __graft_entry__ import build

    torch.cuda.set_device(local_rank)
    dev = local_rank
    if rank == 0:
        build()
    if world > 1:
        dist.barrier()
        build()
    work = make_phen_workload(rank, args.shots, args.ps)
    shots_per_step = sum(sh.B for _, _, sh in work)
    res = precision_forms(work, dev, args.steps, args.warmup, world, rank, args.workspace_gb,
                          None if (rank != 0 or args.no_cpu_baseline) else args.cpu_seconds,
                          e2e_args=args if (rank == 0 and not args.no_e2e) else None)
    forms = res["forms"]
    main_form = forms["fp16"]
    line = {
        "metric": METRIC, "value": main_form["value"], "unit": "syndromes/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": main_form["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "msg_storage": "f16",
        "data": "synthetic",
        "config": {"workload": PHEN_WORKLOAD, "code": "[[144,12,12]] phenomenological DEM, 936 x 2592, 6912 edges",
                   "shots_per_p_per_gpu": args.shots, "syndromes_per_step_per_gpu": shots_per_step,
                   "l2": "flushed before every timed step (256 MiB write outside the step events)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "launch_shapes": res["launch_shapes"]},
        "roofline": main_form["roofline"], "gpu_launches": main_form["gpu_launches"], "clocks": main_form["clocks"],
        "forms": forms,
        "fp16_vs_plain_fp32": main_form["value"] / forms["fp32"]["value"],
    }
    if res["e2e"] is not None:
        line["e2e"] = res["e2e"]
    if "cpu_baseline" in res:
        line["cpu_baseline"] = res["cpu_baseline"]
        line["fp64_agreement"] = res["fp64_agreement"]
    if rank == 0:
        print(json.dumps(line), flush=True)


def unrolled_bytes_per_launch(kind: int, E: int, N: int, M: int, Bp: int, T: int) -> float:
    """Algorithmic HBM bytes of one launch of an unrolled pass, averaged over
    the launches of a training step (forward, recomputed segments, adjoint).
    Per-edge arrays are float32 [E][Bp], per-node arrays [N][Bp]; bit planes
    take one bit per shot and row."""
    EB, NB = 4.0 * E * Bp, 4.0 * N * Bp
    if kind == 3:      # check pass: E(t-1) in, D(t) out, syndrome bits
        return 2 * EB + M * Bp / 8
    if kind == 4:      # error pass: D(t) in, E(t) out; the recomputed half also writes Lambda(t)
        return 2 * EB + NB / 2 + N * Bp / 8
    if kind == 5:      # error adjoint: gE(t) (t < T) and E(t) in, Lambda(t) in, gD(t) out, error bits
        return EB * (1 + (T - 1) / T) + NB + EB + N * Bp / 8
    if kind == 6:      # check adjoint: E(t-1) and gD(t) in, gE(t-1) out (t > 1), syndrome bits
        return 2 * EB + EB * (T - 1) / T + M * Bp / 8
    raise ValueError(kind)


def run_unrolled(args, rank: int, world: int, local_rank: int):
    """Training steps of the unrolled decoder (forward + adjoint + Adam) on the
    phenomenological DEM, then the learned weights judged by the plain and
    the beam decoder's LER on held-out shots."""
    import torch
    import torch.distributed as dist

    from __graft_entry__ import build
    from paper_2512_07057_gb300 import decoder as D
    from paper_2512_07057_gb300 import unrolled as G
    from paper_2512_07057_gb300 import workloads as W

    torch.cuda.set_device(local_rank)
    dev = local_rank
    if rank == 0:
        build()
    if world > 1:
        dist.barrier()
        build()
    prob = W.bb_phenomenological(12, 6, 12, UNR_P, UNR_P)
    T, k, Bn = UNR_T, UNR_K, UNR_B
    tr = G.UnrolledTrainer(prob, Bn, T, k, device=dev)
    nb = args.warmup + 2 * args.steps
    batches = [G.batch_tensors(prob, Bn, W.shot_seed(f"unrolled_bench_r{rank}", i), dev)[:2] for i in range(nb)]
    w = torch.full((T, prob.n_edges), ALPHA, dtype=torch.float32, device=f"cuda:{dev}", requires_grad=True)
    opt = torch.optim.Adam([w], lr=UNR_LR)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=f"cuda:{dev}")

    def step(i):
        s_t, e_t = batches[i]
        opt.zero_grad(set_to_none=True)
        loss = G.unrolled_loss(w, tr, s_t, e_t)[0]
        loss.backward()
        opt.step()
        return loss

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize(dev)

    def region(profiled: bool, first: int):
        tr.dec.profile(profiled)
        tr.dec.profile_read_kinds()
        sampler = ClockSampler(dev) if (rank == 0 and not profiled) else None
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        if sampler:
            sampler.start()
            time.sleep(0.3)
        for q in range(args.steps):
            flush.fill_(float(q))
            ev[q][0].record(stream)
            step(first + q)
            ev[q][1].record(stream)
        torch.cuda.synchronize(dev)
        clk = sampler.stop() if sampler else None
        prof = tr.dec.profile_read_kinds()
        tr.dec.profile(False)
        return [a.elapsed_time(b) for a, b in ev], clk, prof

    ms_steps, clocks, _ = region(False, args.warmup)
    _, _, prof = region(True, args.warmup + args.steps)
    ms_total = float(sum(ms_steps))
    if world > 1:
        t = torch.tensor([ms_total], dtype=torch.float64, device=f"cuda:{dev}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    E, N, M = prob.n_edges, prob.N, prob.M
    Bp = (Bn + 511) // 512 * 512
    names = {3: "k_u_check", 4: "k_u_var", 5: "k_u_bvar", 6: "k_u_bcheck"}
    per_kind = {names[kd]: {"ms_per_step": float(prof["ms"][kd]) / args.steps,
                            "launches_per_step": float(prof["launches"][kd]) / args.steps} for kd in names}
    dom = max(names, key=lambda kd: prof["ms"][kd])
    launch_ms = float(prof["ms"][dom]) / max(1, int(prof["launches"][dom]))
    alg = unrolled_bytes_per_launch(dom, E, N, M, Bp, T)
    pk, pk_kind = peaks()
    hbm = float(pk.get("hbm_gbs", 6800.0))
    achieved = alg / (launch_ms * 1e-3) / 1e9
    roofline = {"kernel": names[dom], "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": None, "algorithmic_bytes_per_launch": alg, "launch_ms": launch_ms,
                "kernel_share": float(prof["ms"][dom] / max(prof["ms"][3:7].sum(), 1e-9)),
                "peak_source": f"hbm_gbs ({pk_kind})",
                "measured_in": "second timed region: same steps, each pass launched between CUDA events"}
    tr_rec = _traffic_record(names[dom], E)
    if tr_rec is not None and tr_rec[1] == "launch":
        roofline["traffic"] = tr_rec[0]
        roofline["traffic_source"] = "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, averaged over " \
                                     "the launches of one training step of this workload"
    steps_s = ms_total * 1e-3
    value = world * Bn * args.steps / steps_s
    # edge updates: forward T iterations, the recomputed T, the adjoint T (check + error pass each)
    upd = 3.0 * T * E * Bn
    line = {
        "metric": METRIC, "value": value, "unit": "training syndromes/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": UNR_WORKLOAD, "code": "[[144,12,12]] phenomenological DEM, 936 x 2592, 6912 edges",
                   "batch": Bn, "T": T, "ckpt_every": k, "weights": T * E, "optimizer": f"Adam lr={UNR_LR}",
                   "l2": "flushed before every timed step (256 MiB write outside the step events)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "edge_updates_per_s": world * upd * args.steps / steps_s,
        "kernels": per_kind, "roofline": roofline, "clocks": clocks,
        # per step: forward 2 bit-plane + 1 initial-message + T check + T error + 1 loss kernels; backward
        # T recomputed check + T recomputed error + T error-adjoint + T check-adjoint + 1 gradient kernels
        "gpu_launches": (6 * T + 5) * args.steps,
        "timed_launches_per_step": {"check": float(prof["launches"][3]) / args.steps,
                                    "error": float(prof["launches"][4]) / args.steps,
                                    "error_adjoint": float(prof["launches"][5]) / args.steps,
                                    "check_adjoint": float(prof["launches"][6]) / args.steps},
    }
    if rank == 0 and not args.no_e2e:
        line["e2e"] = _unrolled_e2e(tr, w, opt, prob, Bn, args, dev)
    if rank == 0:
        line["ler_judgement"] = _judge_weights(prob, args, dev)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = _unrolled_cpu_baseline(prob, T, args.cpu_seconds)
    tr.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def _unrolled_e2e(tr, w, opt, prob, Bn, args, dev):
    """Training steps with each batch copied from pinned host memory and the loss read back."""
    import torch

    from paper_2512_07057_gb300 import unrolled as G
    from paper_2512_07057_gb300 import workloads as W
    host = []
    for i in range(args.steps + 1):
        sh = W.sample_shots(prob, Bn, W.shot_seed("unrolled_bench_e2e", i), keep_errors=True)
        host.append((torch.from_numpy(sh.syndromes.view(np.int32)).pin_memory(),
                     torch.from_numpy(sh.errors.view(np.int32)).pin_memory()))
    h2d = host[0][0].numel() * 4 + host[0][1].numel() * 4

    def step(i):
        s_t = host[i][0].to(f"cuda:{dev}", non_blocking=True)
        e_t = host[i][1].to(f"cuda:{dev}", non_blocking=True)
        opt.zero_grad(set_to_none=True)
        loss = G.unrolled_loss(w, tr, s_t, e_t)[0]
        loss.backward()
        opt.step()
        return float(loss.detach())            # device -> host read of the step's loss

    step(0)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for i in range(1, args.steps + 1):
        step(i)
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    return {"value": Bn * args.steps / dt, "unit": "training syndromes/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": 4, "api": "UnrolledLoss (torch.autograd) over bsd_unrolled_forward/backward"}


def _judge_weights(prob, args, dev):
    """Train the weights, then decode held-out shots with the plain decoder
    (BP alone, T iterations) and the beam decoder, with the scale 0.625 and
    with the learned weights."""
    import torch

    from paper_2512_07057_gb300 import decoder as D
    from paper_2512_07057_gb300 import unrolled as G
    from paper_2512_07057_gb300 import workloads as W
    t0 = time.perf_counter()
    wl, hist = G.train_weights(prob, T=UNR_T, ckpt_every=UNR_K, batch=UNR_B, steps=args.train_steps, lr=UNR_LR,
                               init=ALPHA, tag="unrolled_judge_train", device=dev)
    train_s = time.perf_counter() - t0
    # objectives that weight the late iterations (the plain decoder reads its
    # hard decision at the last one): the last term alone, and c_t = t / T
    variants = {"learned": wl}
    for vname, c in (("learned_last_iteration", np.eye(UNR_T)[-1]),
                     ("learned_linear_in_t", np.arange(1, UNR_T + 1) / UNR_T)):
        variants[vname], _ = G.train_weights(prob, T=UNR_T, ckpt_every=UNR_K, batch=UNR_B, steps=args.train_steps,
                                             lr=UNR_LR, init=ALPHA, tag="unrolled_judge_train", device=dev,
                                             iter_weights=c)
    # the loss on one fixed held-out batch, with the initial and the learned weights
    tr = G.UnrolledTrainer(prob, UNR_B, UNR_T, UNR_K, device=dev)
    vs, ve, _ = G.batch_tensors(prob, UNR_B, W.shot_seed("unrolled_judge_validation", 0), dev)
    val = {}
    for wname, wts in (("scale_0.625", np.full_like(wl, ALPHA)), *variants.items()):
        lv = tr.forward(torch.from_numpy(wts).to(f"cuda:{dev}"), vs, ve).cpu().numpy()
        val[wname] = {"loss": float(lv[0]), "loss_last_iteration": float(lv[-1])}
    tr.close()
    sh = W.sample_shots(prob, args.judge_shots, W.shot_seed("unrolled_judge_heldout", 0))
    synd = D.to_torch_words(sh.syndromes, dev)
    out = {"train_steps": args.train_steps, "train_s": train_s, "train_loss_first10": float(np.mean(hist[:10])),
           "train_loss_last10": float(np.mean(hist[-10:])), "validation": val, "held_out_shots": args.judge_shots,
           "weights_mean": float(wl.mean()), "weights_std": float(wl.std())}
    for name, params in (("plain_bp_T20", D.make_params(ms_scale=ALPHA, max_rounds=0, initial_iters=UNR_T)),
                         ("beam64_640iters", D.make_params(PHEN_PRESET, ms_scale=ALPHA))):
        dec = D.BeamSearchDecoder(prob, params, device=dev)
        res = {}
        for wname, wts in (("scale_0.625", None), *variants.items()):
            dec.set_weights(wts)
            o = dec.decode(synd)
            torch.cuda.synchronize(dev)
            st = D.from_torch_words(o.status)
            fails = int(round(ler_of(prob, sh, D.from_torch_words(o.obs_flips), st & 7) * sh.B))
            lo, hi = wilson(fails, sh.B)
            res[wname] = {"ler": fails / sh.B, "failures": fails, "wilson95": [lo, hi],
                          "not_converged": int(((st & 7) == 4).sum())}
        # a change is significant when the Wilson intervals do not overlap
        base = res["scale_0.625"]["wilson95"]
        for wname in variants:
            iv = res[wname]["wilson95"]
            res[wname]["differs_from_scale"] = bool(iv[1] < base[0] or iv[0] > base[1])
        dec.close()
        out[name] = res
    return out


def _unrolled_cpu_baseline(prob, T, target_s):
    """The double-precision autograd reference (forward + backward) on the host cores."""
    import torch

    from oracle import unrolled as U
    from paper_2512_07057_gb300 import workloads as W
    tab = U.Tables(prob)
    n = 8
    sh = W.sample_shots(prob, n, "unrolled_cpu", keep_errors=True)
    s, e = W.unpack_bits(sh.syndromes, prob.M), W.unpack_bits(sh.errors, prob.N)
    w0 = np.full((T, prob.n_edges), ALPHA)
    t0 = time.perf_counter()
    reps = 0
    while True:
        U.unrolled_grad(tab, s, e, w0)
        reps += 1
        if time.perf_counter() - t0 > target_s / 3:
            break
    dt = time.perf_counter() - t0
    return {"value": n * reps / dt, "unit": "training syndromes/s", "cores": torch.get_num_threads(),
            "kind": "oracle", "sample": f"{reps} forward+backward passes of {n} shots, T={T}, float64 autograd "
                                        f"reference, {dt:.1f} s"}


def synthetic_widths(prob, sh, dev, steps: int, warmup: int, world: int, rank: int, workspace_gb: float,
                     cpu_seconds: float | None, e2e_args=None) -> dict:
    """The 936 x 8800 synthetic DEM decoded with beam widths 8, 32 and 64 (the
    matching Table I presets) on the same syndromes: the throughput over the
    three, each width's kernel times, LER and roofline; with cpu_seconds the
    double-precision oracle on a bounded prefix per width."""
    import torch
    import torch.distributed as dist

    from paper_2512_07057_gb300 import decoder as D
    synd = D.to_torch_words(sh.syndromes, dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=f"cuda:{dev}")
    stream = torch.cuda.current_stream(dev)
    res = {"per_width": {}, "launch_shapes": {}}
    decs, outs = [], []
    for preset in SYN_PRESETS:
        d = D.BeamSearchDecoder(prob, D.make_params(preset, ms_scale=ALPHA,
                                                    workspace_bytes=int(workspace_gb * (1 << 30))), device=dev)
        decs.append(d)
        outs.append(d.alloc_outputs(sh.B))
        res["launch_shapes"][preset] = autotune(d, synd, 16384)

    def run_region(ds, os_):
        def step():
            for d, o in zip(ds, os_):
                d.decode(synd, o, stream=stream)
        for _ in range(warmup):
            flush.fill_(1.0)
            step()
        torch.cuda.synchronize(dev)
        tr_args = (ds, step, flush, stream, dev, steps, world, rank)
        ms_steps, _, clocks, prof_graph = timed_region(*tr_args, profiled=False, sample_clocks=True)
        _, _, _, prof = timed_region(*tr_args, profiled=True, sample_clocks=False)
        ms_total = float(sum(ms_steps))
        if world > 1:
            t = torch.tensor([ms_total], dtype=torch.float64, device=f"cuda:{dev}")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms_total = float(t.item())
        return ms_total, clocks, prof_graph, prof

    # all three widths in one step (the headline of this workload)
    ms_total, clocks, prof_graph, prof = run_region(decs, outs)
    roofline, exec_iters = alu_roofline(prof, prob.n_edges, dev, "small case of the same DEM",
                                        shots=len(decs) * sh.B * steps, M=prob.M)
    for preset, d, o, pr in zip(SYN_PRESETS, decs, outs, prof):
        st = D.from_torch_words(o.status)
        it = D.from_torch_words(o.iters).astype(np.int64)
        res["per_width"][preset] = {
            "ler": ler_of(prob, sh, D.from_torch_words(o.obs_flips), st & 7),
            "seed_converged": float(((st & 7) == 1).mean()), "beam_converged": float(((st & 7) == 2).mean()),
            "failed": float(((st & 7) == 4).mean()), "mean_alg_iters": float(it.mean()),
            "kernel_ms_per_step": kernel_ms(pr, steps)}
    steps_s = ms_total * 1e-3
    res.update(value=world * len(decs) * sh.B * steps / steps_s, ms_per_step=ms_total / steps, clocks=clocks,
               roofline=roofline, gpu_launches=int(sum(pr["kernel_launches"] for pr in prof_graph)),
               exec_bp_iters_per_step={"seed": float(exec_iters[0]) / steps, "round": float(exec_iters[1]) / steps,
                                       "seed_batched": float(exec_iters[2]) / steps})
    # each width timed alone, with its own roofline
    for preset, d, o in zip(SYN_PRESETS, decs, outs):
        ms_w, _, _, prof_w = run_region([d], [o])
        rl, _ = alu_roofline(prof_w, prob.n_edges, dev, "small case of the same DEM", shots=sh.B * steps, M=prob.M)
        res["per_width"][preset].update(value=world * sh.B * steps / (ms_w * 1e-3), ms_per_step=ms_w / steps,
                                        roofline=rl)
    # binary16 message storage at w = 32, timed alone beside the single-
    # precision decoder of the same width: the batch streams its messages, so
    # half the bytes per message is where 16-bit storage can pay
    from paper_2512_07057_gb300 import binding as BB
    d16 = D.BeamSearchDecoder(prob, D.make_params("beam32_340iters", ms_scale=ALPHA, msg_precision=BB.BSD_FP16,
                                                  workspace_bytes=int(workspace_gb * (1 << 30))), device=dev)
    o16 = d16.alloc_outputs(sh.B)
    res["launch_shapes"]["beam32_340iters_fp16"] = autotune(d16, synd, 16384)
    ms16, _, _, prof16 = run_region([d16], [o16])
    rl16, _ = alu_roofline(prof16, prob.n_edges, dev, "small case of the same DEM", shots=sh.B * steps,
                           msg_bytes=2, M=prob.M)
    st16 = D.from_torch_words(o16.status)
    ref32 = outs[SYN_PRESETS.index("beam32_340iters")]
    same = (D.from_torch_words(o16.corrections) == D.from_torch_words(ref32.corrections)).all(axis=1)
    fp32_ms = res["per_width"]["beam32_340iters"]["ms_per_step"]
    res["fp16_beam32"] = {
        "value": world * sh.B * steps / (ms16 * 1e-3), "ms_per_step": ms16 / steps, "msg_bytes": 2,
        "speedup_vs_fp32_same_width": fp32_ms / (ms16 / steps),
        "ler": ler_of(prob, sh, D.from_torch_words(o16.obs_flips), st16 & 7),
        "near_tie_rerun_fraction": float(((st16 & BB.BSD_STATUS_FP32_RERUN) != 0).mean()),
        "corrections_equal_to_fp32_fraction": float(same.mean()),
        "kernel_ms_per_step": kernel_ms(prof16[0], steps), "roofline": rl16}
    d16.close()
    if e2e_args is not None:
        res["e2e"] = e2e_host(decs, [(w, prob, sh) for w in SYN_PRESETS], e2e_args, dev)
    for d in decs:
        d.close()
    if cpu_seconds:
        tot_n = tot_t = 0.0
        for preset in SYN_PRESETS:
            base, run = cpu_baseline_of([(preset, prob, sh)], cpu_seconds / 3, preset, single_s=1.5)
            res["per_width"][preset]["cpu_baseline"] = base
            tot_n += run["n"]
            tot_t += run["dt"]
        res["cpu_baseline"] = {"value": tot_n / tot_t, "unit": "syndromes/s", "cores": cores(), "kind": "oracle",
                               "sample": "the per-width samples together (per_width.*.cpu_baseline), "
                                         "double-precision oracle"}
    return res


def run_synthetic(args, rank: int, world: int, local_rank: int):
    """The 936 x 8800 synthetic DEM decoded with beam widths 8, 32 and 64 (the
    matching Table I presets), 10^6 seeded shots each per step."""
    import torch
    import torch.distributed as dist

    from __graft_entry__ import build
    from paper_2512_07057_gb300 import workloads as W

    torch.cuda.set_device(local_rank)
    dev = local_rank
    if rank == 0:
        build()
    if world > 1:
        dist.barrier()
        build()
    prob = W.synthetic_dem()
    sh = W.sample_shots(prob, args.shots, W.shot_seed("synthetic_dem", rank))
    res = synthetic_widths(prob, sh, dev, args.steps, args.warmup, world, rank, args.workspace_gb,
                           None if (rank != 0 or args.no_cpu_baseline) else args.cpu_seconds,
                           e2e_args=args if (rank == 0 and not args.no_e2e) else None)
    line = {
        "metric": METRIC, "value": res["value"], "unit": "syndromes/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": SYN_WORKLOAD, "code": f"synthetic DEM {prob.M} x {prob.N}, {prob.n_edges} edges",
                   "shots_per_width_per_gpu": sh.B, "syndromes_per_step_per_gpu": len(SYN_PRESETS) * sh.B,
                   "l2": "flushed before every timed step (256 MiB write outside the step events)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "launch_shapes": res["launch_shapes"]},
        "exec_bp_iters_per_step": res["exec_bp_iters_per_step"],
        "roofline": res["roofline"], "gpu_launches": res["gpu_launches"],
        "per_width": res["per_width"], "clocks": res["clocks"], "fp16_beam32": res["fp16_beam32"],
    }
    if "e2e" in res:
        line["e2e"] = res["e2e"]
    if "cpu_baseline" in res:
        line["cpu_baseline"] = res["cpu_baseline"]
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_xyz(args, rank: int, world: int, local_rank: int):
    """XYZ decoding (H with both stabilizer types) against XZ decoding (the X
    and Z components decoded separately) of the same depolarizing shots, with
    the beam decoder and with plain BP; the line's value is the XYZ beam
    decoder's throughput."""
    import torch
    import torch.distributed as dist

    from __graft_entry__ import build
    from paper_2512_07057_gb300 import decoder as D
    from paper_2512_07057_gb300 import workloads as W

    torch.cuda.set_device(local_rank)
    dev = local_rank
    if rank == 0:
        build()
    if world > 1:
        dist.barrier()
        build()
    nshots = args.shots if args.shots != 1_000_000 else XYZ_SHOTS
    budget = int(args.workspace_gb * (1 << 30)) // 4
    work, decs, synd, outs, tuned = [], [], [], [], {}
    for p in XYZ_PS:
        prob = W.bb_xyz_code_capacity(12, 6, p)
        sh = W.sample_shots(prob, nshots, W.shot_seed(f"bb144_xyz_p{p}", rank))
        work.append((p, prob, sh))
        d = D.BeamSearchDecoder(prob, D.make_params(XYZ_PRESET, ms_scale=ALPHA, workspace_bytes=budget), device=dev)
        synd.append(D.to_torch_words(sh.syndromes, dev))
        decs.append(d)
        outs.append(d.alloc_outputs(sh.B))
        tuned[str(p)] = autotune(d, synd[-1], 16384)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=f"cuda:{dev}")
    stream = torch.cuda.current_stream(dev)

    def step():
        for d, s_, o in zip(decs, synd, outs):
            d.decode(s_, o, stream=stream)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize(dev)
    tr_args = (decs, step, flush, stream, dev, args.steps, world, rank)
    ms_steps, _, clocks, prof_graph = timed_region(*tr_args, profiled=False, sample_clocks=True)
    _, _, _, prof = timed_region(*tr_args, profiled=True, sample_clocks=False)
    ms_total = float(sum(ms_steps))
    if world > 1:
        t = torch.tensor([ms_total], dtype=torch.float64, device=f"cuda:{dev}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    roofline, _ = alu_roofline(prof, work[0][1].n_edges, dev, "small case")
    # LER: XYZ and XZ, beam decoder and plain BP (max_rounds 0, the preset's first run)
    per_p = {}
    for (p, prob, sh), o, s_ in zip(work, outs, synd):
        fail_xyz = _failures(prob, sh, o)
        zp, xp = W.bb_xz_parts(12, 6, p)
        s1, s2 = W.split_bits(sh.syndromes, prob.M, zp.M)
        o1, o2 = W.split_bits(sh.obs, prob.K, zp.K)
        res = {"xyz_beam": float(fail_xyz.mean())}
        plain = D.BeamSearchDecoder(prob, D.make_params(XYZ_PRESET, ms_scale=ALPHA, max_rounds=0,
                                                        workspace_bytes=budget), device=dev)
        res["xyz_plain_bp"] = float(_failures(prob, sh, plain.decode(s_)).mean())
        plain.close()
        for mode, mr in (("beam", None), ("plain_bp", 0)):
            fails = np.zeros(sh.B, bool)
            for part, sp, op in ((zp, s1, o1), (xp, s2, o2)):
                kw = {} if mr is None else {"max_rounds": 0}
                dd = D.BeamSearchDecoder(part, D.make_params(XYZ_PRESET, ms_scale=ALPHA, workspace_bytes=budget,
                                                             **kw), device=dev)
                fails |= _failures(part, W.Shots(syndromes=sp, obs=op, errors=None),
                                   dd.decode(D.to_torch_words(sp, dev)))
                dd.close()
            res[f"xz_{mode}"] = float(fails.mean())
        res["xz_over_xyz_beam"] = res["xz_beam"] / res["xyz_beam"] if res["xyz_beam"] > 0 else None
        per_p[str(p)] = res
    steps_s = ms_total * 1e-3
    line = {
        "metric": METRIC, "value": world * sum(sh.B for _, _, sh in work) * args.steps / steps_s,
        "unit": "syndromes/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_total / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": XYZ_WORKLOAD, "code": "[[144,12,12]] BB, H = [H_X on (Z,Y); H_Z on (X,Y)], "
                                                     "144 x 432, 1728 edges",
                   "shots_per_p_per_gpu": nshots, "l2": "flushed before every timed step (256 MiB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU", "launch_shapes": tuned},
        "roofline": roofline, "gpu_launches": int(sum(pr["kernel_launches"] for pr in prof_graph)),
        "ler": per_p, "clocks": clocks,
    }
    if rank == 0 and not args.no_cpu_baseline:
        r, n, dt = oracle_rate(work, args.cpu_seconds, cores(), XYZ_PRESET)
        line["cpu_baseline"] = {"value": r, "unit": "syndromes/s", "cores": cores(), "kind": "oracle",
                                "sample": f"first {n} shots of each p batch, double-precision oracle, {dt:.1f} s"}
    if rank == 0 and not args.no_e2e:
        line["e2e"] = e2e_host(decs, work, args, dev)
    if rank == 0:
        print(json.dumps(line), flush=True)
    for d in decs:
        d.close()


def _failures(prob, sh, out):
    """Logical failures per shot: a wrong observable vector or no converged correction."""
    import torch

    from paper_2512_07057_gb300 import decoder as D
    from paper_2512_07057_gb300 import workloads as W
    torch.cuda.synchronize()
    st = D.from_torch_words(out.status) & 7
    o = W.unpack_bits(D.from_torch_words(out.obs_flips)[:, :(prob.K + 31) // 32], prob.K)
    t = W.unpack_bits(sh.obs, prob.K)
    return (o != t).any(1) | (st == 4)


def run_latency(args, rank: int, world: int, local_rank: int):
    """Low-latency mode: each syndrome decoded alone (B = 1) as soon as it is
    submitted; latency = host wall time from the call to the correction and
    status being readable on the host.  Two paths: the syndrome resident on
    the device (decode + a 12-byte device-to-host read of status and the first
    correction words), and host buffers end to end (bsd_decode_host).  Each
    with the small-chunk graph (grids sized to one shot) and without it."""
    import torch

    from __graft_entry__ import build
    from paper_2512_07057_gb300 import decoder as D
    from paper_2512_07057_gb300 import workloads as W

    torch.cuda.set_device(local_rank)
    dev = local_rank
    if rank == 0:
        build()
    cases = [("bb144_cc_p0.03", W.bb144_code_capacity(0.03), "beam32_340iters"),
             ("phenom_p0.003", W.bb_phenomenological(12, 6, 12, 3e-3, 3e-3), "beam32_340iters"),
             ("synthetic_dem", W.synthetic_dem(), "beam32_340iters")]
    n = args.steps * LAT_PER_STEP
    stream = torch.cuda.current_stream(dev)
    results, all_mean = {}, []
    for name, prob, preset in cases:
        sh = W.sample_shots(prob, n + 64, W.shot_seed(f"latency_{name}", rank))
        synd = D.to_torch_words(sh.syndromes, dev)
        res = {}
        for mode, sb in (("small_graph", 0), ("full_grid", -1)):
            d = D.BeamSearchDecoder(prob, D.make_params(preset, ms_scale=ALPHA, workspace_bytes=1 << 30,
                                                        small_batch=sb), device=dev)
            out = d.alloc_outputs(1)
            host = torch.empty(3, dtype=torch.int32).pin_memory()
            lat = np.zeros(n)
            for i in range(-32, n):                       # 32 warm-up decodes
                k = (i + 64) % (n + 64)
                t0 = time.perf_counter()
                d.decode(synd[k:k + 1], out, stream=stream)
                host[0:1].copy_(out.status, non_blocking=True)
                host[1:3].copy_(out.corrections[0, :2], non_blocking=True)
                stream.synchronize()
                if i >= 0:
                    lat[i] = time.perf_counter() - t0
            hs = torch.from_numpy(sh.syndromes.view(np.int32)).pin_memory()
            WN, WK = (prob.N + 31) // 32, max((prob.K + 31) // 32, 1)
            hc = torch.empty(WN, dtype=torch.int32).pin_memory()
            ho = torch.empty(WK, dtype=torch.int32).pin_memory()
            hst = torch.empty(1, dtype=torch.int32).pin_memory()
            lat_h = np.zeros(n)
            row = hs.shape[1] * 4
            for i in range(-32, n):
                k = (i + 64) % (n + 64)
                t0 = time.perf_counter()
                d.decode_host_ptrs(hs.data_ptr() + k * row, 1, hc.data_ptr(), ho.data_ptr(), hst.data_ptr(), None,
                                   stream=stream)
                if i >= 0:
                    lat_h[i] = time.perf_counter() - t0
            # the request loop (bsd_serve_*): host buffers in and out, no
            # launch for a syndrome whose seed BP ends the search
            lat_s = None
            if mode == "small_graph":
                from paper_2512_07057_gb300 import binding as BB
                d.serve_start(idle_ms=1000)
                lat_s = np.zeros(n)
                vp = lambda a: C.c_void_p(a)
                for i in range(-32, n):
                    k = (i + 64) % (n + 64)
                    t0 = time.perf_counter()
                    BB.bsd_serve_decode(d.h, vp(hs.data_ptr() + k * row), vp(hc.data_ptr()), vp(ho.data_ptr()),
                                        vp(hst.data_ptr()), None)
                    if i >= 0:
                        lat_s[i] = time.perf_counter() - t0
                d.serve_stop()
            d.close()
            us = lambda a, q: float(np.quantile(a, q) * 1e6)
            stats = lambda a: {"mean": float(a.mean() * 1e6), "p50": us(a, 0.5), "p99": us(a, 0.99),
                               "p99.9": us(a, 0.999), "max": float(a.max() * 1e6)}
            res[mode] = {"device_resident_us": stats(lat), "host_buffers_us": stats(lat_h)}
            if lat_s is not None:
                res[mode]["request_loop_us"] = stats(lat_s)
        results[name] = {"preset": preset, "syndromes": n, **res}
        all_mean.append(res["small_graph"]["request_loop_us"]["mean"])
    mean_us = float(np.mean(all_mean))
    line = {"metric": METRIC, "value": 1e6 / mean_us, "unit": "syndromes/s (one at a time)", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_us * LAT_PER_STEP / 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": LAT_WORKLOAD, "step": f"{LAT_PER_STEP} single-syndrome decodes",
                       "timer": "host wall clock per syndrome, submit to result on the host",
                       "value_from": "request loop (bsd_serve_decode), mean over the three cases",
                       "l2": "not flushed: consecutive single decodes, the latency setting"},
            "latency": results,
            "context": "the paper reports 99.9 percentile decoding times per syndrome on one CPU core for its "
                       "circuit-level [[144,12,12]] workload (Tables II-III); that workload is not available here"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_num_results(args, rank: int, world: int, local_rank: int):
    """num_results > 1: the best-LER preset of Table I (32 results, the
    minimum-weight one returned) against the same beam with the first
    result; throughput, LER, iterations and where the time goes (the
    selection kernel holds the deduplication of results)."""
    import torch
    import torch.distributed as dist

    from __graft_entry__ import build
    from paper_2512_07057_gb300 import decoder as D
    from paper_2512_07057_gb300 import workloads as W

    torch.cuda.set_device(local_rank)
    dev = local_rank
    if rank == 0:
        build()
    if world > 1:
        dist.barrier()
        build()
    nshots = args.shots if args.shots != 1_000_000 else NR_SHOTS
    work = []
    for p in NR_PS:
        prob = W.bb144_code_capacity(p)
        work.append((p, prob, W.sample_shots(prob, nshots, W.shot_seed(f"bb144_cc_p{p}", rank))))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=f"cuda:{dev}")
    stream = torch.cuda.current_stream(dev)
    forms = {}
    for preset in NR_PRESETS:
        decs, synd, outs, tuned = [], [], [], {}
        for p, prob, sh in work:
            d = D.BeamSearchDecoder(prob, D.make_params(preset, ms_scale=ALPHA,
                                                        workspace_bytes=int(args.workspace_gb * (1 << 30)) // 2),
                                    device=dev)
            decs.append(d)
            synd.append(D.to_torch_words(sh.syndromes, dev))
            outs.append(d.alloc_outputs(sh.B))
            tuned[str(p)] = autotune(d, synd[-1], 16384)

        def step():
            for d, s_, o in zip(decs, synd, outs):
                d.decode(s_, o, stream=stream)

        for _ in range(args.warmup):
            flush.fill_(1.0)
            step()
        torch.cuda.synchronize(dev)
        tr_args = (decs, step, flush, stream, dev, args.steps, world, rank)
        ms_steps, _, clocks, prof_graph = timed_region(*tr_args, profiled=False, sample_clocks=True)
        _, _, _, prof = timed_region(*tr_args, profiled=True, sample_clocks=False)
        ms_total = float(sum(ms_steps))
        if world > 1:
            t = torch.tensor([ms_total], dtype=torch.float64, device=f"cuda:{dev}")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms_total = float(t.item())
        roofline, exec_iters = alu_roofline(prof, work[0][1].n_edges, dev, "16000-shot case")
        per_p = {}
        for (p, prob, sh), o, pr in zip(work, outs, prof):
            st = D.from_torch_words(o.status)
            it = D.from_torch_words(o.iters).astype(np.int64)
            per_p[str(p)] = {"ler": ler_of(prob, sh, D.from_torch_words(o.obs_flips), st & 7),
                             "seed_converged": float(((st & 7) == 1).mean()),
                             "beam_converged": float(((st & 7) == 2).mean()),
                             "failed": float(((st & 7) == 4).mean()), "mean_alg_iters": float(it.mean()),
                             "kernel_ms_per_step": kernel_ms(pr, args.steps)}
        forms[preset] = {"value": world * sum(sh.B for _, _, sh in work) * args.steps / (ms_total * 1e-3),
                         "unit": "syndromes/s", "ms_per_step": ms_total / args.steps, "roofline": roofline,
                         "exec_bp_iters_per_step": {"seed": float(exec_iters[0]) / args.steps,
                                                    "round": float(exec_iters[1]) / args.steps},
                         "gpu_launches": int(sum(pr["kernel_launches"] for pr in prof_graph)), "clocks": clocks,
                         "per_p": per_p, "launch_shapes": tuned}
        for d in decs:
            d.close()
    main = forms[NR_PRESETS[1]]
    line = {"metric": METRIC, "value": main["value"], "unit": "syndromes/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": NR_WORKLOAD, "shots_per_p_per_gpu": nshots,
                       "l2": "flushed before every timed step (256 MiB write outside the step events)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": main["roofline"], "gpu_launches": main["gpu_launches"], "clocks": main["clocks"],
            "forms": forms, "one_result_over_32_results": forms[NR_PRESETS[0]]["value"] / main["value"]}
    if rank == 0 and not args.no_cpu_baseline:
        r, n, dt = oracle_rate(work, args.cpu_seconds, cores(), NR_PRESETS[1])
        line["cpu_baseline"] = {"value": r, "unit": "syndromes/s", "cores": cores(), "kind": "oracle",
                                "sample": f"first {n} shots of each p batch, beam64_32res_640iters, double-precision "
                                          f"oracle, {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def e2e_host(decs, work, args, dev):
    """Same metric through bsd_decode_host: pinned host syndromes in, host results out."""
    import torch
    bufs = []
    h2d = d2h = 0
    for d, (p, prob, sh) in zip(decs, work):
        s = torch.from_numpy(sh.syndromes.view(np.int32)).pin_memory()
        WN, WK = (prob.N + 31) // 32, max((prob.K + 31) // 32, 1)
        c = torch.empty((sh.B, WN), dtype=torch.int32).pin_memory()
        o = torch.empty((sh.B, WK), dtype=torch.int32).pin_memory()
        st = torch.empty(sh.B, dtype=torch.int32).pin_memory()
        it = torch.empty(sh.B, dtype=torch.int32).pin_memory()
        bufs.append((d, s, c, o, st, it, sh.B))
        h2d += s.numel() * 4
        d2h += (c.numel() + o.numel() + st.numel() + it.numel()) * 4
    stream = torch.cuda.current_stream(dev)

    def step():
        for d, s, c, o, st, it, nb in bufs:
            d.decode_host_ptrs(s.data_ptr(), nb, c.data_ptr(), o.data_ptr(), st.data_ptr(), it.data_ptr(),
                               stream=stream)

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    shots = sum(b[-1] for b in bufs)
    return {"value": shots * args.steps / dt, "unit": "syndromes/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "api": "bsd_decode_host (pinned host buffers)"}


def _traffic_record(kernel: str, edges: int, msg_bytes: int = 0):
    """(bytes per unit of work, unit) recorded for `kernel` on a problem with
    `edges` edges (and, where the record names it, `msg_bytes` bytes per
    stored message), if the kernel sources the record names are unchanged
    since the capture; the unit is a candidate-iteration (decoder kernels), a
    launch (the unrolled passes) or a shot (the seed stage)."""
    import glob
    import re
    for path in glob.glob(os.path.join(ROOT, "profiles", f"{kernel}_traffic_*.md")):
        txt = open(path).read()
        h = re.search(r"^source_hash: (\w+)$", txt, re.M)
        k = re.search(r"^kernel: (\w+)$", txt, re.M)
        b = re.search(r"^bytes_per_(candidate_iteration|launch|shot): ([0-9.]+)$", txt, re.M)
        e = re.search(r"^edges: (\d+)$", txt, re.M)
        mb = re.search(r"^msg_bytes: (\d+)$", txt, re.M)
        src = re.search(r"^sources: (.+)$", txt, re.M)
        if e is not None and int(e.group(1)) != edges:
            continue
        if mb is not None and msg_bytes and int(mb.group(1)) != msg_bytes:
            continue
        files = src.group(1).split() if src else None
        if h and k and b and k.group(1) == kernel and h.group(1) == _source_hash(files):
            return float(b.group(2)), b.group(1)
    return None


def _memory_record(kernel: str, edges: int, msg_bytes: int = 0):
    """The DRAM throughput and L2 hit rate that ncu measured for one launch of
    `kernel` (profiles/<kernel>_memory_*.md) on a problem with `edges` edges,
    if the kernel sources the record names are unchanged since the capture."""
    import glob
    import re
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", f"{kernel}_memory_*.md"))):
        txt = open(path).read()
        f = {m.group(1): m.group(2).strip() for m in re.finditer(r"^(\w+): (.+)$", txt, re.M)}
        if f.get("kernel") != kernel or "dram_bytes" not in f or "duration_us" not in f:
            continue
        if "edges" in f and int(f["edges"]) != edges:
            continue
        if "msg_bytes" in f and msg_bytes and int(f["msg_bytes"]) != msg_bytes:
            continue
        if f.get("source_hash") != _source_hash(f["sources"].split() if "sources" in f else None):
            continue
        dram_b, dur = float(f["dram_bytes"]), float(f["duration_us"]) * 1e-6
        return {"dram_gbs": dram_b / dur / 1e9, "l2_hit": float(f["l2_hit_pct"]) / 100.0,
                "dram_bytes_captured": dram_b, "duration_us_captured": dur * 1e6, "case": f.get("case", ""),
                "record": os.path.relpath(path, ROOT)}
    return None


def _source_hash(files=None) -> str:
    """sha256[:16] over the named files of the CUDA sources (all of them by default)."""
    import hashlib
    d = os.path.join(ROOT, "paper_2512_07057_gb300", "csrc")
    h = hashlib.sha256()
    for f in (files if files else sorted(os.listdir(d))):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def main():
    global NO_AUTOTUNE
    args = parse()
    NO_AUTOTUNE = args.no_autotune
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        if args.workload == "phenom_precision":
            run_precision(args, rank, world, local_rank)
        elif args.workload == "unrolled_training":
            run_unrolled(args, rank, world, local_rank)
        elif args.workload == "synthetic_dem":
            run_synthetic(args, rank, world, local_rank)
        elif args.workload == "xyz":
            run_xyz(args, rank, world, local_rank)
        elif args.workload == "latency":
            run_latency(args, rank, world, local_rank)
        elif args.workload == "num_results":
            run_num_results(args, rank, world, local_rank)
        else:
            run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
