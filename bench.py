#!/usr/bin/env python
"""QAOA max-cut benchmark: layers/s of the whole hot path on one B300 (or N independent replicas).

One step = the whole path once: reset to |+>^n (launch control), p levels of {cost phase with
the on-the-fly cut count, RX mixer on every qubit}, and <C> with the norm reduced in FP64 and
read back to the host.  Default workload: near-3-regular graph on n = 33 vertices (one degree-2
vertex, since a 3-regular graph on an odd vertex count does not exist), seed 0, p = 8 seeded
levels, complex64 state of 2^33 amplitudes (64 GiB), larger than L2, so no L2 flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--n 33] [--p 8]
  python bench.py --serve      # request-serving mode (qaoa_submit / qaoa_poll), its own JSON line
  python bench.py --grad       # adjoint-gradient mode (qaoa_gradient), its own JSON line

Prints ONE JSON line on rank 0.  On one GPU the default line also carries the rest of the metric,
measured after the headline on the same GPU (`--no-extra` skips them): `n30` (3-regular n = 30,
p = 8: layers/s and the pass roofline), `grad` (adjoint gradients/s on G(24, 0.5), p = 10) and
`serve` (the request stream at 2000/s and at a sustainable 300/s: the server against the plain
one-request-at-a-time C API, requests/s and p50/p99 latency).  `--impl reference` times the CPU
oracle (gate-level complex128 simulator, the paper's Algorithm 1) on a bounded sample of the same
workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2312_03019_b300 import inputs as I  # noqa: E402

METRIC = "QAOA layers/s"
UNIT = "layers/s"
# DRAM bytes (read + write) per launch of each read+write pass kind (the library's profile
# categories: [0] the mixer-only pass (group 0 at n <= 33), [1] the fused boundary pass with the cost phase,
# [2] the last pass with <C>), complex64, unit weights, per amplitude, from one ncu capture of
# the same kernel build at n = 28 (the full-size state is too large for a multi-metric capture),
# against 16 B per amplitude algorithmic (4.2950 GB per launch at n = 28): 4.2362, 4.2352 and
# 4.2360 GB.  A pass's last writes are still in L2 when it ends.  A pass reads and writes every
# amplitude once, so the traffic scales with 2^n.
NCU_TRAFFIC_BY_KIND = (4.2362e9 / 2 ** 28, 4.2352e9 / 2 ** 28, 4.2360e9 / 2 ** 28)
NOMINAL_HBM_GBS = 7700.0  # B300 HBM3e, nominal (the fractions are also given against it)
PASS_KINDS = ("tile_kernel, mixer-only pass (read+write; the group-0 pass at n <= 33)",
              "tile_kernel, fused boundary pass with the cost phase (read+write)",
              "tile_kernel, last pass with <C> (read+write)")
SYNTH_KIND = "tile_kernel, first pass (synthesises |+>, write only)"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=33)
    ap.add_argument("--p", type=int, default=8)
    ap.add_argument("--prec", choices=["c64", "c128"], default="c64")
    ap.add_argument("--cpu-sample-n", type=int, default=26)
    ap.add_argument("--cpu-sample-seconds", type=float, default=10.0,
                    help="the CPU baseline times oracle levels at --cpu-sample-n until this much time has passed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the untimed complex128 rerun that gives the line's error against FP64")
    ap.add_argument("--weighted", action="store_true",
                    help="edge weights U[0.1, 2] on the same graph (Algorithm 2 path), for context")
    ap.add_argument("--cpu-report", action="store_true",
                    help="time the CPU oracle on the host's cores (all threads and one) at the small configurations")
    ap.add_argument("--grad", action="store_true",
                    help="gradient mode: d<C>/d(gamma, beta) by qaoa_gradient on G(24, 0.5), p = 10")
    ap.add_argument("--grad-n", type=int, default=24,
                    help="--grad: vertices of the G(n, 0.5) graph (default 24, the gradient workload)")
    ap.add_argument("--grad-p", type=int, default=10, help="--grad: levels (default 10)")
    ap.add_argument("--serve", action="store_true",
                    help="serving mode: an open-loop Poisson request stream through qaoa_submit/qaoa_poll")
    ap.add_argument("--serve-requests", type=int, default=4096)
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-budget-gib", type=float, default=64.0)
    ap.add_argument("--serve-sustain-rate", type=float, default=300.0,
                    help="second arrival rate of the serving comparison, one the GPU keeps up with")
    ap.add_argument("--extra-serve-requests", type=int, default=1024,
                    help="requests per arrival rate in the default line's serving block")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the n=30, gradient and serving blocks of the default line")
    return ap.parse_args()


def workload(n: int, p: int, weighted: bool = False):
    g = I.regular3(n, 0)
    if weighted:
        g = I.random_weights(g, seed=0, lo=0.1, hi=2.0)
    gamma, beta = I.angles(p, 0)
    return g, gamma, beta


def workload_name(g, p, prec):
    fam = "near-3-regular (one degree-2 vertex)" if g.n % 2 else "3-regular"
    if g.weights is not None:
        fam += " edge-weighted U[0.1, 2]"
    elem = "complex64" if prec == "c64" else "complex128"
    cut = "weighted C(z) in fixed point on the fly" if g.weights is not None else "cut values on the fly"
    return (f"{fam} graph n={g.n}, |E|={g.m}, seed 0, p={p} seeded levels, {elem} state of 2^{g.n} "
            f"amplitudes, {cut}, <C> and norm reduced in FP64")


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# --------------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------------- CPU oracle

def oracle_level_seconds(n_s: int, p_levels: int = 1):
    """Time `p_levels` oracle levels (cost layer + mixer layer, gate by gate) at n_s."""
    import oracle
    g, gamma, beta = workload(n_s, p_levels)
    psi = oracle.initial_state(n_s)
    t0 = time.perf_counter()
    for k in range(p_levels):
        psi = oracle.cost_layer(g, gamma[k], psi)
        psi = oracle.mixer_layer(n_s, beta[k], psi)
    return time.perf_counter() - t0, g


def gates_per_level(g):
    return 3 * g.m + 1 + g.n  # CNOT-RZ-CNOT per edge, global phase, one RX per qubit


def oracle_layers_per_s(n_target: int, m_target_graph, n_s: int, min_seconds: float):
    """Oracle layers/s at n_target extrapolated from levels timed at n_s (as many as fit in
    about min_seconds, at most 8): every gate streams the whole state, so time scales with 2^n
    times the gate count."""
    import oracle
    levels, total, gs = 0, 0.0, None
    while levels < 8 and (levels == 0 or total < min_seconds):
        t, gs = oracle_level_seconds(n_s)
        levels += 1
        total += t
    scale = (2.0 ** (n_target - n_s)) * gates_per_level(m_target_graph) / gates_per_level(gs)
    return levels / (total * scale), total, levels, gs, oracle.threads()


def cpu_baseline_block(args, g_target):
    v, t, levels, gs, cores = oracle_layers_per_s(g_target.n, g_target, args.cpu_sample_n, args.cpu_sample_seconds)
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"{levels} oracle levels (gate-level complex128, Algorithm 1) on the same graph family at "
                       f"n={gs.n} (|E|={gs.m}) took {t:.2f} s on {cores} threads; scaled to n={g_target.n} "
                       f"by 2^n x gate count ({gates_per_level(gs)} -> {gates_per_level(g_target)} gates/level)")}


def paper_method_block(g_target, n_s: int = 24):
    """The paper's own CPU method (Opt_u: launch control, Algorithm 2 + 3 cost layer, mixer gate
    by gate, OpenMP) timed for one level at n_s on the same graph family, scaled to the target
    size by 2^n x n (its per-level work: n popcounts per amplitude and n mixer passes)."""
    import baseline
    gs = I.regular3(n_s, 0)
    ga, be = I.angles(1, 0)
    baseline.run(gs, ga, be)  # warm-up (page faults, thread start)
    t0 = time.perf_counter()
    baseline.run(gs, ga, be)
    t = time.perf_counter() - t0
    scale = (2.0 ** (g_target.n - n_s)) * g_target.n / n_s
    return {"value": 1.0 / (t * scale), "unit": UNIT, "cores": baseline.threads(), "kind": "paper method (Opt_u)",
            "sample": (f"one level of Opt_u (launch control + Algorithm 2/3 + gate-by-gate mixer, OpenMP) on "
                       f"3-regular n={n_s} took {t:.3f} s (includes the launch-control fill); scaled to "
                       f"n={g_target.n} by 2^n x n"),
            "measured_layers_per_s_at_sample": 1.0 / t}


# --------------------------------------------------------------------------------- reference arm

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    g, gamma, beta = workload(args.n, args.p)
    import oracle
    warm = max(3, args.warmup)
    n_s = args.cpu_sample_n
    for _ in range(warm):
        oracle_level_seconds(n_s)
    times = []
    gs = None
    for _ in range(args.steps):
        t, gs = oracle_level_seconds(n_s)
        times.append(t)
    scale = (2.0 ** (args.n - n_s)) * gates_per_level(g) / gates_per_level(gs)
    t_step = statistics.mean(times) * scale  # one layer at the target size
    value = 1.0 / t_step
    cores = oracle.threads()
    rec = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": warm, "ms_per_step": t_step * 1e3 * args.p,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": (f"oracle levels timed at n={n_s} (|E|={gs.m}, same graph family), value "
                                f"extrapolated to: " + workload_name(g, args.p, "c128")),
                   "n": args.n, "p": args.p, "edges": g.m, "sample_n": n_s, "sample_edges": gs.m,
                   "extrapolated_to_n": args.n, "extrapolated": True,
                   "extrapolation": "time x 2^(n - sample_n) x (gates per level at n) / (gates per level at sample_n)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": (f"each step: one oracle level at n={n_s} (|E|={gs.m}, same family) on {cores} "
                                    f"threads, scaled to n={args.n} by 2^n x gate count (extrapolated, not "
                                    f"an n={args.n} timing)")},
        "measured_ms_per_level_at_sample_n": statistics.mean(times) * 1e3,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(rec), flush=True)
    return 0


# --------------------------------------------------------------------------------- replicas

def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest of every rank's x (the slowest replica's time): an all-reduce MAX over the
    process group (NCCL on the GPUs, gloo in the CPU tests), x itself on a single process."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_rank: float, seconds_max: float, world: int) -> float:
    """Whole-job rate of `world` independent replicas: every rank's units over the slowest time."""
    return world * units_per_rank / seconds_max


# --------------------------------------------------------------------------------- our arm

def roofline_from_profile(prof, g, elem, known_traffic, ms_total):
    """The roofline object of the dominant pass kind and the fraction of peak per layer, from the
    library's per-pass CUDA events over a timed region of ms_total milliseconds."""
    peak, peak_kind = measured_peaks()
    if prof["pass_launches"] <= 0:
        return None, None
    # the dominant kernel: the pass kind with the most event time in the timed steps (one
    # instantiation of tile_kernel each); the all-pass mean is given beside it
    bytes_per_launch = 2.0 * elem * (1 << g.n)
    kinds = []
    for c, name in enumerate(PASS_KINDS):
        L = prof["kind_launches"][c]
        if not L:
            continue
        ms = prof["kind_ms"][c] / L
        ach = bytes_per_launch / (ms / 1e3) / 1e9
        kinds.append({"kernel": name, "launches": L, "launch_ms": ms, "achieved": ach, "frac": ach / peak,
                      "frac_nominal": ach / NOMINAL_HBM_GBS,
                      "share_of_timed_ms": prof["kind_ms"][c] / ms_total,
                      "traffic": NCU_TRAFFIC_BY_KIND[c] * (1 << g.n) if known_traffic else None})
    if prof["synth_launches"]:
        ms = prof["synth_ms"] / prof["synth_launches"]
        ach = bytes_per_launch / 2 / (ms / 1e3) / 1e9
        kinds.append({"kernel": SYNTH_KIND, "launches": prof["synth_launches"], "launch_ms": ms, "achieved": ach,
                      "frac": ach / peak, "frac_nominal": ach / NOMINAL_HBM_GBS,
                      "share_of_timed_ms": prof["synth_ms"] / ms_total, "traffic": None})
    dom = max((k for k in kinds if k["kernel"] != SYNTH_KIND), key=lambda d: d["launch_ms"] * d["launches"])
    mean_ms = prof["pass_ms"] / prof["pass_launches"]
    roof = {"bound": "hbm", "achieved": dom["achieved"], "peak": peak, "unit": "GB/s", "frac": dom["frac"],
            "traffic": dom["traffic"], "peak_kind": f"{peak_kind} copy bandwidth", "kernel": dom["kernel"],
            "peak_nominal": NOMINAL_HBM_GBS, "frac_nominal": dom["achieved"] / NOMINAL_HBM_GBS,
            "bytes_per_launch": bytes_per_launch, "launch_ms": dom["launch_ms"], "launches": dom["launches"],
            "all_read_write_passes": {"launches": prof["pass_launches"], "launch_ms": mean_ms,
                                      "achieved": bytes_per_launch / (mean_ms / 1e3) / 1e9,
                                      "frac": bytes_per_launch / (mean_ms / 1e3) / 1e9 / peak},
            "per_kind": kinds}
    # every byte the step's passes move (read+write passes and the write-only first pass) over
    # the passes' event time: the fraction of peak per layer
    moved = prof["pass_bytes"] + prof["synth_bytes"]
    layer_frac = moved / ((prof["pass_ms"] + prof["synth_ms"]) / 1e3) / 1e9 / peak
    return roof, layer_frac


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:  # one replica per GPU: bind the group to this rank's device
        dist.init_process_group("nccl", device_id=dev)

    from paper_2312_03019_b300 import build as bld
    bld.build()
    from paper_2312_03019_b300 import binding as B

    g, gamma, beta = workload(args.n, args.p, args.weighted)
    warm = max(3, args.warmup)
    st = B.QAOAState(g, args.prec, device=dev)
    stream = st.stream

    def step():
        st.reset()
        st.apply_layers(gamma, beta)
        return st.expectation()

    for _ in range(warm):
        step()

    def barrier():
        if world > 1:
            dist.barrier(device_ids=[local])

    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    gpu_id = f"GPU-{uuid}" if uuid is not None else str(local)
    sampler = ClockSampler(gpu_id)

    B.qaoa_profile_enable(st.handle, True)
    barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    results = []
    for _ in range(args.steps):
        results.append(step())
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    prof = B.qaoa_profile_read(st.handle)
    B.qaoa_profile_enable(st.handle, False)

    ms_max = max_over_ranks(ms, world, dev)
    value = replica_rate(args.steps * args.p, ms_max / 1e3, world)

    # end to end through the public API with host inputs and a host result
    e2e = None
    if not args.no_e2e:
        for _ in range(2):
            h = B.qaoa_state_init(g, args.prec, st.buffer.data_ptr(), st.nbytes, stream.cuda_stream)
            B.qaoa_apply_layers(h, gamma, beta)
            B.qaoa_expectation(h)
            B.qaoa_state_free(h)
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            h = B.qaoa_state_init(g, args.prec, st.buffer.data_ptr(), st.nbytes, stream.cuda_stream)
            B.qaoa_apply_layers(h, gamma, beta)
            B.qaoa_expectation(h)
            B.qaoa_state_free(h)
        torch.cuda.synchronize(dev)
        el = time.perf_counter() - t0
        e2e = {"value": replica_rate(args.steps * args.p, max_over_ranks(el, world, dev), world), "unit": UNIT,
               "h2d_bytes_per_step": int(8 * g.m + 16 * args.p), "d2h_bytes_per_step": 16,
               "note": "graph and angles go host to device as kernel parameters; <C> and norm come back"}

    peak, peak_kind = measured_peaks()
    elem = 8 if args.prec == "c64" else 16
    roof, layer_frac = roofline_from_profile(prof, g, elem, args.prec == "c64" and g.weights is None, ms_max)
    state_gbs = value * 2.0 * elem * (1 << g.n) / 1e9

    rec = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": warm,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.prec == "c64" else "f64", "data": "synthetic",
        "config": {"workload": workload_name(g, args.p, args.prec), "n": g.n, "p": args.p, "edges": g.m,
                   "state_bytes": elem << g.n, "l2": "state larger than L2 (no flush needed)",
                   "parallelism": f"{world} independent replicas" if world > 1 else "single GPU"},
        "state_gbs_algorithmic": state_gbs,
        "hbm_frac_algorithmic": state_gbs / world / peak,
        "hbm_frac_passes": layer_frac,
        "passes_per_step": (prof["pass_launches"] + prof["synth_launches"]) / args.steps,
        "roofline": roof,
        "gpu_launches": prof["kernel_launches"],
        "clocks": clocks,
        "e2e": e2e,
        "expectation": results[-1][0], "norm": results[-1][1],
    }
    if rank == 0 and not args.no_accuracy:
        rec["accuracy"] = accuracy_block(B, g, gamma, beta, st, args.prec, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        del st
        torch.cuda.empty_cache()
        rec["cpu_baseline"] = cpu_baseline_block(args, g)
        rec["cpu_paper_method"] = paper_method_block(g)
    if rank == 0 and world == 1 and not args.no_extra:
        # the rest of the metric on the same GPU, after the headline: n = 30, the adjoint
        # gradient workload and the serving workload (each untimed by the headline's clock)
        st = None
        torch.cuda.empty_cache()
        t0 = time.perf_counter()
        if args.n != 30:
            rec["n30"] = size_block(B, 30, 8, "c64", steps=10, warmup=3)
        rec["grad"] = grad_block(B, "c64", False, 10, 3, not args.no_accuracy)
        # the same at a size where neither state fits in L2 (G(28, 0.5), p = 6; timing only)
        g28 = grad_block(B, "c64", False, 4, 3, False, n=28, p=6)
        rec["grad"]["n28"] = {k: g28[k] for k in ("value", "unit", "ms_per_gradient", "ms_per_forward",
                                                  "gradient_over_forward")}
        rec["grad"]["n28"]["workload"] = g28["config"]["workload"]
        rec["serve"] = serve_block(B, count=args.extra_serve_requests,
                                   rates=(args.serve_rate, args.serve_sustain_rate), prec="c64")
        rec["extra_blocks_s"] = time.perf_counter() - t0
    if rank == 0:
        print(json.dumps(rec), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def size_block(B, n, p, prec="c64", steps=10, warmup=3):
    """Layers/s and the pass kernels' roofline on (near-)3-regular n, seed 0, p seeded levels:
    the same step as the headline (reset, p levels, <C> read back), device-timed with CUDA events
    on the library's stream."""
    import torch
    g, gamma, beta = workload(n, p)
    st = B.QAOAState(g, prec)

    def step():
        st.reset()
        st.apply_layers(gamma, beta)
        return st.expectation()

    for _ in range(max(3, warmup)):
        step()
    B.qaoa_profile_enable(st.handle, True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st.stream)
    for _ in range(steps):
        c, nrm = step()
    e1.record(st.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = B.qaoa_profile_read(st.handle)
    B.qaoa_profile_enable(st.handle, False)
    elem = 8 if prec == "c64" else 16
    roof, layer_frac = roofline_from_profile(prof, g, elem, prec == "c64", ms)
    st.close()
    torch.cuda.empty_cache()
    value = steps * p / (ms / 1e3)
    peak, _ = measured_peaks()
    return {"metric": METRIC, "value": value, "unit": UNIT, "steps": steps, "ms_per_step": ms / steps,
            "config": {"workload": workload_name(g, p, prec), "n": n, "p": p, "edges": g.m,
                       "state_bytes": elem << n},
            "hbm_frac_algorithmic": value * 2.0 * elem * (1 << n) / 1e9 / peak, "hbm_frac_passes": layer_frac,
            "roofline": roof, "expectation": c, "norm": nrm}


def accuracy_block(B, g, gamma, beta, st, prec, dev):
    """The error of this line's result against FP64: after the timed region, the same circuit is
    run once more in complex64 on `st` and once in complex128 on the same GPU (the tests pin the
    complex128 path to the p = 1 closed form at these sizes), and the two states are compared on
    the device in chunks.  Untimed."""
    import torch
    if prec != "c64":
        return {"reference": "none: this run is complex128 (FP64 throughout)"}
    need = (16 << g.n) + (6 << 30)
    free, _ = torch.cuda.mem_get_info(dev)
    if free < need:
        return {"unavailable": f"the complex128 rerun needs {need / 2**30:.0f} GiB, {free / 2**30:.0f} GiB free"}
    st.reset()
    st.apply_layers(gamma, beta)
    c64, n64 = st.expectation()
    ref = B.QAOAState(g, "c128", device=dev)
    try:
        ref.apply_layers(gamma, beta)
        c128, n128 = ref.expectation()
        t64, t128 = st.as_tensor(), ref.as_tensor()
        ip = torch.zeros((), dtype=torch.complex128, device=dev)
        worst = 0.0
        chunk = 1 << 27
        for i in range(0, t64.numel(), chunk):
            a = t64[i:i + chunk].to(torch.complex128)
            b = t128[i:i + chunk]
            ip += torch.vdot(b, a)
            worst = max(worst, (a - b).abs().max().item())
            del a, b
        fid = abs(ip.item()) ** 2 / (n64 * n128)
        del t64, t128
    finally:
        ref.close()
        torch.cuda.empty_cache()
    return {"reference": "the same circuit in complex128 on this GPU", "expectation": c64,
            "expectation_ref": c128, "abs_err": c64 - c128, "rel_err": (c64 - c128) / c128 if c128 else None,
            "norm_err": n64 - 1.0, "fidelity_deficit": 1.0 - fid,
            "max_amp_err_rel": worst * 2.0 ** (g.n / 2), "untimed": True}


def serve_stream(B, reqs, cfg):
    """Submit every request at its arrival time (open loop), then collect all results.
    Latency and makespan come from the server's own clock (t_submit, t_done)."""
    sv = B.qaoa_server_create(**cfg)
    try:
        # warm-up: one request of each kind and size, so graph capture and first-use costs stay out
        seen = {}
        for r in reqs:
            seen.setdefault((r.graph.n, r.want_grad), r)
        warm = [B.qaoa_submit(sv, r.graph, r.gamma, r.beta, r.want_grad) for r in seen.values()]
        while warm:
            warm = [t for t in warm if B.qaoa_poll(sv, t) is None]
            time.sleep(0.001)
        base = B.qaoa_server_stats_read(sv)
        t0 = B.qaoa_server_time(sv)
        tickets = []
        for r in reqs:
            while B.qaoa_server_time(sv) - t0 < r.arrival_s:
                pass
            while True:
                try:
                    tickets.append(B.qaoa_submit(sv, r.graph, r.gamma, r.beta, r.want_grad))
                    break
                except B.QAOAError as e:
                    if e.status != B.QAOA_ERR_AGAIN:
                        raise
                    time.sleep(0.0002)
        res = {}
        while len(res) < len(tickets):
            for t in tickets:
                if t not in res:
                    out = B.qaoa_poll(sv, t)
                    if out is not None:
                        res[t] = out
            time.sleep(0.002)
        stats = B.qaoa_server_stats_read(sv)
    finally:
        B.qaoa_server_destroy(sv)
    done = [res[t] for t in tickets]
    bad = [d for d in done if d["status"] != 0]
    if bad:
        raise RuntimeError(f"{len(bad)} requests failed")
    lat = sorted(d["t_done"] - d["t_submit"] for d in done)
    span = max(d["t_done"] for d in done) - min(d["t_submit"] for d in done)
    q = lambda f: lat[min(len(lat) - 1, int(f * len(lat)))] * 1e3
    stats = {k: stats[k] - base.get(k, 0) if k != "arena_peak_bytes" else stats[k] for k in stats}
    return {"requests_per_s": len(done) / span, "p50_ms": q(0.50), "p99_ms": q(0.99), "makespan_s": span,
            "stats": stats}, done


def plain_stream(B, reqs, prec="c64"):
    """The same open-loop stream run one request at a time through the plain C API (no server):
    each request, once it has arrived, gets qaoa_state_init on a preallocated device buffer,
    qaoa_apply_layers + qaoa_expectation (or qaoa_gradient) and qaoa_state_free, in arrival order.
    Latency = completion - scheduled arrival, on the host clock."""
    import torch
    nmax = max(r.graph.n for r in reqs)
    nbytes = B.qaoa_state_bytes(nmax, prec)
    buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    work = torch.empty(nbytes, dtype=torch.uint8, device="cuda") if any(r.want_grad for r in reqs) else None
    stream = torch.cuda.current_stream().cuda_stream

    def one(r):
        h = B.qaoa_state_init(r.graph, prec, buf.data_ptr(), nbytes, stream)
        try:
            if r.want_grad:
                c, dg, db = B.qaoa_gradient(h, r.gamma, r.beta, work.data_ptr(), nbytes)
            else:
                B.qaoa_apply_layers(h, r.gamma, r.beta)
                c, _ = B.qaoa_expectation(h)
                dg = db = None
        finally:
            B.qaoa_state_free(h)
        return c, dg, db

    seen = {}
    for r in reqs:  # warm-up: one request of each size and kind, as for the server
        if (r.graph.n, r.want_grad) not in seen:
            seen[(r.graph.n, r.want_grad)] = one(r)
    torch.cuda.synchronize()
    out = []
    t0 = time.perf_counter()
    for r in reqs:
        while time.perf_counter() - t0 < r.arrival_s:
            pass
        c, dg, db = one(r)
        out.append({"expectation": c, "d_gamma": dg, "d_beta": db,
                    "latency": time.perf_counter() - t0 - r.arrival_s})
    span = time.perf_counter() - t0
    lat = sorted(d["latency"] for d in out)
    q = lambda f: lat[min(len(lat) - 1, int(f * len(lat)))] * 1e3
    del buf, work
    torch.cuda.empty_cache()
    return {"requests_per_s": len(out) / span, "p50_ms": q(0.50), "p99_ms": q(0.99), "makespan_s": span}, out


SERVE_CFG = dict(prec="c64", max_inflight=64, queue_capacity=8192, max_batch=64, streams=8, use_graphs=True)


def serve_block(B, count=1024, rates=(2000.0, 300.0), budget_gib=64.0, prec="c64"):
    """The serving workload (Poisson arrivals, n ~ U{14..28}, half 3-regular and half G(n, 0.3),
    p ~ U{1..6}, 25 % with gradient, complex64) at each arrival rate: the server
    (qaoa_submit / qaoa_poll) against the plain one-request-at-a-time C API on the same stream,
    with the largest difference between their results."""
    import numpy as np
    rows = []
    for rate in rates:
        reqs = I.request_stream(count=count, rate_hz=rate, seed=0).requests
        cfg = dict(SERVE_CFG, prec=prec, hbm_budget_bytes=int(budget_gib * (1 << 30)))
        served, done = serve_stream(B, reqs, cfg)
        plain, pdone = plain_stream(B, reqs, prec)
        diff_c = max(abs(a["expectation"] - b["expectation"]) / max(1, r.graph.m)
                     for a, b, r in zip(done, pdone, reqs))
        diff_g = max([float(np.max(np.abs(np.concatenate([a["d_gamma"] - b["d_gamma"], a["d_beta"] - b["d_beta"]]))))
                      for a, b, r in zip(done, pdone, reqs) if r.want_grad] or [0.0])
        rows.append({"arrival_rate_hz": rate, "requests": len(reqs), "served": served, "plain_c_api": plain,
                     "speedup_vs_plain": served["requests_per_s"] / plain["requests_per_s"],
                     "max_diff_C_over_edges": diff_c, "max_diff_grad": diff_g})
    return {"metric": "QAOA serving throughput and latency", "unit": "requests/s",
            "config": {"workload": f"{count} seeded requests (the first of the 4096-request stream's draws), "
                                   "n 14-28 (half 3-regular, half G(n,0.3)), p 1-6, 25% with gradient",
                       "prec": prec, "hbm_budget_gib": budget_gib,
                       "server": {k: v for k, v in SERVE_CFG.items() if k != "prec"},
                       "plain_c_api": "qaoa_state_init / apply_layers / expectation (or qaoa_gradient) / "
                                      "state_free per request, in arrival order, one at a time"},
            "rates": rows}


def run_cpu_report(args):
    """The oracle (gate-level complex128, Algorithm 1) timed on this host with all threads and
    with one: 3-regular n=10, p=1 (gamma 0.4, beta 0.3); one level of G(26, 0.5) (one thread:
    one level at n=20, scaled by 2^n x gate count); the FP64 adjoint gradient of G(14, 0.5),
    p=10."""
    import oracle
    allt = oracle.threads()
    rows = []

    def timed(fn, reps=1):
        fn()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        return (time.perf_counter() - t0) / reps

    for threads in (allt, 1):
        oracle.set_threads(threads)
        g1, ga1, be1 = I.workload_n10_regular3_p1()
        t1 = timed(lambda: oracle.expectation(g1, oracle.qaoa_state(g1, ga1, be1)), reps=20)
        g2, ga2, be2 = I.workload_gnp26_p4()
        if threads == 1:
            gs = I.gnp(20, 0.5, 0)
            ts, _ = oracle_level_seconds_graph(gs, ga2[0], be2[0])
            t2 = ts * 2.0 ** 6 * gates_per_level(g2) / gates_per_level(gs)
            how = "one level at n=20 scaled by 2^n x gate count"
        else:
            t2, _ = oracle_level_seconds_graph(g2, ga2[0], be2[0])
            how = "one level measured"
        g4 = I.gnp(14, 0.5, 0)
        ga4, be4 = I.angles(10, 0)
        t4 = timed(lambda: oracle.adjoint_gradient(g4, ga4, be4), reps=3)
        rows.append({"threads": threads, "n10_p1_ms": t1 * 1e3, "gnp26_level_s": t2, "gnp26_level": how,
                     "gnp14_p10_adjoint_ms": t4 * 1e3})
    oracle.set_threads(allt)
    print(json.dumps({"mode": "cpu-report", "kind": "oracle", "host_threads": allt, "rows": rows}), flush=True)
    return 0


def oracle_level_seconds_graph(g, gamma, beta):
    """One oracle level (cost layer, gate by gate, and mixer layer) on graph g."""
    import oracle
    psi = oracle.initial_state(g.n)
    t0 = time.perf_counter()
    psi = oracle.cost_layer(g, gamma, psi)
    psi = oracle.mixer_layer(g.n, beta, psi)
    return time.perf_counter() - t0, g


def grad_block(B, prec="c64", weighted=False, steps=10, warmup=3, accuracy=True, n=24, p=10):
    """Adjoint gradients per second on G(24, 0.5), seed 0, p = 10 (20 parameters), through
    qaoa_gradient (forward levels, lambda = C psi, reverse sweep; host-synchronous per call),
    beside the forward evaluation of the same circuit and the 4p forward evaluations central
    differences would need.  Other sizes: G(n, 0.5), seed 0, with p seeded levels."""
    import numpy as np
    import torch

    if (n, p) == (24, 10):
        g, gamma, beta = I.workload_gnp24_p10()
    else:
        g = I.gnp(n, 0.5, 0)
        gamma, beta = I.angles(p, 0)
    if weighted:  # the same graph with seeded U[0.1, 2] edge weights (Algorithm 2 path)
        g = I.random_weights(g, seed=0, lo=0.1, hi=2.0)
    s = B.QAOAState(g, prec)
    work = torch.empty(s.nbytes, dtype=torch.uint8, device="cuda")
    warm, K = max(3, warmup), max(steps, 10)

    def grad():
        return B.qaoa_gradient(s.handle, gamma, beta, work.data_ptr(), s.nbytes)

    def forward():
        s.reset()
        s.apply_layers(gamma, beta)
        return s.expectation()

    for _ in range(warm):
        grad()
        forward()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K):
        c, dg, db = grad()
    t_grad = (time.perf_counter() - t0) / K
    t0 = time.perf_counter()
    for _ in range(K):
        forward()
    t_fwd = (time.perf_counter() - t0) / K
    p = len(gamma)
    rec = {"metric": "QAOA adjoint gradients/s", "value": 1.0 / t_grad, "unit": "gradients/s",
           "higher_is_better": True, "steps": K, "warmup": warm, "dtype": "f32" if prec == "c64" else "f64",
           "config": {"workload": f"G({n}, 0.5) seed 0{' with edge weights U[0.1, 2]' if weighted else ''}, "
                                  f"|E|={g.m}, p={p} seeded levels ({2 * p} parameters), "
                                  f"{'complex64' if prec == 'c64' else 'complex128'}, host-timed calls"},
           "ms_per_gradient": t_grad * 1e3, "ms_per_forward": t_fwd * 1e3,
           "gradient_over_forward": t_grad / t_fwd,
           "speedup_vs_central_differences": 4 * p * t_fwd / t_grad,
           "expectation": c}
    s.close()
    del work
    if prec == "c64" and accuracy:  # the same gradient in complex128 (untimed)
        r = B.QAOAState(g, "c128")
        try:
            c2, dg2, db2 = r.gradient(gamma, beta)
        finally:
            r.close()
        ref = np.concatenate([dg2, db2])
        err = np.abs(np.concatenate([dg, db]) - ref)
        rec["accuracy"] = {"reference": "the same gradient in complex128 on this GPU", "abs_err_C": c - c2,
                           "max_abs_err_grad": float(err.max()),
                           "max_err_grad_rel": float(err.max() / max(1e-300, np.abs(ref).max())), "untimed": True}
    torch.cuda.empty_cache()
    return rec


def run_grad(args):
    import torch

    if not torch.cuda.is_available():
        raise SystemExit("the gradient benchmark needs a CUDA device")
    from paper_2312_03019_b300 import build as bld
    bld.build()
    from paper_2312_03019_b300 import binding as B

    rec = grad_block(B, args.prec, args.weighted, args.steps, args.warmup, not args.no_accuracy, args.grad_n,
                     args.grad_p)
    rec.update({"n_gpus": 1, "mode": "grad", "data": "synthetic"})
    print(json.dumps(rec), flush=True)
    return 0


def serve_accuracy(B, reqs, done, samples=32):
    """Error of served results against FP64: a seeded sample of the requests is run alone in
    complex128 (QAOAState, and its adjoint gradient where the request asked for one) and
    compared with what the server returned.  Untimed."""
    import numpy as np
    import torch
    rng = np.random.default_rng(0)
    pick = sorted(rng.choice(len(reqs), size=min(samples, len(reqs)), replace=False).tolist())
    worst_c, worst_g, ngrad = 0.0, 0.0, 0
    for i in pick:
        r, d = reqs[i], done[i]
        s = B.QAOAState(r.graph, "c128")
        try:
            if r.want_grad:
                c, dg, db = s.gradient(r.gamma, r.beta)
                scale = max(1.0, float(np.max(np.abs(np.concatenate([dg, db])))))
                err = max(np.max(np.abs(d["d_gamma"] - dg)), np.max(np.abs(d["d_beta"] - db))) / scale
                worst_g = max(worst_g, float(err))
                ngrad += 1
            else:
                s.apply_layers(r.gamma, r.beta)
                c, _ = s.expectation()
            worst_c = max(worst_c, abs(d["expectation"] - c) / max(1, r.graph.m))
        finally:
            s.close()
    torch.cuda.empty_cache()
    return {"reference": "the same requests run alone in complex128 on this GPU", "sampled": len(pick),
            "with_gradient": ngrad, "max_abs_err_C_over_edges": worst_c,
            "max_grad_err_rel": worst_g if ngrad else None, "untimed": True}


def run_serve(args):
    import torch

    if not torch.cuda.is_available():
        raise SystemExit("the serving benchmark needs a CUDA device")
    from paper_2312_03019_b300 import binding as B

    stream = I.request_stream(count=args.serve_requests, rate_hz=args.serve_rate, seed=0)
    reqs = stream.requests
    budget = int(args.serve_budget_gib * (1 << 30))
    served, done = serve_stream(B, reqs, dict(hbm_budget_bytes=budget, prec=args.prec, max_inflight=64,
                                              queue_capacity=8192, max_batch=64, streams=8, use_graphs=True))
    serial, done_serial = serve_stream(B, reqs, dict(hbm_budget_bytes=budget, prec=args.prec, max_inflight=1,
                                                     queue_capacity=8192, max_batch=1, streams=1, use_graphs=False))
    # the two configurations must agree request by request (same kernels, same reduction order)
    for a, b in zip(done, done_serial):
        if a["expectation"] != b["expectation"]:
            raise RuntimeError("served and serial results differ")
    plain, _ = plain_stream(B, reqs, args.prec)
    rec = {"metric": "QAOA serving throughput", "value": served["requests_per_s"], "unit": "requests/s",
           "higher_is_better": True, "n_gpus": 1, "dtype": "f32" if args.prec == "c64" else "f64",
           "data": "synthetic", "mode": "serve",
           "config": {"workload": f"{len(reqs)} requests, Poisson {args.serve_rate:g}/s, n 14-28 "
                                  "(half 3-regular, half G(n,0.3)), p 1-6, 25% with gradient",
                      "prec": args.prec, "hbm_budget_gib": args.serve_budget_gib},
           "served": served, "serial": serial, "plain_c_api": plain,
           "speedup_vs_serial": served["requests_per_s"] / serial["requests_per_s"],
           "speedup_vs_plain": served["requests_per_s"] / plain["requests_per_s"]}
    if args.prec == "c64" and not args.no_accuracy:
        rec["accuracy"] = serve_accuracy(B, reqs, done)
    print(json.dumps(rec), flush=True)
    return 0


def main():
    args = parse_args()
    if args.serve:
        return run_serve(args)
    if args.grad:
        return run_grad(args)
    if args.cpu_report:
        return run_cpu_report(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
