#!/usr/bin/env python
"""Benchmark of the Glasma + CPIC hot path on GB300.

Workload (one "step"): 64 Glasma events of uneven lattices (16 each of 128^2,
256^2, 384^2, 512^2; L = 10 fm; g^2 mu ~ U[1.5, 2.5] GeV), each with 10k charm
quarks, evolved in FP32 (FP64 accumulators) from tau = dtau to tau = 1 fm/c:
a full run of the batch, every event to its own step count (103..410).
Metric: site-updates/s (value) and particle-steps/s, whole job over N GPUs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--mode graph|persistent|eager|per_event]
  python bench.py --impl reference ...   (the FP64 CPU oracle on the host cores)
  python bench.py --workload warm_start  (tau = 0+ link solve of 16 events at 1024^2: Newton
                                          iterations and wall time, cold vs learned warm start)
  python bench.py --workload single_512  (one 512^2 event, 100k charm + 100k beauty, FP32 and
                                          FP64, nearest-grid-point and cloud-in-cell gathers)
  python bench.py --workload jets        (4 events of 1024^2, 1M massless partons each)
  python bench.py --workload scans       (the p_T and p_x scans of Figs. 1-2)
  python bench.py --workload correlators (the estimators of Eqs. 4-5 on a 1024^2 event)

N > 1: launched by torchrun, one rank per GPU; each rank runs an independent
replica batch (different event seeds), no data-path collective ("weak").
"""
import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Glasma site-updates/s & Wong particle-steps/s on 1 GB300 vs plain, at fixed tol"
WORKLOAD = ("64 MV events, 16 each of 128^2/256^2/384^2/512^2 (L=10 fm, g2mu~U[1.5,2.5] GeV), "
            "10k charm/event, FP32 fields+particles with FP64 accumulators, tau 0->1 fm/c")
HBARC_GEV_FM = 0.1973269804
BYTES_PER_SITE = 448  # algorithmic bytes of one FP32 site-update (12-real links, read + write once)
BYTES_PER_PARTICLE = 132  # algorithmic bytes of one FP32 particle-step (state read + write, p0 read)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--mode", default="auto", choices=["auto", "graph", "persistent", "eager", "per_event"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--g2mu", type=float, default=2.0, help="MV scale g^2 mu (GeV) of the scans workload")
    p.add_argument("--field-variant", type=int, default=-1,
                   help="fixed field tile variant (default: tuned on the batch)")
    p.add_argument("--push-variant", type=int, default=-1, help="fixed push kernel with --field-variant")
    p.add_argument("--workload", default="batch", choices=["batch", "warm_start", "correlators", "single_512", "scans", "jets"],
                   help="batch: the 64-event coupled evolution (default); warm_start: the tau = 0+ link "
                        "solve of 16 events at 1024^2, cold vs learned warm start; correlators: the lattice-"
                        "correlator estimators of Eqs. 4-5 on a 1024^2 event; single_512: one 512^2 event with "
                        "100k charm + 100k beauty, FP32 and FP64; scans: the p_T and p_x scans of Figs. 1-2; "
                        "jets: 4 events of 1024^2 with 1M partons each")
    return p.parse_args()


# ---------------------------------------------------------------- distributed plumbing
def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(v, ws):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- peaks, traffic
def measured_peak():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the field kernel's device code (su3.cuh, field.cuh); kernels_field.cu only
    instantiates tile shapes, which the profile summary names."""
    h = hashlib.sha256()
    for f in ("su3.cuh", "field.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2307_07999_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic_per_site():
    """DRAM bytes per site of the field kernel from the committed ncu summary, if it was
    taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "field_step_fp32_ncu.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    m = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    b = re.search(r"dram_bytes_per_site:\s*([0-9.]+)", txt)
    if not m or not b or m.group(1) != kernel_source_hash():
        return None
    return float(b.group(1))


# ---------------------------------------------------------------- CPU baseline: the FP64 oracle
def oracle_prepare(rank=0):
    """The oracle's own initial state of one 256^2 event of the batch and its 10k charm
    quarks at their formation step (the sample the CPU timings run on)."""
    import oracle as O
    from paper_2307_07999_gb300 import workloads as W

    evs, pps = W.batched_uneven(rank=rank)
    e = 16  # first 256^2 event
    gp, pp = evs[e], pps[e]
    n = gp.n
    a_fm = gp.L_fm / n
    a = a_fm / W.HBARC
    st, iters, fails = O.glasma_init(n, gp.n_sheets, gp.g2mu_GeV * a, gp.m_ir_GeV * a, gp.seed, gp.dtau_over_a)
    P = O.particles_init(pp.n_particles, n, pp.mass_GeV * a, 0, 0.0, pp.p_max_GeV * a, pp.seed)
    n_form = int(round(pp.tau_form_fm / (gp.dtau_over_a * a_fm)))
    n_steps = int(math.ceil(gp.tau_end_fm / (gp.dtau_over_a * a_fm) - 1e-9))
    while st.step < n_form:
        st = O.field_step(st, gp.dtau_over_a)
    return {"O": O, "gp": gp, "pp": pp, "n": n, "a": a, "st0": st, "P0": P, "n_steps": n_steps}


def oracle_pass(ctx):
    """One pass of the oracle's coupled FP64 evolution tau_form -> tau_end from the
    prepared state; returns (coupled steps, seconds)."""
    O, gp, pp, a = ctx["O"], ctx["gp"], ctx["pp"], ctx["a"]
    st, P = ctx["st0"].copy(), ctx["P0"].copy()
    t0 = time.perf_counter()
    steps = 0
    while st.step < ctx["n_steps"]:
        nx = O.field_step(st, gp.dtau_over_a)
        O.push(P, st, nx, gp.dtau_over_a, pp.mass_GeV * a)
        st = nx
        steps += 1
    return steps, time.perf_counter() - t0


def oracle_sample(budget_s=15.0, rank=0, single_thread=False):
    """The oracle as it stands on a bounded sample of the workload: one 256^2 event of
    the batch with its 10k charm quarks, coupled steps from tau_form until the budget
    is spent.  Returns site-updates/s, particle-steps/s and the sample description."""
    ctx = oracle_prepare(rank)
    O, gp, pp, a, n = ctx["O"], ctx["gp"], ctx["pp"], ctx["a"], ctx["n"]
    # the coupled evolution from tau_form to tau_end, repeated from the same state at
    # tau_form until the budget is spent (each pass runs to the end)
    t0 = time.perf_counter()
    steps = passes = 0
    while time.perf_counter() - t0 < budget_s or passes == 0:
        k, _ = oracle_pass(ctx)
        steps += k
        passes += 1
    dt = time.perf_counter() - t0
    cores = O.set_threads(0)
    out = {
        "site_updates_per_s": n * n * steps / dt,
        "particle_steps_per_s": pp.n_particles * steps / dt,
        "cores": cores,
        "sample": f"one {n}^2 event of the batch + its {pp.n_particles} charm quarks: {passes} pass(es) of the "
                  f"coupled FP64 evolution tau_form -> tau_end ({steps} steps, {dt:.1f} s)",
        "seconds": dt,
    }
    if not single_thread:
        return out
    # one thread: the first coupled steps from tau_form (about 5 s)
    O.set_threads(1)
    st, P = ctx["st0"].copy(), ctx["P0"].copy()
    t1 = time.perf_counter()
    steps1 = 0
    while (time.perf_counter() - t1 < 5.0 or steps1 == 0) and st.step < ctx["n_steps"]:
        nx = O.field_step(st, gp.dtau_over_a)
        O.push(P, st, nx, gp.dtau_over_a, pp.mass_GeV * a)
        st = nx
        steps1 += 1
    dt1 = time.perf_counter() - t1
    O.set_threads(cores)
    out["single_thread"] = {"site_updates_per_s": n * n * steps1 / dt1, "particle_steps_per_s": pp.n_particles * steps1 / dt1,
                            "sample": f"the first {steps1} coupled steps from tau_form on one thread ({dt1:.1f} s)"}
    return out


def run_reference(args, ws, rank):
    """The oracle as the reference arm: its own initial state prepared once (untimed), then
    each step one pass of the coupled FP64 evolution of the 256^2 sample event from
    tau_form to tau_end (a fixed bounded sample, a few seconds on the host cores)."""
    if rank != 0:
        return
    ctx = oracle_prepare(rank)
    n, pp = ctx["n"], ctx["pp"]
    per_step = []
    for i in range(args.warmup + args.steps):
        k, dt = oracle_pass(ctx)
        if i >= args.warmup:
            per_step.append((k, dt))
    steps = sum(k for k, _ in per_step)
    secs = sum(dt for _, dt in per_step)
    v = n * n * steps / secs
    ps = pp.n_particles * steps / secs
    cores = ctx["O"].set_threads(0)
    sample = (f"one {n}^2 event of the batch + its {pp.n_particles} charm quarks: per step one pass of the coupled "
              f"FP64 evolution tau_form -> tau_end ({per_step[0][0]} coupled steps)")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "site-updates/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * secs / len(per_step),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "particle_steps_per_s": ps,
        "config": {"workload": WORKLOAD, "oracle_sample": sample},
        "cpu_baseline": {"value": v, "unit": "site-updates/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "site-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def run_ours(args, ws, rank, local):
    import torch

    import paper_2307_07999_gb300 as G
    from paper_2307_07999_gb300 import workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    evs, pps = W.batched_uneven(rank=rank)
    with torch.cuda.stream(stream):
        B = G.Batch(evs, pps, device=dev, stream=stream)
        ic_fail = B.init()
        if args.field_variant >= 0:
            # a fixed tile shape and push kernel (profiling runs: the tuner's timings are
            # distorted under a profiler, so the shape the plain run chose is given here)
            B.set_variant(args.field_variant)
            B.set_push_variant(max(args.push_variant, 0))
            tile_v = args.field_variant
            tile_ms = [float("nan")] * G.field_tile_variants(G.GLASMA_FP32)
        else:
            # tile shape of the batched field kernel: timed on this batch, fastest kept
            tile_v, tile_ms = B.tune(steps=8)
    su, ps = B.work()
    shapes = [G.field_tile_shape(G.GLASMA_FP32, v) for v in range(len(tile_ms))]
    tile = shapes[tile_v]

    def timed(mode, K, W_):
        for _ in range(W_):
            B.run(mode)
        torch.cuda.synchronize()
        barrier(ws)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            B.run(mode)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
        return e0.elapsed_time(e1) / K

    modes = ["graph", "persistent"] if args.mode == "auto" else [args.mode]
    best = None
    for m in modes:
        try:
            t = timed(m, 1, 1)
        except G.GlasmaError as ex:
            print(f"mode {m} unavailable: {ex}", file=sys.stderr)
            continue
        if best is None or t < best[1]:
            best = (m, t)
    mode = best[0]

    # the field launches of the timed runs bracketed by event-record nodes in the graph
    in_graph_timing = mode in ("graph", "eager")
    if in_graph_timing:
        B.set_graph_timing(True)
    clk = ClockSampler(local)
    clk.start()
    ms = timed(mode, args.steps, args.warmup)
    clocks = clk.stop()
    graph_t = B.graph_times() if in_graph_timing else None
    ms = max_over_ranks(ms, ws)
    value = su * ws / (ms / 1000.0)
    pvalue = ps * ws / (ms / 1000.0)
    launches = B.launches(mode) * args.steps

    # end to end through the public API, right after the device-timed steps (same GPU state):
    # H2D of the initial state from pinned host memory, the run, D2H of every event's
    # broadening table, each step
    # The host-to-device copy of step k+1's state runs on a copy stream into a device
    # staging buffer while step k runs; each step then imports from the staging buffer
    # (device to device, on the batch stream).  Every step's H2D is inside the timed
    # region (the first one is not overlapped).
    nbytes = B.state_bytes()
    host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    B.export_state(host)
    staging = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    copy_stream = torch.cuda.Stream(device=dev)

    def e2e(K):
        d2h = 0
        staged = torch.cuda.Event()
        with torch.cuda.stream(copy_stream):
            staging.copy_(host, non_blocking=True)
            staged.record(copy_stream)
        for k in range(K):
            stream.wait_event(staged)
            B.import_state(staging)
            loaded = torch.cuda.Event()
            loaded.record(stream)
            B.run(mode)
            if k + 1 < K:
                copy_stream.wait_event(loaded)
                with torch.cuda.stream(copy_stream):
                    staging.copy_(host, non_blocking=True)
                    staged = torch.cuda.Event()
                    staged.record(copy_stream)
            tabs = [B.broadening(e) for e in range(B.E)]
            d2h = sum(t.nbytes for t in tabs)
        return d2h

    e2e(1)
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    d2h = e2e(args.steps)
    torch.cuda.synchronize()
    barrier(ws)
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1000.0 / args.steps, ws)

    # per-kernel durations (CUDA events around every launch, on the batch stream).  The dominant
    # kernel is the batched field step (448 B per site-update)
    pmode = "graph"
    if in_graph_timing:
        B.set_graph_timing(False)
    prof = B.profile(pmode)  # site counts per launch (and eager launch times)
    if graph_t is not None:
        # durations of the field launches of the last timed run (event-record nodes)
        field_ms, n_launch, _ = graph_t
        per_launch_ms = field_ms / n_launch
        share, other_ms, timing_src = field_ms / ms, ms - field_ms, "event-record nodes in the timed graph runs"
    else:
        per_launch_ms = prof["main_ms"] / prof["main_launches"]
        share = prof["main_ms"] / (prof["main_ms"] + prof["other_ms"])
        other_ms, timing_src = prof["other_ms"], "CUDA events around every launch of an eager run"
    bytes_per_launch = (BYTES_PER_SITE * prof["main_sites"] + BYTES_PER_PARTICLE * prof["main_particle_steps"]) \
        / prof["main_launches"]
    achieved = bytes_per_launch / (per_launch_ms / 1000.0) / 1e9
    peak, peak_kind = measured_peak()
    tps = ncu_traffic_per_site()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": (tps * prof["main_sites"] / prof["main_launches"] if tps else None),
                "kernel": f"k_field_step_tiles<{tile[0]},{tile[1]},{tile[2]}>",
                "peak_kind": f"{peak_kind} HBM copy (burst)",
                "algorithmic_bytes_per_launch": bytes_per_launch, "ms_per_launch": per_launch_ms,
                "launch_timing": timing_src,
                "share_of_step": share,
                "other_kernels_ms_per_run": other_ms}
    # the whole step against the same peak, algorithmic bytes 448 per site-update and
    # 132 per particle-step (the particle state; the gather's field reads not counted)
    whole = (BYTES_PER_SITE * su + BYTES_PER_PARTICLE * ps) / (ms / 1000.0) / 1e9
    roofline["whole_step"] = {"achieved": whole, "frac": whole / peak, "unit": "GB/s"}
    # the push's own roofline: its time per run is the step minus the field launches;
    # algorithmic bytes 132 per particle-step (particle state read + written), the field
    # reads of its gather listed beside them (35 groups of 32 B around the cell, or the
    # 18-group record of the record push, which the field launch also writes)
    if other_ms > 0:
        pa = BYTES_PER_PARTICLE * ps / (other_ms / 1000.0) / 1e9
        rec_push = B.push_variant == 2
        roofline["push"] = {"achieved": pa, "frac": pa / peak, "unit": "GB/s", "ms_per_run": other_ms,
                            "particle_steps_per_s": ps / (other_ms / 1000.0),
                            "algorithmic_bytes_per_particle_step": BYTES_PER_PARTICLE,
                            "gather_bytes_per_particle_step": 18 * 32 if rec_push else 35 * 32,
                            "gather": ("one 576 B record per particle (written by the field launch for occupied cells)"
                                       if rec_push else "35 field groups of 32 B around the particle's cell")}

    # plain one-event-per-launch GPU path on the same GPU
    plain = None
    if not args.no_plain:
        pms = timed("per_event", 1, 1)
        plain = {"value": su / (pms / 1000.0), "unit": "site-updates/s", "ms_per_step": pms,
                 "speedup_of_batched": pms / ms}


    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        r = oracle_sample(budget_s=15.0, single_thread=True)
        cpu = {"value": r["site_updates_per_s"], "unit": "site-updates/s", "cores": r["cores"], "kind": "oracle",
               "sample": r["sample"], "particle_steps_per_s": r["particle_steps_per_s"],
               "single_thread": r["single_thread"]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "site-updates/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "particle_steps_per_s": pvalue,
            "config": {"workload": WORKLOAD, "mode": mode,
                       "field_tile": f"{tile[0]}x{tile[1]}, {tile[2]} CTAs/SM " + ("(fixed)" if args.field_variant >= 0 else "(autotuned)"),
                       "push_kernel": {0: "fields through L1 (128-thread blocks, 3 per SM)",
                                       1: "fields staged in shared memory (32-thread blocks)",
                                       2: "gather records written by the field launch (128-thread blocks, 4 per SM)",
                                       3: "split: gather + contracted forces (3 blocks per SM), then the move (4 per SM)"}
                       .get(B.push_variant, "?")
                                      + (" (fixed)" if args.field_variant >= 0 else " (autotuned)"),
                       **({"persistent_kernel": "one cooperative launch: 32x4 field tiles dealt out statically, "
                                                "particle blocks through an atomic counter, 3 CTAs/SM; the field "
                                                "tile and push kernel above are the graph path's"}
                          if mode == "persistent" else {}),
                       "tile_tuning_ms_per_8_steps": ({f"{a}x{b}/{c}": round(t, 3) for (a, b, c), t in zip(shapes, tile_ms)}
                                                      if args.field_variant < 0 else None),
                       "site_updates_per_step": su,
                       "particle_steps_per_step": ps, "l2": "inputs larger than L2 (3.5 GB of field state)",
                       "ic_unconverged_links": ic_fail, "parallelism": f"{ws} independent replica batch(es)"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "plain_one_event_per_launch": plain,
            "e2e": {"value": su * ws / (e2e_ms / 1000.0), "unit": "site-updates/s", "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                    "pipeline": "H2D of step k+1 (pinned host -> device staging, copy stream) overlaps step k"},
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- learned warm start of the tau = 0+ solve
WS_EVAL, WS_TRAIN, WS_N = 16, 5, 1024


def run_warm_start(args, ws, rank, local):
    """Newton iterations per link and wall time of the tau = 0+ link solve to residual
    <= 1e-12, cold start (U1 U2) vs the learned warm start, on 16 MV events at 1024^2
    (L = 10 fm, g^2 mu = 2 GeV).  The network is trained first, by the library's own
    BF16 kernels, on the Newton-solved links of 5 other events (10.5M links)."""
    import torch

    import paper_2307_07999_gb300 as G
    from paper_2307_07999_gb300 import workloads as W

    torch.cuda.set_device(local)
    L, g2mu = 10.0, 2.0

    def event(seed):
        return G.Glasma(WS_N, L, g2mu_GeV=g2mu, precision=G.GLASMA_FP32, tau_end_fm=1.0, seed=seed, newton_tol=1e-12)

    t0 = time.perf_counter()
    Xs, Ts = [], []
    for e in range(WS_TRAIN):
        g = event(W.event_seed(5, 100 + e, rank))
        f, _, _ = g.init()
        X, T = G.ic_dataset(g)
        Xs.append(X)
        Ts.append(T)
        del g
    X, T = torch.cat(Xs), torch.cat(Ts)
    del Xs, Ts
    perm = torch.randperm(X.shape[0], device=X.device, generator=torch.Generator(device=X.device).manual_seed(rank))
    X, T = X[perm].contiguous(), T[perm].contiguous()
    net = G.WarmStartNet(seed=11 + rank)
    net.fit_scales(X, T)
    l0, _ = net.loss_grad(X[:65536], T[:65536])
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    loss = net.train(X, T, epochs=4, batch=4096, lr=2e-3)
    loss = net.train(X, T, epochs=4, batch=4096, lr=5e-4)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    n_train = X.shape[0]
    del X, T, perm

    def timed_init(g, warm):
        torch.cuda.synchronize()
        a = time.perf_counter()
        r = G.init_warm(g, net) if warm else g.init()
        torch.cuda.synchronize()
        return r, (time.perf_counter() - a) * 1000.0

    rows = []
    for e in range(WS_EVAL):
        seed = W.event_seed(5, e, rank)
        for warm in (False, True):
            g = event(seed)
            if e == 0:
                timed_init(g, warm)  # first-use costs (cuFFT plans, module loads) out of the timing
            (f, it, mx), ms = timed_init(g, warm)
            U = g.get_state()[0] if e == 0 else None
            rows.append((e, warm, f, it, mx, ms, U))
            del g
    cold = [r for r in rows if not r[1]]
    warm = [r for r in rows if r[1]]
    same = float(np.abs(cold[0][6] - warm[0][6]).max())
    it_c = statistics.mean(r[3] for r in cold)
    it_w = statistics.mean(r[3] for r in warm)
    ms_c = statistics.mean(r[5] for r in cold)
    ms_w = statistics.mean(r[5] for r in warm)
    links = 2 * WS_N * WS_N * WS_EVAL
    if rank == 0:
        line = {
            "metric": "tau=0+ link solve: Newton iterations per link to residual <= 1e-12, learned warm start",
            "value": it_w, "unit": "iterations/link", "n_gpus": ws, "steps": WS_EVAL, "warmup": 1,
            "ms_per_step": ms_w, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 Newton, bf16/f32 network", "data": "synthetic",
            "config": {"workload": f"{WS_EVAL} MV events at {WS_N}^2 (L={L} fm, g2mu={g2mu} GeV, m_IR=0.2 GeV, "
                                   f"10 sheets): {links} link solves",
                       "network": "36-128-128-16 tanh, BF16 weights, FP32 accumulation (hand-written kernels)",
                       "training": {"links": n_train, "events": WS_TRAIN, "epochs": 8, "batch": 4096,
                                    "loss_initial": l0, "loss_final": loss, "seconds": t_train,
                                    "dataset_seconds": t1 - t0}},
            "cold": {"iterations_per_link": it_c, "max_iterations": max(r[4] for r in cold),
                     "unconverged": sum(r[2] for r in cold), "ic_ms_per_event": ms_c},
            "warm": {"iterations_per_link": it_w, "max_iterations": max(r[4] for r in warm),
                     "unconverged": sum(r[2] for r in warm), "ic_ms_per_event": ms_w},
            "iteration_ratio": it_w / it_c, "ic_time_ratio": ms_w / ms_c,
            "same_roots_max_abs_diff_event0": same,
        }
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- lattice-correlator estimators
CORR_BYTES_PER_SITE = 10 * 32 + 2 * 48 * 4 + 18 * 4  # field groups read, I and J read + written, W read (FP32)


def run_correlators(args, ws, rank, local):
    """One FP32 MV event at 1024^2 (L = 10 fm) evolved to 1 fm/c with the static and
    lightlike estimators attached from tau = dtau: time per step of the field step alone
    and of field step + estimators (CUDA events, inputs > L2), and the estimators at the
    end of the Glasma stage."""
    import torch

    import paper_2307_07999_gb300 as G

    torch.cuda.set_device(local)
    n, L = 1024, 10.0
    stream = torch.cuda.Stream()

    def event():
        g = G.Glasma(n, L, precision=G.GLASMA_FP32, tau_end_fm=1.0, seed=(5 << 32) + 500 + rank, reunit_every=64,
                     stream=stream)
        assert g.init()[0] == 0
        return g

    def timed(g, k):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.step(k)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    g = event()
    g.step(args.warmup)
    ms_field = timed(g, 100)
    del g
    g = event()
    c = G.Correlators(g, tau_start_fm=0.0, ox0=0.5)
    g.step(args.warmup)
    ms_both = timed(g, 100)
    n_steps = int(math.ceil(1.0 / (0.125 * L / n) - 1e-9))
    g.step(n_steps - (1 + args.warmup + 100))  # the state is at step 1 after init
    tab = c.table()
    ms_corr = ms_both - ms_field
    achieved = CORR_BYTES_PER_SITE * n * n / (ms_corr / 1000.0) / 1e9
    peak, kind = measured_peak()
    i03 = int(np.argmin(np.abs(tab[:, 0] - 0.3)))
    if rank == 0:
        line = {
            "metric": "lattice-correlator estimators (Eqs. 4-5): site-steps/s", "value": n * n / (ms_corr / 1000.0),
            "unit": "site-steps/s", "n_gpus": ws, "steps": 100, "warmup": args.warmup, "ms_per_step": ms_corr,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 sums)",
            "data": "synthetic",
            "config": {"workload": f"one MV event at {n}^2 (L={L} fm, g2mu=2 GeV), static + lightlike estimators "
                                   "at every site, tau_start = dtau", "l2": "inputs larger than L2"},
            "field_step_ms": ms_field, "field_plus_estimators_ms": ms_both,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "algorithmic_bytes_per_site": CORR_BYTES_PER_SITE,
                         "peak_kind": f"{kind} HBM copy (burst)"},
            "estimators_at_tau_0.3fm_GeV2": {"tau_fm": tab[i03, 0], "static": tab[i03, 1:4].tolist(),
                                             "lightlike": tab[i03, 4:7].tolist()},
        }
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- one event at paper scale, FP32 and FP64
SINGLE_512_SORT_EVERY = 16  # counting sort of the quarks by cell, every 16 steps


def run_single_512(args, ws, rank, local):
    """One MV event on 512^2 (L = 10 fm, g2mu = 2 GeV, m = 0.2 GeV, 10 sheets) with 100k
    charm (1.5 GeV) and 100k beauty (4.7 GeV) quarks, |p_T| ~ U[0, 5] GeV, formed at
    1/(2M), evolved from tau = dtau to 1 fm/c (409 coupled steps), in FP32 and in FP64, the
    quarks sorted by cell every 16 steps.
    A step is one whole run; every run restarts from the same initial state (uploaded
    untimed).  Also: the FP32 field step alone (roofline) and the FP32-vs-FP64 errors of
    <dp_i^2>, kappa and the anisotropy <dp_L^2>/<dp_T^2>."""
    import torch

    import paper_2307_07999_gb300 as G

    torch.cuda.set_device(local)
    n, L, NP = 512, 10.0, 100000
    species = [(1.5, (2 << 32) + 11 + 1000 * rank), (4.7, (2 << 32) + 12 + 1000 * rank)]
    seed = (2 << 32) + 1000 * rank
    stream = torch.cuda.Stream()
    g0 = G.Glasma(n, L, precision=G.GLASMA_FP64, tau_end_fm=1.0, seed=seed, stream=stream)
    fails = g0.init()[0]
    U, E, phi, pi, _ = g0.get_state()
    del g0
    n_steps = int(math.ceil(1.0 / (0.125 * L / n) - 1e-9))

    def setup(prec, interp=0):
        g = G.Glasma(n, L, precision=prec, tau_end_fm=1.0, seed=seed, reunit_every=(64 if prec else 0),
                     stream=stream)
        cs = [G.CPIC(g, NP, m, HBARC_GEV_FM / (2 * m), p_min_GeV=0.0, p_max_GeV=5.0, seed=ps, interp=interp,
                     bin_every=SINGLE_512_SORT_EVERY)
              for m, ps in species]
        return g, cs

    def one_run(g, cs):
        g.set_state(U, E, phi, pi, 1)
        for c in cs:
            c.init()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        G.push_many(cs, n_steps - 1)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    out = {}
    for prec in (G.GLASMA_FP32, G.GLASMA_FP64):
        g, cs = setup(prec)
        for _ in range(args.warmup):
            one_run(g, cs)
        sampler = ClockSampler(local) if prec == G.GLASMA_FP32 else None
        if sampler:
            sampler.start()
        barrier(ws)
        ms = [one_run(g, cs) for _ in range(args.steps)]
        clocks = sampler.stop() if sampler else None
        tabs = [c.broadening() for c in cs]
        psteps = sum(int(t[1:, 4].sum()) for t in tabs)
        g.set_state(U, E, phi, pi, 1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.step(100)
        e1.record(stream)
        torch.cuda.synchronize()
        out[prec] = dict(ms=max_over_ranks(statistics.mean(ms), ws), tabs=tabs, psteps=psteps,
                         field_ms=e0.elapsed_time(e1) / 100, clocks=clocks, diag=g.diagnostics())
        del cs, g
    # the same run with the cloud-in-cell gather: one timed run per precision, and its errors
    cic = {}
    for prec in (G.GLASMA_FP32, G.GLASMA_FP64):
        g, cs = setup(prec, interp=1)
        one_run(g, cs)
        cic[prec] = dict(ms=max_over_ranks(one_run(g, cs), ws), tabs=[c.broadening() for c in cs])
        del cs, g
    f32, f64 = out[G.GLASMA_FP32], out[G.GLASMA_FP64]
    su = n * n * (n_steps - 1)
    errs = {}
    cic_errs = {}
    for name, t32, t64 in zip(("charm", "beauty"), cic[G.GLASMA_FP32]["tabs"], cic[G.GLASMA_FP64]["tabs"]):
        den = lambda a: max(np.abs(a).max(), 1e-300)
        k32, k64 = G.kappa_qhat(t32)[:, 1:], G.kappa_qhat(t64)[:, 1:]
        cic_errs[name] = {"dp2": float(np.abs(t32[:, 1:4] - t64[:, 1:4]).max() / den(t64[:, 1:4])),
                          "kappa": float(np.abs(k32 - k64).max() / den(k64))}
    for name, t32, t64 in zip(("charm", "beauty"), f32["tabs"], f64["tabs"]):
        den = lambda a: max(np.abs(a).max(), 1e-300)
        k32, k64 = G.kappa_qhat(t32)[:, 1:], G.kappa_qhat(t64)[:, 1:]
        a32, a64 = G.anisotropy(t32)[1:, 1], G.anisotropy(t64)[1:, 1]
        errs[name] = {"dp2": float(np.abs(t32[:, 1:4] - t64[:, 1:4]).max() / den(t64[:, 1:4])),
                      "kappa": float(np.abs(k32 - k64).max() / den(k64)),
                      "anisotropy": float(np.abs(a32 - a64).max() / den(a64)),
                      "final_anisotropy": float(a64[-1]),
                      "kappa_T_peak_GeV2_per_fm": float((k64[:, 0] + k64[:, 1]).max()),
                      "kappa_L_peak_GeV2_per_fm": float(k64[:, 2].max())}
    peak, kind = measured_peak()
    field_bw = BYTES_PER_SITE * n * n / (f32["field_ms"] / 1000.0) / 1e9
    whole_bw = (BYTES_PER_SITE * su + BYTES_PER_PARTICLE * f32["psteps"]) / (f32["ms"] / 1000.0) / 1e9
    if rank == 0:
        line = {
            "metric": "Glasma site-updates/s & Wong particle-steps/s, one 512^2 event, FP32 vs FP64",
            "value": su * ws / (f32["ms"] / 1000.0), "unit": "site-updates/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": f32["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (FP64 accumulators)", "data": "synthetic",
            "particle_steps_per_s": f32["psteps"] * ws / (f32["ms"] / 1000.0),
            "config": {"workload": "one MV event on 512^2 (L=10 fm, g2mu=2 GeV, m=0.2 GeV, 10 sheets), 100k charm "
                                   "(1.5 GeV) + 100k beauty (4.7 GeV), |p_T|~U[0,5] GeV, tau_form=1/(2M), tau "
                                   "dtau->1 fm/c (409 steps)",
                       "l2": "inputs larger than L2 (67.1 MB per FP32 field buffer, 58.7 MB of it state, x 2 read "
                             "per step, 30 MB of particles)", "ic_unconverged_links": int(fails),
                       "sort_every": SINGLE_512_SORT_EVERY},
            "fp64": {"ms_per_step": f64["ms"], "site_updates_per_s": su * ws / (f64["ms"] / 1000.0),
                     "particle_steps_per_s": f64["psteps"] * ws / (f64["ms"] / 1000.0),
                     "field_step_ms": f64["field_ms"], "fp32_speedup": f64["ms"] / f32["ms"]},
            "fp32_vs_fp64": errs,
            "cloud_in_cell": {"fp32_ms_per_run": cic[G.GLASMA_FP32]["ms"], "fp64_ms_per_run": cic[G.GLASMA_FP64]["ms"],
                              "fp32_vs_fp64": cic_errs},
            "fp32_monitors": {"gauss_rel": f32["diag"][0], "unitarity": f32["diag"][5]},
            "roofline": {"bound": "hbm", "achieved": field_bw, "peak": peak, "unit": "GB/s", "frac": field_bw / peak,
                         "traffic": None, "kernel": "k_field_step<float> (one event)",
                         "peak_kind": f"{kind} HBM copy (burst)", "field_step_ms": f32["field_ms"],
                         "whole_step": {"achieved": whole_bw, "frac": whole_bw / peak, "unit": "GB/s"}},
            "clocks": f32["clocks"],
        }
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- parameter scans of Figs. 1 and 2
def run_scans(args, ws, rank, local):
    """The heavy-quark and jet scans of Figs. 1-2 as multi-ensemble jobs: on each of 4 MV
    events (512^2, L = 10 fm, g2mu = 2 GeV), 4 beauty ensembles (m = 4.2 GeV as in Fig. 1,
    |p_T| = 0, 2, 5, 10 GeV with isotropic azimuth, tau_form = 1/(2m)) and 4 quark-jet
    ensembles (m = 1.5 GeV, p_x = 1, 2, 5, 10 GeV along x, tau_form = 0: pushed from the
    first step after tau = 0+), 25k particles each, pushed together (cpic_push_many) in
    FP32 to 1 fm/c.  Reports, pooled over the events: peak of the total kappa = kappa_T +
    kappa_L (heavy quarks) or qhat = qhat_y + qhat_z (jets) and its delta tau, and the
    anisotropy at delta tau = 0.3 fm/c.  The paper's printed values are quoted as context
    only: its lattice parameters are not given."""
    import torch

    import paper_2307_07999_gb300 as G

    torch.cuda.set_device(local)
    n, L, NP, n_ev = 512, 10.0, 25000, 4
    hq = [(4.2, p, HBARC_GEV_FM / (2 * 4.2)) for p in (0.0, 2.0, 5.0, 10.0)]
    jets = [(1.5, p, 0.0) for p in (1.0, 2.0, 5.0, 10.0)]
    stream = torch.cuda.Stream()
    tabs = [[] for _ in range(len(hq) + len(jets))]
    ctabs = []  # lattice-correlator estimators (Eqs. 4-5) of each event, from the beauty formation step
    n_steps = int(math.ceil(1.0 / (0.125 * L / n) - 1e-9))
    ms_total, psteps = 0.0, 0
    for e in range(n_ev):
        g = G.Glasma(n, L, g2mu_GeV=args.g2mu, precision=G.GLASMA_FP32, tau_end_fm=1.0,
                     seed=(6 << 32) + e + 1000 * rank, reunit_every=64, stream=stream)
        assert g.init()[0] == 0
        cs = []
        for k, (m, p, tf) in enumerate(hq + jets):
            jet = k >= len(hq)
            c = G.CPIC(g, NP, m, tf, p_min_GeV=p, p_max_GeV=p, init_kind=1 if jet else 0,
                       seed=((6 << 32) + 100 * e + k + 1000 * rank) ^ 0x5A5A5A5A5A5A5A5A)
            c.init()
            cs.append(c)
        corr = G.Correlators(g, tau_start_fm=hq[0][2], ox0=0.5)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        G.push_many(cs, n_steps - 1)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_total += e0.elapsed_time(e1)
        for k, c in enumerate(cs):
            t = c.broadening()
            tabs[k].append(t)
            psteps += int(t[1:, 4].sum())
        ctabs.append(corr.table())
        del corr, cs, g

    def pooled(ts):
        out = ts[0].copy()
        cnt = sum(t[:, 4] for t in ts)
        out[:, 1:4] = sum(t[:, 1:4] * t[:, 4:5] for t in ts) / np.where(cnt > 0, cnt, 1.0)[:, None]
        out[:, 4] = cnt
        return out

    res = {"heavy_quarks": [], "jets": []}
    for k, (m, p, tf) in enumerate(hq + jets):
        jet = k >= len(hq)
        t = pooled(tabs[k])
        kq = G.kappa_qhat(t)
        dtau = t[:, 0] - t[0, 0]
        tot = kq[:, 2] + kq[:, 3] if jet else kq[:, 1] + kq[:, 2] + kq[:, 3]
        i = int(np.argmax(tot))
        a = G.anisotropy(t, "jet" if jet else "hq")
        j = int(np.argmin(np.abs(dtau - 0.3)))
        entry = {"mass_GeV": m, ("p_x_GeV" if jet else "p_T_GeV"): p, "tau_form_fm": round(tf, 4),
                 "peak_GeV2_per_fm": float(tot[i]), "peak_delta_tau_fm": float(dtau[i]),
                 "anisotropy_at_0.3fm": float(a[j, 1]), "anisotropy_at_end": float(a[-1, 1]),
                 "dp2_at_end_GeV2": t[-1, 1:4].tolist()}
        res["jets" if jet else "heavy_quarks"].append(entry)
    # the paper's qualitative claims (Sec. 2): static quarks (Eq. 4) less anisotropic than
    # dynamical ones at p_T = 0 and more than the fastest; dynamical jets more anisotropic
    # than lightlike ones (Eq. 5); late kappa_L < 0 (heavy quarks)
    ct = sum(ctabs) / len(ctabs)
    jc = int(np.argmin(np.abs((ct[:, 0] - ct[0, 0]) - 0.3)))
    static_an = float(ct[jc, 3] / (ct[jc, 1] + ct[jc, 2]))
    light_an = float(ct[jc, 6] / ct[jc, 5])
    hq_an = [e["anisotropy_at_0.3fm"] for e in res["heavy_quarks"]]
    jet_an = [e["anisotropy_at_0.3fm"] for e in res["jets"]]
    late_kl = []
    for k in range(len(hq)):
        q = G.kappa_qhat(pooled(tabs[k]))
        late_kl.append(float(q[q[:, 0] >= 0.7, 3].mean()))
    checks = {"static_anisotropy_at_0.3fm": static_an, "lightlike_anisotropy_at_0.3fm": light_an,
              "static_less_anisotropic_than_pT0": static_an < hq_an[0],
              "pT10_less_anisotropic_than_static": hq_an[-1] < static_an,
              "anisotropy_ordered_with_1/pT": all(a > b for a, b in zip(hq_an, hq_an[1:])),
              "jets_more_anisotropic_than_lightlike": all(a > light_an for a in jet_an),
              "late_kappa_L_GeV2_per_fm (tau >= 0.7 fm/c, p_T = 0/2/5/10)": late_kl}
    if rank == 0:
        line = {
            "metric": "parameter scans of Figs. 1-2: particle-steps/s (8 ensembles x 25k on 4 events of 512^2)",
            "value": psteps * ws / (ms_total / 1000.0), "unit": "particle-steps/s", "n_gpus": ws, "steps": 1,
            "warmup": 0, "ms_per_step": ms_total, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (FP64 accumulators)", "data": "synthetic",
            "config": {"workload": f"4 MV events of 512^2 (L=10 fm, g2mu={args.g2mu:g} GeV); beauty m=4.2 GeV p_T in "
                                   "{0,2,5,10} GeV (tau_form=1/2m), quarks m=1.5 GeV p_x in {1,2,5,10} GeV "
                                   "(tau_form=0); 25k each, FP32 to 1 fm/c"},
            "results": res,
            "qualitative_checks": checks,
            "paper_context": {"kappa_total_peak_GeV2_per_fm": "19-22 at delta tau 0.03-0.05 fm/c (beauty, m=4.2 GeV)",
                              "qhat_total_peak_GeV2_per_fm": "24-30 at tau 0.04 fm/c",
                              "note": "Q_s = 2 GeV there, lattice parameters not given: qualitative only"},
        }
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- jets at 1024^2
JETS_SORT_EVERY = 16  # counting sort of the partons by cell, every 16 steps


def run_jets(args, ws, rank, local):
    """Jets: 4 MV events of 1024^2 (L = 10 fm, g2mu = 2 GeV, m = 0.2 GeV, 10 sheets), each
    probed by 1M massless partons along +x in three ensembles of |p_x| = 2, 5, 10 GeV
    (333,334 / 333,333 / 333,333), formed at 0.3 fm/c, FP32 (FP64 sums) to 1 fm/c: 819
    coupled steps per event, the partons pushed from step 246 and sorted by cell every 16
    steps (a field buffer is larger than L2 here; sorted, neighbouring partons share the
    field lines of their gathers).  A step is the whole job
    (all 4 events from their initial states, uploaded untimed); value = site-updates/s,
    particle-steps/s beside it; q^_y, q^_z at tau = 0.5 fm/c and their peak."""
    import torch

    import paper_2307_07999_gb300 as G

    torch.cuda.set_device(local)
    n, L, n_ev = 1024, 10.0, 4
    counts = [333334, 333333, 333333]
    stream = torch.cuda.Stream()
    n_steps = int(math.ceil(1.0 / (0.125 * L / n) - 1e-9))
    states = []
    for e in range(n_ev):
        g = G.Glasma(n, L, precision=G.GLASMA_FP32, tau_end_fm=1.0, seed=(4 << 32) + e + 1000 * rank,
                     reunit_every=64, stream=stream)
        g.init()
        states.append(g.export_state())
    g = G.Glasma(n, L, precision=G.GLASMA_FP32, tau_end_fm=1.0, seed=4 << 32, reunit_every=64, stream=stream)
    cs = [G.CPIC(g, cnt, 0.0, 0.3, p_min_GeV=p, p_max_GeV=p, init_kind=1, bin_every=JETS_SORT_EVERY,
                 seed=((4 << 32) + 7919 * (k + 1) + 1000 * rank) ^ 0x5A5A5A5A5A5A5A5A)
          for k, (p, cnt) in enumerate(zip((2.0, 5.0, 10.0), counts))]

    def job():
        ms, tabs = 0.0, []
        for e in range(n_ev):
            g.import_state(states[e])
            for c in cs:
                c.init()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            G.push_many(cs, n_steps - 1)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            tabs.append([c.broadening() for c in cs])
        return ms, tabs

    for _ in range(args.warmup):
        job()
    clk = ClockSampler(local)
    clk.start()
    barrier(ws)
    runs = [job() for _ in range(args.steps)]
    clocks = clk.stop()
    ms = max_over_ranks(statistics.mean(r[0] for r in runs), ws)
    tabs = runs[-1][1]
    su = n_ev * n * n * (n_steps - 1)
    ps = sum(int(t[1:, 4].sum()) for ev in tabs for t in ev)
    # field step alone (single-event kernel), for the roofline
    g.import_state(states[0])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step(200)
    e1.record(stream)
    torch.cuda.synchronize()
    field_ms = e0.elapsed_time(e1) / 200
    peak, kind = measured_peak()
    field_bw = BYTES_PER_SITE * n * n / (field_ms / 1000.0) / 1e9
    whole_bw = (BYTES_PER_SITE * su + BYTES_PER_PARTICLE * ps) / (ms / 1000.0) / 1e9
    # the pushes (and sorts) of a job: its time minus its field steps timed alone
    push_ms = max(ms - su / (n * n) * field_ms, 1e-9)
    push_bw = BYTES_PER_PARTICLE * ps / (push_ms / 1000.0) / 1e9
    qh = {}
    for k, p in enumerate((2.0, 5.0, 10.0)):
        cnt = sum(ev[k][:, 4] for ev in tabs)
        pooled = tabs[0][k].copy()
        pooled[:, 1:4] = sum(ev[k][:, 1:4] * ev[k][:, 4:5] for ev in tabs) / np.where(cnt > 0, cnt, 1.0)[:, None]
        q = G.kappa_qhat(pooled)
        i5 = int(np.argmin(np.abs(q[:, 0] - 0.5)))
        tot = q[:, 2] + q[:, 3]
        qh[f"p_x={p:g} GeV"] = {"qhat_y_at_0.5fm": float(q[i5, 2]), "qhat_z_at_0.5fm": float(q[i5, 3]),
                                "qhat_total_peak": float(tot.max()), "peak_tau_fm": float(q[int(tot.argmax()), 0]),
                                "anisotropy_at_end": float(G.anisotropy(pooled, "jet")[-1, 1])}
    if rank == 0:
        line = {
            "metric": "jets at 1024^2: Glasma site-updates/s & Wong particle-steps/s (4 events x 1M partons)",
            "value": su * ws / (ms / 1000.0), "unit": "site-updates/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (FP64 accumulators)", "data": "synthetic",
            "particle_steps_per_s": ps * ws / (ms / 1000.0),
            "config": {"workload": "4 MV events of 1024^2 (L=10 fm, g2mu=2 GeV), 1M massless partons each along +x, "
                                   "|p_x| in {2,5,10} GeV by thirds, tau_form=0.3 fm/c, FP32 to 1 fm/c (819 steps)",
                       "sort_every": JETS_SORT_EVERY,
                       "l2": "inputs larger than L2 (268 MB per FP32 field buffer, 235 MB of it state, 60 MB of partons per event)"},
            "site_updates_per_step": su, "particle_steps_per_step": ps,
            "roofline": {"bound": "hbm", "achieved": field_bw, "peak": peak, "unit": "GB/s", "frac": field_bw / peak,
                         "traffic": None, "kernel": "k_field_step<float> (one event)", "field_step_ms": field_ms,
                         "peak_kind": f"{kind} HBM copy (burst)",
                         "whole_step": {"achieved": whole_bw, "frac": whole_bw / peak, "unit": "GB/s"},
                         "push": {"ms_per_job": push_ms, "share_of_job": push_ms / ms, "achieved": push_bw,
                                  "frac": push_bw / peak, "unit": "GB/s",
                                  "algorithmic_bytes_per_particle_step": BYTES_PER_PARTICLE,
                                  "timing": "derived: the job's time minus its field steps at the field step's own "
                                            "time (pushes, sorts and launch gaps)"}},
            "qhat_GeV2_per_fm": qh,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.workload == "warm_start":
        run_warm_start(args, ws, rank, local)
    elif args.workload == "correlators":
        run_correlators(args, ws, rank, local)
    elif args.workload == "single_512":
        run_single_512(args, ws, rank, local)
    elif args.workload == "scans":
        run_scans(args, ws, rank, local)
    elif args.workload == "jets":
        run_jets(args, ws, rank, local)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
