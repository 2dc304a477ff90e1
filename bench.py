"""Benchmark: Kalman-filter track reconstruction throughput on one GB300 (or N, weak scaling).

One step is one pass of the whole hot path over one batch of synthetic events: build the hit
index of every event, find tracks from every seed (beam search, K candidates), and fit every found
track, all through the C ABI, captured once in a CUDA graph and replayed. The workload is the
batched uneven-event configuration: 100 events with 2,000-20,000 tracks each (about 1.07 M seeds),
17 barrel layers at r = 4..68 cm with 0.02 X0 each, 3.8 T, pT 0.5-10 GeV, |eta| < 1, hit
resolution 0.01 cm (r phi) and 0.1 cm (z); finding with chi2 < 30, K = 6, one miss allowed.
The metric is seeds per second through the step (every seed is found and its track fitted).
Other workloads (--workload): hi_occ (barrel + disks, noise 100%, K = 8; --steering for the
region steering lists), material (r-z material map and energy loss), field (parametrised field),
duplicates (module overlaps and combinatorial seeds; the step adds seed cleaning before finding
and duplicate-track removal after it).

Besides the device-timed step the line carries the end-to-end figure (host copies in and out,
pipelined on their own streams), the roofline of every step kernel (the finder's DRAM traffic from
the committed ncu capture while its sources and flags match), the clocks seen during the timed
region, and the learned proposal against plain finding.

The FP64 oracle runs only in the CPU baseline leg (and as the whole reference arm, --impl
reference), on a bounded sample of the same workload, on the host cores.

Prints one JSON line.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "KF finding seeds/s & fitting tracks/s on 1 GB300; learned vs plain at <=0.5% eff loss"
UNIT = "seeds/s"
WORKLOAD = "fit_batched"

# Algorithmic FP32 operation counts per unit of work, counted from the formulas the path
# evaluates (fused multiply-add = 2 flops, special functions and divisions not counted):
#   propagation to the next surface incl. path search (3 Newton steps) ...... 150
#   covariance transport J C J^T, projection onto the surface, scattering ... 320
#   Kalman update (measurement, S = H C H^T + V, gain, state, covariance) .... 260
#   chi2 of one hit in a search window ...................................... 20
#   seed from three hits ..................................................... 80
FLOP_PROP, FLOP_TRANSPORT, FLOP_UPDATE, FLOP_CHI2, FLOP_SEED = 150, 320, 260, 20, 80
# Learned proposal network 14 -> 64 -> 64 -> 1 per sample: forward 2 (14*64 + 64*64 + 64); backward
# 2 (64*64 + 64*64 + 64*14 + 64) for the weight gradients and the hidden-layer back-propagation
# (bias sums, ReLU masks and the sigmoid not counted).
FLOP_MLP_FWD = 2 * (14 * 64 + 64 * 64 + 64)
FLOP_MLP_BWD = 2 * (64 * 64 + 64 * 64 + 64 * 14 + 64)
# Both network kernels run their contractions on the tensor cores with every operand split into
# three bf16 parts and six MMAs per product (FP32-faithful), so their roofline is the measured bf16
# tensor peak / 6. MMA flops they issue per sample (M = 128 samples per tile, inputs padded to 16):
# forward 6 x 2 (16 x 64 + 64 x 64); loss-gradient adds E2 W2 (6 x 2 x 64 x 64) and the weight-gradient
# product [e2 | e1]^T [h1 | x | 1 | 0] (6 x 2 x 128 x 96).
MLP_SPLIT_MMAS = 6
MMA_MLP_FWD = MLP_SPLIT_MMAS * 2 * (16 * 64 + 64 * 64)
MMA_MLP_GRAD = MMA_MLP_FWD + MLP_SPLIT_MMAS * 2 * (64 * 64 + 128 * 96)
# DRAM traffic of the finder measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum of one
# launch, or of adaptive capacity's two passes, per seed) on a smaller case of each workload (30
# events of the 100-event workload, 40 of the barrel + disk workload; profiles/k_find_tracks_*),
# keyed by workload (and adaptive capacity, and the learned proposal's top_n and score margin), valid
# while the finder's sources and build flags are the ones profiled (SHA-1 over FIND_SOURCES);
# otherwise reported as null.
FIND_SOURCES = ("paper_1906_02253_gb300/csrc/find.cu", "paper_1906_02253_gb300/csrc/find_kernel.cuh",
                "paper_1906_02253_gb300/csrc/find_learned.cu", "paper_1906_02253_gb300/csrc/kf_math.cuh",
                "paper_1906_02253_gb300/csrc/find_launch.cuh", "paper_1906_02253_gb300/csrc/mlp.cuh",
                "paper_1906_02253_gb300/build.py")
FIND_PROFILE = {"sources_sha1": "37e3a4f5b5505e80f57304bd1472dadac3fc4110",
                "dram_bytes_per_seed": {"fit_100ev_uneven_17layers_ms": (125605888 + 35233024) / 302063,
                                        "find_200ev_barrel_disks_noise100": (144240128 + 31036672) / 211523,
                                        "find_200ev_barrel_disks_noise100_adaptive4":
                                            (170531328 + 35969024 + 128829952 + 27841280) / 211523,
                                        "find_200ev_barrel_disks_noise100_adaptive2":
                                            (168316416 + 38796544 + 159785216 + 35333632) / 211523,
                                        "find_200ev_barrel_disks_noise100_adaptive2_learned2_0.7":
                                            (154265088 + 31579648 + 42024960 + 3967232) / 211523}}
# Hit index: algorithmic HBM bytes per hit (read 8 B of (phi, z); write 8 B sorted, 4 B id, 16 B search
# record) plus, per (event, surface), the bin offsets (4 B per bin + 1) and the phi sub-bin offsets (16 B per bin).
INDEX_BYTES_PER_HIT = 36
INDEX_BYTES_PER_BIN = 4 + 16


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) < 9:
                continue
            for k, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(k)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "fallback": True}


# ------------------------------------------------------------------------------------------------
# Oracle legs (host cores only)
# ------------------------------------------------------------------------------------------------

def calibration_events(n_events: int) -> int:
    """Events whose seeds the autotuner times: a quarter of the batch, at least 10. Adaptive capacity
    needs enough seeds in its second pass to fill the GPU before it can win on a subset."""
    return min(n_events, max(10, n_events // 4))


def oracle_sample(wl, batch, n_seeds_max: int, clean: bool = False, n_threads: int = 0, learned=None):
    """Run the FP64 oracle (index + find + fit of the found tracks; with ``clean``, seed cleaning
    before finding and duplicate removal after it) on the first seeds of the batch, all host
    cores; ``learned`` = (weights, mean, sd, top_n, score_margin) finds with the learned proposal.
    Returns (seconds, n_seeds, counters, threads)."""
    import numpy as np
    import oracle

    g = oracle.Geometry(wl)
    seeds, st = batch.seeds()
    ev = batch.track_event[st]
    n = min(n_seeds_max, len(st))
    last_ev = int(ev[n - 1])
    sub = np.nonzero(ev <= last_ev)[0][:n]
    t0 = time.perf_counter()
    if clean:
        keep = oracle.clean_seeds(seeds[sub], ev[sub], oracle.seed_params(g, batch, seeds[sub]))
        sub = sub[keep != 0]
    lk = {}
    if learned is not None:
        w, mean, sd, top_n, margin = learned
        lk = dict(mlp=(np.asarray(w, np.float64), np.asarray(mean, np.float64), np.asarray(sd, np.float64)),
                  top_n=top_n, score_margin=margin)
    f = oracle.find(g, batch, seeds[sub], ev[sub], n_threads=n_threads, **lk)
    if clean:
        oracle.remove_duplicates(f["hits"], f["n_hits"], f["chi2"], f["p"][:, 4], f["p"][:, 5], ev[sub])
    oracle.fit(g, batch.hits, batch.hit_surface, f["hits"], n_threads=n_threads)
    dt = time.perf_counter() - t0
    threads = n_threads if n_threads > 0 else (os.cpu_count() or 1)
    if clean:
        return dt, len(keep), f["counters"], threads
    return dt, len(sub), f["counters"], threads


def network_file(name: str) -> str:
    """The trained network of a workload (paper_1906_02253_gb300/data/mlp_<name>.npz), else the
    barrel-geometry network."""
    path = os.path.join(ROOT, "paper_1906_02253_gb300", "data", f"mlp_{name}.npz")
    return path if os.path.exists(path) else MLP_FILE


def learned_arg(args, name: str):
    """--learned TOP_N[:MARGIN] as (weights, mean, sd, top_n, margin, file) with the workload's
    network, or None."""
    if not getattr(args, "learned", ""):
        return None
    import numpy as np
    top_n, _, margin = args.learned.partition(":")
    path = network_file(name)
    z = np.load(path)
    return z["weights"], z["mean"], z["sd"], int(top_n), float(margin or 0.0), os.path.basename(path)


def run_reference(args, wl, batch):
    """The reference arm: the oracle as it stands, on the host cores, one bounded sample per step."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    per_step = args.ref_seeds
    clean = args.clean or getattr(wl, "combinatorial_seeds", False)
    lrn = learned_arg(args, args.workload)
    lrn = lrn[:5] if lrn else None
    for _ in range(args.warmup):
        oracle_sample(wl, batch, min(per_step, 2000), clean, learned=lrn)
    times, n = [], 0
    for _ in range(args.steps):
        dt, n, _, cores = oracle_sample(wl, batch, per_step, clean, learned=lrn)
        times.append(dt)
    value = n / statistics.mean(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * statistics.mean(times),
            "higher_is_better": True, "scaling": args.scaling, "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded generator)",
            "config": {"workload": wl.name, "sample": f"first {n} seeds of the batch (index, "
                       + ("seed cleaning, find, duplicate removal, fit)" if clean else "find, fit)"),
                       "finder": (f"learned proposal, top_n {lrn[3]}, score margin {lrn[4]:g}" if lrn
                                  else "plain (full window)")},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n} seeds per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------------

def measure_workload(args, wl, batch, full: bool = True, mlp_name: str = None, e2e: bool = None):
    """The step (index, seed states, find, fit; with seed cleaning and duplicate removal on
    combinatorial seeds) on one workload: device-timed graph replays, per-part times, efficiency,
    the learned proposal against plain finding and the rooflines. `e2e` (default: `full`) adds the
    end-to-end measurement through host buffers, `full` the single-thread oracle figure. Returns
    the JSON object (and, under "_ctx", the device state the further measurements reuse)."""
    e2e = full if e2e is None else e2e
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1906_02253_gb300 as kf

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    kf.load_library()
    g = kf.Geometry(wl)
    host = kf.to_device_event_batch(batch, device="cpu")
    n_seeds = host["seed_hits"].shape[1]
    n_hits = batch.n_hits
    lmax = wl.lmax
    import synth
    steer = synth.steering_tables(wl, 0.4, 1.8, endcap_barrels=3) if args.steering else None
    clean = args.clean or getattr(wl, "combinatorial_seeds", False)

    # Device inputs and preallocated outputs.
    d = {k: v.to(dev) for k, v in host.items() if isinstance(v, torch.Tensor)}
    seed_keep = track_keep = dws = None
    if clean:  # seed cleaning before finding, duplicate removal after it
        seed_keep = torch.ones(n_seeds, dtype=torch.int32, device=dev)
        track_keep = torch.ones(n_seeds, dtype=torch.int32, device=dev)
        dws = torch.empty(max(kf.dedup_workspace_size(n_seeds, lmax, n_hits), 256), dtype=torch.uint8,
                          device=dev)
    # --learned: the step's finder runs the learned proposal with the workload's network
    lrn = learned_arg(args, mlp_name or args.workload)
    mlp_buf = kf.mlp_buffer(lrn[0], lrn[1], lrn[2], device=dev) if lrn else None
    prm = kf.find_params(wl.chi2_cut, wl.k_max, wl.max_miss, lmax, args.block, args.blocks_per_sm,
                         steering_tables=steer, seed_keep=seed_keep, adaptive_capacity=args.adaptive,
                         mlp=mlp_buf, top_n=lrn[3] if lrn else 0, score_margin=lrn[4] if lrn else 0.0)
    idx = kf.HitIndex(g, batch.n_events, n_hits, dev)
    fout = dict(hits=torch.empty((lmax, n_seeds), dtype=torch.int32, device=dev),
                nhits=torch.empty(n_seeds, dtype=torch.int32, device=dev),
                chi2=torch.empty(n_seeds, dtype=torch.float32, device=dev),
                state=torch.empty((6, n_seeds), dtype=torch.float32, device=dev),
                cov=torch.empty((21, n_seeds), dtype=torch.float32, device=dev),
                status=torch.empty(n_seeds, dtype=torch.int32, device=dev))
    fit_out = dict(state=torch.empty((6, n_seeds), dtype=torch.float32, device=dev),
                   cov=torch.empty((21, n_seeds), dtype=torch.float32, device=dev),
                   chi2=torch.empty(n_seeds, dtype=torch.float32, device=dev),
                   ndof=torch.empty(n_seeds, dtype=torch.int32, device=dev),
                   status=torch.empty(n_seeds, dtype=torch.int32, device=dev))
    wsb = torch.empty(max(kf.find_workspace_size(n_seeds, prm), 256), dtype=torch.uint8, device=dev)
    max_slab = host["max_slab_hits"]
    stream = torch.cuda.Stream(device=dev)
    # Autotune (block size, candidate capacity, adaptive capacity) of the finder and the fit's block size on a
    # calibration subset: the seeds of the first quarter of the events (outside the timed region).
    tuning = {}
    fit_block = 0
    if not args.no_autotune:
        with torch.cuda.stream(stream):
            kf.build_hit_index(g, d["hits"], d["slab_offsets"], batch.n_events, max_slab, index=idx, stream=stream)
            if clean:
                kf.clean_seeds(g, d["hits"], d["hit_surface"], d["seed_hits"], d["seed_event"], keep=seed_keep,
                               workspace=dws, stream=stream)
            n_cal = int(np.searchsorted(host["seed_event"].numpy(), calibration_events(batch.n_events)))
            cal_s = d["seed_hits"][:, :n_cal].contiguous()
            cal_e = d["seed_event"][:n_cal].contiguous()
            prm, ms_find = kf.autotune_find(g, idx, d["hits"], d["hit_surface"], cal_s, cal_e, prm, stream=stream)
            cal = kf.find_tracks(g, idx, d["hits"], d["hit_surface"], cal_s, cal_e, prm, stream=stream)
            fit_block, ms_fit = kf.autotune_fit(g, d["hits"], d["hit_surface"], cal["hits"], stream=stream)
        torch.cuda.synchronize()
        tuning = {"calibration_seeds": n_cal, "find_block_threads": prm.block_threads,
                  "find_k_capacity": prm.k_capacity, "find_adaptive_capacity": prm.adaptive_capacity,
                  "find_ms": ms_find, "fit_block_threads": fit_block, "fit_ms": ms_fit}
        # the tuned configuration's workspace (adaptive capacity adds its overflow list)
        wsb = torch.empty(max(kf.find_workspace_size(n_seeds, prm), 256), dtype=torch.uint8, device=dev)
    parts = ["index"] + (["clean"] if clean else []) + ["find"] + (["dedup"] if clean else []) + ["fit"]

    def step(s, events=None, dd=None, fo=None, fi=None):
        """One step on stream s; dd, fo, fi: input, finder-output and fit-output buffers (default
        the main set)."""
        dd = d if dd is None else dd
        fo = fout if fo is None else fo
        fi = fit_out if fi is None else fi

        def mark(i):
            if events:
                events[i].record(s)
        mark(0)
        kf.build_hit_index(g, dd["hits"], dd["slab_offsets"], batch.n_events, max_slab, index=idx, stream=s)
        mark(1)
        if clean:
            kf.clean_seeds(g, dd["hits"], dd["hit_surface"], dd["seed_hits"], dd["seed_event"], keep=seed_keep,
                           workspace=dws, stream=s)
            mark(2)
        kf.find_tracks(g, idx, dd["hits"], dd["hit_surface"], dd["seed_hits"], dd["seed_event"], prm, out=fo,
                       workspace=wsb, stream=s)
        mark(parts.index("find") + 1)
        if clean:
            kf.remove_duplicates(fo["hits"], fo["nhits"], fo["chi2"], fo["state"], dd["seed_event"], n_hits,
                                 keep=track_keep, workspace=dws, stream=s)
            mark(parts.index("dedup") + 1)
        kf.fit_tracks(g, dd["hits"], dd["hit_surface"], fo["hits"], out=fi, block_threads=fit_block, stream=s)
        mark(len(parts))

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step(stream)
    torch.cuda.synchronize()

    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        step(stream)
    torch.cuda.synchronize()

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 126 MB L2

    def timed_steps(k, fn):
        times = []
        for _ in range(k):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
            times.append((a, b))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in times]

    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_steps = timed_steps(args.steps, graph.replay)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    from paper_1906_02253_gb300 import shard
    ms_step = shard.max_over_ranks(statistics.mean(t_steps), device=dev)
    # index, seed states, find, fit kernels (plus one memset node); adaptive capacity: a second find
    # pass; cleaning: count, 3 scan kernels, fill, seed directions, decision; duplicate removal:
    # count, 3 scan kernels, fill, decision
    # learned proposal: the weight-fragment kernel before the finder
    launches_per_step = 4 + (1 if prm.adaptive_capacity > 0 else 0) + (7 + 6 if clean else 0) + (1 if lrn else 0)

    # Per-part durations: the same launches eager, events on the launching stream.
    kern = {k: [] for k in parts}
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(parts) + 1)]
            step(stream, ev)
        torch.cuda.synchronize()
        for i, k in enumerate(parts):
            kern[k].append(ev[i].elapsed_time(ev[i + 1]))
    kern_ms = {k: statistics.mean(v) for k, v in kern.items()}

    res_host = dict(hits=torch.empty((lmax, n_seeds), dtype=torch.int32).pin_memory())
    h2d = d2h = 0
    ms_e2e = ms_e2e_serial = None
    if e2e:
        # End to end through the public API with host buffers: H2D of the step's inputs from pinned
        # memory, the calls, D2H of the step's result (found hit lists, fitted states, chi2). Serial:
        # copy in, compute (the calls issued one by one), copy out on one stream. Pipelined: copies
        # on their own streams with two buffer sets, so the H2D of step i+1 and the D2H of step i-1
        # overlap the compute of step i (every step's copies stay inside the timed region), the
        # calls of each set's step captured once and replayed as a graph.
        pinned = {k: host[k].pin_memory() for k in ("hits", "hit_surface", "slab_offsets", "seed_hits", "seed_event")}
        res_host = dict(hits=torch.empty((lmax, n_seeds), dtype=torch.int32).pin_memory(),
                        state=torch.empty((6, n_seeds), dtype=torch.float32).pin_memory(),
                        chi2=torch.empty(n_seeds, dtype=torch.float32).pin_memory())
        h2d = sum(t.numel() * t.element_size() for t in pinned.values())
        d2h = sum(t.numel() * t.element_size() for t in res_host.values())

        def copy_out(fo, fi):
            res_host["hits"].copy_(fo["hits"], non_blocking=True)
            res_host["state"].copy_(fi["state"], non_blocking=True)
            res_host["chi2"].copy_(fi["chi2"], non_blocking=True)

        def e2e_step():
            for k, t in pinned.items():
                d[k].copy_(t, non_blocking=True)
            step(stream)
            copy_out(fout, fit_out)

        t_e2e = timed_steps(args.steps, e2e_step)
        ms_e2e_serial = shard.max_over_ranks(statistics.mean(t_e2e), device=dev)

        sets = [(d, fout, fit_out), ({k: torch.empty_like(d[k]) for k in pinned},
                                     {k: torch.empty_like(v) for k, v in fout.items()},
                                     {k: torch.empty_like(v) for k, v in fit_out.items()})]
        s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
        # the step's calls on each buffer set, captured once (the first set's is the timed graph's)
        # and replayed, so that the host only enqueues copies and one graph launch per step
        graph1 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph1, stream=stream):
            step(stream, dd=sets[1][0], fo=sets[1][1], fi=sets[1][2])
        torch.cuda.synchronize()
        set_graphs = (graph, graph1)

        def e2e_pipeline(k):
            k = max(1, k)
            ev_in, ev_c, ev_out = ([torch.cuda.Event() for _ in range(k)] for _ in range(3))
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            s_in.wait_event(t0)
            s_out.wait_event(t0)
            for i in range(k):
                dd, fo, fi = sets[i % 2]
                with torch.cuda.stream(s_in):
                    if i >= 2:
                        s_in.wait_event(ev_c[i - 2])  # step i-2 has read this input set
                    for key, t in pinned.items():
                        dd[key].copy_(t, non_blocking=True)
                    ev_in[i].record(s_in)
                stream.wait_event(ev_in[i])
                if i >= 2:
                    stream.wait_event(ev_out[i - 2])  # step i-2's results in this output set are read back
                with torch.cuda.stream(stream):
                    set_graphs[i % 2].replay()
                ev_c[i].record(stream)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(ev_c[i])
                    copy_out(fo, fi)
                    ev_out[i].record(s_out)
            stream.wait_event(ev_out[k - 1])
            t1.record(stream)
            torch.cuda.synchronize()
            return t0.elapsed_time(t1) / k

        e2e_pipeline(min(args.warmup, 3))
        ms_e2e = shard.max_over_ranks(e2e_pipeline(args.steps), device=dev)

    # Result sanity on the last step (efficiency of the found tracks, host logic only).
    from paper_1906_02253_gb300 import metrics
    if not e2e:
        res_host["hits"].copy_(fout["hits"])
    eff, fake = metrics.efficiency(batch, host["seed_track"], res_host["hits"].numpy().T,
                                   fout["nhits"].cpu().numpy())
    dups = None
    if clean:
        nh_all = fout["nhits"].cpu().numpy()
        hl = res_host["hits"].numpy().T
        sk, tk = seed_keep.cpu().numpy(), track_keep.cpu().numpy()
        dups = {"seeds": n_seeds, "seeds_kept": int(sk.sum()), "tracks_kept": int((sk * tk).sum())}
        for nm, k in (("after_cleaning", sk), ("after_cleaning_and_removal", sk * tk)):
            e, dr, fr = metrics.track_rates(batch, host["seed_track"], hl, nh_all, k)
            dups[nm] = {"efficiency": e, "duplicate_rate": dr, "fake_rate": fr}
        eff, fake = dups["after_cleaning_and_removal"]["efficiency"], dups["after_cleaning_and_removal"]["fake_rate"]
    fit_ok = float((fit_out["status"] == 0).float().mean().item())

    learned = None
    if not args.no_learned and not lrn:  # (with --learned the step's finder is no longer plain)
        learned = compare_learned(args, kf, g, idx, d, prm, fout, wsb, stream, batch, host, eff, fake, kern_ms["find"],
                                  mlp_name or args.workload)

    # whole job: the seeds of every rank (their events differ) over the slowest rank's time
    job_seeds = shard.sum_over_ranks(n_seeds, device=dev)
    value = job_seeds / (ms_step / 1000.0)
    e2e_value = job_seeds / (ms_e2e / 1000.0) if ms_e2e else None
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": args.scaling,
           "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded generator, no datasets)",
           "config": {"workload": wl.name, "events": batch.n_events, "seeds": n_seeds, "hits": n_hits,
                      "layers": len(wl.surfaces), "k_max": wl.k_max, "chi2_cut": wl.chi2_cut,
                      "step": ("hit index + seed cleaning + find + duplicate removal + fit" if clean
                               else "hit index + find + fit") + ", one CUDA graph",
                      "l2": "flushed between steps (256 MB write)",
                      "next_surface": "region steering (eta edges 0.4, 1.8)" if args.steering else "geometric rule",
                      "finder": (f"learned proposal, top_n {lrn[3]}, score margin {lrn[4]:g}, network {lrn[5]}"
                                 if lrn else "plain (full window)"),
                      "parallelism": (f"one fixed batch split over {ws} GPU(s) by LPT on track counts"
                                      if args.scaling == "strong" else f"every GPU its own events ({ws} GPU(s))")
                                     + ", no collective"},
           "gpu_launches": launches_per_step * args.steps, "autotune": tuning,
           "kernel_ms": kern_ms, "efficiency": eff, "fake_rate": fake, "fit_ok_fraction": fit_ok,
           "fit_tracks_per_s": job_seeds / (kern_ms["fit"] / 1000.0),
           "find_seeds_per_s": job_seeds / (kern_ms["find"] / 1000.0),
           }
    if e2e:
        out["e2e"] = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                      "ms_per_step": ms_e2e, "pipelined": "H2D of step i+1 and D2H of step i-1 on their own "
                      "streams overlap step i (two buffer sets, each set's step a captured graph of the "
                      "library calls); L2: the H2D rewrites the inputs each step",
                      "serial_ms_per_step": ms_e2e_serial,
                      "serial_value": job_seeds / (ms_e2e_serial / 1000.0)}
    out["clocks"] = clk.summary()
    if learned is not None:
        out["learned_vs_plain"] = learned
    if dups is not None:
        out["duplicates"] = dups

    # CPU baseline (oracle on a bounded sample) and the finder's algorithmic work per seed.
    counters = None
    if rank == 0 and not args.no_cpu_baseline:
        dt, n, counters, cores = oracle_sample(wl, batch, args.cpu_seeds, clean, learned=lrn[:5] if lrn else None)
        out["cpu_baseline"] = {"value": n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"first {n} seeds of the batch: index, "
                                         + ("seed cleaning, find, duplicate removal, " if clean else "find, ")
                                         + f"fit of the found tracks (FP64, {dt:.1f} s)"}
        counters = np.asarray(counters, np.float64) / n
        if full:
            dt1, n1, _, _ = oracle_sample(wl, batch, min(20000, n), clean, n_threads=1,
                                          learned=lrn[:5] if lrn else None)
            out["cpu_baseline"]["single_thread"] = {"value": n1 / dt1, "unit": UNIT, "cores": 1,
                                                    "sample": f"first {n1} seeds ({dt1:.1f} s)"}
    out["roofline"] = roofline(kern_ms, counters, n_seeds, n_hits, batch, fit_out, out["clocks"],
                               adaptive=prm.adaptive_capacity, learned=f"_learned{lrn[3]}_{lrn[4]:g}" if lrn else "")
    out["_ctx"] = dict(kf=kf, g=g, d=d, host=host, idx=idx, prm=prm, fout=fout, fit_out=fit_out, stream=stream,
                       flush=flush, n_seeds=n_seeds, batch=batch, wl=wl, learned=learned)
    return out


MLP_FILE = os.path.join(ROOT, "paper_1906_02253_gb300", "data", "mlp_learned.npz")


def compare_learned(args, kf, g, idx, d, prm, fout, wsb, stream, batch, host, eff_plain, fake_plain, ms_plain,
                    mlp_name):
    """Learned proposal vs the plain finder on the same batch and K: finder seeds/s (CUDA events on
    the launching stream, L2 flushed between runs), efficiency and fake rate, for several top_n.
    Each learned configuration is autotuned on its own (block size and candidate capacity of the
    learned instance) on the same calibration seeds as plain finding."""
    import numpy as np
    import torch
    from paper_1906_02253_gb300 import metrics

    path = network_file(mlp_name)
    if not os.path.exists(path):
        return {"unavailable": "no trained network in paper_1906_02253_gb300/data"}
    z = np.load(path)
    buf = kf.mlp_buffer(z["weights"], z["mean"], z["sd"], device=d["hits"].device)
    n = host["seed_hits"].shape[1]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=d["hits"].device)
    n_cal = int(np.searchsorted(host["seed_event"].numpy(), calibration_events(batch.n_events)))
    cal_s = d["seed_hits"][:, :n_cal].contiguous()
    cal_e = d["seed_event"][:n_cal].contiguous()
    res = {"network": json.loads(str(z["info"])), "network_file": os.path.basename(path), "k_max": prm.k_max,
           "plain": {"find_seeds_per_s": n / (ms_plain / 1000.0), "efficiency": eff_plain, "fake_rate": fake_plain,
                     "block_threads": prm.block_threads, "k_capacity": prm.k_capacity,
                     "adaptive_capacity": prm.adaptive_capacity}}
    best = None
    # top_n rule on the passing hits, score margins, and (window) the top_n of the whole window's box
    # ranked before the chi2 cut
    for top_n, margin, window in ((1, 0.0, False), (2, 0.0, False), (4, 0.0, False), (2, 0.5, False),
                                  (2, 0.7, False), (2, 1.0, False), (2, 2.0, False), (2, 0.0, True),
                                  (4, 0.0, True), (2, 0.5, True), (2, 0.7, True)):
        lp = kf.find_params(prm.chi2_cut, prm.k_max, prm.max_miss, prm.lmax, 0, 0, mlp=buf, top_n=top_n,
                            score_margin=margin, window_ranking=window)
        lp.steering, lp._steer_ref = prm.steering, getattr(prm, "_steer_ref", None)  # same next-surface rule
        lp.seed_keep, lp._keep_ref = prm.seed_keep, getattr(prm, "_keep_ref", None)  # same seeds
        lw = torch.empty(max(kf.find_workspace_size(n, lp), 256), dtype=torch.uint8, device=d["hits"].device)
        if not args.no_autotune:
            with torch.cuda.stream(stream):
                lp, _ = kf.autotune_find(g, idx, d["hits"], d["hit_surface"], cal_s, cal_e, lp, stream=stream)
            torch.cuda.synchronize()
            # the tuned configuration's workspace (adaptive capacity adds its overflow list)
            lw = torch.empty(max(kf.find_workspace_size(n, lp), 256), dtype=torch.uint8, device=d["hits"].device)
        times = []
        for i in range(args.warmup + args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                kf.find_tracks(g, idx, d["hits"], d["hit_surface"], d["seed_hits"], d["seed_event"], lp, out=fout,
                               workspace=lw, stream=stream)
                b.record(stream)
            torch.cuda.synchronize()
            if i >= args.warmup:
                times.append(a.elapsed_time(b))
        e, f = metrics.efficiency(batch, host["seed_track"], fout["hits"].cpu().numpy().T, fout["nhits"].cpu().numpy())
        r = {"find_seeds_per_s": n / (statistics.mean(times) / 1000.0), "find_ms": statistics.mean(times),
             "efficiency": e, "fake_rate": f, "efficiency_loss": eff_plain - e,
             "block_threads": lp.block_threads, "k_capacity": lp.k_capacity,
             "adaptive_capacity": lp.adaptive_capacity}
        r["speedup_vs_plain"] = r["find_seeds_per_s"] / res["plain"]["find_seeds_per_s"]
        name = f"top_n={top_n}" + (f",margin={margin:g}" if margin > 0 else "") + (",window" if window else "")
        res[name] = r
        if r["efficiency_loss"] <= 0.005 and (best is None or r["find_seeds_per_s"] > res[best]["find_seeds_per_s"]):
            best = name
    res["best_within_0.5pct_eff_loss"] = best
    res["_mlp"] = (z["weights"], z["mean"], z["sd"])
    return res


def learned_roofline(batch, wl, res, n_sample: int = 20000):
    """Roofline of the learned finder (top_n = 2): the plain finder's algorithmic flops per seed with
    the counts of learned finding, plus 10,112 flops per network evaluation, all counted by the
    oracle's learned finding on the first seeds of the batch."""
    import numpy as np
    import oracle
    import torch
    w, mean, sd = res["_mlp"]
    seeds, st = batch.seeds()
    n = min(n_sample, len(st))
    f = oracle.find(oracle.Geometry(wl), batch, seeds[:n], batch.track_event[st][:n],
                    mlp=(np.asarray(w, np.float64), np.asarray(mean, np.float64), np.asarray(sd, np.float64)),
                    top_n=2)
    c = np.asarray(f["counters"], np.float64) / n
    n_prop, n_pass, n_upd, n_scan, n_win, n_mlp = c
    per_seed = FLOP_SEED + n_prop * (FLOP_PROP + FLOP_TRANSPORT) + n_upd * FLOP_UPDATE + n_win * FLOP_CHI2 + n_mlp * FLOP_MLP_FWD
    r = res["top_n=2"]
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    alu_peak = props.multi_processor_count * 128 * 2 * _peaks().get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    ach = per_seed * r["find_seeds_per_s"] / 1e12
    return {"kernel": "k_find_tracks (learned, top_n=2)", "bound": "alu", "achieved": ach, "peak": alu_peak,
            "unit": "TFLOP/s", "frac": ach / alu_peak,
            "work_per_seed": {"propagations": n_prop, "updates": n_upd, "chi2": n_win, "network_evaluations": n_mlp,
                              "flop": per_seed, "sample_seeds": n}}


def _timed(args, stream, flush, fn, reps=None):
    """Mean CUDA-event time (ms) of fn on `stream`, L2 flushed before each run, after warm-up."""
    import torch
    times = []
    reps = args.steps if reps is None else reps
    for i in range(args.warmup + reps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        if i >= args.warmup:
            times.append(a.elapsed_time(b))
    return statistics.mean(times)


def _alu_peak():
    import torch
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    mhz = _peaks().get("sm_max_mhz", 2070.0)
    return props.multi_processor_count * 128 * 2 * mhz * 1e6 / 1e12, mhz


def fit_line(args, kf, wl, batch, stream, flush, d=None):
    """Fitting over the known hit sequences of a workload's generated tracks (the fitting configs):
    every track of every event in one CUDA-graph launch of kf_fit_tracks with its autotuned block
    size, L2 flushed between replays; tracks/s, the fit's roofline (FP32 ALU) and the FP64 oracle's
    fit on the host cores."""
    import numpy as np
    import torch
    import oracle
    dev = torch.device("cuda", torch.cuda.current_device())
    g = kf.Geometry(wl)
    if d is None:
        d = {k: v.to(dev) for k, v in kf.to_device_event_batch(batch, device="cpu").items() if isinstance(v, torch.Tensor)}
    th = d["track_hits"]
    n = th.shape[1]
    out = dict(state=torch.empty((6, n), dtype=torch.float32, device=dev),
               cov=torch.empty((21, n), dtype=torch.float32, device=dev),
               chi2=torch.empty(n, dtype=torch.float32, device=dev),
               ndof=torch.empty(n, dtype=torch.int32, device=dev),
               status=torch.empty(n, dtype=torch.int32, device=dev))
    with torch.cuda.stream(stream):
        blk, _ = kf.autotune_fit(g, d["hits"], d["hit_surface"], th, stream=stream)
        for _ in range(args.warmup):
            kf.fit_tracks(g, d["hits"], d["hit_surface"], th, out=out, block_threads=blk, stream=stream)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        kf.fit_tracks(g, d["hits"], d["hit_surface"], th, out=out, block_threads=blk, stream=stream)
    torch.cuda.synchronize()
    ms = _timed(args, stream, flush, graph.replay)
    ok = out["status"] == 0
    n_fit = int(ok.sum().item())
    n_steps = float(((out["ndof"][ok].double() + 5.0) / 2.0 - 1.0).sum().item())
    flops = n_fit * (FLOP_SEED + FLOP_UPDATE) + n_steps * (FLOP_PROP + FLOP_TRANSPORT + FLOP_UPDATE)
    peak, mhz = _alu_peak()
    ach = flops / (ms / 1000.0) / 1e12
    res = {"workload": wl.name, "events": batch.n_events, "tracks": n, "layers": len(wl.surfaces),
           "metric": "fitting tracks/s (known hit sequences, one CUDA graph launch)", "value": n / (ms / 1000.0),
           "unit": "tracks/s", "ms": ms, "block_threads": blk, "fit_ok_fraction": n_fit / max(n, 1),
           "roofline": {"kernel": "k_fit_tracks", "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                        "frac": ach / peak, "peak_note": f"FP32 {mhz:.0f} MHz", "flop_per_track": flops / max(n_fit, 1)}}
    if not args.no_cpu_baseline:
        m = min(n, args.fit_cpu_tracks)
        t0 = time.perf_counter()
        oracle.fit(oracle.Geometry(wl), batch.hits, batch.hit_surface, batch.track_hits[:m])
        dt = time.perf_counter() - t0
        res["cpu_baseline"] = {"value": m / dt, "unit": "tracks/s", "cores": os.cpu_count() or 1, "kind": "oracle",
                               "sample": f"first {m} tracks of the batch (FP64 fit, {dt:.2f} s)"}
    return res


def secondary_rooflines(args, kf, ctx, learned):
    """Rooflines of the kernels besides index, finder and fit, each timed live with CUDA events on
    its stream: the seed states (FP32 ALU), the network's forward and loss-gradient kernels on a
    synthetic feature batch (tensor cores), seed cleaning and duplicate removal on the module-overlap
    workload (HBM, their algorithmic bytes), and the learned finder."""
    import numpy as np
    import torch
    import synth
    peak, mhz = _alu_peak()
    hbm = _peaks()["hbm_gbs"]
    stream, flush, d, g, batch = ctx["stream"], ctx["flush"], ctx["d"], ctx["g"], ctx["batch"]
    n = ctx["n_seeds"]
    res = {}
    st_out = (torch.empty((28, n), dtype=torch.float32, device=d["hits"].device),
              torch.empty(n, dtype=torch.int32, device=d["hits"].device))
    ms = _timed(args, stream, flush, lambda: kf.seed_states(g, d["hits"], d["hit_surface"], d["seed_hits"],
                                                            d["seed_event"], batch.n_events, out=st_out, stream=stream))
    per = FLOP_SEED + 2 * (FLOP_PROP + FLOP_TRANSPORT) + 3 * FLOP_UPDATE
    ach = per * n / (ms / 1000.0) / 1e12
    res["seed_states"] = {"kernel": "k_seed_states", "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                          "frac": ach / peak, "ms": ms, "flop_per_seed": per, "seeds": n}
    # network kernels on 2^20 synthetic feature rows
    rows = 1 << 20
    gen = torch.Generator(device=d["hits"].device).manual_seed(7)
    feats = torch.randn((rows, 14), generator=gen, device=d["hits"].device)
    labels = (torch.rand(rows, generator=gen, device=d["hits"].device) > 0.5).float()
    params = kf.mlp_buffer(synth.mlp_init(5), np.zeros(14), np.ones(14), device=d["hits"].device)
    logits = torch.empty(rows, device=d["hits"].device)
    grad = torch.empty(kf.MLP_PARAMS, device=d["hits"].device)
    loss = torch.empty(1, device=d["hits"].device)
    pk = _peaks()
    bf16 = pk.get("bf16_tflops") or 1900.0
    split_peak = bf16 / MLP_SPLIT_MMAS
    for key, kern, fn, alg, mma in (
            ("mlp_forward", "k_mlp_forward", lambda: kf.mlp_forward(params, feats, out=logits, stream=stream),
             FLOP_MLP_FWD, MMA_MLP_FWD),
            ("mlp_loss_grad", "k_mlp_loss_grad",
             lambda: kf.mlp_loss_grad(params, feats, labels, grad=grad, loss=loss, stream=stream),
             FLOP_MLP_FWD + FLOP_MLP_BWD, MMA_MLP_GRAD)):
        ms = _timed(args, stream, flush, fn)
        ach = alg * rows / (ms / 1000.0) / 1e12
        mma_t = mma * rows / (ms / 1000.0) / 1e12
        res[key] = {"kernel": kern, "bound": "tensor", "achieved": ach, "peak": split_peak, "unit": "TFLOP/s",
                    "frac": ach / split_peak, "ms": ms, "rows": rows, "flop_per_row": alg,
                    "peak_basis": ("measured bf16 tensor peak / 6 (three-part bf16 split, six MMAs per product)"
                                   if "bf16_tflops" in pk else "fallback bf16 peak / 6"),
                    "mma_tflops": mma_t, "mma_frac_of_bf16_peak": mma_t / bf16, "mma_flop_per_row": mma}
    # seed cleaning and duplicate removal on the module-overlap workload
    wd = synth.workload("duplicates")
    bd = synth.generate(wd)
    hd = kf.to_device_event_batch(bd, device="cpu")
    dd = {k: v.to(d["hits"].device) for k, v in hd.items() if isinstance(v, torch.Tensor)}
    gd = kf.Geometry(wd)
    nd = dd["seed_hits"].shape[1]
    keep = torch.ones(nd, dtype=torch.int32, device=d["hits"].device)
    dws = torch.empty(max(kf.dedup_workspace_size(nd, wd.lmax, bd.n_hits), 256), dtype=torch.uint8,
                      device=d["hits"].device)
    ms = _timed(args, stream, flush, lambda: kf.clean_seeds(gd, dd["hits"], dd["hit_surface"], dd["seed_hits"],
                                                            dd["seed_event"], keep=keep, workspace=dws, stream=stream))
    # bytes: seed hit ids and event (16), the three hits (24), keep (4), the inverted index (three
    # references per seed, counted, filled and read: 3 x 12), its offsets (4 per hit, scanned twice)
    nbytes = nd * (16 + 24 + 4 + 36) + bd.n_hits * 8
    ach = nbytes / (ms / 1000.0) / 1e9
    res["seed_cleaning"] = {"kernel": "k_count_users, scan, k_fill_users, k_seed_dirs, k_clean_seeds", "bound": "hbm",
                            "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "ms": ms, "seeds": nd,
                            "bytes": nbytes}
    prm = kf.find_params(wd.chi2_cut, wd.k_max, wd.max_miss, wd.lmax, seed_keep=keep)
    fo = kf.find_tracks(gd, kf.build_hit_index(gd, dd["hits"], dd["slab_offsets"], bd.n_events, hd["max_slab_hits"]),
                        dd["hits"], dd["hit_surface"], dd["seed_hits"], dd["seed_event"], prm)
    tkeep = torch.ones(nd, dtype=torch.int32, device=d["hits"].device)
    ms = _timed(args, stream, flush, lambda: kf.remove_duplicates(fo["hits"], fo["nhits"], fo["chi2"], fo["state"],
                                                                  dd["seed_event"], bd.n_hits, keep=tkeep,
                                                                  workspace=dws, stream=stream))
    # bytes: hit lists (lmax x 4), hits, chi2, direction, event, keep (24), the inverted index
    # (lmax references per track, counted, filled and read: lmax x 12), offsets (8 per hit)
    nbytes = nd * (wd.lmax * 16 + 24) + bd.n_hits * 8
    ach = nbytes / (ms / 1000.0) / 1e9
    res["duplicate_removal"] = {"kernel": "k_count_users, scan, k_fill_users, k_remove_duplicates", "bound": "hbm",
                                "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "ms": ms,
                                "tracks": nd, "bytes": nbytes}
    if learned is not None and "top_n=2" in learned and not args.no_cpu_baseline:
        res["learned_find"] = learned_roofline(batch, ctx["wl"], learned)
    return res


def run_gpu(args, wl, batch):
    import numpy as np
    import torch
    ws, rank, local = _dist()
    out = measure_workload(args, wl, batch, full=True)
    ctx = out.pop("_ctx")
    extras = ws == 1 and not args.no_extras
    if extras:
        import synth
        kf = ctx["kf"]
        # the largest configuration: barrel + disks, noise 100%, K = 8, plain and learned, autotuned
        wh = synth.workload("hi_occ")
        bh = synth.generate(wh)
        hi = measure_workload(args, wh, bh, full=False, mlp_name="hi_occ", e2e=True)
        hctx = hi.pop("_ctx")
        for k in ("metric", "n_gpus", "steps", "warmup", "higher_is_better", "scaling", "vs_baseline", "data"):
            hi.pop(k, None)
        out["hi_occ"] = hi
        del hctx
        torch.cuda.empty_cache()
        # the same step with the learned finder (top 2, score margin 0.7), autotuned on its own
        import copy
        la = copy.copy(args)
        la.learned, la.no_learned, la.cpu_seeds = "2:0.7", True, min(args.cpu_seeds, 50000)
        hl = measure_workload(la, wh, bh, full=False, mlp_name="hi_occ", e2e=True)
        hl.pop("_ctx")
        out["hi_occ"]["learned_step"] = {k: hl[k] for k in ("value", "unit", "ms_per_step", "e2e", "efficiency", "fake_rate",
                                                         "kernel_ms", "autotune", "gpu_launches", "roofline")
                                         if k in hl}
        out["hi_occ"]["learned_step"]["finder"] = hl["config"]["finder"]
        out["hi_occ"]["learned_step"]["vs_plain_step"] = hl["value"] / hi["value"]
        torch.cuda.empty_cache()
        # fitting over known hit sequences: the 1-event, 10-layer workload and the 100-event batch
        out["fit_known_hits"] = {
            "fit_small": fit_line(args, kf, synth.workload("fit_small"), synth.generate("fit_small"), ctx["stream"],
                                  ctx["flush"]),
            "fit_batched": fit_line(args, kf, wl, batch, ctx["stream"], ctx["flush"], d=ctx["d"]),
        }
        out["roofline"]["secondary"] = secondary_rooflines(args, kf, ctx, ctx["learned"])
    for blk in (out, out.get("hi_occ", {})):
        lv = blk.get("learned_vs_plain")
        if isinstance(lv, dict):
            lv.pop("_mlp", None)
    if rank == 0:
        print(json.dumps(out), flush=True)


def find_sources_sha1() -> str:
    import hashlib
    h = hashlib.sha1()
    for f in FIND_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def roofline(kern_ms, counters, n_seeds, n_hits, batch, fit_out, clocks, adaptive=0, learned=""):
    """Roofline of every step kernel, and of the dominant one at the top level. The finder and the
    fit are FP32-ALU bound (no dense contraction): peak = SMs x 128 FP32 lanes x 2 flop x max SM
    clock. The index is HBM bound."""
    import torch
    peaks = _peaks()
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    alu_peak = props.multi_processor_count * 128 * 2 * sm_mhz * 1e6 / 1e12
    # context: the FP32 rate a plain FMA stream reaches on this GPU (the library's probe kernel)
    import paper_1906_02253_gb300 as kf
    fma_rate = kf.fp32_fma_rate()
    per = {}
    n_slabs = batch.n_events * len(batch.wl.surfaces)
    n_bins = max(s.n_phi * s.n_2nd for s in batch.wl.surfaces)
    nbytes = INDEX_BYTES_PER_HIT * n_hits + n_slabs * (INDEX_BYTES_PER_BIN * n_bins + 4)
    ach = nbytes / (kern_ms["index"] / 1000.0) / 1e9
    per["index"] = {"kernel": "k_build_hit_index", "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": ach / peaks["hbm_gbs"], "traffic": None}
    # fit of the found tracks: N hits give N - 1 propagation steps (ndof = 2 N - 5)
    ok = fit_out["status"] == 0
    n_fit = int(ok.sum().item())
    n_steps = float(((fit_out["ndof"][ok].double() + 5.0) / 2.0 - 1.0).sum().item())
    flops = n_fit * (FLOP_SEED + FLOP_UPDATE) + n_steps * (FLOP_PROP + FLOP_TRANSPORT + FLOP_UPDATE)
    ach = flops / (kern_ms["fit"] / 1000.0) / 1e12
    per["fit"] = {"kernel": "k_fit_tracks", "bound": "alu", "achieved": ach, "peak": alu_peak, "unit": "TFLOP/s",
                  "frac": ach / alu_peak, "traffic": None, "peak_note": f"FP32 {sm_mhz:.0f} MHz",
                  "fma_probe_tflops": fma_rate}
    if counters is None:
        per["find"] = {"kernel": "k_find_tracks", "bound": "alu", "achieved": None, "peak": alu_peak,
                       "unit": "TFLOP/s", "frac": None, "traffic": None}
    else:
        # chi2 work: the hits of the windows the finder scans (limited to the phi sub-bins they touch)
        n_prop, n_pass, n_upd, n_scan, n_win = counters[:5]
        per_seed = FLOP_SEED + n_prop * (FLOP_PROP + FLOP_TRANSPORT) + n_upd * FLOP_UPDATE + n_win * FLOP_CHI2
        n_mlp = counters[5] if learned and len(counters) > 5 else 0.0
        per_seed += n_mlp * FLOP_MLP_FWD  # network evaluations (on the tensor cores, counted as FP32 flops)
        ach = per_seed * n_seeds / (kern_ms["find"] / 1000.0) / 1e12
        # profiled per configuration: one pass, or adaptive capacity's two passes together
        key = batch.wl.name + (f"_adaptive{adaptive}" if adaptive else "") + learned
        bytes_seed = FIND_PROFILE["dram_bytes_per_seed"].get(key)
        profiled = find_sources_sha1() == FIND_PROFILE["sources_sha1"] and bytes_seed is not None
        traffic = bytes_seed * n_seeds if profiled else None
        per["find"] = {"kernel": "k_find_tracks", "bound": "alu", "achieved": ach, "peak": alu_peak,
                       "unit": "TFLOP/s", "frac": ach / alu_peak, "traffic": traffic,
                       "traffic_unit": "bytes per launch (ncu, scaled by seeds)", "peak_note": f"FP32 {sm_mhz:.0f} MHz",
                       "fma_probe_tflops": fma_rate,
                       "work_per_seed": {"propagations": n_prop, "updates": n_upd, "chi2": n_win,
                                         "chi2_whole_bins": n_scan, "network_evaluations": n_mlp,
                                         "flop": per_seed}}
    dom = max(("index", "find", "fit"), key=lambda k: kern_ms[k])
    out = dict(per[dom])
    out["per_kernel"] = {k: {kk: v[kk] for kk in ("kernel", "bound", "achieved", "peak", "unit", "frac")}
                         for k, v in per.items()}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="kfgb", choices=["kfgb", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--events", type=int, default=None, help="override the number of events")
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--cpu-seeds", type=int, default=10 ** 9, help="oracle sample for the CPU baseline")
    ap.add_argument("--ref-seeds", type=int, default=200000, help="oracle sample per reference step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-vs-plain comparison")
    ap.add_argument("--learned", default="", metavar="TOP_N[:MARGIN]",
                    help="the step's finder with the learned proposal (the workload's trained network), e.g. 2:0.7")
    ap.add_argument("--no-autotune", action="store_true", help="default launch configuration")
    ap.add_argument("--adaptive", type=int, default=0,
                    help="with --no-autotune: the finder's adaptive capacity (first-pass slots; 0 = one pass)")
    ap.add_argument("--clean", action="store_true",
                    help="seed cleaning and duplicate-track removal in the step (on for combinatorial seeds)")
    ap.add_argument("--steering", action="store_true",
                    help="region steering lists (5 eta regions) instead of the geometric next-surface rule")
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="weak: every rank its own events; strong: one fixed batch split over the ranks (LPT)")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the main step (no high-occupancy block, fit lines or secondary rooflines)")
    ap.add_argument("--fit-cpu-tracks", type=int, default=200000, help="oracle sample of the fit lines")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    ws, rank, local = _dist()
    if args.impl == "reference" and rank != 0:
        return  # the reference arm runs on rank 0 only
    if ws > 1 and args.impl != "reference":
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import synth
    over = {"n_events": args.events} if args.events else {}
    from paper_1906_02253_gb300 import shard
    if args.scaling == "weak":
        # every rank processes its own events (different seed), no data exchange
        wl = synth.workload(args.workload, seed=shard.rank_seed(synth.WORKLOADS[args.workload].seed, rank), **over)
        batch = synth.generate(wl)
    else:
        # one fixed batch; each rank takes its share of the events (greedy LPT on track counts)
        import numpy as np
        wl = synth.workload(args.workload, **over)
        batch = synth.generate(wl)
        if ws > 1 and args.impl != "reference":
            counts = np.bincount(batch.track_event, minlength=batch.n_events)
            batch = batch.select_events(shard.shard_events(counts, ws, rank))
            wl = batch.wl
    if args.impl == "reference":
        run_reference(args, wl, batch)
        return
    run_gpu(args, wl, batch)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
