#!/usr/bin/env python
"""Benchmark: dJFA vs JFA frames of a moving-seed Voronoi simulation on GB300.

One step = one simulation timestep of the hot path.  By default that is one
point of the 8192 x 8192 sweep: a 8192 x 8192 grid with 2^18 uniform seeds
moving by uniform integers in [-4, 4] per axis (``--seeds S --max-disp D``
select another point; ``--workload single2048`` the 2048 x 2048, 16384-seed
workload): the seed move (Algorithm 1's SimulateParticles), the stamp and the
dJFA passes of Eq. 4 (6 passes at the default point, the first two Von
Neumann).  The same trajectory is also run with a full JFA frame per step (13
passes, Eq. 2) for the speedup, and every 10th frame both are scored against
each other (the paper's similarity, Section VI-A) and against the exact
diagram (distance-correct pixels).

Printed: one JSON line (rank 0).  ``value`` is whole-job dJFA throughput in
Gpixel-passes/s from CUDA events around each step (inputs resident in HBM, L2
flushed between steps); ``e2e`` is the same metric through the Python/C API
with host buffers (displacements in, label map out, every step).

``--impl reference`` times the CPU oracle on the same workload instead.
Under torchrun every rank runs an independent replica (its own seeds); there
is no data-path collective.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gpixel-passes/s and ms/frame, dJFA vs JFA at stated similarity; % of HBM peak"
UNIT = "Gpixel-passes/s"
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 512 << 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="sweep8192",
                    help="sweep8192 (default; --seeds and --max-disp pick the point), single2048, single256, "
                         "batched256, serve1000, churn2048")
    ap.add_argument("--seeds", type=int, default=None,
                    help="sweep8192: seed count (2^10, 2^14, 2^18 (default), 2^22)")
    ap.add_argument("--max-disp", type=int, default=None, help="sweep8192: maximum move per axis (1, 4 (default), 16)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="bounded CPU-oracle sample for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-labels", choices=["packed", "24", "32"], default="packed",
                    help="end-to-end read-back: labels bit-packed at the fewest bits the seed count needs "
                         "(default; 19 bits a pixel for 2^18 seeds), 24-bit labels (3 B a pixel, up to "
                         "16777215 seeds) or the int32 map")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip vd_autotune (the pass launch-shape search) before the timed steps")
    ap.add_argument("--metric", choices=["euclid", "manhattan"], default="euclid",
                    help="dJFA distance: euclid (dJFAe) or manhattan (dJFAm, scored against Euclidean JFA)")
    ap.add_argument("--extra", type=int, default=0, help="extra dJFA passes after the schedule (0, 1, 2)")
    ap.add_argument("--rates", default="2000,5000,10000,20000",
                    help="serve1000: Poisson request rates (per second)")
    ap.add_argument("--duration", type=float, default=1.0, help="serve1000: seconds of arrivals per rate")
    ap.add_argument("--churn", type=int, default=164, help="churn2048: seeds removed and inserted per step")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


_SWEEP = {}
_DJFA_METRIC = {}


def workload(name):
    """(w, h, seeds, timesteps, max displacement) of a named workload."""
    from paper_2209_00117_gb300 import inputs

    if name == "sweep8192":
        sw = inputs.SWEEP8192
        s = _SWEEP.get("seeds") or sw["seeds"][2]
        d = _SWEEP.get("max_disp") or sw["max_disp"][1]
        if s not in sw["seeds"] or d not in sw["max_disp"]:
            raise SystemExit(f"sweep8192 takes --seeds in {sw['seeds']} and --max-disp in {sw['max_disp']}")
        return sw["side"], sw["side"], s, sw["steps"], d
    if name not in inputs.SINGLE:
        raise SystemExit(f"unknown workload {name}; choose from {sorted(inputs.SINGLE)} or sweep8192")
    w, h, s, steps, d = inputs.SINGLE[name]
    return w, h, s, steps, d


def workload_key(name, s, d):
    """Name of a workload in lines and in profiles/traffic.txt."""
    return name if name != "sweep8192" else f"sweep8192_s{s}_d{d}"


def l2_note(w, h, gpu):
    """How the timed steps avoid a warm L2: two int32 maps larger than the
    129 MB L2 need nothing more; smaller ones are flushed between steps."""
    if 4 * w * h > (129 << 20):
        return (f"inputs larger than L2 (two {4 * w * h >> 20} MB label maps a simulation); "
                f"the GPU arm also writes {L2_FLUSH_BYTES >> 20} MB between timed steps, outside the step events")
    if gpu:
        return f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MB write, outside the step events)"
    return "host memory"


def config_dict(name, w, h, s, d, n_jfa, n_djfa, world, l2):
    return {
        "workload": f"{name}: {w}x{h} int32 label map, {s} uniform seeds, moves uniform in "
                    f"[-{d},{d}] per axis, clamped; dJFA (Eq. 4) vs JFA (Eq. 2) per frame",
        "grid": [w, h], "seeds": s, "max_disp": d,
        "passes": {"jfa": n_jfa, "djfa": n_djfa, "djfa_von_neumann": 2},
        "djfa_metric": _DJFA_METRIC.get("name", "euclid"), "djfa_extra_passes": _DJFA_METRIC.get("extra", 0),
        "l2": l2,
        "parallelism": "replicas" if world > 1 else "single",
    }


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.dev = device_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", str(self.dev)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# multi-rank aggregation (replicas: no data-path collective)
# ---------------------------------------------------------------------------

def max_over_ranks(pg, value, device):
    """The largest `value` over all ranks (the slowest rank sets the job time)."""
    if pg is None:
        return value
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_gpx(pixel_passes_per_step, steps, world, t_max_ms):
    """Gpixel-passes/s of the whole job: every rank's units over the max time."""
    return pixel_passes_per_step * steps * world / (t_max_ms * 1e-3) / 1e9


def owned(n_items, world, rank):
    """The simulations rank `rank` of `world` owns: indices i with
    i % world == rank.  Every simulation belongs to exactly one rank, and the
    ranks' shares differ by at most one."""
    return list(range(rank, n_items, world))


def sum_over_ranks(pg, value, device):
    """The sum of `value` over all ranks (host-side aggregation of counts)."""
    if pg is None:
        return value
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


def gather_arrays(pg, arr):
    """Every rank's 1-D float array, concatenated in rank order (host objects:
    latencies and the like, never device data)."""
    arr = np.asarray(arr, dtype=np.float64)
    if pg is None:
        return arr
    parts = [None] * pg.get_world_size()
    pg.all_gather_object(parts, arr)
    return np.concatenate(parts) if parts else arr


def latency_summary(lat):
    """p50 / p99 / mean (ms) of a latency array in seconds."""
    lat = np.asarray(lat, dtype=np.float64)
    return {"p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "mean_ms": 1e3 * float(lat.mean())}


# ---------------------------------------------------------------------------
# roofline inputs
# ---------------------------------------------------------------------------

def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback (6.8 TB/s, earlier GB300 copy measurement)"


# the sources of the timed pass kernels: the plain pass and the
# position-tagged passes of a dJFA frame
PASS_SOURCES = ("vd_kernels.cuh", "vd_pass_pk.cuh")


def kernel_source_hash():
    h = hashlib.sha256()
    for name in PASS_SOURCES:
        with open(os.path.join(ROOT, "paper_2209_00117_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kind, workload_name):
    """DRAM bytes per launch of a kernel kind from the committed ncu summary
    (profiles/traffic.txt), or None when absent or taken on other kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    cur = kernel_source_hash()
    with open(p) as f:
        for line in f:
            t = line.split()
            # lines taken on earlier kernel source stay as history; the one
            # whose hash matches the current source counts
            if len(t) >= 4 and not line.startswith("#") and t[0] == kind and t[1] == workload_name and t[3] == cur:
                return float(t[2])
    return None


# ---------------------------------------------------------------------------
# the CPU oracle (baseline leg and reference arm)
# ---------------------------------------------------------------------------

def cpu_oracle_run(name, steps, seconds, seed=0, warmup=0, threads=None):
    """Times oracle dJFA steps on the host cores on the same trajectory; stops
    after `steps` timed steps or `seconds` of timed work, whichever first.
    `threads` limits the oracle's OpenMP threads for this run (None: all)."""
    import oracle
    from paper_2209_00117_gb300 import inputs

    oracle.build()
    if threads is not None:
        prev = oracle.get_threads()
        oracle.set_threads(threads)
        try:
            return cpu_oracle_run(name, steps, seconds, seed=seed, warmup=warmup)
        finally:
            oracle.set_threads(prev)
    w, h, s, _, d = workload(name)
    xy = inputs.uniform_seeds(w, h, s, seed=seed)
    total = warmup + steps
    disp = inputs.displacements(s, d, total, seed=seed)
    t0 = time.perf_counter()
    lab = oracle.jfa(w, h, xy)  # frame 0: the chain's start (timed apart from the dJFA steps)
    t_jfa = time.perf_counter() - t0
    n_pass = len(oracle.djfa_schedule(w, h, s, d, vn_waves=2))
    done, t_acc = 0, 0.0
    for i in range(total):
        t0 = time.perf_counter()
        xy = oracle.move(w, h, xy, disp[i])
        lab = oracle.djfa_step(w, h, xy, lab, d_max=d, vn_waves=2)
        dt = time.perf_counter() - t0
        if i >= warmup:
            done += 1
            t_acc += dt
            if t_acc >= seconds:
                break
    gpx = w * h * n_pass * done / t_acc / 1e9
    return {"value": gpx, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
            "sample": f"{done} dJFA steps (move + stamp + {n_pass} passes) of the {name} trajectory "
                      f"after an untimed JFA frame 0, plain C oracle with OpenMP",
            "ms_per_step": 1e3 * t_acc / max(done, 1), "steps": done, "jfa_ms_per_frame": 1e3 * t_jfa}


def apply_tuning(vd, sim, chosen):
    """Puts a vd_autotune choice on another context of the same workload."""
    for name, v in chosen.items():
        sim.set_option(getattr(vd, "OPT_" + name.upper()), v)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w, h, s, _, d = workload(args.workload)
    import oracle

    res = cpu_oracle_run(args.workload, args.steps, float("inf"), seed=0, warmup=args.warmup)
    n_jfa = len(oracle.jfa_schedule(w, h))
    n_djfa = len(oracle.djfa_schedule(w, h, s, d, vn_waves=2))
    line = {
        "impl": "reference", "metric": METRIC, "value": res["value"], "unit": UNIT,
        "n_gpus": world, "steps": res["steps"], "warmup": args.warmup,
        "ms_per_step": res["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": config_dict(workload_key(args.workload, s, d), w, h, s, d, n_jfa, n_djfa, world,
                              l2_note(w, h, gpu=False)),
        "cpu_baseline": {k: res[k] for k in ("value", "unit", "cores", "kind", "sample")},
        "e2e": {"value": res["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import torch

    from paper_2209_00117_gb300 import build, inputs, vd

    rank, world, local = dist_env()
    build.build()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
        pg = dist

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    w, h, s, _, d = workload(args.workload)
    wkey = workload_key(args.workload, s, d)
    K, W = args.steps, args.warmup
    if W < 3:
        raise SystemExit("--warmup must be >= 3")
    total = W + K
    seed = rank  # independent replica per rank
    xy = inputs.uniform_seeds(w, h, s, seed=seed)
    disp_host = inputs.displacements(s, d, total, seed=seed)
    n_jfa = len(vd.jfa_schedule(w, h))
    n_djfa = len(vd.djfa_schedule(w, h, s, d, vn_waves=2, extra=args.extra))
    px = w * h
    metric = vd.MANHATTAN if args.metric == "manhattan" else vd.EUCLID

    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    disp_dev = torch.from_numpy(disp_host).to(f"cuda:{local}")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=f"cuda:{local}")
    exact_dist = torch.empty((h, w), dtype=torch.int32, device=f"cuda:{local}")

    dj = vd.VoronoiSim(w, h, s, stream=stream)
    jf = vd.VoronoiSim(w, h, s, stream=stream)
    for sim in (dj, jf):
        sim.set_seeds(xy)
        sim.set_option(vd.OPT_USE_GRAPHS, 1)
    dj.jfa(metric=metric)  # frame 0 of the dJFA chain
    tuned = None
    if not args.no_autotune:
        # the library's launch-shape search on this simulation's own steps
        # (state restored afterwards); its choice stays in force
        chosen, cand_ms = dj.autotune(d_max=d, max_disp=d, vn_waves=2, metric=metric, rng_seed=12345, steps=4)
        tuned = {"chosen": chosen, "candidate_ms_per_step": [round(t, 4) for t in cand_ms]}

    def djfa_step(i):
        # move + stamp + passes: one vd_step call (one graph)
        dj.step(disp_dev[i], d_max=d, vn_waves=2, extra=args.extra, metric=metric)

    def jfa_step(i):
        jf.move(disp_dev[i])
        jf.jfa()

    for i in range(W):
        djfa_step(i)
        jfa_step(i)
    torch.cuda.synchronize()

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    sims = []
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    l0 = dj.launches + jf.launches
    t0 = time.perf_counter()
    for j in range(K):
        i = W + j
        flush.zero_()
        ev[j][0].record(stream)
        djfa_step(i)
        ev[j][1].record(stream)
        flush.zero_()
        ev[j][2].record(stream)
        jfa_step(i)
        ev[j][3].record(stream)
        if (j + 1) % 10 == 0 or j == K - 1:
            # scored between steps, outside the step events; the dJFA map against
            # the exact diagram in its own metric, the JFA map in Euclidean
            dj.exact(None, exact_dist, metric=metric)
            ne_d, _ = dj.similarity(exact_dist=exact_dist, metric=metric)
            nm = dj.match_count(jf)
            if metric != vd.EUCLID:
                dj.exact(None, exact_dist, metric=vd.EUCLID)
            ne_j, _ = jf.similarity(exact_dist=exact_dist)
            sims.append((j + 1, nm, ne_d, ne_j))
    barrier()
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    launches = dj.launches + jf.launches - l0
    t_djfa = sum(e[0].elapsed_time(e[1]) for e in ev)  # ms
    t_jfa = sum(e[2].elapsed_time(e[3]) for e in ev)

    dev = f"cuda:{local}"
    t_djfa_max = max_over_ranks(pg, t_djfa, dev)
    t_jfa_max = max_over_ranks(pg, t_jfa, dev)
    value = whole_job_gpx(px * n_djfa, K, world, t_djfa_max)
    jfa_value = whole_job_gpx(px * n_jfa, K, world, t_jfa_max)

    # --- per-kernel timing for the roofline: the same trajectory replayed with
    #     events around every launch (eager launches, L2 flushed between steps)
    pr = vd.VoronoiSim(w, h, s, stream=stream)
    pr.set_seeds(xy)
    if tuned:
        apply_tuning(vd, pr, tuned["chosen"])
    pr.jfa(metric=metric)
    for i in range(W):
        pr.step(disp_dev[i], d_max=d, vn_waves=2, extra=args.extra, metric=metric)
    pr.set_option(vd.OPT_PROFILE, 1)
    pr.profile_reset()
    for j in range(K):
        flush.zero_()
        pr.step(disp_dev[W + j], d_max=d, vn_waves=2, extra=args.extra, metric=metric)
    prof = pr.profile()
    pr.close()
    dom = max(prof, key=lambda k: prof[k]["ms"])
    pd = prof[dom]
    n_dom = max(pd["launches"], 1)
    avg_ms_eager = pd["ms"] / n_dom
    if dom in ("pass", "fused"):
        alg_bytes = 8.0 * px + 8.0 * s  # read + write one int32 per pixel, the seed table once
    elif dom == "fill":
        alg_bytes = 4.0 * px
    else:
        alg_bytes = 16.0 * s
    peak, peak_src = hbm_peak()
    tot_ms = sum(v["ms"] for v in prof.values())
    share = pd["ms"] / tot_ms if tot_ms > 0 else 1.0
    # The dominant kernel's mean launch time in the timed region: the timed
    # (graph-replayed, event-bracketed) dJFA frame time, times that kernel's
    # share of GPU time in an eager replay of the same steps with events around
    # every launch, divided by its launches per frame.  Its time x launches per
    # step is then at most ms_per_step by construction.
    per_step = n_dom / K
    live_ms = (t_djfa / K) * share / per_step
    achieved = alg_bytes / (live_ms * 1e-3) / 1e9
    eager_gbs = alg_bytes / (avg_ms_eager * 1e-3) / 1e9
    roofline = {
        "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
        "traffic": recorded_traffic(dom, wkey),
        "kernel": dom, "alg_bytes_per_launch": alg_bytes, "avg_launch_us": live_ms * 1e3,
        "launches_per_step": per_step,
        "kernel_ms_per_step": live_ms * per_step,
        "peak_source": peak_src,
        "share": {k: round(v["ms"] / tot_ms, 4) for k, v in prof.items() if tot_ms > 0},
        "measured": "timed-region dJFA frame time (CUDA events around each graph-replayed step on the launching "
                    "stream) x the kernel's share of GPU time in an eager replay of the same K steps with CUDA "
                    "events around every launch / its launches per step",
        "eager_replay": {"avg_launch_us": avg_ms_eager * 1e3, "achieved": eager_gbs, "frac": eager_gbs / peak,
                         "method": "CUDA events around every launch (eager, serialised launches)"},
    }

    # --- end to end through the API with host buffers
    e2e = None
    if not args.no_e2e:
        ee = vd.VoronoiSim(w, h, s, stream=stream)
        ee.set_seeds(xy)
        ee.set_option(vd.OPT_USE_GRAPHS, 1)
        if tuned:
            apply_tuning(vd, ee, tuned["chosen"])
        ee.jfa(metric=metric)
        pin_disp = torch.from_numpy(disp_host).pin_memory()
        # the map comes back bit-packed at the fewest bits the labels need (the
        # copy to the host is the bound of this leg: 19 bits a pixel for 2^18
        # seeds instead of 32), or as 24-bit labels, or as the int32 map
        if args.e2e_labels == "packed":
            bits = vd.label_bits(s)
        else:
            bits = 24 if args.e2e_labels == "24" and s <= 0xFFFFFF else 32
        if args.e2e_labels == "packed":
            pin_out = [torch.empty((px * bits + 7) // 8, dtype=torch.uint8).pin_memory() for _ in range(2)]
            read_back = lambda out: ee.labels_packed_async(out, bits)  # noqa: E731
        elif bits == 24:
            pin_out = [torch.empty(3 * h * w, dtype=torch.uint8).pin_memory() for _ in range(2)]
            read_back = ee.labels24_async
        else:
            pin_out = [torch.empty((h, w), dtype=torch.int32).pin_memory() for _ in range(2)]
            read_back = ee.labels_async
        for i in range(W):
            ee.step(pin_disp[i], d_max=d, vn_waves=2, extra=args.extra, metric=metric)
            read_back(pin_out[i % 2])
        ee.wait_labels()
        barrier()
        t_e2e = time.perf_counter()
        for j in range(K):
            # inputs in from pinned memory; every step's map copied out while
            # the next step computes (two read-back slots)
            ee.step(pin_disp[W + j], d_max=d, vn_waves=2, extra=args.extra, metric=metric)
            read_back(pin_out[j % 2])
        ee.wait_labels()
        barrier()
        te = max_over_ranks(pg, 1e3 * (time.perf_counter() - t_e2e), dev)
        # the last step's map, widened on the host, equals the context's own
        if args.e2e_labels == "packed":
            assert np.array_equal(vd.unpack_labels(pin_out[(K - 1) % 2].numpy(), h, w, bits, rows_per_chunk=256),
                                  ee.labels())
        elif bits == 24:
            assert np.array_equal(vd.widen24(pin_out[(K - 1) % 2].numpy(), h, w), ee.labels())
        ee.close()
        e2e = {"value": whole_job_gpx(px * n_djfa, K, world, te), "unit": UNIT,
               "h2d_bytes_per_step": int(s * 2 * 4), "d2h_bytes_per_step": int((px * bits + 7) // 8),
               "ms_per_step": te / K, "labels": f"{bits}-bit" + (" packed" if args.e2e_labels == "packed" else ""),
               "timing": "host wall clock around K steps (pinned displacements in, every step's whole label map "
                         f"read back as {bits}-bit labels, read-back overlapped with the next step)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res = cpu_oracle_run(args.workload, K, args.cpu_seconds, seed=0)
        cpu = {k: res[k] for k in ("value", "unit", "cores", "kind", "sample")}
        cpu["ms_per_step"] = res["ms_per_step"]
        cpu["jfa_ms_per_frame"] = res["jfa_ms_per_frame"]
        if w * h <= (1 << 24):
            # the same oracle on one core, a shorter bounded sample
            one = cpu_oracle_run(args.workload, K, args.cpu_seconds / 3, seed=0, threads=1)
            cpu["single_thread"] = {"value": one["value"], "ms_per_step": one["ms_per_step"], "steps": one["steps"],
                                    "jfa_ms_per_frame": one["jfa_ms_per_frame"]}

    last = sims[-1] if sims else (0, 0, 0, 0)
    similarity = {
        "frames_scored": [f for f, *_ in sims],
        "djfa_vs_jfa_pct": [round(100.0 * nm / px, 4) for _, nm, _, _ in sims],
        "djfa_exact_pct": [round(100.0 * ne / px, 4) for _, _, ne, _ in sims],
        "jfa_exact_pct": [round(100.0 * ne / px, 4) for _, _, _, ne in sims],
        "last_counts": {"frame": last[0], "pixels": px, "djfa_match_jfa": last[1],
                        "djfa_distance_correct": last[2], "jfa_distance_correct": last[3]},
    }
    dj.close()
    jf.close()
    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": t_djfa_max / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": config_dict(wkey, w, h, s, d, n_jfa, n_djfa, world, l2_note(w, h, gpu=True)),
        "ms_per_frame": {"djfa": t_djfa_max / K, "jfa": t_jfa_max / K},
        "jfa": {"value": jfa_value, "unit": UNIT, "ms_per_step": t_jfa_max / K},
        "speedup_djfa_vs_jfa": t_jfa_max / t_djfa_max,
        # the pass-count ratio beside the measured speedup: a speedup well
        # above it would mean a slow JFA arm rather than fewer passes
        "pass_ratio_jfa_vs_djfa": n_jfa / n_djfa,
        "ms_per_pass": {"djfa": t_djfa_max / K / n_djfa, "jfa": t_jfa_max / K / n_jfa},
        "similarity": similarity,
        "roofline": roofline,
        "autotune": tuned,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "wall_s_timed_region": wall,
    }
    print(json.dumps(line))
    if pg is not None:
        pg.destroy_process_group()
    return 0


def init_ranks():
    """(rank, world, local, process group or None): NCCL ranks under a
    multi-rank launch, used only for host-side aggregation and barriers."""
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
        pg = dist
    return rank, world, local, pg


def run_batched(args):
    """256 independent simulations (sides in {256, 512, 1024, 2048}, seeds
    uniform in [64, side^2/64], moves in [-2, 2]) stepped as one batch per
    timestep, against the same simulations run one by one with one launch per
    pass (plain JFA frames, and unbatched dJFA frames).  Under N ranks each
    rank steps its own disjoint share of the 256 (simulation i on rank
    i % N): no data-path collective, the counts and times are aggregated on
    the host (sum of work, maximum of time)."""
    import torch

    from paper_2209_00117_gb300 import build, inputs, vd

    build.build()
    rank, world, local, pg = init_ranks()
    dev = f"cuda:{local}"
    K, W, D = args.steps, args.warmup, 2
    pop = inputs.batched_population(256, seed=0)
    mine = owned(len(pop), world, rank)
    shapes = [(pop[i].w, pop[i].h, pop[i].s) for i in mine]
    xys = [inputs.uniform_seeds(w, h, s_, seed=i) for i, (w, h, s_) in zip(mine, shapes)]
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    b = vd.VoronoiBatch(shapes, stream=stream)
    b.set_seeds(np.concatenate(xys))
    b.jfa()
    b.configure(d_max=D)
    if args.no_autotune:
        # the autotuner's usual choice: launch per round, 4 rows a thread
        b.set_option(vd.BOPT_ROWS_PER_THREAD, 4)
        best, cand_ms = None, []
    else:
        best, cand_ms = b.autotune(steps=3, max_disp=D, rng_seed=0)
    px, pp, n_seeds = b.work()
    for _ in range(W):
        b.step(None, max_disp=D, rng_seed=0)
    b.synchronize()
    if pg is not None:
        pg.barrier()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e[0].record(stream)
    for _ in range(K):
        b.step(None, max_disp=D, rng_seed=0)
    e[1].record(stream)
    b.synchronize()
    t_batch = max_over_ranks(pg, e[0].elapsed_time(e[1]), dev)
    steps_done = W + K

    # the same simulations one by one, one launch per pass: JFA frames and dJFA frames
    sims = []
    for j, (w, h, s_) in enumerate(shapes):
        c = vd.VoronoiSim(w, h, s_, stream=stream)
        c.set_seeds(xys[j])
        c.set_option(vd.OPT_USE_GRAPHS, 0)
        sims.append(c)
    K1 = max(1, min(K, 5))

    def per_sim_steps(frame, n_steps, step0):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for t in range(n_steps):
            for j, c in enumerate(sims):
                c.move(None, max_disp=D, rng_seed=0, stream_id=j, step=step0 + t)
                frame(c)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n_steps

    # bring the contexts to the batch's frame with JFA (timing the last K1 steps)
    for c in sims:
        c.jfa()
    per_sim_steps(lambda c: c.jfa(), steps_done - K1, 0)
    t_jfa = max_over_ranks(pg, per_sim_steps(lambda c: c.jfa(), K1, steps_done - K1), dev)
    # similarity of the batch's dJFA maps to same-frame JFA maps, on the GPU
    match = 0
    for j, (w, h, _) in enumerate(shapes):
        lab = torch.empty((h, w), dtype=torch.int32, device=dev)
        b.labels(j, out=lab)
        match += sims[j].similarity(ref_labels=lab)[1]
    # unbatched dJFA, one launch per pass, from the JFA maps
    t_djfa_alone = max_over_ranks(pg, per_sim_steps(lambda c: c.djfa_step(d_max=D), K1, steps_done), dev)
    pp_jfa = sum(w * h * len(vd.jfa_schedule(w, h)) for (w, h, _) in shapes)
    for c in sims:
        c.close()
    b.close()
    # whole-job sums of this rank's work (host-side aggregation)
    px_all = sum_over_ranks(pg, px, dev)
    pp_all = sum_over_ranks(pg, pp, dev)
    pp_jfa_all = sum_over_ranks(pg, pp_jfa, dev)
    seeds_all = sum_over_ranks(pg, n_seeds, dev)
    match_all = sum_over_ranks(pg, match, dev)
    sims_all = sum_over_ranks(pg, len(shapes), dev)
    if pg is not None:
        pg.destroy_process_group()
    if rank != 0:
        return 0
    line = {
        "workload": "batched256: 256 independent simulations, sides uniform in {256, 512, 1024, 2048}, "
                    "seeds uniform in [64, side^2/64], moves uniform in [-2, 2]",
        "metric": METRIC, "unit": UNIT, "steps": K, "warmup": W, "dtype": "int32", "data": "synthetic",
        "n_gpus": world, "scaling": "strong", "simulations": int(sims_all),
        "parallelism": f"simulation i on rank i % {world}" if world > 1 else "single",
        "pixels": int(px_all), "seeds": int(seeds_all), "pixel_passes_per_step": int(pp_all),
        "batched_djfa": {"value": pp_all / (t_batch / K * 1e-3) / 1e9, "ms_per_step": t_batch / K,
                         "launch_shape": {"candidate": best, "candidate_ms": cand_ms,
                                          "mode": "persistent" if b_mode(best) else "per round (graph)"}},
        "unbatched_djfa_one_launch_per_pass": {"value": pp_all / (t_djfa_alone * 1e-3) / 1e9,
                                               "ms_per_step": t_djfa_alone},
        "plain_jfa_one_launch_per_pass": {"value": pp_jfa_all / (t_jfa * 1e-3) / 1e9, "ms_per_step": t_jfa},
        "speedup_batched_djfa_vs_plain_jfa": t_jfa / (t_batch / K),
        "similarity_djfa_vs_jfa_pct": round(100.0 * match_all / px_all, 4),
        "l2": "working set (2 maps per simulation) is larger than L2",
    }
    print(json.dumps(line))
    return 0


def b_mode(candidate):
    """Autotuner candidates 3 .. 14 are the persistent launch shapes (0 .. 2
    and 15, 16 launch per round; None: not autotuned, launch per round)."""
    return candidate is not None and 3 <= candidate <= 14


def run_serve(args):
    """1000 resident simulations (sides in {512, 1024, 2048, 4096}, density as
    the batched workload) admitted under an 80 GB HBM budget, then Poisson
    request traces at each rate: p50 / p99 step latency and steps/s.  Under N
    ranks simulation i lives on rank i % N, each with its own server and an
    80 GB budget of its own GPU; a rank replays the requests of the one
    shared trace that target its simulations, and the latencies are merged on
    the host (percentiles of all ranks' latencies together)."""
    import torch

    from paper_2209_00117_gb300 import build, inputs, vd

    build.build()
    rank, world, local, pg = init_ranks()
    dev = f"cuda:{local}"
    D = 2
    pop = inputs.batched_population(1000, sides=(512, 1024, 2048, 4096), seed=0)
    mine = owned(len(pop), world, rank)
    srv = vd.VoronoiServer(max_sims=len(mine), hbm_budget_bytes=80 * 10**9, d_max=D, max_disp=D, rng_seed=0)
    sid = {}  # global simulation index -> this rank's server id
    refused = 0
    from paper_2209_00117_gb300._native import VDError

    t0 = time.perf_counter()
    for i in mine:
        p = pop[i]
        try:
            sid[i] = srv.add_sim(p.w, p.h, inputs.uniform_seeds(p.w, p.h, p.s, seed=i))
        except VDError:
            refused += 1
    t_admit = time.perf_counter() - t0
    st = srv.stats()
    admitted = sorted(sid)
    admitted_all = gather_arrays(pg, np.asarray(admitted, np.float64)).astype(np.int64)
    out = []
    for rate in [float(r) for r in args.rates.split(",")]:
        n = max(1, int(rate * args.duration))
        arr = inputs.poisson_arrivals(rate, n, seed=int(rate))
        # the one trace over every admitted simulation, split by owner
        tgt = admitted_all[inputs.request_targets(n, len(admitted_all), seed=int(rate))]
        keep = np.fromiter((t % world == rank for t in tgt), dtype=bool, count=n)
        a_mine = arr[keep]
        t_mine = np.asarray([sid[int(t)] for t in tgt[keep]], np.int32)
        if pg is not None:
            pg.barrier()
        lat = srv.run_trace(a_mine, t_mine) if len(a_mine) else np.zeros(0)
        span = float(np.max(a_mine + lat)) if len(a_mine) else 0.0
        lat_all = gather_arrays(pg, lat)
        span_all = max_over_ranks(pg, span, dev)
        out.append({"rate_per_s": rate, "requests": n, **latency_summary(lat_all),
                    "steps_per_s": n / span_all})
    st2 = srv.stats()
    srv.close()
    used = sum_over_ranks(pg, st["used_bytes"], dev)
    refused_all = sum_over_ranks(pg, refused, dev)
    launches = sum_over_ranks(pg, st2["launches"] - st["launches"], dev)
    steps_done = sum_over_ranks(pg, st2["steps_done"], dev)
    t_admit = max_over_ranks(pg, t_admit, dev)
    if pg is not None:
        pg.destroy_process_group()
    if rank != 0:
        return 0
    print(json.dumps({
        "workload": "serve1000: 1000 resident simulations, sides uniform in {512, 1024, 2048, 4096}, seeds "
                    "uniform in [64, side^2/64], dJFA step requests (moves in [-2, 2]) as Poisson streams",
        "unit": "steps/s and ms", "dtype": "int32", "data": "synthetic", "n_gpus": world,
        "parallelism": f"simulation i on rank i % {world}, one server per GPU" if world > 1 else "single",
        "admitted": int(len(admitted_all)), "refused": int(refused_all), "hbm_used_gb": used / 1e9,
        "hbm_budget_gb_per_gpu": st["budget_bytes"] / 1e9, "admit_s": t_admit,
        "kernel_launches": int(launches), "steps": int(steps_done),
        "rates": out}))
    return 0


def run_churn(args):
    """Seed churn on the 2048^2, 16384-seed simulation: every step moves the
    seeds, removes `--churn` random seeds and inserts as many new ones
    (vd_update_seeds), then runs the frame (the repair schedule after a
    removal).  Against plain dJFA steps of the same simulation."""
    import torch

    from paper_2209_00117_gb300 import build, inputs, vd

    rank, world, local = dist_env()
    build.build()
    torch.cuda.set_device(local)
    w = h = 2048
    s, D, K, W = 16384, 2, args.steps, args.warmup
    c = args.churn
    g = np.random.default_rng(rank)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    sim = vd.VoronoiSim(w, h, s, stream=stream)
    sim.set_option(vd.OPT_USE_GRAPHS, 1)
    sim.set_seeds(inputs.uniform_seeds(w, h, s, seed=rank))
    sim.jfa()

    def plain(t):
        sim.move(None, max_disp=D, rng_seed=rank, stream_id=0, step=t)
        sim.djfa_step(d_max=D)

    def churn(t):
        sim.move(None, max_disp=D, rng_seed=rank, stream_id=0, step=t)
        remove = g.choice(sim.n_seeds, size=c, replace=False).astype(np.int32)
        add = np.stack([g.integers(0, w, c), g.integers(0, h, c)], axis=1).astype(np.int32)
        t0 = time.perf_counter()
        sim.update_seeds(remove, add)
        t_upd.append(time.perf_counter() - t0)
        sim.djfa_step(d_max=D)

    def timed(fn, step0):
        for i in range(W):
            fn(step0 + i)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(K):
            fn(step0 + W + i)
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / K * 1e3

    t_upd = []
    ms_plain = timed(plain, 0)
    t_upd.clear()
    ms_churn = timed(churn, 10 * (K + W))
    upd_ms = 1e3 * float(np.mean(t_upd[W:])) if len(t_upd) > W else None
    lab = sim.labels()
    ex_l, ex_d = sim.exact()
    n_exact, _ = sim.similarity(exact_dist=ex_d)
    print(json.dumps({
        "workload": f"churn2048: 2048x2048 int32 map, 16384 seeds, moves in [-{D},{D}], {c} seeds removed and "
                    f"{c} inserted per step (vd_update_seeds), each step's frame the repair schedule",
        "unit": "ms per step (host wall clock, K steps)", "steps": K, "warmup": W, "dtype": "int32",
        "data": "synthetic", "churn_per_step": c,
        "ms_per_step_plain_djfa": ms_plain, "ms_per_step_with_churn": ms_churn,
        "ms_update_seeds_alone": upd_ms,
        "empty_pixels_after": int((lab < 0).sum()),
        "distance_correct_pct_after": round(100.0 * n_exact / (w * h), 4),
    }))
    sim.close()
    return 0


def free_port():
    import socket

    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def launch_ranks(n):
    """Runs this command as n ranks, one process per GPU, through
    torch.distributed.run on 127.0.0.1; returns the launcher's exit status."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.run(cmd).returncode


def main():
    args = parse_args()
    if args.gpus < 1:
        raise SystemExit("--gpus must be >= 1")
    if "WORLD_SIZE" in os.environ:
        _, world, _ = dist_env()
        if world != args.gpus:
            raise SystemExit(f"--gpus {args.gpus} but this launch has WORLD_SIZE={world} ranks")
    elif args.gpus > 1:
        return launch_ranks(args.gpus)
    if args.workload == "batched256":
        return run_batched(args)
    if args.workload == "churn2048":
        return run_churn(args)
    if args.workload == "serve1000":
        return run_serve(args)
    _SWEEP["seeds"] = args.seeds
    _SWEEP["max_disp"] = args.max_disp
    _DJFA_METRIC["name"] = args.metric
    _DJFA_METRIC["extra"] = args.extra
    if args.extra not in (0, 1, 2):
        raise SystemExit("--extra takes 0, 1 or 2")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
