"""Benchmark: batched Kalman-filter track finding + duplicate removal + re-fit.

Workload: PU-200-like batch, 100 events x 8,000 generated tracks, 17 barrel
layers, 20% noise hits, up to 10 candidates per seed (synthetic, seeded).
One step = bin hits, find tracks for every seed, remove duplicates, re-fit the
kept tracks and take the gradient of their summed chi2 with respect to the
layer alignment offsets (adjoint of the fit), replayed as one captured CUDA
graph over the whole batch.

Prints one JSON line: seeds/s (whole job), candidate-layer steps/s, the plain
per-event launch form for comparison, the end-to-end rate through the C ABI
with host buffers, the FP32 roofline of the find kernel, the same step with
seed cleaning and the kinematic pre-cuts of duplicate removal switched on
(timed separately, with the cleaning stage's memory roofline) and the FP64
oracle's rate on the host cores (bounded sample).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "seeds/s and candidate-layer KF updates/s at PU-200, batched vs plain; % FP32 peak"
UNIT = "seeds/s"
L2_BYTES = 129 * 1024 * 1024

# Algorithmic operations per unit of work (an FMA counts 2): the operation
# census of the oracle's own step functions (trivial operations dropped, shared
# ones and symmetric results counted once) on states of the same workload,
# stored by the census script beside the oracle and read here as data.  Per
# candidate-layer step (propagation, transport, frame, z window), per hit in
# the search window, per kept hit-child (update), per scattering, per seed fit
# and per hit of the re-fit; window hits per step from the oracle's count of
# hits inside each prediction's chi2-ellipse bounding box.
with open(os.path.join(ROOT, "oracle", "flop_census.json")) as _f:
    CENSUS = json.load(_f)
F_STEP = CENSUS["flops"]["F_STEP"]
F_HIT = CENSUS["flops"]["F_HIT"]
F_UPDATE = CENSUS["flops"]["F_UPDATE"]
F_MS = CENSUS["flops"]["F_MS"]
F_SEED = CENSUS["flops"]["F_SEED"]
WINDOW_HITS_PER_STEP = CENSUS["window_hits_per_step"]
# Steps onto endcap disks (plane step, (r-phi, r) frame and r window, disk
# update and scattering), counted apart on a barrel-plus-endcap event.
F_DISK_STEP = CENSUS["disks"]["flops"]["F_DISK_STEP"]
F_DISK_HIT = CENSUS["disks"]["flops"]["F_DISK_HIT"]
F_DISK_UPDATE = CENSUS["disks"]["flops"]["F_DISK_UPDATE"]
F_DISK_MS = CENSUS["disks"]["flops"]["F_DISK_MS"]
WINDOW_HITS_PER_DISK_STEP = CENSUS["disks"]["window_hits_per_disk_step"]

# DRAM traffic (read + write) of one k_find launch on the 100-event batch,
# scaled by events from an ncu capture of the same kernel on 20 of its events
# (191.46 MB: 169.83 read + 21.62 written).
# None whenever k_find changes until it is captured again.
FIND_TRAFFIC_BYTES = 191.46e6 * 5

# Duplicate handling measured beside the headline step (Sec. 4.2): seed
# cleaning on kinematics alone (eta, phi0 within 0.01, pT within 20%) and
# duplicate removal with pre-cuts (eta, phi0 within 0.02, pT within 30%).
DUP_CFG = dict(seed_clean=1, seed_deta=0.01, seed_dphi=0.01, seed_dpt=0.2, seed_min_shared=0,
               dup_deta=0.02, dup_dphi=0.02, dup_dpt=0.3)
# Algorithmic HBM bytes of seed cleaning per seed: k_sc_kin reads the order
# entry, five state values and three hit indices and writes 32 B of
# kinematics and hits (68 B); k_sc_conflicts reads its own 32 B and writes a
# conflict count and state (37 B; neighbours come from L2); k_sc_resolve reads
# order and state twice, writes the new order entry and keep flag (15 B).
CLEAN_BYTES_PER_SEED = 68 + 37 + 15
# DRAM traffic (read + write) of the three seed-cleaning kernels per 100-event
# batch, scaled by events from an ncu capture on 20 of its events (17.57 MB;
# ncu flushes the caches before each kernel, so this is the cold-cache figure).
# Set to None whenever those kernels change until they are captured again.
CLEAN_TRAFFIC_BYTES = 17.57e6 * 5

FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0


def _measured_peak(key, fallback):
    """(value, source) of a measured peak of this GPU model, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key]), "measured"
    except (OSError, KeyError, ValueError):
        return fallback, "fallback"


def sm_count(dev=0):
    import torch
    return torch.cuda.get_device_properties(dev).multi_processor_count


def fp32_peak_tflops(n_sm, mhz=SM_MAX_MHZ):
    return n_sm * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while running."""

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([s.strip() for s in line.split(",")])

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[0]))
                mx.append(float(s[1]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, s[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(value, device):
    """Largest value over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_alignment_over_ranks(g_align, chi2_total, device):
    """The one exchange of the multi-GPU path: every rank fits its own events,
    and the alignment gradient [n_layers][2] and the summed chi2 are added
    over ranks (one all-reduce of 2 n_layers + 1 values).  Returns the sums;
    the identity without a process group."""
    import torch
    import torch.distributed as dist
    v = np.concatenate([np.asarray(g_align, np.float64).ravel(), [float(chi2_total)]])
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        t = torch.from_numpy(v).to(device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        v = t.cpu().numpy()
    return v[:-1].reshape(np.shape(g_align)), float(v[-1])


def make_inputs(name, rank, n_events=None, **overrides):
    from synth import make_batch
    # per-rank distinct events: shift the configuration seed by the rank
    from synth.events import CONFIGS
    seed = CONFIGS[name]["seed"] + 7919 * rank
    return make_batch(name, n_events=n_events, seed=seed, **overrides)


# Parameterized field of the field-map step: Bz 10% weaker at |z| = 120 cm
# and 5% weaker at r = 110 cm than at the centre.
FIELD_MAP = dict(field_cz=-0.10 / 120.0 ** 2, field_cr=-0.05 / 110.0 ** 2)


def tracker_for(b, **cfg):
    from paper_1906_11744_gb300 import Tracker, make_config, make_detector
    d = b.det
    disks = dict(disk_z=tuple(d.disk_z), disk_rmin=d.disk_rmin, disk_rmax=d.disk_rmax, disk_x0=d.disk_x0,
                 disk_eloss=d.disk_eloss, sigma_r=d.sigma_r, eta_barrel=d.eta_barrel) if getattr(d, "disk_z", ()) else {}
    det = make_detector(d.radius, d.x0, d.z_max, d.bz, d.sigma_rphi, d.sigma_z, eloss=getattr(d, "eloss", None),
                        field_cz=getattr(d, "field_cz", 0.0), field_cr=getattr(d, "field_cr", 0.0), **disks)
    c = dict(max_cands=b.cfg["max_cands"])
    c.update(cfg)
    return Tracker(det, make_config(**c))


def _oracle_event(b, e, threads, ex):
    """The FP64 oracle on one whole event: find (seed ranges on `threads`
    host threads; the oracle's C++ calls release the interpreter lock),
    duplicate removal of the event, re-fit of the kept tracks with the
    gradient of their summed chi2 (track ranges on the threads).  Returns
    (seeds, candidate-layer steps)."""
    import oracle
    prm, cov, sh = b.event_seeds(e)
    ns = prm.shape[1]
    cuts = np.linspace(0, ns, threads + 1).astype(int)
    parts = list(ex.map(lambda k: oracle.find_event(b, e, seeds=(int(cuts[k]), int(cuts[k + 1]))), range(threads)))
    hits = np.concatenate([r["hits"] for r in parts])
    n_found = np.concatenate([r["n_found"] for r in parts])
    chi2 = np.concatenate([r["chi2"] for r in parts])
    steps = sum(r["counters"]["steps"] for r in parts)
    keep = oracle.dedup(hits, n_found, chi2, 0.5)
    x, y, z, lay = b.event_hits(e)
    k = np.nonzero(keep)[0]
    kc = np.array_split(k, threads)
    list(ex.map(lambda ks: oracle.fit_grad(b.det, prm[:, ks], cov[:, ks], hits[ks], n_found[ks], x, y, z, lay,
                                           b.align) if len(ks) else None, kc))
    return ns, steps


def oracle_sample(b, budget_s=15.0, threads=None):
    """The oracle on whole events of the batch, one after the other, each
    spread over `threads` host threads, until about budget_s seconds."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    oracle.build()
    threads = threads or os.cpu_count() or 1
    t0 = time.perf_counter()
    seeds = steps = events = 0
    with ThreadPoolExecutor(threads) as ex:
        for e in range(b.n_events):
            s_, st_ = _oracle_event(b, e, threads, ex)
            seeds += s_
            steps += st_
            events += 1
            if time.perf_counter() - t0 > budget_s:
                break
    dt = time.perf_counter() - t0
    return dict(value=seeds / dt, unit=UNIT, cores=threads, kind="oracle", seconds=dt,
                sample=f"{events} of {b.n_events} events ({seeds} seeds), find + dedup + fit + chi2 gradient, "
                       f"FP64, {threads} host thread{'s' if threads > 1 else ''}",
                steps_per_s=steps / dt)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    b = make_inputs(args.config, 0, n_events=min(args.ref_events, 100))
    times = []
    seeds = 0
    for _ in range(args.warmup + args.steps):
        r = oracle_sample(b, budget_s=args.ref_budget / max(1, args.steps))
        times.append(r)
    timed = times[args.warmup:]
    value = statistics.mean(t["value"] for t in timed)
    seeds = sum(int(t["sample"].split("(")[1].split()[0]) for t in timed)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1000.0 * statistics.mean(t["seconds"] for t in timed),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": workload_desc(args.config)},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": timed[0]["cores"], "kind": "oracle",
                            "sample": timed[0]["sample"]},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def mixed_pileup(args, rank, dev, stream, flush_l2):
    """The batching comparison on 64 events of uneven pileup (20-200, 1,000 to
    10,000 seeds each, N = 6): one captured graph over the batch (launch shape
    from the autotuner, whose full table is returned) against plain
    per-event launches without a graph, the same step (bin, find, duplicate
    removal, fit, adjoint) and L2 flush as the headline."""
    import torch
    from paper_1906_11744_gb300 import KF_FIT_FOUND
    b = make_inputs("c2", rank)
    d_in = {k: torch.from_numpy(np.ascontiguousarray(getattr(b, k))).to(dev)
            for k in ("x", "y", "z", "layer", "params", "cov", "seed_hits")}

    def loaded(**cfg):
        t = tracker_for(b, **cfg)
        t.load_hits(b.hit_off, d_in["x"], d_in["y"], d_in["z"], d_in["layer"], stream)
        t.load_seeds(b.seed_off, d_in["params"], d_in["cov"], d_in["seed_hits"], stream)
        t.set_alignment(b.align, stream)
        return t

    def timed(step):
        for _ in range(args.warmup):
            step()
        stream.synchronize()
        ea = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        eb = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        for k in range(args.steps):
            flush_l2()
            ea[k].record(stream)
            step()
            eb[k].record(stream)
        stream.synchronize()
        return max_over_ranks(sum(a.elapsed_time(c) for a, c in zip(ea, eb)), dev) / args.steps

    tb = loaded(persistent=1, per_event=0)
    tune = tb.autotune(stream)
    best = tune[np.argmin(tune[:, 4])]
    tb.close()
    tb = loaded(persistent=1, per_event=0, lanes_per_seed=int(best[0]), block_threads=int(best[1]),
                find_regcap=int(best[3]))
    tb.capture_graph(with_adjoint=True, stream=stream)
    ms_b = timed(lambda: tb.launch_graph(stream))
    tb.close()
    tp = loaded(persistent=0, per_event=1, lanes_per_seed=int(best[0]))
    g_plain = torch.empty((b.det.n_layers, 2), dtype=torch.float32, device=dev)

    def plain_step():
        tp.find_tracks(stream)
        tp.remove_duplicates(stream)
        tp.fit_tracks(KF_FIT_FOUND, stream=stream)
        tp.fit_adjoint(g_plain, stream=stream)

    ms_p = timed(plain_step)
    tp.close()
    n = b.n_seeds * (int(os.environ.get("WORLD_SIZE", "1")))
    per_ev = np.diff(b.seed_off)
    return {"workload": workload_desc("c2"), "seeds_per_step": int(b.n_seeds),
            "seeds_per_event_min_max": [int(per_ev.min()), int(per_ev.max())],
            "batched": {"value": n / (ms_b / 1e3), "unit": UNIT, "ms_per_step": ms_b,
                        "form": "one CUDA graph per step over the 64 events, persistent finding kernel"},
            "plain": {"value": n / (ms_p / 1e3), "unit": UNIT, "ms_per_step": ms_p,
                      "form": "per-event launches of bin/find/dedup, one fit and one adjoint launch, no graph"},
            "batched_over_plain": ms_p / ms_b,
            "autotune": {"columns": ["lanes_per_seed", "block_threads", "persistent", "register_cap", "find_ms"],
                         "rows": [[float(v) for v in r] for r in tune],
                         "pick": [float(v) for v in best]}}


def workload_desc(name):
    from synth.events import CONFIGS
    c = CONFIGS[name]
    tr = c["tracks"] if c["tracks"] != "pileup" else f"50xPU{c['pileup_range']}"
    return (f"{name}: {c['n_events']} events x {tr} tracks, {c['n_layers']} barrel layers, "
            f"{int(100 * c['noise'])}% noise, N={c['max_cands']} candidates, 64x1024 eta-phi bins")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c4")
    ap.add_argument("--events", type=int, default=None, help="override the number of events")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--find-shape", default=None,
                    help="lanes,threads,persistent,regcap of the finding kernel (skips the autotuner)")
    ap.add_argument("--no-oracle", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-dup", action="store_true", help="skip the duplicate-handling step")
    ap.add_argument("--no-material", action="store_true", help="skip the material-map step")
    ap.add_argument("--no-field", action="store_true", help="skip the parameterized-field step")
    ap.add_argument("--no-endcap", action="store_true", help="skip the barrel-plus-endcap step (c6)")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-pileup (64 events, PU 20-200) step")
    ap.add_argument("--oracle-budget", type=float, default=15.0)
    ap.add_argument("--ref-budget", type=float, default=60.0)
    ap.add_argument("--ref-events", type=int, default=20)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1906_11744_gb300 import KF_FIT_FOUND

    b = make_inputs(args.config, rank, n_events=args.events)
    n_seeds = b.n_seeds
    stream = torch.cuda.Stream(device=dev)
    tt = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    d_in = dict(x=tt(b.x), y=tt(b.y), z=tt(b.z), layer=tt(b.layer), params=tt(b.params),
                cov=tt(b.cov), seed_hits=tt(b.seed_hits))
    torch.cuda.synchronize()

    shape = {}
    if args.find_shape:
        lanes, threads, pers, regcap = (int(v) for v in args.find_shape.split(","))
        shape = dict(lanes_per_seed=lanes, block_threads=threads, persistent=pers, find_regcap=regcap)
        args.no_autotune = True
    t = tracker_for(b, **{"persistent": 1, "per_event": 0, **shape})
    t.load_hits(b.hit_off, d_in["x"], d_in["y"], d_in["z"], d_in["layer"], stream)
    t.load_seeds(b.seed_off, d_in["params"], d_in["cov"], d_in["seed_hits"], stream)
    t.set_alignment(b.align, stream)
    tune = None
    if not args.no_autotune:
        tune = t.autotune(stream)
    t.set_stage_timing(True)
    t.capture_graph(with_adjoint=True, stream=stream)
    n_kernels = t.graph_kernel_count()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def flush_l2():
        with torch.cuda.stream(stream):
            flush.fill_(1.0)

    for _ in range(args.warmup):
        t.launch_graph(stream)
    stream.synchronize()
    counters = t.counters(stream)

    ev_a = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_b = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stage = {"bin": 0.0, "find": 0.0, "dedup": 0.0, "fit": 0.0, "adjoint": 0.0}
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    for k in range(args.steps):
        flush_l2()
        ev_a[k].record(stream)
        t.launch_graph(stream)
        ev_b[k].record(stream)
        st = t.stage_ms(stream)  # synchronizes the stream
        for key in stage:
            stage[key] += st[key]
    torch.cuda.synchronize()
    clocks.stop()
    step_ms = [a.elapsed_time(bb) for a, bb in zip(ev_a, ev_b)]
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(total_ms, dev)
    seeds_all = n_seeds * world
    value = seeds_all * args.steps / (total_ms / 1e3)

    # the one exchange of the multi-GPU path, after the timed steps: the
    # alignment gradient and the fit chi2 summed over ranks
    from paper_1906_11744_gb300 import kf_get_gradient
    g_rank = np.zeros((b.det.n_layers, 2), np.float32)
    kf_get_gradient(t.ctx, g_align=g_rank, stream=stream)
    fit_last = t.get_fit(stream=stream)
    chi2_rank = float(fit_last["chi2"][fit_last["status"] == 0].astype(np.float64).sum())
    g_sum, chi2_sum = sum_alignment_over_ranks(g_rank, chi2_rank, dev)
    exchange = {"values": int(g_sum.size + 1), "chi2_total": chi2_sum, "g_align_abs_max": float(np.abs(g_sum).max()),
                "form": "all-reduce (sum) of the alignment gradient and the fit chi2 over ranks, after the timed steps"}
    steps_per_s = counters["steps"] * world * args.steps / (total_ms / 1e3)

    # roofline of the find kernel (ALU bound: FP32 FMA pipe)
    find_ms = stage["find"] / args.steps
    # counters (steps, updates, holes, seeds) equal the oracle's on the same
    # inputs (tests); window hits from the oracle's rate per step
    find_flops = (counters["steps"] * (F_STEP + WINDOW_HITS_PER_STEP * F_HIT) + counters["updates"] * F_UPDATE
                  + (counters["updates"] + counters["holes"]) * F_MS + counters["seeds"] * F_SEED)
    achieved = find_flops / (find_ms / 1e3) / 1e12
    n_sm = sm_count(dev)
    peak = fp32_peak_tflops(n_sm)
    traffic = None
    if FIND_TRAFFIC_BYTES is not None and args.config == "c4" and not args.events:
        traffic = FIND_TRAFFIC_BYTES
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": "k_find",
                "flops_per_launch": find_flops, "find_ms": find_ms,
                "flops_per_unit": {"step": F_STEP, "window_hit": F_HIT, "window_hits_per_step": WINDOW_HITS_PER_STEP,
                                   "update": F_UPDATE, "scatter": F_MS, "seed_fit": F_SEED,
                                   "source": "oracle operation census (oracle/flop_census.json)"},
                "peak_note": f"{n_sm} SMs (device) x 128 FP32 lanes x 2 x 2070 MHz (unit counts x max clock)"}

    # plain per-event launches (no graph), same work
    plain = None
    if not args.no_plain:
        tp = tracker_for(b, persistent=0, per_event=1,
                         lanes_per_seed=int(tune[np.argmin(tune[:, 4])][0]) if tune is not None and len(tune) else 0)
        tp.load_hits(b.hit_off, d_in["x"], d_in["y"], d_in["z"], d_in["layer"], stream)
        tp.load_seeds(b.seed_off, d_in["params"], d_in["cov"], d_in["seed_hits"], stream)
        tp.set_alignment(b.align, stream)

        g_plain = torch.empty((b.det.n_layers, 2), dtype=torch.float32, device=dev)

        def plain_step():
            tp.find_tracks(stream)
            tp.remove_duplicates(stream)
            tp.fit_tracks(KF_FIT_FOUND, stream=stream)
            tp.fit_adjoint(g_plain, stream=stream)

        for _ in range(args.warmup):
            plain_step()
        stream.synchronize()
        pa = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        pb = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        for k in range(args.steps):
            flush_l2()
            pa[k].record(stream)
            plain_step()
            pb[k].record(stream)
        stream.synchronize()
        pms = sum(a.elapsed_time(bb) for a, bb in zip(pa, pb))
        plain = {"value": seeds_all * args.steps / (pms / 1e3), "unit": UNIT,
                 "ms_per_step": pms / args.steps,
                 "form": "per-event launches of bin/find/dedup, one fit and one adjoint launch, no graph"}
        tp.close()

    # mixed pileup: 64 events of pileup 20-200, batched graph against plain per-event launches
    mixed = None
    if not args.no_mixed and args.config == "c4":
        mixed = mixed_pileup(args, rank, dev, stream, flush_l2)

    # the same step with seed cleaning and the kinematic pre-cuts of duplicate removal
    dup = None
    if not args.no_dup:
        best = {} if tune is None else dict(
            lanes_per_seed=int(tune[np.argmin(tune[:, 4])][0]), block_threads=int(tune[np.argmin(tune[:, 4])][1]),
            persistent=int(tune[np.argmin(tune[:, 4])][2]), find_regcap=int(tune[np.argmin(tune[:, 4])][3]))
        td = tracker_for(b, **{"persistent": 1, "per_event": 0, **(shape or best), **DUP_CFG})
        td.load_hits(b.hit_off, d_in["x"], d_in["y"], d_in["z"], d_in["layer"], stream)
        td.load_seeds(b.seed_off, d_in["params"], d_in["cov"], d_in["seed_hits"], stream)
        td.set_alignment(b.align, stream)
        td.set_stage_timing(True)
        td.capture_graph(with_adjoint=True, stream=stream)
        for _ in range(args.warmup):
            td.launch_graph(stream)
        stream.synchronize()
        dc = td.counters(stream)
        da = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        db = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        dstage = {}
        for k in range(args.steps):
            flush_l2()
            da[k].record(stream)
            td.launch_graph(stream)
            db[k].record(stream)
            for key, v in td.stage_ms(stream).items():
                dstage[key] = dstage.get(key, 0.0) + v
        stream.synchronize()
        dms = max_over_ranks(sum(a.elapsed_time(bb) for a, bb in zip(da, db)), dev)
        trk = td.get_tracks(stream=stream)
        clean_ms = dstage["seed_clean"] / args.steps
        clean_gbs = n_seeds * CLEAN_BYTES_PER_SEED / (clean_ms / 1e3) / 1e9
        hbm_peak = _measured_peak("hbm_gbs", 6800.0)
        dup = {"value": seeds_all * args.steps / (dms / 1e3), "unit": UNIT, "ms_per_step": dms / args.steps,
               "cuts": DUP_CFG, "stage_ms": {k: v / args.steps for k, v in dstage.items()},
               "seeds_dropped_per_step": int(n_seeds - dc["seeds"]),
               "tracks_kept_per_step": int(trk["keep"].sum()),
               "tracks_kept_without": None,
               "gpu_launches": td.graph_kernel_count() * args.steps,
               "roofline_seed_clean": {"bound": "hbm", "achieved": clean_gbs, "peak": hbm_peak[0],
                                       "unit": "GB/s", "frac": clean_gbs / hbm_peak[0], "peak_source": hbm_peak[1],
                                       "bytes_per_seed": CLEAN_BYTES_PER_SEED,
                                       "traffic": (CLEAN_TRAFFIC_BYTES if CLEAN_TRAFFIC_BYTES is not None
                                                   and args.config == "c4" and not args.events else None)}}
        td.close()
        dup["tracks_kept_without"] = int(t.get_tracks(stream=stream)["keep"].sum())

    # the same step with a material map (thickness per layer at 9 z nodes, 0.01-0.03 X0)
    mat = None
    if not args.no_material:
        best = shape or ({} if tune is None else dict(
            lanes_per_seed=int(tune[np.argmin(tune[:, 4])][0]), block_threads=int(tune[np.argmin(tune[:, 4])][1]),
            persistent=int(tune[np.argmin(tune[:, 4])][2]), find_regcap=int(tune[np.argmin(tune[:, 4])][3])))
        tm = tracker_for(b, **{"persistent": 1, "per_event": 0, **best})
        tm.load_hits(b.hit_off, d_in["x"], d_in["y"], d_in["z"], d_in["layer"], stream)
        tm.load_seeds(b.seed_off, d_in["params"], d_in["cov"], d_in["seed_hits"], stream)
        tm.set_alignment(b.align, stream)
        x0_map = np.random.default_rng(17).uniform(0.01, 0.03, size=(b.det.n_layers, 9)).astype(np.float32)
        tm.set_material(x0_map, stream)
        tm.set_stage_timing(True)
        tm.capture_graph(with_adjoint=True, stream=stream)
        for _ in range(args.warmup):
            tm.launch_graph(stream)
        stream.synchronize()
        ma = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        mb = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        mstage = {}
        for k in range(args.steps):
            flush_l2()
            ma[k].record(stream)
            tm.launch_graph(stream)
            mb[k].record(stream)
            for key, v in tm.stage_ms(stream).items():
                mstage[key] = mstage.get(key, 0.0) + v
        stream.synchronize()
        mms = max_over_ranks(sum(a.elapsed_time(bb) for a, bb in zip(ma, mb)), dev)
        mat = {"value": seeds_all * args.steps / (mms / 1e3), "unit": UNIT, "ms_per_step": mms / args.steps,
               "map": "thickness per layer at 9 z nodes over [-z_max, z_max], uniform 0.01-0.03 X0, linear between",
               "stage_ms": {k: v / args.steps for k, v in mstage.items()},
               "gpu_launches": tm.graph_kernel_count() * args.steps}
        tm.close()

    # the same workload in a parameterized field (events simulated through it)
    fld = None
    if not args.no_field:
        best = shape or ({} if tune is None else dict(
            lanes_per_seed=int(tune[np.argmin(tune[:, 4])][0]), block_threads=int(tune[np.argmin(tune[:, 4])][1]),
            persistent=int(tune[np.argmin(tune[:, 4])][2]), find_regcap=int(tune[np.argmin(tune[:, 4])][3])))
        bf = make_inputs(args.config, rank, n_events=args.events, **FIELD_MAP)
        df = dict(x=tt(bf.x), y=tt(bf.y), z=tt(bf.z), layer=tt(bf.layer), params=tt(bf.params),
                  cov=tt(bf.cov), seed_hits=tt(bf.seed_hits))
        tf = tracker_for(bf, **{"persistent": 1, "per_event": 0, **best})
        tf.load_hits(bf.hit_off, df["x"], df["y"], df["z"], df["layer"], stream)
        tf.load_seeds(bf.seed_off, df["params"], df["cov"], df["seed_hits"], stream)
        tf.set_alignment(bf.align, stream)
        tf.set_stage_timing(True)
        tf.capture_graph(with_adjoint=True, stream=stream)
        for _ in range(args.warmup):
            tf.launch_graph(stream)
        stream.synchronize()
        fa = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        fb = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        fstage = {}
        for k in range(args.steps):
            flush_l2()
            fa[k].record(stream)
            tf.launch_graph(stream)
            fb[k].record(stream)
            for key, v in tf.stage_ms(stream).items():
                fstage[key] = fstage.get(key, 0.0) + v
        stream.synchronize()
        fms = max_over_ranks(sum(a.elapsed_time(bb) for a, bb in zip(fa, fb)), dev)
        fld = {"value": bf.n_seeds * world * args.steps / (fms / 1e3), "unit": UNIT, "ms_per_step": fms / args.steps,
               "field": "Bz(r, z) = 3.8 T (1 + cz z^2 + cr r^2), cz = %.3e, cr = %.3e cm^-2 (10%% weaker at |z| = 120 cm, "
                        "5%% at r = 110 cm), taken at each propagation's start" % (FIELD_MAP["field_cz"],
                                                                                    FIELD_MAP["field_cr"]),
               "counters_per_step": tf.counters(stream),
               "stage_ms": {k: v / args.steps for k, v in fstage.items()},
               "gpu_launches": tf.graph_kernel_count() * args.steps}
        tf.close()
        del df

    # PU-200-like barrel plus endcaps (c6: 20 events x 8,000 tracks, |eta| < 2.4, seven disks
    # per side): finding over the region plans, duplicate removal, fit and adjoint in one graph
    endcap = None
    endcap_batch = None
    if not args.no_endcap:
        be = make_inputs("c6", rank)
        de = dict(x=tt(be.x), y=tt(be.y), z=tt(be.z), layer=tt(be.layer), params=tt(be.params),
                  cov=tt(be.cov), seed_hits=tt(be.seed_hits))
        best_e = shape or ({} if tune is None else dict(
            lanes_per_seed=int(tune[np.argmin(tune[:, 4])][0]), block_threads=int(tune[np.argmin(tune[:, 4])][1]),
            persistent=int(tune[np.argmin(tune[:, 4])][2]), find_regcap=int(tune[np.argmin(tune[:, 4])][3])))
        te = tracker_for(be, **{"persistent": 1, "per_event": 0, **best_e})
        te.load_hits(be.hit_off, de["x"], de["y"], de["z"], de["layer"], stream)
        te.load_seeds(be.seed_off, de["params"], de["cov"], de["seed_hits"], stream)
        te.set_alignment(be.align, stream)
        te.set_stage_timing(True)
        te.capture_graph(with_adjoint=True, stream=stream)
        for _ in range(args.warmup):
            te.launch_graph(stream)
        stream.synchronize()
        ea = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        eb = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        estage = {}
        for k in range(args.steps):
            flush_l2()
            ea[k].record(stream)
            te.launch_graph(stream)
            eb[k].record(stream)
            for key, v in te.stage_ms(stream).items():
                estage[key] = estage.get(key, 0.0) + v
        stream.synchronize()
        ems = max_over_ranks(sum(a.elapsed_time(bb) for a, bb in zip(ea, eb)), dev)
        eta0 = -np.log(np.tan(0.5 * be.params[5].astype(np.float64)))
        trk = te.get_tracks()
        lay_all = be.layer
        n_disk_hits = 0
        for e in range(be.n_events):
            a0, a1 = be.seed_off[e], be.seed_off[e + 1]
            h = trk["hits"][a0:a1]
            lay_e = lay_all[be.hit_off[e]:be.hit_off[e + 1]]
            n_disk_hits += int((lay_e[h[h >= 0]] >= be.det.n_layers).sum())
        ec = te.counters(stream)
        # roofline of the disk finding kernel: barrel and disk steps, updates
        # and scatterings at their own census counts (the disk counters are
        # parts of the totals; barrel window hits at the barrel batch's rate)
        e_find_ms = estage["find"] / args.steps
        nd, ndu, ndh = ec["disk_steps"], ec["disk_updates"], ec["disk_holes"]
        e_flops = ((ec["steps"] - nd) * (F_STEP + WINDOW_HITS_PER_STEP * F_HIT)
                   + nd * (F_DISK_STEP + WINDOW_HITS_PER_DISK_STEP * F_DISK_HIT)
                   + (ec["updates"] - ndu) * F_UPDATE + ndu * F_DISK_UPDATE
                   + (ec["updates"] - ndu + ec["holes"] - ndh) * F_MS + (ndu + ndh) * F_DISK_MS
                   + ec["seeds"] * F_SEED)
        e_ach = e_flops / (e_find_ms / 1e3) / 1e12
        endcap_batch = be
        endcap = {"workload": "c6: %d events x 8,000 tracks, |eta| < 2.4, 17 barrel layers + 2 x 7 disks "
                              "(|z| 130-250 cm, r 15-110 cm), 20%% noise, N=10" % be.n_events,
                  "roofline": {"bound": "alu", "achieved": e_ach, "peak": peak, "unit": "TFLOP/s",
                               "frac": e_ach / peak, "traffic": None, "kernel": "k_find (disk variant)",
                               "flops_per_launch": e_flops, "find_ms": e_find_ms,
                               "flops_per_unit": {"disk_step": F_DISK_STEP, "disk_window_hit": F_DISK_HIT,
                                                  "window_hits_per_disk_step": WINDOW_HITS_PER_DISK_STEP,
                                                  "disk_update": F_DISK_UPDATE, "disk_scatter": F_DISK_MS,
                                                  "source": "oracle operation census (oracle/flop_census.json)"}},
                  "find_shape": best_e or None,
                  "value": be.n_seeds * world * args.steps / (ems / 1e3), "unit": UNIT,
                  "ms_per_step": ems / args.steps,
                  "forward_seed_fraction": float(np.mean(np.abs(eta0) >= be.det.eta_barrel)),
                  "found_disk_hits_per_step": n_disk_hits,
                  "counters_per_step": ec,
                  "stage_ms": {k: v / args.steps for k, v in estage.items()},
                  "gpu_launches": te.graph_kernel_count() * args.steps}
        te.close()
        del de

    # end to end through the C ABI with host buffers (pinned), host<->device copies inside.
    # Two contexts: while one step's graph runs, the next step's inputs are uploaded (and
    # checked) through the other context, and its graph starts as soon as this one ends
    # (graphs never run at the same time), while this step's results are downloaded.
    # Every step's uploads and result downloads stay inside the timed region.  The serial
    # form (one context) is kept beside.
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
        h = dict(x=pin(b.x), y=pin(b.y), z=pin(b.z), layer=pin(b.layer), params=pin(b.params),
                 cov=pin(b.cov), seed_hits=pin(b.seed_hits))
        L = b.det.n_layers
        from paper_1906_11744_gb300 import kf_get_fit, kf_get_gradient, kf_get_tracks

        def host_outs():
            return (dict(hits=torch.empty((n_seeds, L), dtype=torch.int32).pin_memory(),
                         n_found=torch.empty(n_seeds, dtype=torch.int32).pin_memory(),
                         chi2=torch.empty(n_seeds, dtype=torch.float32).pin_memory(),
                         keep=torch.empty(n_seeds, dtype=torch.uint8).pin_memory()),
                    dict(params=torch.empty((6, n_seeds), dtype=torch.float32).pin_memory(),
                         chi2=torch.empty(n_seeds, dtype=torch.float32).pin_memory(),
                         status=torch.empty(n_seeds, dtype=torch.int32).pin_memory()),
                    torch.empty((L, 2), dtype=torch.float32).pin_memory())

        best = shape or ({} if tune is None else dict(
            lanes_per_seed=int(tune[np.argmin(tune[:, 4])][0]), block_threads=int(tune[np.argmin(tune[:, 4])][1]),
            persistent=int(tune[np.argmin(tune[:, 4])][2]), find_regcap=int(tune[np.argmin(tune[:, 4])][3])))
        t2 = tracker_for(b, **{"persistent": 1, "per_event": 0, **best})
        stream2 = torch.cuda.Stream(device=dev)
        t2.load_hits(b.hit_off, d_in["x"], d_in["y"], d_in["z"], d_in["layer"], stream2)
        t2.load_seeds(b.seed_off, d_in["params"], d_in["cov"], d_in["seed_hits"], stream2)
        t2.set_alignment(b.align, stream2)
        t2.capture_graph(with_adjoint=True, stream=stream2)
        lanes = [(t, stream, host_outs()), (t2, stream2, host_outs())]

        def upload(i):  # synchronizes this context's stream only
            c, st, _ = lanes[i]
            c.load_hits(b.hit_off, h["x"], h["y"], h["z"], h["layer"], st)
            c.load_seeds(b.seed_off, h["params"], h["cov"], h["seed_hits"], st)

        def launch(i):
            c, st, _ = lanes[i]
            c.launch_graph(st)

        def collect(i):  # downloads into pinned host buffers (each call synchronizes)
            c, st, (outs, fouts, g_host) = lanes[i]
            kf_get_tracks(c.ctx, **outs, stream=st)
            kf_get_fit(c.ctx, **fouts, stream=st)
            kf_get_gradient(c.ctx, g_align=g_host, stream=st)

        def run_serial(n):
            for _ in range(n):
                upload(0)
                launch(0)
                collect(0)

        def run_pipelined(n):
            upload(0)
            launch(0)
            for k in range(n):
                if k + 1 < n:
                    upload((k + 1) % 2)  # beside graph k
                    # graph k+1 right after graph k (one graph at a time), so that
                    # step k's downloads below run beside it
                    done = torch.cuda.Event()
                    done.record(lanes[k % 2][1])
                    lanes[(k + 1) % 2][1].wait_event(done)
                    launch((k + 1) % 2)
                collect(k % 2)

        run_serial(2)
        run_pipelined(2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run_serial(args.steps)
        torch.cuda.synchronize()
        serial_s = max_over_ranks(time.perf_counter() - t0, dev)
        t0 = time.perf_counter()
        run_pipelined(args.steps)
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0, dev)
        t2.close()
        outs, fouts, g_host = lanes[0][2]
        bi = sum(v.numel() * v.element_size() for v in h.values())
        bo = sum(v.numel() * v.element_size() for v in outs.values()) + \
            sum(v.numel() * v.element_size() for v in fouts.values()) + g_host.numel() * 4
        e2e = {"value": seeds_all * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bo, "ms_per_step": 1e3 * e2e_s / args.steps,
               "form": "two contexts: uploads of step k+1 and downloads of step k-1 overlap the graph of step k; graphs run one at a time",
               "serial": {"value": seeds_all * args.steps / serial_s, "ms_per_step": 1e3 * serial_s / args.steps,
                          "form": "one context: upload, graph, download in sequence"}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_oracle:
        cpu = oracle_sample(b, budget_s=args.oracle_budget)            # all host cores
        one = oracle_sample(b, budget_s=1.0, threads=1)                   # one event, one core
        cpu["single_core_value"] = one["value"]
        cpu["single_core_sample"] = one["sample"]
        if endcap is not None and endcap_batch is not None:  # the oracle beside the endcap step
            ce = oracle_sample(endcap_batch, budget_s=5.0)
            endcap["cpu_baseline"] = {k: ce[k] for k in ("value", "unit", "cores", "kind", "sample")}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": workload_desc(args.config) + (f" (events={args.events})" if args.events else ""),
                          "seeds_per_gpu": n_seeds, "hits_per_gpu": b.n_hits,
                          "l2": "flushed (2x L2 write) before every timed step",
                          "launch": "one CUDA graph per step: bin (5 kernels) + find + dedup + fit (track order, FP32 pass, careful pass) + adjoint (FP32 pass, careful-list passes in double and FP32, finish: 4)",
                          "find_shape": shape or None,
                          "autotuned": None if tune is None else {
                              "lanes_per_seed": int(tune[np.argmin(tune[:, 4])][0]),
                              "block_threads": int(tune[np.argmin(tune[:, 4])][1]),
                              "persistent": int(tune[np.argmin(tune[:, 4])][2]),
                              "register_cap": int(tune[np.argmin(tune[:, 4])][3]),
                              "candidates_tried": int(len(tune))}},
               "candidate_layer_steps_per_s": steps_per_s,
               "stage_ms": {k: v / args.steps for k, v in stage.items()},
               "counters_per_step": counters,
               "plain": plain,
               "e2e": e2e,
               "gpu_launches": n_kernels * args.steps,
               "roofline": roofline,
               "alignment_exchange": exchange,
               "mixed_pileup": mixed,
               "dup_handling": dup,
               "material_map": mat,
               "field_map": fld,
               "endcap": endcap,
               "cpu_baseline": None if cpu is None else {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample",
                                                                            "single_core_value", "single_core_sample")},
               "clocks": clocks.summary()}
        print(json.dumps(out))
    t.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
