#!/usr/bin/env python
"""Throughput benchmark of the lubrication correction (pairs per second).

One step = one pass of the whole path over one suspension, enqueued on one
stream: lub_pairs_build (cell list + Sec. III A pre-filters), then
lub_correct (the closest points of Sec. III A, then Sec. III B and the
Appendix: resistance, forces and their scatter to the particles), captured
once into a CUDA graph and replayed.

Headline workload (N=1): the large dense run, 1,048,576 spheroids (aspect
ratio log-uniform in [1/3, 3]) at volume fraction 0.5 in a 1024^3 cube
periodic in x and y between two plane walls (a growth packing), mixed
precision, learned warm start, every particle moved by a seeded random rigid
motion (lub_random_motion, outside the timed step) between steps.  Beside it,
on the same motions: the plain form (Newton from the line of centres), the
paper's temporal warm start and the network on every pair; the same step with
several steps and motions per graph; per-kernel rooflines from the library's
kernel trace; the end-to-end step through the public API with host buffers;
the FP64 oracle on a sample of the same pairs on the host cores.  Secondary
workloads: the 32,768-particle mixed suspension, fresh pairs (learned against
plain, with the network's break-even), the 256-suspension ensemble.
Under torchrun each rank runs its own independent copy (another seed): weak
scaling with no collective in the data path.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the host cores instead (the reference arm).
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "lubrication pair-corrections/s at 1e-5 rel. err; learned vs plain GPU form"
WORKLOAD = ("large dense run: N=1048576 spheroids, aspect ratio log-uniform [1/3,3], equivalent radius 4.96, "
            "phi=0.5 (growth packing of a 128x128x1024 slab tiled 8x8), cube 1024^3 periodic in x,y between plane "
            "walls at z=0 and z=1024, pairs with possible gap < 1 (Delta_L=1), mixed precision, learned warm start; "
            "seeded rigid motions dr~N(0,0.01^2), dtheta~N(0,0.005^2) between steps")
WORKLOAD_32K = ("mixed suspension: N=32768 (50% spheres r=4.5, 50% oblates 6,6,3), phi=0.3, periodic cube "
                "L=357.7, 90% of particles attached to an earlier one at a gap log-uniform in [1e-4,1], "
                "pairs with possible gap < 1 (Delta_L=1)")

# Algorithmic work per unit: what the method computes or moves, counted from
# the per-pair formulas (not from executed instructions).  A float-float
# operation counts as 10 FP32 FLOP (TwoSum/TwoProduct and renormalisation).
FP32_NEWTON_FLOP = 170.0        # one FP32 Newton iteration on the sphere (2 support functions, gradient, 2x2 Hessian)
FF_GAP_STEP_FP32_FLOP = 2400.0  # gap (70 FLOP) + one Newton step (170 FLOP) in float-float, x10
FP64_NEWTON_FLOP = 170.0        # one FP64 Newton iteration (FP64 mode)
FP64_GAP_FLOP = 70.0            # the FP64 gap
RES_FP32_FLOP = 1300.0          # K2 per pair: 2 surface frames, eigenproblem, cubic rotation, 16 K elements, K~,
                                # forces (900) + the normal velocity in float-float (40 FLOP x 10) + scatter
PAIRS_BYTES_PER_PARTICLE = 64.0  # pose + shape read once (48 B) + cell index and sorted index, two passes (16 B)
PAIRS_BYTES_PER_PAIR = 8.0       # (i, j) written
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from ncu
# captures, valid while the kernel's sources hash to the recorded value
# (one ncu capture of dram__bytes_read.sum + dram__bytes_write.sum per kernel
# over `bench.py --only large --steps 3`, the last of its three steps)
TRAFFIC = {
    "large": {"sources": "f33b023ddd56a8f2",
              "bytes": {"pairs_build": 274182656, "k_closest_mixed": 372022272, "k_resistance_apply": 496749056}},
}
TRAFFIC_SOURCES = ("closest.cu", "pair_force.cuh", "resistance.cu", "pairs.cu", "ff.cuh", "lub_internal.cuh",
                   "mlp_infer.cuh", "scan.cu", "scan_tile.cuh", "apply.cu")
# the form of the timed step: lub_pairs_build, then lub_correct (closest
# points, resistance and scatter in one call)
STEP_FORM = "fused"
# the timed step writes every output: the per-particle force and torque sums,
# the normals, gaps, statuses, iteration counts and the per-pair forces and
# lever arms; the same step without the last two (optional outputs) is
# reported beside it
PAIR_FORCES = True
MOTION_SEED = 777
SIG_R, SIG_T = 0.01, 0.005


def sources_hash():
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_1308_6482_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--large-n", type=int, default=1 << 20)
    ap.add_argument("--graph-steps", type=int, default=10, help="steps (with their motions) per graph, even")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-secondary", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--learned-pairs", type=int, default=1 << 20)
    ap.add_argument("--ens-n", type=int, default=256, help="suspensions in the ensemble workload")
    ap.add_argument("--ens-steps", type=int, default=100)
    ap.add_argument("--n", type=int, default=32768, help="particles of the mixed suspension (secondary)")
    ap.add_argument("--mlp-engine", default="mma_sync", choices=["mma_sync", "tcgen05"],
                    help="tensor-core engine of the network in --only learned")
    ap.add_argument("--only", default=None, choices=["large", "step", "ensemble", "learned", "probe"],
                    help="run only that workload eagerly, a few steps, and print a summary (for profilers; no "
                         "bench line)")
    return ap.parse_args()


def peaks(lub=None, dev=None):
    """Roofline denominators: HBM (a STREAM-style copy) and BF16 (cuBLAS) from
    MEASURED_PEAKS.json, measured on these GPUs, FP32 and FP64 from the
    library's FMA-chain probe run now on this GPU (lub_probe_peak)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    out = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "src": "fallback"}
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        out.update(d)
        out["src"] = "measured"
    if lub is not None:
        ctx = lub.Context()
        out["fp32_tflops"] = lub.lub_probe_peak(ctx.h, lub.LUB_PROBE_FP32)
        out["fp64_tflops"] = lub.lub_probe_peak(ctx.h, lub.LUB_PROBE_FP64)
        out["alu_src"] = "lub_probe_peak (FMA chains, 8 blocks of 256 per SM), measured in this run"
    return out


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
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "50", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
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
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(ms_per_step, units, ws, device):
    """Whole-job figures of independent replicas: the slowest rank's time per
    step (max over ranks) and the units all ranks processed (sum).  Identity
    for one rank; any torch.distributed backend (NCCL on the GPUs, gloo in the
    CPU tests)."""
    if ws <= 1:
        return float(ms_per_step), float(units)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms_per_step)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), float(c.item())


def rank_seed(rank):
    """Each rank steps its own suspension: the workload seed of rank r."""
    return 2 + 1000 * rank


def ensemble_shard(n_susp, ws, rank):
    """Suspensions of the ensemble run by `rank` of `ws`: s with s mod ws == rank."""
    return list(range(rank, n_susp, ws))


def make_workload(n, seed):
    import gen
    return gen.config_mixed_suspension(N=n, phi=0.3, seed=seed)


def event_pairs(torch, k):
    return [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]


def graph_of(torch, stream, fn):
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        fn()
    stream.synchronize()
    return g


def large_pipeline(lub, parts, dom, dev, rmax, warm, net, packed=False):
    P = lub.DeviceParticles(parts, dev, max_semi_axis=rmax, packed=packed)
    pl = lub.Pipeline(P, dom, lub.default_params(precision="mixed", warm_start=warm), capacity=1024, device=dev)
    if warm in (lub.LUB_WARM_MLP, lub.LUB_WARM_MLP_ALL):
        net.install(pl.ctx)
    npairs = pl.build_pairs()
    pl._alloc(int(npairs * 1.3) + 4096, dev)
    pl.build_pairs()
    # launch shapes timed on this workload's own step (lub_autotune)
    pl.tuned = pl.autotune(reps=3)
    return P, pl


def run_steps(lub, torch, np, pl, P, stream, flush, steps, warmup):
    """One CUDA graph of one step (STEP_FORM).  Per step: the seeded
    motion of every particle and an L2 flush, outside the events, then the
    graph between two events.  Returns ms [steps], pair counts [steps], the
    mean Newton iterations per pair and the capacity overflows."""
    with torch.cuda.stream(stream):
        pl.step(form=STEP_FORM, pair_forces=PAIR_FORCES, stream=stream)
        pl.step(form=STEP_FORM, pair_forces=PAIR_FORCES, stream=stream)
    stream.synchronize()
    g = graph_of(torch, stream, lambda: pl.step(form=STEP_FORM, pair_forces=PAIR_FORCES, stream=stream))
    dev = P.t["x"].device
    counts = torch.zeros(steps, dtype=torch.int32, device=dev)
    its = torch.zeros(steps, dtype=torch.float64, device=dev)
    idx = torch.arange(pl.cap, device=dev)
    ev = event_pairs(torch, steps)
    with torch.cuda.stream(stream):
        for k in range(warmup):
            lub.lub_random_motion(pl.ctx.h, P.c, MOTION_SEED, k, SIG_R, SIG_T, stream=stream)
            flush.zero_()
            g.replay()
        for k in range(steps):
            lub.lub_random_motion(pl.ctx.h, P.c, MOTION_SEED, warmup + k, SIG_R, SIG_T, stream=stream)
            flush.zero_()
            ev[k][0].record(stream)
            g.replay()
            ev[k][1].record(stream)
            counts[k].copy_(pl.d_count[0])
            m = torch.clamp(pl.d_count[0], max=pl.cap)
            its[k] = (pl.iters.double() * (idx < m)).sum() / m
    stream.synchronize()
    ms = np.array([a.elapsed_time(b) for a, b in ev])
    cnt = counts.cpu().numpy().astype(np.float64)
    del g
    return ms, cnt, float(its.mean().item()), int((cnt > pl.cap).sum())


def run_multi(lub, torch, np, pl, P, stream, G, replays, step0):
    """One CUDA graph of G steps, each preceded by its seeded motion (the
    motions' step index kept on the device, so every replay moves on).  The
    inputs are larger than the L2 cache; no flush inside the graph.  Returns
    ms per step (motions included)."""
    ctr = torch.tensor([step0, 0], dtype=torch.int64, device=P.t["x"].device)

    def body():
        for j in range(G):
            lub.lub_random_motion(pl.ctx.h, P.c, MOTION_SEED, 0, SIG_R, SIG_T, step_dev=ctr[j % 2:],
                                  next_dev=ctr[(j + 1) % 2:], stream=stream)
            pl.step(form=STEP_FORM, pair_forces=PAIR_FORCES, stream=stream)

    with torch.cuda.stream(stream):
        pl.step(form=STEP_FORM, pair_forces=PAIR_FORCES, stream=stream)
    stream.synchronize()
    g = graph_of(torch, stream, body)
    ev = event_pairs(torch, replays)
    with torch.cuda.stream(stream):
        g.replay()
        for a, b in ev:
            a.record(stream)
            g.replay()
            b.record(stream)
    stream.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev])) / G
    del g
    return ms


def kernels_in_step(form=None, precision="mixed"):
    # lub_pairs_build: zeroing of its counters, cells count, scan, cells fill,
    # sweep, FP64 test of the candidates within the sweep's margin, scan,
    # compaction = 8.  lub_correct (the fused form), mixed:
    # particle table (which also clears the sums and the work list), FP32
    # stage, work-list FP64 solves, resistance with scatter = 4; FP64: zeroing
    # and the one pass = 2.  The merged form (lub_closest_points, then
    # lub_resistance_apply), mixed: 3 + 3 (zeroing and a second particle
    # table); FP64: 1 + 2.
    form = form or STEP_FORM
    if form == "fused":
        return 8 + (4 if precision == "mixed" else 2)
    if precision == "mixed":
        return 8 + 3 + 3
    return 8 + 1 + 2


def rooflines(kernel_ms, call_ms, npairs, n, mean_it, pk, traffic):
    """Per kernel: algorithmic work per launch over the kernel's event-timed
    duration, against the measured peak of its pipe."""
    out = {}
    b = n * PAIRS_BYTES_PER_PARTICLE + npairs * PAIRS_BYTES_PER_PAIR
    ach = b / (call_ms["pairs_build"] * 1e-3) / 1e9
    out["pairs_build"] = {
        "kernel": "lub_pairs_build (8 kernels; k_pairs_sweep %.0f%% of the call)"
                  % (100 * kernel_ms["sweep"] / call_ms["pairs_build"]),
        "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": ach / pk["hbm_gbs"],
        "traffic": traffic.get("pairs_build"), "algorithmic_bytes": b, "ms": call_ms["pairs_build"],
        "peak_src": "hbm_gbs of MEASURED_PEAKS.json (%s)" % pk["src"]}
    f = npairs * (mean_it * FP32_NEWTON_FLOP + FF_GAP_STEP_FP32_FLOP)
    ach = f / (kernel_ms["closest"] * 1e-3) / 1e12
    out["k_closest_mixed"] = {
        "kernel": "k_closest_mixed (FP32 Newton + float-float gap and step)", "bound": "alu", "achieved": ach,
        "peak": pk["fp32_tflops"], "unit": "TFLOP/s (FP32)", "frac": ach / pk["fp32_tflops"],
        "traffic": traffic.get("k_closest_mixed"), "algorithmic_flop": f, "ms": kernel_ms["closest"],
        "peak_src": pk["alu_src"]}
    f = npairs * RES_FP32_FLOP
    ach = f / (kernel_ms["resistance"] * 1e-3) / 1e12
    out["k_resistance_apply"] = {
        "kernel": "k_resistance_apply (geometry, K~, forces, scatter)", "bound": "alu", "achieved": ach,
        "peak": pk["fp32_tflops"], "unit": "TFLOP/s (FP32)", "frac": ach / pk["fp32_tflops"],
        "traffic": traffic.get("k_resistance_apply"), "algorithmic_flop": f, "ms": kernel_ms["resistance"],
        "peak_src": pk["alu_src"]}
    return out


def traffic_for(workload):
    """Recorded per-launch DRAM bytes of a workload's kernels, or {} when the
    sources changed since the capture (the figures would be stale)."""
    rec = TRAFFIC.get(workload)
    if not rec or rec.get("sources") != sources_hash():
        return {}
    return rec["bytes"]


def large_headline(args, lub, torch, np, dev, stream, flush, ws, rank, pk):
    import gen
    from paper_1308_6482_gb300.mlp import WarmStartMLP

    t0 = time.perf_counter()
    parts, dom = gen.large_config(N=args.large_n, seed=6 + 1000 * rank)
    t_gen = time.perf_counter() - t0
    n = len(parts["x"])
    rmax = float(max(parts["r_par"].max(), parts["r_perp"].max())) + 0.05
    net = WarmStartMLP.load(device=dev)
    forms = (("learned", lub.LUB_WARM_MLP), ("plain", lub.LUB_WARM_NONE), ("temporal", lub.LUB_WARM_PREVIOUS),
             ("learned_every_pair", lub.LUB_WARM_MLP_ALL))
    res = {}
    sampler = None
    pairs0 = None
    tuned_shapes = None
    for name, warm in forms:
        P, pl = large_pipeline(lub, parts, dom, dev, rmax, warm, net)
        if name == "learned":
            tuned_shapes = {k: list(v) for k, v in pl.tuned.items()}
        if pairs0 is None:
            m0 = min(pl.count(), pl.cap)
            pairs0 = (pl.pair_i[:m0].cpu().numpy(), pl.pair_j[:m0].cpu().numpy())
        steps = args.steps if name != "learned_every_pair" else max(10, min(args.steps, 100))
        if name == "learned":
            sampler = ClockSampler(int(str(dev).split(":")[-1]) if ":" in str(dev) else 0)
            sampler.start()
            time.sleep(0.2)
            if ws > 1:
                import torch.distributed as dist
                dist.barrier()
            torch.cuda.synchronize()
        t_w = time.perf_counter()
        ms, cnt, it, over = run_steps(lub, torch, np, pl, P, stream, flush, steps, args.warmup)
        wall = time.perf_counter() - t_w
        if name == "learned":
            if ws > 1:
                dist.barrier()
            clocks = sampler.stop()
        fb = float(((pl.status[:min(pl.count(), pl.cap)] & lub.LUB_ST_FP64) != 0).float().mean().item())
        step_ms, pairs = aggregate(float(ms.mean()), float(cnt.mean()), ws, dev)
        res[name] = {"ms_per_step": step_ms, "pairs_per_s": pairs / (step_ms * 1e-3), "pairs_per_step": pairs,
                     "newton_iters_per_pair": it, "fp64_fallback_fraction": fb, "steps": steps,
                     "capacity_overflows": over, "wall_s": wall}
        if name == "learned":
            # per-kernel times (library trace) and per-call times of eager steps
            K = 20
            lub.lub_trace_enable(pl.ctx.h, 1)
            evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
            with torch.cuda.stream(stream):
                for k in range(K):
                    lub.lub_random_motion(pl.ctx.h, P.c, MOTION_SEED, 10 ** 6 + k, SIG_R, SIG_T, stream=stream)
                    flush.zero_()
                    evs[k][0].record(stream)
                    pl.build_pairs(sync_count=False, grow=False, stream=stream)
                    evs[k][1].record(stream)
                    pl.closest(stream=stream)
                    evs[k][2].record(stream)
                    pl.resistance_apply(stream=stream)
                    evs[k][3].record(stream)
            stream.synchronize()
            call_ms = {c: float(np.mean([evs[k][q].elapsed_time(evs[k][q + 1]) for k in range(K)]))
                       for q, c in enumerate(("pairs_build", "closest", "resistance_apply"))}
            kernel_ms = {}
            for q, name_k in ((lub.LUB_TRACE_SWEEP, "sweep"), (lub.LUB_TRACE_CLOSEST, "closest"),
                              (lub.LUB_TRACE_RESISTANCE, "resistance")):
                tot, nl = lub.lub_trace_read(pl.ctx.h, q)
                kernel_ms[name_k] = tot / max(nl, 1)
            lub.lub_trace_enable(pl.ctx.h, 0)
            npairs_traced = float(min(pl.count(), pl.cap))
            # the step with several steps (and their motions) per graph
            multi_ms = run_multi(lub, torch, np, pl, P, stream, args.graph_steps, max(5, steps // args.graph_steps),
                                 2 * 10 ** 6)
            # the other forms of the same step (the same calls, the same motions)
            other_ms = {}
            # the forms of the step measured side by side (20 graph replays each, the
            # motions inside the loop): the timed one, the same without the
            # per-pair forces and lever arms, and the two forms of separate calls
            for f2 in ("fused", "fused_without_pair_forces", "merged", "calls"):
                pf = PAIR_FORCES if f2 == "fused" else f2 != "fused_without_pair_forces"
                g2 = graph_of(torch, stream, lambda f2=f2, pf=pf: pl.step(form=f2.split("_with")[0], pair_forces=pf,
                                                                          stream=stream))
                e2 = event_pairs(torch, 20)
                with torch.cuda.stream(stream):
                    for k, (a, b) in enumerate(e2):
                        lub.lub_random_motion(pl.ctx.h, P.c, MOTION_SEED, 4 * 10 ** 6 + k, SIG_R, SIG_T,
                                              stream=stream)
                        flush.zero_()
                        a.record(stream)
                        g2.replay()
                        b.record(stream)
                stream.synchronize()
                other_ms[f2] = float(np.mean([a.elapsed_time(b) for a, b in e2[3:]]))
                del g2
            # the motion kernel alone
            evm = event_pairs(torch, 20)
            with torch.cuda.stream(stream):
                for k, (a, b) in enumerate(evm):
                    a.record(stream)
                    lub.lub_random_motion(pl.ctx.h, P.c, MOTION_SEED, 3 * 10 ** 6 + k, SIG_R, SIG_T, stream=stream)
                    b.record(stream)
            stream.synchronize()
            motion_ms = float(np.mean([a.elapsed_time(b) for a, b in evm]))
        del pl, P
        torch.cuda.empty_cache()
    lead = res["learned"]
    roof = rooflines(kernel_ms, call_ms, npairs_traced, n, lead["newton_iters_per_pair"], pk, traffic_for("large"))
    dom_k = max(("sweep", "closest", "resistance"), key=lambda k: kernel_ms[k])
    dominant = {"sweep": "pairs_build", "closest": "k_closest_mixed", "resistance": "k_resistance_apply"}[dom_k]
    out = {"value": lead["pairs_per_s"], "ms_per_step": lead["ms_per_step"], "pairs_per_step": lead["pairs_per_step"],
           "particles": n, "clocks": clocks, "forms": res, "call_ms": call_ms, "kernel_ms": kernel_ms,
           "other_forms_ms_per_step": other_ms, "autotuned_shapes": tuned_shapes,
           "steps_per_graph": {"1": lead["ms_per_step"], str(args.graph_steps): multi_ms,
                               "motion_ms": motion_ms,
                               "note": "%d steps per graph: ms per step with each step's seeded motion inside the "
                                       "graph (1 step per graph: the motion runs outside the events)"
                                       % args.graph_steps},
           "roofline": dict(roof[dominant], name=dominant), "rooflines": roof, "generation_s": t_gen,
           "speedup_learned_vs_plain": lead["pairs_per_s"] / res["plain"]["pairs_per_s"],
           "speedup_learned_vs_temporal": lead["pairs_per_s"] / res["temporal"]["pairs_per_s"]}
    return out, parts, dom, pairs0, rmax, net


def e2e_large(args, lub, torch, np, parts, dom, dev, stream, rmax, net):
    """The same metric through the public API with host buffers: every step
    copies the packed pinned host particles to the device (one copy), runs the
    step and copies force and torque back to pinned host memory (one copy),
    one CUDA graph per step, the host waiting for every step's result."""
    Pk, ple = large_pipeline(lub, parts, dom, dev, rmax, lub.LUB_WARM_MLP, net, packed=True)
    hblob = Pk.host_blob(parts, torch.empty(Pk.blob.numel(), dtype=torch.uint8).pin_memory())
    hout = torch.empty(ple.ft_particles.numel(), dtype=ple.ft_particles.dtype).pin_memory()
    bi = hblob.numel()
    bo = hout.numel() * hout.element_size()
    Ke = max(10, min(args.steps, 50))

    # the velocities (last in the packed layout) are read only by the
    # correction, so their part of the copy runs on a side stream beside the
    # pair build and joins before lub_correct; the poses and shapes go first
    off_v = Pk.layout["vx"][0]
    side = torch.cuda.Stream(device=dev)
    fork, join = torch.cuda.Event(), torch.cuda.Event()

    def e2e_step():
        Pk.blob[:off_v].copy_(hblob[:off_v], non_blocking=True)
        # the velocities after the poses (the two would share the link)
        fork.record(stream)
        side.wait_event(fork)
        with torch.cuda.stream(side):
            Pk.blob[off_v:].copy_(hblob[off_v:], non_blocking=True)
            join.record(side)
        ple.build_pairs(sync_count=False, grow=False, stream=stream)
        stream.wait_event(join)
        ple.step(build=False, form=STEP_FORM, pair_forces=PAIR_FORCES, stream=stream)
        hout.copy_(ple.ft_particles, non_blocking=True)

    with torch.cuda.stream(stream):
        for _ in range(3):
            e2e_step()
    stream.synchronize()
    ge = graph_of(torch, stream, e2e_step)
    for _ in range(3):
        ge.replay()
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_e = time.perf_counter()
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(Ke):
            ge.replay()
            stream.synchronize()
        e1.record(stream)
    stream.synchronize()
    host_ms = (time.perf_counter() - t_e) * 1e3 / Ke
    e2e_ms = e0.elapsed_time(e1) / Ke
    npairs = float(min(ple.count(), ple.cap))
    del ge, ple, Pk
    return {"value": npairs / (e2e_ms * 1e-3), "unit": "pairs/s", "h2d_bytes_per_step": int(bi),
            "d2h_bytes_per_step": int(bo), "ms_per_step": e2e_ms, "host_wall_ms_per_step": host_ms,
            "how": "packed pinned host particles -> device (two copies: poses and shapes, then the velocities on a "
                   "side stream beside the pair build, which does not read them), the step (learned warm start), "
                   "force+torque -> pinned host (one copy), one CUDA graph per step, host synchronised on every "
                   "step's result"}


def cpu_model():
    """The host CPU's model name and architecture, as the OS reports them."""
    import platform
    name = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                name = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not name:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        name = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return "%s (%s)" % (name or "unknown", platform.machine())


def cpu_baseline(parts, dom, pairs0, budget_s=20.0):
    """The FP64 oracle, as it stands, on the host cores: closest points,
    forces and sums of the same workload's pairs (the list the GPU built from
    the initial poses), whole passes until the budget; the O(N^2) candidate
    scan of the paper's pre-filters timed separately on one 16,384-particle
    tile of the packing."""
    import numpy as np

    import oracle
    cores = os.cpu_count()
    pi, pj = pairs0
    P = oracle.Particles(parts)
    t0 = time.perf_counter()
    passes = 0
    while True:
        cp = oracle.closest(P, dom, pi, pj)
        pf = oracle.pair_force(P, dom, None, pi, pj, cp)
        oracle.apply(P.n, pi, pj, pf["FT"], pf["lever"])
        passes += 1
        el = time.perf_counter() - t0
        if el > budget_s / 2 or passes >= 5:
            break
    value = passes * len(pi) / el
    n0 = min(16384, P.n)
    tile = {k: np.asarray(v)[:n0] for k, v in parts.items()}
    tdom = dict(dom)
    L = dom["L"]
    tdom["L"] = (L[0] / 8, L[1] / 8, L[2]) if P.n == 1 << 20 else L
    t1 = time.perf_counter()
    ci, _ = oracle.candidates(tile, tdom, 1.0)
    t_scan = time.perf_counter() - t1
    return {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle", "cpu": cpu_model(),
            "sample": "all %d pairs of the first step, %d pass(es) of closest points + forces + sums (%d OpenMP "
                      "threads), %.1f s" % (len(pi), passes, cores, el),
            "candidate_scan": {"pairs_per_s": len(ci) / t_scan, "particles": n0, "pairs": int(len(ci)), "s": t_scan,
                               "note": "O(N^2) pre-filter of Sec. III A, 1 thread, on one tile of the packing"}}


def suspension_32k(args, lub, torch, np, dev, stream, flush, ws, rank, pk):
    """The 32,768-particle mixed suspension (the paper-scale workload): the
    merged step as one graph, the other forms of the step, the "normal only"
    model, the link-based comparison model and the sub-stepped integrator."""
    parts, dom = make_workload(args.n, rank_seed(rank))
    prm = lub.default_params(precision="mixed")
    pl = lub.Pipeline(parts, dom, prm, device=dev)
    npairs = pl.build_pairs()
    pl._alloc(int(npairs * 1.1) + 1024, dev)
    npairs = pl.build_pairs()
    with torch.cuda.stream(stream):
        shapes = pl.autotune(reps=5, stream=stream)
    stream.synchronize()

    def time_graph(fn, K):
        with torch.cuda.stream(stream):
            fn()
        stream.synchronize()
        g = graph_of(torch, stream, fn)
        ev = event_pairs(torch, K)
        with torch.cuda.stream(stream):
            for _ in range(3):
                flush.zero_()
                g.replay()
            for a, b in ev:
                flush.zero_()
                a.record(stream)
                g.replay()
                b.record(stream)
        stream.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in ev]))

    K = max(20, min(args.steps, 200))
    forms = {f: time_graph(lambda f=f: pl.step(form=f, pair_forces=(PAIR_FORCES if f == STEP_FORM else True),
                                               stream=stream), K)
             for f in ("merged", "calls", "fused")}
    res = pl.results()
    # per-call and per-kernel times of eager steps
    lub.lub_trace_enable(pl.ctx.h, 1)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(50)]
    with torch.cuda.stream(stream):
        for e in evs:
            flush.zero_()
            e[0].record(stream)
            pl.build_pairs(sync_count=False, grow=False, stream=stream)
            e[1].record(stream)
            pl.closest(stream=stream)
            e[2].record(stream)
            pl.resistance_apply(stream=stream)
            e[3].record(stream)
    stream.synchronize()
    call_ms = {c: float(np.mean([e[q].elapsed_time(e[q + 1]) for e in evs]))
               for q, c in enumerate(("pairs_build", "closest", "resistance_apply"))}
    kernel_ms = {}
    for q, nm in ((lub.LUB_TRACE_SWEEP, "sweep"), (lub.LUB_TRACE_CLOSEST, "closest"),
                  (lub.LUB_TRACE_RESISTANCE, "resistance")):
        tot, nl = lub.lub_trace_read(pl.ctx.h, q)
        kernel_ms[nm] = tot / max(nl, 1)
    lub.lub_trace_enable(pl.ctx.h, 0)
    roof = rooflines(kernel_ms, call_ms, npairs, args.n, float(np.mean(res["iters"])), pk, traffic_for("32k"))
    # "normal only" model (K~33 alone, Sec. IV C)
    pln = lub.Pipeline(lub.DeviceParticles(parts, dev), dom, lub.default_params(precision="mixed", model="normal"),
                       capacity=pl.cap, device=dev)
    pln.build_pairs()
    normal_ms = time_graph(lambda: pln.step(form=STEP_FORM, pair_forces=PAIR_FORCES, stream=stream), 50)
    del pln
    # the link-based model of Ding and Aidun (Sec. II) on the same pair list
    with torch.cuda.stream(stream):
        F_l, T_l, nl_l = pl.links(0.6, stream=stream)
    stream.synchronize()
    e5 = event_pairs(torch, 20)
    with torch.cuda.stream(stream):
        for a, b in e5:
            flush.zero_()
            a.record(stream)
            pl.links(0.6, stream=stream)
            b.record(stream)
    stream.synchronize()
    link_ms = float(np.mean([a.elapsed_time(b) for a, b in e5]))
    nl_host = nl_l[:npairs].cpu().numpy()
    # particle sub-stepping (Sec. II) with the contact branch: one LB step =
    # the pair build and 10 sub-steps, one graph per LB step
    pls = lub.Pipeline(lub.DeviceParticles(parts, dev), dom,
                       lub.default_params(precision="mixed", h_c=0.01, eps_c=100.0), capacity=pl.cap, device=dev)
    pls.build_pairs()
    gf = torch.Generator(device=dev)
    gf.manual_seed(99)
    fext = 0.01 * torch.randn(3 * pls.n, generator=gf, device=dev, dtype=torch.float32)
    lb_ms = time_graph(lambda: pls.substeps(10, 1.0, 0.1, f_ext=fext, stream=stream), 20)
    pairs_s = min(pls.count(), pls.cap)
    del pls
    ms, pairs_all = aggregate(forms[STEP_FORM], npairs, ws, dev)
    return {"workload": WORKLOAD_32K, "ms_per_step": ms, "pairs_per_s": pairs_all / (ms * 1e-3),
            "pairs_per_step": int(npairs), "forms_ms_per_step": forms, "call_ms": call_ms, "kernel_ms": kernel_ms,
            "rooflines": roof, "newton_iters_mean": float(np.mean(res["iters"])),
            "autotuned_shapes": {k: list(v) for k, v in shapes.items()} if shapes else None,
            "normal_only_model_ms_per_step": normal_ms,
            "comparison_link_model": {"ms_per_call": link_ms, "pairs_per_s": npairs / (link_ms * 1e-3),
                                      "links_per_pair": float(nl_host.mean()),
                                      "note": "Eq. methods:dlub on a unit lattice, D3Q19 links, q_bar = 0.6, FP64 "
                                              "per link, the step's pair list, one warp per pair"},
            "substepping": {"ms_per_lb_step": lb_ms, "substeps": 10, "pairs": pairs_s,
                            "pair_corrections_per_s": 10 * pairs_s / (lb_ms * 1e-3),
                            "note": "h_c=0.01, eps_c=100, dt=0.1, density 1, external force N(0,0.01^2)"},
            "l2": "flushed between timed steps (256 MB write outside the step events)"}


def learned_vs_plain(args, lub, torch, np, dev, stream, flush, steps=20, warmup=3):
    """The learned warm start against the plain (line-of-centres) start on
    fresh spheroid pairs: aspect ratios log-uniform in [1/3, 3], gaps
    log-uniform in [1e-4, 1] x the pair's smallest semi-axis, a seed the
    training set never used.  Times lub_closest_points alone, L2 flushed
    between calls; checks that the forms reach the same gaps (equal
    accuracy); and the network's break-even: its own time against the time
    of the Newton iterations it saves."""
    import gen
    from paper_1308_6482_gb300.mlp import WarmStartMLP

    parts, dom, pi, pj = gen.pair_stream(args.learned_pairs, seed=9100, kind="aspect", gap_range=(1e-4, 1.0),
                                         gap_scale="min_axis")
    m = len(pi)
    net = WarmStartMLP.load(device=dev)
    P = lub.DeviceParticles(parts, dev)
    out = {"workload": "%d fresh spheroid pairs, aspect ratios log-uniform [1/3,3], gap log-uniform "
                       "[1e-4,1] x min semi-axis" % m, "steps": steps}

    def timed(fn):
        ev = event_pairs(torch, steps)
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                flush.zero_()
                fn()
            for a, b in ev:
                flush.zero_()
                a.record(stream)
                fn()
                b.record(stream)
        stream.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in ev]))

    for prec in ("fp64", "mixed"):
        res = {}
        forms = [("plain", "none", "mma_sync"), ("learned_every_pair", "mlp_all", "mma_sync"),
                 ("learned_every_pair_tcgen05", "mlp_all", "tcgen05")]
        if prec == "mixed":
            forms.append(("learned", "mlp", "mma_sync"))
        net_ms = {}
        for form, warm, engine in forms:
            prm = lub.default_params(precision=prec, warm_start=warm)
            pl = lub.Pipeline(P, dom, prm, capacity=m, device=dev)
            if warm != "none":
                net.install(pl.ctx)
                lub.lub_mlp_engine(pl.ctx.h, engine)
            pl.set_pairs(pi, pj)
            ms = timed(lambda: pl.closest(stream=stream))
            if warm == "mlp_all" and engine not in net_ms:
                pq = torch.zeros(4 * pl.cap, dtype=torch.float32, device=dev)
                net_ms[engine] = timed(lambda: lub.lub_mlp_predict(pl.ctx.h, pl.P.c, pl.D, pl.pair_i, pl.pair_j,
                                                                   pl.d_count, pl.cap, pq, stream=stream))
            it = pl.iters[:m].cpu().numpy().astype(np.float64)
            stt = pl.status[:m].cpu().numpy()
            res[form] = {"pairs_per_s": m / (ms * 1e-3), "ms": ms, "newton_iters_mean": float(it.mean()),
                         "warp_max_iters_mean": float(it[:m - m % 32].reshape(-1, 32).max(1).mean()),
                         "fp64_fallback_fraction": float(np.mean((stt & lub.LUB_ST_FP64) != 0)),
                         "h": pl.gap[:m].cpu().numpy(), "status": stt}
            del pl
        h0, s0 = res["plain"].pop("h"), res["plain"].pop("status")
        for form in list(res):
            if form == "plain":
                continue
            h1, s1 = res[form].pop("h"), res[form].pop("status")
            res[form]["max_abs_gap_difference"] = float(np.abs(h1 - h0).max())
            res[form]["status_equal_fraction"] = float(np.mean((s0 & 7) == (s1 & 7)))
            res[form]["speedup"] = res[form]["pairs_per_s"] / res["plain"]["pairs_per_s"]
        # break-even: the network against the iterations it saves.  With the
        # tcgen05 engine the network is a launch of its own and the solve is
        # the plain form's kernel started from the network's normals, so
        # (that call) - (the network alone) is the solve from the learned start
        saved = res["plain"]["newton_iters_mean"] - res["learned_every_pair"]["newton_iters_mean"]
        solve_warm = res["learned_every_pair_tcgen05"]["ms"] - net_ms["tcgen05"]
        gain = res["plain"]["ms"] - solve_warm
        per_iter = gain / saved if saved > 0 else None
        res["break_even"] = {
            "network_ms": net_ms, "network_us_per_million_pairs": {k: v * 1e3 / (m / 1e6) for k, v in net_ms.items()},
            "iterations_saved_per_pair": saved, "solve_from_learned_start_ms": solve_warm,
            "solve_from_line_of_centres_ms": res["plain"]["ms"], "solve_time_saved_ms": gain,
            "ms_per_newton_iteration_of_all_pairs": per_iter,
            "iterations_the_network_costs": (net_ms["mma_sync"] / per_iter) if per_iter and per_iter > 0 else None,
            "note": "the network pays when the solve time it saves exceeds its own time (lub_mlp_predict); "
                    "solve_from_learned_start_ms = the tcgen05 form's call minus its network launch"}
        out[prec] = res
    return out


def ensemble_bench(args, lub, torch, np, dev, stream, flush, ws=1, rank=0):
    """Batched ensemble: args.ens_n independent periodic suspensions of mixed
    spheroids (growth packings, aspect ratio log-uniform [1/3, 3], phi uniform
    [0.1, 0.5], pair counts log-uniform [1e3, 2e5]) stepped together, one
    launch per stage for all suspensions, launch shapes from the autotuner,
    every particle moved by a seeded rigid motion (lub_random_motion) between
    steps: one graph per step (motion outside the events) and several steps
    with their motions per graph; the warm starts in both precisions; the same
    suspensions stepped one by one.  Under torchrun the suspensions shard over
    the ranks (suspension s on rank s mod N, no exchange)."""
    import gen
    from paper_1308_6482_gb300.mlp import WarmStartMLP

    t0 = time.perf_counter()
    sus, meta = gen.ensemble(n_susp=args.ens_n, seed=4)
    sus = [sus[b] for b in ensemble_shard(len(sus), ws, rank)]
    t_gen = time.perf_counter() - t0
    parts, doms, off = lub.make_ensemble(sus)
    rmax = float(max(parts["r_par"].max(), parts["r_perp"].max())) + 0.05
    net = WarmStartMLP.load(device=dev)

    def make(warm, precision, shapes=None, tune=False):
        P = lub.DeviceParticles(parts, dev, max_semi_axis=rmax, batch_offsets=off)
        pl = lub.Pipeline(P, doms, lub.default_params(precision=precision, warm_start=warm), capacity=1024,
                          device=dev)
        if warm in (lub.LUB_WARM_MLP, lub.LUB_WARM_MLP_ALL):
            net.install(pl.ctx)
        if shapes:
            for q, (blk, per) in enumerate(shapes):
                lub.lub_set_launch_shape(pl.ctx.h, q, blk, per)
        npairs = pl.build_pairs()
        pl._alloc(int(npairs * 1.3) + 4096, dev)
        pl.build_pairs()
        if tune:
            with torch.cuda.stream(stream):
                pl.autotune(reps=2, stream=stream)
            stream.synchronize()
        return P, pl

    t1 = time.perf_counter()
    P, pl = make(lub.LUB_WARM_NONE, "mixed", tune=True)
    shapes = [lub.lub_get_launch_shape(pl.ctx.h, q) for q in range(lub.LUB_TUNE_COUNT)]
    ms, cnt, it_plain, over = run_steps(lub, torch, np, pl, P, stream, flush, args.ens_steps, 3)
    multi = run_multi(lub, torch, np, pl, P, stream, args.graph_steps, max(3, args.ens_steps // args.graph_steps),
                      5 * 10 ** 6)
    del pl, P
    t_run = time.perf_counter() - t1
    warm_forms = {}
    for prec in ("mixed", "fp64"):
        for name, warm in (("plain", lub.LUB_WARM_NONE), ("temporal", lub.LUB_WARM_PREVIOUS),
                           ("learned", lub.LUB_WARM_MLP), ("learned_every_pair", lub.LUB_WARM_MLP_ALL)):
            if prec == "mixed" and name == "plain":
                continue
            if prec == "fp64" and name == "learned_every_pair":
                continue  # the same as learned in FP64
            steps_w = max(10, args.ens_steps // (4 if prec == "mixed" else 10))
            Pw, plw = make(warm, prec, shapes=shapes)
            msw, cntw, itw, _ = run_steps(lub, torch, np, plw, Pw, stream, flush, steps_w, 3)
            del plw, Pw
            wms, wpairs = aggregate(float(msw.mean()), float(cntw.mean()), ws, dev)
            warm_forms["%s_%s" % (name, prec)] = {"ms_per_step": wms, "pairs_per_s": wpairs / (wms * 1e-3),
                                                  "newton_iters_per_pair": itw, "steps": len(msw)}
    # the same suspensions one by one: their own calls, eager (a few steps)
    prm = lub.default_params(precision="mixed")
    sep = [lub.Pipeline(lub.DeviceParticles(p, dev), d, prm, device=dev) for p, d in sus]
    for q in sep:
        q.build_pairs()
    Ks = 3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        for q in sep:
            q.step(form=STEP_FORM, pair_forces=PAIR_FORCES, stream=stream)
        flush.zero_()
        e0.record(stream)
        for _ in range(Ks):
            for q in sep:
                q.step(form=STEP_FORM, pair_forces=PAIR_FORCES, stream=stream)
        e1.record(stream)
    stream.synchronize()
    sep_ms = e0.elapsed_time(e1) / Ks
    sep_pairs = float(sum(q.count() for q in sep))
    del sep
    step_ms, all_pairs = aggregate(float(ms.mean()), float(cnt.mean()), ws, dev)
    multi_ms, _ = aggregate(multi, 0.0, ws, dev)
    sep_ms, sep_pairs = aggregate(sep_ms, sep_pairs, ws, dev)
    n_all = aggregate(0.0, float(len(parts["x"])), ws, dev)[1]
    return {
        "workload": "%d periodic suspensions (growth packings), phi uniform [0.1,0.5], aspect ratio log-uniform "
                    "[1/3,3], pair counts log-uniform [1e3,2e5]; %d particles, %d steps of seeded rigid motions "
                    "(dr ~ N(0,0.01^2), dtheta ~ N(0,0.005^2))" % (args.ens_n, int(n_all), args.ens_steps),
        "precision": "mixed", "pairs_per_step_mean": all_pairs, "ms_per_step": step_ms,
        "pairs_per_s": all_pairs / (step_ms * 1e-3), "newton_iters_per_pair": it_plain,
        "capacity_overflows": over, "ranks": ws,
        "steps_per_graph": {"1": step_ms, str(args.graph_steps): multi_ms,
                            "note": "ms per step; %d steps per graph include each step's seeded motion "
                                    "(lub_random_motion) inside the graph" % args.graph_steps},
        "launch": "one launch per stage for all suspensions (pair build, closest points, resistance with scatter)",
        "autotuned_shapes": {lub.TUNE_NAMES[q]: list(v) for q, v in enumerate(shapes)},
        "autotune_and_run_s": t_run, "generation_s": t_gen, "warm_starts": warm_forms,
        "separate_calls": {"ms_per_step": sep_ms, "pairs_per_s": sep_pairs / (sep_ms * 1e-3),
                           "launches_per_step": "per suspension, eager"},
        "speedup_vs_separate": float((all_pairs / step_ms) / (sep_pairs / sep_ms)),
    }


def only_leg(args, lub, torch, np, dev, stream):
    """A few eager steps of one workload with no graph, tuning or timing: a
    short, fixed launch sequence for a profiler."""
    import gen
    from paper_1308_6482_gb300.mlp import WarmStartMLP
    if args.only == "probe":
        # the ALU roofline denominators: lub_probe_peak repeated, with the SM
        # clocks sampled while it runs
        ctx = lub.Context()
        props = torch.cuda.get_device_properties(dev)
        clocks = ClockSampler(dev.index or 0)
        clocks.start()
        runs = {"fp32": [], "fp64": []}
        for _ in range(max(3, args.steps)):
            runs["fp32"].append(lub.lub_probe_peak(ctx.h, lub.LUB_PROBE_FP32))
            runs["fp64"].append(lub.lub_probe_peak(ctx.h, lub.LUB_PROBE_FP64))
        clk = clocks.stop()
        return {"device": props.name, "sms": props.multi_processor_count,
                "tflops": {k: {"median": float(np.median(v)), "min": float(np.min(v)), "max": float(np.max(v)),
                               "runs": len(v)} for k, v in runs.items()},
                "clocks": clk,
                "method": "8 independent FMA chains per thread, 8 blocks of 256 threads per SM, 2^17 (FP32) / "
                          "2^12 (FP64) iterations, best of 3 timed launches after one warm-up (CUDA events)"}
    if args.only == "large":
        parts, dom = gen.large_config(N=args.large_n, seed=6)
        rmax = float(max(parts["r_par"].max(), parts["r_perp"].max())) + 0.05
        P, pl = large_pipeline(lub, parts, dom, dev, rmax, lub.LUB_WARM_MLP, WarmStartMLP.load(device=dev))
    elif args.only == "step":
        parts, dom = make_workload(args.n, rank_seed(0))
        pl = lub.Pipeline(parts, dom, lub.default_params(precision="mixed"), device=dev)
        npairs = pl.build_pairs()
        pl._alloc(int(npairs * 1.1) + 1024, dev)
        P = pl.P
    elif args.only == "ensemble":
        sus, _ = gen.ensemble(n_susp=args.ens_n, seed=4)
        parts, doms, off = lub.make_ensemble(sus)
        P = lub.DeviceParticles(parts, dev, batch_offsets=off)
        pl = lub.Pipeline(P, doms, lub.default_params(precision="mixed"), capacity=1024, device=dev)
        npairs = pl.build_pairs()
        pl._alloc(int(npairs * 1.3) + 4096, dev)
    else:  # learned: fresh pairs, the network on every pair (mixed)
        parts, dom, pi, pj = gen.pair_stream(args.learned_pairs, seed=9100, kind="aspect", gap_range=(1e-4, 1.0),
                                             gap_scale="min_axis")
        pl = lub.Pipeline(parts, dom, lub.default_params(precision="mixed", warm_start="mlp_all"),
                          capacity=len(pi), device=dev)
        WarmStartMLP.load(device=dev).install(pl.ctx)
        lub.lub_mlp_engine(pl.ctx.h, args.mlp_engine)
        pl.set_pairs(pi, pj)
        with torch.cuda.stream(stream):
            for _ in range(args.steps):
                pl.closest(stream=stream)
        stream.synchronize()
        return {"pairs": len(pi), "steps": args.steps}
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            pl.step(form=STEP_FORM, pair_forces=PAIR_FORCES, stream=stream)
    stream.synchronize()
    return {"pairs": int(min(pl.count(), pl.cap)), "steps": args.steps}


def run_ours(args):
    import numpy as np
    import torch

    import paper_1308_6482_gb300 as lub

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    if args.only:
        leg = only_leg(args, lub, torch, np, dev, stream)
        if rank == 0:
            print(json.dumps({"only": args.only, args.only: leg}))
        return
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    pk = peaks(lub, dev)
    head, parts, dom, pairs0, rmax, net = large_headline(args, lub, torch, np, dev, stream, flush, ws, rank, pk)
    e2e = None if args.no_e2e else e2e_large(args, lub, torch, np, parts, dom, dev, stream, rmax, net)
    secondary = {}
    if not args.no_secondary:
        secondary["mixed_suspension_32k"] = suspension_32k(args, lub, torch, np, dev, stream, flush, ws, rank, pk)
        secondary["learned_vs_plain_fresh_pairs"] = learned_vs_plain(args, lub, torch, np, dev, stream, flush)
        secondary["ensemble"] = ensemble_bench(args, lub, torch, np, dev, stream, flush, ws, rank)
    lead = head["forms"]["learned"]
    out = {
        "metric": METRIC, "value": head["value"], "unit": "pairs/s", "n_gpus": ws, "steps": lead["steps"],
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+ff32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": "mixed (FP32; float-float gap, normal and normal velocity; "
                                                      "FP64 for pairs the FP32 Newton fails)",
                   "form": "lub_pairs_build, then lub_correct (closest points, resistance, scatter), one CUDA "
                           "graph per step",
                   "warm_start": "learned (LUB_WARM_MLP: the network starts the FP64 solves; FP32 Newton from the "
                                 "line of centres)",
                   "particles": head["particles"], "pairs_per_step": head["pairs_per_step"],
                   "l2": "inputs larger than L2 (about 0.5 GB per step) and a 256 MB flush between timed steps",
                   "cuda_graph": True, "parallelism": "independent replicas" if ws > 1 else "1 GPU",
                   "forms": head["forms"], "speedup_learned_vs_plain": head["speedup_learned_vs_plain"],
                   "speedup_learned_vs_temporal": head["speedup_learned_vs_temporal"],
                   "steps_per_graph": head["steps_per_graph"], "call_ms": head["call_ms"],
                   "other_forms_ms_per_step": head["other_forms_ms_per_step"], "autotuned_shapes": head["autotuned_shapes"],
                   "kernel_ms": head["kernel_ms"], "generation_s": head["generation_s"]},
        "roofline": head["roofline"], "rooflines": head["rooflines"], "peaks": {
            k: pk.get(k) for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained", "fp32_tflops", "fp64_tflops",
                                   "src", "alu_src")},
        "clocks": head["clocks"], "gpu_launches": kernels_in_step() * lead["steps"], "e2e": e2e,
        "secondary": secondary,
    }
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        out["cpu_baseline"] = cpu_baseline(parts, dom, pairs0)
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on the host cores, on the same
    workload and metric: the growth-packed slab the large run tiles 8 x 8
    (16,384 spheroids, its pairs are the large run's pairs up to the
    tiling), the oracle's own O(N^2) pre-filter as set-up, then each step the
    closest points, forces and sums of a sample of its pairs sized so the run
    stays within about a minute."""
    ws, rank, local = dist_setup()
    if rank != 0:
        return
    import gen
    import oracle
    parts, dom = gen.large_config(N=args.large_n, seed=6, base_only=True)
    P = oracle.Particles(parts)
    pi, pj = oracle.candidates(P, dom, 1.0)
    t0 = time.perf_counter()
    m0 = min(len(pi), 8192)
    cp = oracle.closest(P, dom, pi[:m0], pj[:m0])
    oracle.pair_force(P, dom, None, pi[:m0], pj[:m0], cp)
    per_pair = (time.perf_counter() - t0) / m0
    m = int(max(256, min(len(pi), 60.0 / max(1, args.steps + args.warmup) / per_pair)))
    for _ in range(args.warmup):
        cp = oracle.closest(P, dom, pi[:m], pj[:m])
        pf = oracle.pair_force(P, dom, None, pi[:m], pj[:m], cp)
        oracle.apply(P.n, pi[:m], pj[:m], pf["FT"], pf["lever"])
    ts = time.perf_counter()
    for _ in range(args.steps):
        cp = oracle.closest(P, dom, pi[:m], pj[:m])
        pf = oracle.pair_force(P, dom, None, pi[:m], pj[:m], cp)
        oracle.apply(P.n, pi[:m], pj[:m], pf["FT"], pf["lever"])
    el = time.perf_counter() - ts
    value = m * args.steps / el
    cores = os.cpu_count()
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "precision": "fp64 (oracle)", "pairs_per_step": m,
                      "sample": "the 16,384-particle slab of the packing (%d pairs), %d of them per step"
                                % (len(pi), m)},
           "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle", "cpu": cpu_model(),
                            "sample": "%d pairs of the large run's growth-packed slab per step (closest points, "
                                      "forces, sums), %d OpenMP threads" % (m, cores)},
           "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    args = parse()
    if args.graph_steps < 2 or args.graph_steps % 2:
        raise SystemExit("--graph-steps must be even and >= 2")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
