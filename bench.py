#!/usr/bin/env python
"""Throughput benchmark of the lubrication correction (pairs per second).

One step = one pass of the whole path over one suspension: lub_pairs_build
(cell list + Sec. III A pre-filters), lub_closest_points, lub_resistance and
lub_apply, enqueued on one stream.  The step is captured once into a CUDA
graph (built from the same C-ABI calls) and replayed; the L2 cache is flushed
between timed steps by writing a 256 MB buffer outside the step's events.

Workload (N=1): the 32,768-particle mixed suspension (half spheres r = 4.5,
half oblates with semi-axes 6, 6, 3) at volume fraction 0.3 in a periodic
cube, list cut-off 1, mixed precision.  Under torchrun each rank runs its own
independent suspension (different seed): weak scaling with no collective in
the data path.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the host cores instead (the reference arm).
"""
import argparse
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
WORKLOAD = ("mixed suspension: N=32768 (50% spheres r=4.5, 50% oblates 6,6,3), phi=0.3, periodic cube "
            "L=357.7, 90% of particles attached to an earlier one at a gap log-uniform in [1e-4,1], "
            "pairs with possible gap < 1 (Delta_L=1)")

# algorithmic work per unit (what the method must compute or move, counted
# from the per-pair formulas), used for the roofline of the dominant call
FP32_NEWTON_FLOP = 170.0      # one FP32 Newton iteration on the sphere
FP64_GAP_FLOP = 70.0          # the gap: 2 axes from quaternions, 2 support functions, n.d (FP64 mode)
FF_GAP_FP32_FLOP = 4 * 70.0   # the same gap in float-float (mixed): about 4 FP32 operations per operation
FF_STEP_FP32_FLOP = 600.0     # one float-float Newton step (the refinement below the switch, mixed)
FP64_NEWTON_FLOP = 170.0      # one FP64 Newton iteration (FP64 mode)
RES_FP32_FLOP = 900.0         # K2 per pair: 2 surface frames, eigenproblem, cubic rotation, K~, u, forces
PAIRS_BYTES_PER_PARTICLE = 48.0   # pose + shape read once
PAIRS_BYTES_PER_PAIR = 8.0        # (i, j) written
APPLY_BYTES_PER_PAIR = 56.0       # F, T, levers (float) + indices
APPLY_BYTES_PER_PARTICLE = 24.0   # force + torque written
# DRAM bytes per call from one ncu capture of the 32k-particle workload
# (profiles/kernels_mixed_suspension_32k.md: dram__bytes_read.sum +
# dram__bytes_write.sum summed over the pair build's seven kernels, cold cache);
# valid for the kernels profiled there, for that workload only
TRAFFIC_PAIRS_BUILD_32K = 9.1005e6


FORM_NAMES = {"fused": "pair build + fused pass (lub_correct)",
              "merged": "pair build + closest points + resistance with scatter (lub_resistance_apply)",
              "calls": "pair build + closest points + resistance + apply"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="default launch shapes instead of the autotuner's")
    ap.add_argument("--form", default="merged", choices=["calls", "merged", "fused"],
                    help="calls: pair build + closest + resistance + apply; merged: pair build + closest + "
                         "resistance_apply; fused: pair build + lub_correct")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-vs-plain warm-start comparison")
    ap.add_argument("--learned-pairs", type=int, default=1 << 20)
    ap.add_argument("--no-ensemble", action="store_true", help="skip the batched-ensemble workload")
    ap.add_argument("--ens-n", type=int, default=256, help="suspensions in the ensemble workload")
    ap.add_argument("--ens-steps", type=int, default=100)
    ap.add_argument("--no-large", action="store_true", help="skip the large wall-bounded run")
    ap.add_argument("--large-form", default="merged", choices=["calls", "merged", "fused"])
    ap.add_argument("--ens-form", default="merged", choices=["calls", "merged", "fused"])
    ap.add_argument("--large-n", type=int, default=1 << 20)
    ap.add_argument("--large-steps", type=int, default=1000)
    ap.add_argument("--n", type=int, default=32768)
    ap.add_argument("--only", default=None, choices=["step", "large", "ensemble", "learned"],
                    help="run only that workload and print its results (for profiling; no bench line)")
    ap.add_argument("--fp64-switch", type=float, default=1e-3,
                    help="h/a below which pairs get the FP64 Newton refinement (0: none)")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    out = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "src": "fallback"}
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        out.update(d)
        out["src"] = "measured"
    # non-tensor pipes, measured on a GB300 with an FMA-chain probe
    out.setdefault("fp32_tflops", 74.6)
    out.setdefault("fp64_tflops", 1.20)
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
    if args.only:
        stream = torch.cuda.Stream(device=dev)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        leg = {"step": lambda: eager_steps(args, dev, stream),
               "large": lambda: large_bench(args, dev, stream, flush, ws, rank),
               "ensemble": lambda: ensemble_bench(args, dev, stream, flush, ws, rank),
               "learned": lambda: learned_vs_plain(args, dev, stream, flush)}[args.only]()
        if rank == 0:
            print(json.dumps({"only": args.only, args.only: leg}))
        return
    parts, dom = make_workload(args.n, rank_seed(rank))
    prm = lub.default_params(precision=args.precision, fp64_switch=args.fp64_switch)
    pl = lub.Pipeline(parts, dom, prm, device=dev)
    npairs = pl.build_pairs()              # sizes capacity and the context scratch
    pl._alloc(int(npairs * 1.1) + 1024, dev)
    npairs = pl.build_pairs()
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    form = args.form
    fused = form == "fused"
    # launch shapes of this step's kernels from the library's autotuner
    shapes = None
    if not args.no_tune:
        with torch.cuda.stream(stream):
            shapes = pl.autotune(reps=5, stream=stream)
        stream.synchronize()
    # eager step once: per-call launch accounting and results for the work counts
    with torch.cuda.stream(stream):
        pl.step(form=form, stream=stream)
    stream.synchronize()
    res = pl.results()
    mean_it = float(np.mean(res["iters"]))
    fp64_frac = float(np.mean((res["status"] & lub.LUB_ST_FP64) != 0))

    # capture the step into a CUDA graph
    graph = None
    if not args.no_graph:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            pl.step(form=form, stream=stream)
        stream.synchronize()

    calls = {"fused": ("pairs_build", "correct"), "merged": ("pairs_build", "closest", "resistance_apply"),
             "calls": ("pairs_build", "closest", "resistance", "apply")}[form]

    def step_timed(evs):
        # per-call events (used for the roofline) around the calls
        evs[0].record(stream)
        pl.build_pairs(sync_count=False, grow=False, stream=stream)
        evs[1].record(stream)
        if fused:
            pl.correct(stream=stream)
            evs[2].record(stream)
            return
        if form == "merged":
            pl.closest(stream=stream)
            evs[2].record(stream)
            pl.resistance_apply(stream=stream)
            evs[3].record(stream)
            return
        pl.closest(stream=stream)
        evs[2].record(stream)
        pl.resistance(stream=stream)
        evs[3].record(stream)
        pl.apply(stream=stream)
        evs[4].record(stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            if graph is not None:
                graph.replay()
            else:
                pl.step(form=form, stream=stream)
    stream.synchronize()

    # timed region: K steps of the graph, L2 flushed between steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.2)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            if graph is not None:
                graph.replay()
            else:
                pl.step(form=form, stream=stream)
            ends[k].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if ws > 1:
        dist.barrier()
    clocks = sampler.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = float(sum(step_ms))

    # the other forms of the step, graph-replayed with the same flush, for reference
    forms_ms = {}
    if graph is not None:
        for other in ("calls", "merged", "fused"):
            if other == form:
                continue
            g2 = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g2, stream=stream):
                pl.step(form=other, stream=stream)
            stream.synchronize()
            Ko = min(args.steps, 50)
            eo = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(Ko)]
            with torch.cuda.stream(stream):
                for _ in range(3):
                    flush.zero_()
                    g2.replay()
                for a, b in eo:
                    flush.zero_()
                    a.record(stream)
                    g2.replay()
                    b.record(stream)
            stream.synchronize()
            forms_ms[other] = float(np.mean([a.elapsed_time(b) for a, b in eo]))
            del g2

    # the "normal only" model (K~33 alone, Sec. IV C) on the same workload: a
    # second workload of the same path, graph-replayed with the same flush
    normal_ms = None
    if graph is not None:
        pln = lub.Pipeline(lub.DeviceParticles(parts, dev), dom,
                           lub.default_params(precision=args.precision, fp64_switch=args.fp64_switch, model="normal"),
                           capacity=pl.cap, device=dev)
        pln.build_pairs()
        with torch.cuda.stream(stream):
            pln.step(form=form, stream=stream)
        stream.synchronize()
        g3 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g3, stream=stream):
            pln.step(form=form, stream=stream)
        stream.synchronize()
        e3 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(50)]
        with torch.cuda.stream(stream):
            for _ in range(3):
                flush.zero_()
                g3.replay()
            for a, b in e3:
                flush.zero_()
                a.record(stream)
                g3.replay()
                b.record(stream)
        stream.synchronize()
        normal_ms = float(np.mean([a.elapsed_time(b) for a, b in e3]))
        del g3, pln

    # the comparison model of Sec. II: the link-based lubrication of Ding and
    # Aidun (lub_links) on the same pair list, one call per step, L2 flushed
    link = None
    if graph is not None:
        with torch.cuda.stream(stream):
            F_l, T_l, nl_l = pl.links(0.6, stream=stream)
        stream.synchronize()
        e5 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(20)]
        with torch.cuda.stream(stream):
            for a, b in e5:
                flush.zero_()
                a.record(stream)
                pl.links(0.6, stream=stream)
                b.record(stream)
        stream.synchronize()
        link_ms = float(np.mean([a.elapsed_time(b) for a, b in e5]))
        nl_host = nl_l[:npairs].cpu().numpy()
        link = {"ms_per_call": link_ms, "pairs_per_s": npairs / (link_ms * 1e-3),
                "links_per_pair": float(nl_host.mean()), "pairs_with_links": float((nl_host > 0).mean()),
                "note": "Eq. methods:dlub on a unit lattice, D3Q19 links, q_bar = 0.6, FP64 per link; the pair list "
                        "of the step (gaps up to Delta_L = 1), one warp per pair"}

    # particle sub-stepping (Sec. II) on the same workload with the contact
    # branch (h_c = 0.01, eps_c = 100): one LB step = the pair build and 10
    # sub-steps of (closest points, resistance + scatter, rigid update) at
    # dt = 0.1 under a constant external force, one CUDA graph per LB step
    substep = None
    if graph is not None:
        pls = lub.Pipeline(lub.DeviceParticles(parts, dev), dom,
                           lub.default_params(precision=args.precision, fp64_switch=args.fp64_switch, h_c=0.01,
                                              eps_c=100.0), capacity=pl.cap, device=dev)
        pls.build_pairs()
        gf = torch.Generator(device=dev)
        gf.manual_seed(99)
        fext = 0.01 * torch.randn(3 * pls.n, generator=gf, device=dev, dtype=torch.float32)
        with torch.cuda.stream(stream):
            pls.substeps(10, 1.0, 0.1, f_ext=fext, stream=stream)
        stream.synchronize()
        g4 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g4, stream=stream):
            pls.substeps(10, 1.0, 0.1, f_ext=fext, stream=stream)
        stream.synchronize()
        e4 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(20)]
        with torch.cuda.stream(stream):
            for _ in range(3):
                flush.zero_()
                g4.replay()
            for a, b in e4:
                flush.zero_()
                a.record(stream)
                g4.replay()
                b.record(stream)
        stream.synchronize()
        lb_ms = float(np.mean([a.elapsed_time(b) for a, b in e4]))
        pairs_s = min(pls.count(), pls.cap)
        substep = {"ms_per_lb_step": lb_ms, "substeps": 10, "pairs": pairs_s,
                   "pair_corrections_per_s": 10 * pairs_s / (lb_ms * 1e-3),
                   "note": "h_c=0.01, eps_c=100, dt=0.1, density 1, external force N(0,0.01^2); 29 launches per "
                           "LB step in one graph"}
        del g4, pls

    # per-call device times (eager calls, same stream, L2 flushed), for the roofline
    K2 = min(args.steps, 100)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(calls) + 1)] for _ in range(K2)]
    with torch.cuda.stream(stream):
        for k in range(K2):
            flush.zero_()
            step_timed(evs[k])
    stream.synchronize()
    call_ms = {c: float(np.mean([evs[k][q].elapsed_time(evs[k][q + 1]) for k in range(K2)]))
               for q, c in enumerate(calls)}

    # e2e through the public API: host inputs (pinned) -> device, step, force/torque -> host
    e2e = None
    if not args.no_e2e:
        # the user-facing form: particles in one packed device buffer, the
        # step's inputs and outputs moved by one copy each way
        Pk = lub.DeviceParticles(parts, dev, packed=True)
        ple = lub.Pipeline(Pk, dom, prm, capacity=pl.cap, device=dev)
        ple.build_pairs()
        hblob = Pk.host_blob(parts, torch.empty(Pk.blob.numel(), dtype=torch.uint8).pin_memory())
        hout = torch.empty(ple.ft_particles.numel(), dtype=ple.ft_particles.dtype).pin_memory()
        bi = hblob.numel()
        bo = hout.numel() * hout.element_size()
        Ke = min(args.steps, 100)

        def e2e_step():
            Pk.blob.copy_(hblob, non_blocking=True)
            ple.step(form=form, stream=stream)
            hout.copy_(ple.ft_particles, non_blocking=True)

        with torch.cuda.stream(stream):
            for _ in range(3):
                e2e_step()
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # eager: the copies and the step's calls launched one by one
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(Ke):
                e2e_step()
            e1.record(stream)
        stream.synchronize()
        eager_ms = e0.elapsed_time(e1) / Ke
        # graph: the pinned host->device copies, the step and the device->host
        # copies of force and torque captured together and replayed per step;
        # the host waits for every step's result before the next
        ge = torch.cuda.CUDAGraph()
        with torch.cuda.graph(ge, stream=stream):
            e2e_step()
        stream.synchronize()
        for _ in range(3):
            ge.replay()
        stream.synchronize()
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
        del ge
        e2e = {"value": npairs / (e2e_ms * 1e-3), "unit": "pairs/s", "h2d_bytes_per_step": int(bi),
               "d2h_bytes_per_step": int(bo), "ms_per_step": e2e_ms, "host_wall_ms_per_step": host_ms,
               "eager_ms_per_step": eager_ms,
               "how": "packed pinned host particles -> device (one copy), step, force+torque -> pinned host "
                      "(one copy), one CUDA graph per step, host synchronised on every step's result"}

    # max over ranks
    ms_per_step, pairs_all = aggregate(total_ms / args.steps, npairs, ws, dev)
    value = pairs_all / (ms_per_step * 1e-3)

    pk = peaks()
    dom_call = max(call_ms, key=call_ms.get)
    roof = roofline(dom_call, call_ms[dom_call], npairs, args.n, mean_it, fp64_frac, args.precision, pk)
    kernels_per_step = kernels_in_step(args.precision, form)
    out = {
        "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": args.precision, "fp64_switch": args.fp64_switch,
                   "form": {"fused": "pair build + fused pass (lub_correct)",
                            "merged": "pair build + closest points + resistance with scatter (lub_resistance_apply)",
                            "calls": "pair build + closest points + resistance + apply"}[form],
                   "other_forms_ms_per_step": forms_ms,
                   "normal_only_model_ms_per_step": normal_ms,
                   "comparison_link_model": link,
                   "substepping": substep,
                   "pairs_per_step": int(npairs),
                   "particles": args.n, "l2": "flushed between timed steps (256 MB write outside the step events)",
                   "cuda_graph": graph is not None, "parallelism": "independent replicas" if ws > 1 else "1 GPU",
                   "newton_iters_mean": mean_it, "fp64_refined_fraction": fp64_frac,
                   "call_ms": call_ms, "wall_s_timed": wall,
                   "autotuned_shapes": {k: list(v) for k, v in shapes.items()} if shapes else None},
        "roofline": roof, "clocks": clocks, "gpu_launches": kernels_per_step * args.steps,
        "e2e": e2e,
    }
    if not args.no_learned:
        out["learned_vs_plain"] = learned_vs_plain(args, dev, stream, flush)
    if not args.no_ensemble:
        out["ensemble"] = ensemble_bench(args, dev, stream, flush, ws, rank)
    if not args.no_large:
        out["large"] = large_bench(args, dev, stream, flush, ws, rank)
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        out["cpu_baseline"] = cpu_baseline(parts, dom)
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def eager_steps(args, dev, stream):
    """The main workload's step, args.steps times, eagerly on one stream (no
    tuning, no graph): a short, fixed launch sequence for a profiler."""
    import torch

    import paper_1308_6482_gb300 as lub

    parts, dom = make_workload(args.n, rank_seed(0))
    prm = lub.default_params(precision=args.precision, fp64_switch=args.fp64_switch)
    pl = lub.Pipeline(parts, dom, prm, device=dev)
    npairs = pl.build_pairs()
    pl._alloc(int(npairs * 1.1) + 1024, dev)
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            pl.step(form=args.form, stream=stream)
    stream.synchronize()
    return {"pairs": int(npairs), "steps": args.steps, "form": args.form}


def learned_vs_plain(args, dev, stream, flush, steps=20, warmup=3):
    """Learned warm start against the plain (line-of-centres) start on fresh
    spheroid pairs: aspect ratios log-uniform in [1/3, 3], gaps log-uniform in
    [1e-4, 1] x the pair's smallest semi-axis, one seed the training set never
    used.  Times lub_closest_points alone (the network's inference runs inside
    it for the learned form), L2 flushed between calls, and checks that both
    forms reach the same gaps (equal accuracy)."""
    import numpy as np
    import torch

    import gen
    import paper_1308_6482_gb300 as lub
    from paper_1308_6482_gb300.mlp import WarmStartMLP

    parts, dom, pi, pj = gen.pair_stream(args.learned_pairs, seed=9100, kind="aspect", gap_range=(1e-4, 1.0),
                                         gap_scale="min_axis")
    m = len(pi)
    net = WarmStartMLP.load(device=dev)
    P = lub.DeviceParticles(parts, dev)
    out = {"workload": "%d fresh spheroid pairs, aspect ratios log-uniform [1/3,3], gap log-uniform "
                       "[1e-4,1] x min semi-axis" % m, "steps": steps}
    for prec in ("fp64", "mixed"):
        res = {}
        for form in ("plain", "learned", "learned_tcgen05"):
            prm = lub.default_params(precision=prec, warm_start="none" if form == "plain" else "mlp")
            pl = lub.Pipeline(P, dom, prm, capacity=m, device=dev)
            if form != "plain":
                net.install(pl.ctx)
                lub.lub_mlp_engine(pl.ctx.h, "tcgen05" if form == "learned_tcgen05" else "mma_sync")
            pl.set_pairs(pi, pj)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            with torch.cuda.stream(stream):
                for _ in range(warmup):
                    flush.zero_()
                    pl.closest(stream=stream)
                for a, b in ev:
                    flush.zero_()
                    a.record(stream)
                    pl.closest(stream=stream)
                    b.record(stream)
            stream.synchronize()
            ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
            it = pl.iters[:m].cpu().numpy().astype(np.float64)
            res[form] = {"pairs_per_s": m / (ms * 1e-3), "ms": ms, "newton_iters_mean": float(it.mean()),
                         "warp_max_iters_mean": float(it[:m - m % 32].reshape(-1, 32).max(1).mean()),
                         "h": pl.gap[:m].cpu().numpy(), "status": pl.status[:m].cpu().numpy()}
            del pl
        h0, h1 = res["plain"].pop("h"), res["learned"].pop("h")
        s0, s1 = res["plain"].pop("status"), res["learned"].pop("status")
        h2, s2 = res["learned_tcgen05"].pop("h"), res["learned_tcgen05"].pop("status")
        res["max_abs_gap_difference_tcgen05"] = float(np.abs(h2 - h0).max())
        res["speedup_tcgen05"] = res["learned_tcgen05"]["pairs_per_s"] / res["plain"]["pairs_per_s"]
        scale = np.array([max(parts["r_par"][a], parts["r_perp"][a]) + max(parts["r_par"][b], parts["r_perp"][b])
                          for a, b in zip(pi[:4096], pj[:4096])]).max()
        res["max_abs_gap_difference"] = float(np.abs(h1 - h0).max())
        res["gap_scale"] = float(scale)
        res["status_equal_fraction"] = float(np.mean((s0 & 7) == (s1 & 7)))
        res["speedup"] = res["learned"]["pairs_per_s"] / res["plain"]["pairs_per_s"]
        out[prec] = res
    return out


def rigid_motion(P, g, sig_r=0.01, sig_t=0.005):
    """Move every particle by a seeded random rigid motion: dr ~ N(0, sig_r^2)
    per axis, a rotation by a vector ~ N(0, sig_t^2) per axis (torch ops on the
    device; input preparation between steps, not part of the step)."""
    import torch
    n = P.n
    dev = P.t["x"].device
    for k in ("x", "y", "z"):
        P.t[k] += sig_r * torch.randn(n, generator=g, device=dev, dtype=torch.float64)
    th = sig_t * torch.randn((3, n), generator=g, device=dev, dtype=torch.float32)
    a = th.norm(dim=0)
    s = torch.where(a > 0, torch.sin(0.5 * a) / torch.where(a > 0, a, torch.ones_like(a)), 0.5 * torch.ones_like(a))
    dw, dx, dy, dz = torch.cos(0.5 * a), s * th[0], s * th[1], s * th[2]
    w, x, y, z = (P.t[k].clone() for k in ("qw", "qx", "qy", "qz"))
    nw = dw * w - dx * x - dy * y - dz * z
    nx = dw * x + dx * w + dy * z - dz * y
    ny = dw * y - dx * z + dy * w + dz * x
    nz = dw * z + dx * y - dy * x + dz * w
    inv = torch.rsqrt(nw * nw + nx * nx + ny * ny + nz * nz)
    for k, v in (("qw", nw), ("qx", nx), ("qy", ny), ("qz", nz)):
        P.t[k].copy_(v * inv)


def ensemble_bench(args, dev, stream, flush, ws=1, rank=0):
    """Batched ensemble: args.ens_n independent periodic suspensions of mixed
    spheroids (growth packings, aspect ratio log-uniform [1/3, 3], phi uniform
    [0.1, 0.5], pair counts log-uniform [1e3, 2e5]) stepped together: one CUDA graph per
    step (the four calls, one launch per stage for all suspensions), launch
    shapes from the autotuner, every particle moved by a small seeded rigid
    motion between steps.  Against it: the same suspensions stepped one by one
    with their own calls (a few steps), and the same ensemble with the two warm
    starts of the closest-point solve (temporal: the previous step's normals
    carried over; learned: the network).  Under torchrun the suspensions shard
    over the ranks (suspension s on rank s mod N, no exchange)."""
    import numpy as np
    import torch

    import gen
    import paper_1308_6482_gb300 as lub
    from paper_1308_6482_gb300.mlp import WarmStartMLP

    t0 = time.perf_counter()
    sus, meta = gen.ensemble(n_susp=args.ens_n, seed=4)
    sus = [sus[b] for b in ensemble_shard(len(sus), ws, rank)]
    t_gen = time.perf_counter() - t0
    parts, doms, off = lub.make_ensemble(sus)
    rmax = float(max(parts["r_par"].max(), parts["r_perp"].max())) + 0.05
    net = WarmStartMLP.load(device=dev)

    def run(warm, steps, tune=False, shapes=None, precision="mixed"):
        """`steps` graph-replayed steps from the initial poses, the same seeded
        motions for every form; returns (ms [steps], pairs [steps], Newton
        iterations per pair, capacity overflows, the context's shapes)."""
        P = lub.DeviceParticles(parts, dev, max_semi_axis=rmax, batch_offsets=off)
        prm = lub.default_params(precision=precision, warm_start=warm)
        pl = lub.Pipeline(P, doms, prm, capacity=1024, device=dev)
        if warm == lub.LUB_WARM_MLP:
            net.install(pl.ctx)
        if shapes:
            for q, (blk, per) in enumerate(shapes):
                lub.lub_set_launch_shape(pl.ctx.h, q, blk, per)
        npairs = pl.build_pairs()
        pl._alloc(int(npairs * 1.3) + 4096, dev)
        pl.build_pairs()
        with torch.cuda.stream(stream):
            if tune:
                pl.autotune(reps=2, stream=stream)
            pl.step(form=args.ens_form, stream=stream)
            pl.step(form=args.ens_form, stream=stream)
        stream.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            pl.step(form=args.ens_form, stream=stream)
        stream.synchronize()
        g = torch.Generator(device=dev)
        g.manual_seed(12345)
        counts = torch.zeros(steps, dtype=torch.int32, device=dev)
        its = torch.zeros(steps, dtype=torch.float64, device=dev)
        idx = torch.arange(pl.cap, device=dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        with torch.cuda.stream(stream):
            for _ in range(3):
                rigid_motion(P, g)
                graph.replay()
            for k in range(steps):
                rigid_motion(P, g)
                flush.zero_()
                ev[k][0].record(stream)
                graph.replay()
                ev[k][1].record(stream)
                counts[k].copy_(pl.d_count[0])
                m = torch.clamp(pl.d_count[0], max=pl.cap)
                its[k] = (pl.iters.double() * (idx < m)).sum() / m
        stream.synchronize()
        ms = np.array([a.elapsed_time(b) for a, b in ev])
        cnt = counts.cpu().numpy().astype(np.float64)
        sh = [lub.lub_get_launch_shape(pl.ctx.h, q) for q in range(lub.LUB_TUNE_COUNT)]
        return ms, cnt, float(its.mean().item()), int((cnt > pl.cap).sum()), sh

    t1 = time.perf_counter()
    ms, cnt, it_plain, over, shapes = run(lub.LUB_WARM_NONE, args.ens_steps, tune=True)
    t_run = time.perf_counter() - t1
    warm_forms = {}
    for prec in ("mixed", "fp64"):
        for name, warm in (("plain", lub.LUB_WARM_NONE), ("temporal", lub.LUB_WARM_PREVIOUS),
                           ("learned", lub.LUB_WARM_MLP)):
            if prec == "mixed" and name == "plain":
                continue
            steps_w = max(10, args.ens_steps // (4 if prec == "mixed" else 10))
            msw, cntw, itw, _, _ = run(warm, steps_w, shapes=shapes, precision=prec)
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
            q.step(form=args.ens_form, stream=stream)
        flush.zero_()
        e0.record(stream)
        for _ in range(Ks):
            for q in sep:
                q.step(form=args.ens_form, stream=stream)
        e1.record(stream)
    stream.synchronize()
    sep_ms = e0.elapsed_time(e1) / Ks
    sep_pairs = float(sum(q.count() for q in sep))
    step_ms, all_pairs = aggregate(float(ms.mean()), float(cnt.mean()), ws, dev)
    sep_ms, sep_pairs = aggregate(sep_ms, sep_pairs, ws, dev)
    n_all = aggregate(0.0, float(len(parts["x"])), ws, dev)[1]
    return {
        "workload": "%d periodic suspensions (growth packings), phi uniform [0.1,0.5], aspect ratio log-uniform [1/3,3], pair "
                    "counts log-uniform [1e3,2e5]; %d particles, %d steps of seeded rigid motions "
                    "(dr ~ N(0,0.01^2), dtheta ~ N(0,0.005^2))" % (args.ens_n, int(n_all), args.ens_steps),
        "precision": "mixed", "pairs_per_step_mean": all_pairs, "ms_per_step": step_ms,
        "pairs_per_s": all_pairs / (step_ms * 1e-3), "newton_iters_per_pair": it_plain,
        "capacity_overflows": over, "ranks": ws,
        "launch": "one CUDA graph per step (%s), one persistent launch per stage for all suspensions"
                  % FORM_NAMES[args.ens_form],
        "autotuned_shapes": {lub.TUNE_NAMES[q]: list(v) for q, v in enumerate(shapes)},
        "autotune_and_run_s": t_run, "generation_s": t_gen,
        "warm_starts": warm_forms,
        "separate_calls": {"ms_per_step": sep_ms, "pairs_per_s": sep_pairs / (sep_ms * 1e-3),
                           "launches_per_step": "8 per suspension, eager"},
        "speedup_vs_separate": float((all_pairs / step_ms) / (sep_pairs / sep_ms)),
    }


def large_bench(args, dev, stream, flush, ws=1, rank=0):
    """Large run: args.large_n spheroids (aspect ratio log-uniform [1/3, 3]) at
    phi = 0.5 (growth packing) in a 1024^3 cube periodic in x, y between two
    plane walls, mixed
    precision, args.large_steps graph-replayed steps, every particle moved by a
    small seeded rigid motion between steps; then shorter runs with the
    learned and the temporal warm start on the same motions.  Under torchrun
    every rank runs its own copy (another seed): replicas."""
    import numpy as np
    import torch

    import gen
    import paper_1308_6482_gb300 as lub
    from paper_1308_6482_gb300.mlp import WarmStartMLP

    t0 = time.perf_counter()
    parts, dom = gen.large_config(N=args.large_n, seed=6 + 1000 * rank)
    t_gen = time.perf_counter() - t0
    rmax = float(max(parts["r_par"].max(), parts["r_perp"].max())) + 0.05
    net = WarmStartMLP.load(device=dev)

    def run(warm, steps):
        P = lub.DeviceParticles(parts, dev, max_semi_axis=rmax)
        pl = lub.Pipeline(P, dom, lub.default_params(precision="mixed", warm_start=warm), capacity=1024, device=dev)
        if warm == lub.LUB_WARM_MLP:
            net.install(pl.ctx)
        npairs = pl.build_pairs()
        pl._alloc(int(npairs * 1.3) + 4096, dev)
        pl.build_pairs()
        with torch.cuda.stream(stream):
            pl.step(form=args.large_form, stream=stream)
            pl.step(form=args.large_form, stream=stream)
        stream.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            pl.step(form=args.large_form, stream=stream)
        stream.synchronize()
        g = torch.Generator(device=dev)
        g.manual_seed(777)
        counts = torch.zeros(steps, dtype=torch.int32, device=dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        with torch.cuda.stream(stream):
            for _ in range(3):
                rigid_motion(P, g)
                graph.replay()
            for k in range(steps):
                rigid_motion(P, g)
                flush.zero_()
                ev[k][0].record(stream)
                graph.replay()
                ev[k][1].record(stream)
                counts[k].copy_(pl.d_count[0])
        stream.synchronize()
        ms = np.array([a.elapsed_time(b) for a, b in ev])
        cnt = counts.cpu().numpy().astype(np.float64)
        walls = int((pl.pair_j[:min(pl.count(), pl.cap)] < 0).sum().item())
        if warm == lub.LUB_WARM_NONE and args.large_form == "merged":
            # the three calls of the merged step timed one by one (events
            # between the calls, L2 flushed before each step), for the roofline
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            tcall = {"pairs_build": [], "closest": [], "resistance_apply": []}
            with torch.cuda.stream(stream):
                for _ in range(8):
                    flush.zero_()
                    evs[0].record(stream)
                    pl.build_pairs(sync_count=False, grow=False, stream=stream)
                    evs[1].record(stream)
                    pl.closest(stream=stream)
                    evs[2].record(stream)
                    pl.resistance_apply(stream=stream)
                    evs[3].record(stream)
                    stream.synchronize()
                    for q, name in enumerate(tcall):
                        tcall[name].append(evs[q].elapsed_time(evs[q + 1]))
            m = min(pl.count(), pl.cap)
            calls_ms["ms"] = {k: float(np.median(v[2:])) for k, v in tcall.items()}
            calls_ms["pairs"] = m
            calls_ms["mean_it"] = float(pl.iters[:m].float().mean().item())
            calls_ms["fp64_frac"] = float(((pl.status[:m] & lub.LUB_ST_FP64) != 0).float().mean().item())
        return ms, cnt, int((cnt > pl.cap).sum()), walls

    calls_ms = {}
    ms, cnt, over, walls = run(lub.LUB_WARM_NONE, args.large_steps)
    step_ms, pairs = aggregate(float(ms.mean()), float(cnt.mean()), ws, dev)
    out = {"workload": "%d spheroids, aspect ratio log-uniform [1/3,3], phi=0.5 (growth packing), cube %.0f^3 periodic in x,y "
                       "between walls at z=0 and z=L; %d steps of seeded rigid motions"
                       % (len(parts["x"]), dom["L"][0], args.large_steps),
           "precision": "mixed", "form": FORM_NAMES[args.large_form],
           "pairs_per_step_mean": pairs, "wall_pairs_last_step": walls,
           "ms_per_step": step_ms, "pairs_per_s": pairs / (step_ms * 1e-3), "capacity_overflows": over,
           "generation_s": t_gen, "warm_starts": {}}
    if calls_ms:
        # the roofline of the call that takes longest at this size
        pk = peaks()
        dom_call = max(calls_ms["ms"], key=calls_ms["ms"].get)
        roof = roofline(dom_call, calls_ms["ms"][dom_call], calls_ms["pairs"], len(parts["x"]), calls_ms["mean_it"],
                        calls_ms["fp64_frac"], "mixed", pk)
        roof["note"] = "eager calls, events between them, L2 flushed before each step"
        out["call_ms"] = calls_ms["ms"]
        out["roofline"] = roof
    for name, warm in (("learned", lub.LUB_WARM_MLP), ("temporal", lub.LUB_WARM_PREVIOUS)):
        msw, cntw, _, _ = run(warm, max(10, args.large_steps // 10))
        wms, wp = aggregate(float(msw.mean()), float(cntw.mean()), ws, dev)
        out["warm_starts"][name] = {"ms_per_step": wms, "pairs_per_s": wp / (wms * 1e-3), "steps": len(msw)}
    return out


def kernels_in_step(precision, form):
    # lub_pairs_build: zeroing of its counters, cells count, scan, cells fill,
    # sweep, scan, compaction = 7.  Closest points, mixed: zeroing of the work
    # list, float-float positions, FP32 stage, refinement = 4; FP64: 1.
    # merged: zeroing of the sums + lub_resistance_apply = 2; calls:
    # lub_resistance + zeroing + lub_apply (atomic) = 3.  fused (lub_correct):
    # zeroing of the sums, then mixed: zeroing of the work list, positions,
    # FP32 stage, refinement with the forces = 5; FP64: one kernel = 2.
    if form == "fused":
        return 7 + (5 if precision == "mixed" else 2)
    closest = 4 if precision == "mixed" else 1
    return 7 + closest + {"calls": 3, "merged": 2}[form]


def roofline(call, ms, npairs, n, mean_it, fp64_frac, precision, pk):
    t = ms * 1e-3
    if call in ("correct", "closest"):
        # mixed: FP32 Newton, the float-float gap and the float-float refinement
        # of the pairs below the switch, all on the FP32 pipe; FP64 mode: FP64
        # Newton and gap (the fused pass adds the resistance in the mode's precision)
        res = RES_FP32_FLOP if call == "correct" else 0.0
        name = "k_fused (closest + resistance + scatter)" if call == "correct" else "k_closest"
        if precision == "mixed":
            f32 = npairs * (mean_it * FP32_NEWTON_FLOP + FF_GAP_FP32_FLOP + fp64_frac * FF_STEP_FP32_FLOP + res)
            ach = f32 / t / 1e12
            peak = pk["fp32_tflops"]
            return {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s (FP32)",
                    "frac": ach / peak, "traffic": None,
                    "peak_src": "FP32 FMA-chain probe on a GB300 (not in MEASURED_PEAKS.json)"}
        f64 = npairs * (mean_it * FP64_NEWTON_FLOP + FP64_GAP_FLOP + res)
        ach = f64 / t / 1e12
        peak = pk["fp64_tflops"]
        return {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s (FP64)",
                "frac": ach / peak, "traffic": None,
                "peak_src": "FP64 FMA-chain probe on a GB300 (not in MEASURED_PEAKS.json)"}
    if call in ("resistance", "resistance_apply"):
        ach = npairs * RES_FP32_FLOP / t / 1e12
        peak = pk["fp32_tflops"]
        return {"kernel": "k_resistance", "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": None,
                "peak_src": "FP32 FMA-chain probe on a GB300 (not in MEASURED_PEAKS.json)"}
    traffic = None
    if call == "pairs_build":
        b = n * PAIRS_BYTES_PER_PARTICLE + npairs * PAIRS_BYTES_PER_PAIR
        if n == 32768:
            traffic = TRAFFIC_PAIRS_BUILD_32K
    else:
        b = npairs * APPLY_BYTES_PER_PAIR + n * APPLY_BYTES_PER_PARTICLE
    ach = b / t / 1e9
    return {"kernel": call, "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": ach / pk["hbm_gbs"], "traffic": traffic, "peak_src": pk["src"],
            "note": "a chain of small dependent launches over 2.5 MB: latency-bound at this size"
            if call == "pairs_build" else ""}


def cpu_baseline(parts, dom, budget_s=20.0):
    """The FP64 oracle, as it stands, on the host cores: one full step of the
    same workload (pre-filter over all pairs, closest points, forces, sums)."""
    import numpy as np

    import oracle
    cores = os.cpu_count()
    t0 = time.perf_counter()
    P = oracle.Particles(parts)
    pi, pj = oracle.candidates(P, dom, 1.0)
    t1 = time.perf_counter()
    cp = oracle.closest(P, dom, pi, pj)
    pf = oracle.pair_force(P, dom, None, pi, pj, cp)
    f, t = oracle.apply(P.n, pi, pj, pf["FT"], pf["lever"])
    t2 = time.perf_counter()
    return {"value": len(pi) / (t2 - t0), "unit": "pairs/s", "cores": cores, "kind": "oracle",
            "sample": "one full step of the same %d-particle suspension (%d pairs): O(N^2) pre-filter %.2f s "
                      "(1 thread), closest points + forces + sums %.2f s (%d OpenMP threads)"
                      % (P.n, len(pi), t1 - t0, t2 - t1, cores)}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on the host cores, same workload and metric."""
    import numpy as np
    ws, rank, local = dist_setup()
    if rank != 0:
        return
    import oracle
    parts, dom = make_workload(args.n, 2)
    P = oracle.Particles(parts)
    pi, pj = oracle.candidates(P, dom, 1.0)
    # each step: closest points + forces + sums on a contiguous sample of the pair list,
    # sized so the whole run stays within about a minute
    t0 = time.perf_counter()
    m0 = min(len(pi), 4096)
    cp = oracle.closest(P, dom, pi[:m0], pj[:m0])
    pf = oracle.pair_force(P, dom, None, pi[:m0], pj[:m0], cp)
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
           "config": {"workload": WORKLOAD, "precision": "fp64 (oracle)", "pairs_per_step": m},
           "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                            "sample": "%d of the %d pairs per step (closest points, forces, sums)" % (m, len(pi))},
           "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
