"""Benchmark of the Kronecker payoff products on GB300.

A step is one pass of the hot path over one batch: out = A*y and
out' = A^T*x for 1024 strategy vectors of the 1081-hand river endgame
(52-card deck, 5-card board, bets of 0.5 and 1.0 pot, at most 3 aggressive
actions: 57 terminals, 43+43 sequences), FP32.  The metric counts
vector-products (each A*y_b or A^T*x_b is one matvec).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Prints one JSON line (rank 0).
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
sys.path.insert(0, ROOT)

METRIC = "payoff matvecs/sec and HBM GB/s (fraction of peak); solver wall-time to 1e-3 pot"
UNIT = "matvecs/s"
BATCH = 1024
WORKLOAD = "river endgame, 1081 hands, 43+43 sequences, 57 terminals, batch 1024, fp32"
CSRC = os.path.join(ROOT, "paper_2112_03804_gb300", "csrc")
KERNEL = "tma_scan_kernel"
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling runs)")
    ap.add_argument("--workload", default="matvec", choices=["matvec", "batch", "solver", "warmstart", "factors", "libratus", "libratus_solve",
                                                   "turn", "predict"],
                    help="matvec: the headline line; batch / solver / warmstart / factors / libratus: print "
                         "only that measurement")
    ap.add_argument("--games", type=int, default=4096, help="games of the batched workload")
    ap.add_argument("--batch-shape", default=None,
                    help="kernel,warps,grid,schedule: the batched launch shape instead of the autotuner's "
                         "(profiling runs)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the batched and solver measurements in the headline line")
    return ap.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


KERNEL_SOURCES = ("kernels.h", "scan_records.h", "scan_records.cpp", "kernels_tma.cu")


def _kernel_hash():
    """Hash of the benchmarked kernel's code (its sources without comments
    and blank lines: changes whenever the code does, not when a comment
    does)."""
    import re
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        src = open(os.path.join(CSRC, f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        code = "\n".join(line.rstrip() for line in src.splitlines() if line.strip())
        h.update(f.encode())
        h.update(code.encode())
    return h.hexdigest()[:16]


def _traffic(kernel_hash):
    """DRAM bytes per launch from the committed ncu capture, if it was taken
    on the current kernel source."""
    try:
        d = json.load(open(TRAFFIC_FILE))
        if d.get("kernel_sha") == kernel_hash:
            return float(d["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for name, val in zip(names, f[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _workload():
    from paper_2112_03804_gb300 import synth
    return synth.river_spec(seed=2)


def cpu_baseline(spec, seconds: float):
    """The FP64 oracle's direct products (its own OpenMP loop over vectors)
    on this machine's host cores, on a bounded sample of the same workload."""
    from oracle.oracle import OracleGame
    from paper_2112_03804_gb300 import synth
    og = OracleGame(spec)
    cores = os.cpu_count() or 1
    y1 = synth.simplex_vectors(og.sequences(1)["nact"], og.H, 1, seed=3)
    t0 = time.perf_counter()
    og.matvec_A(y1, nthreads=1)
    per_vec = time.perf_counter() - t0
    nvec = max(cores, int(seconds * cores / max(per_vec, 1e-6)) // cores * cores)
    y = synth.simplex_vectors(og.sequences(1)["nact"], og.H, nvec, seed=3)
    t0 = time.perf_counter()
    og.matvec_A(y, nthreads=cores)
    dt = time.perf_counter() - t0
    # the oracle's FP64 RM+ on the tiny game (the solver baseline): the
    # exploitability of the averages every 10 iterations, as the GPU leg
    # checks it, until it is below 1e-3 of the pot
    tiny = OracleGame(synth.tiny_spec())
    t1 = time.perf_counter()
    _, _, _, trace = tiny.rmplus(400, trace_every=10)
    ts = time.perf_counter() - t1
    hit = next((i + 1 for i in range(9, len(trace), 10) if trace[i] < 1e-3), None)
    return {"value": nvec / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{nvec} vectors of A*y on the benchmark game (FP64 oracle, direct sum over "
                      f"terminals and hand pairs), {dt:.1f} s",
            "single_thread": {"value": 1.0 / per_vec, "unit": UNIT, "sample": "1 vector of A*y, 1 thread"},
            "solver": {"game": "tiny Kronecker game (6 one-card hands)", "method": "FP64 RM+ (oracle)",
                       "iters_to_1e-3_pot": hit, "seconds_for_400_iterations_with_checks": ts}}


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return
    spec = _workload()
    from oracle.oracle import OracleGame
    from paper_2112_03804_gb300 import synth
    og = OracleGame(spec)
    cores = os.cpu_count() or 1
    # one step = a bounded sample (one vector per core, both directions)
    ny = cores
    y = synth.simplex_vectors(og.sequences(1)["nact"], og.H, ny, seed=3)
    x = synth.simplex_vectors(og.sequences(0)["nact"], og.H, ny, seed=4)
    for _ in range(args.warmup):
        og.matvec_A(y[:1], nthreads=1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        og.matvec_A(y, nthreads=cores)
        og.matvec_AT(x, nthreads=cores)
    dt = time.perf_counter() - t0
    value = 2 * ny * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD + " (oracle sample: "
                                                             f"{ny}+{ny} vectors per step)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{ny} vectors of A*y and {ny} of A^T*x per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    from paper_2112_03804_gb300 import kps, synth

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    spec = _workload()
    g = kps.Game(spec)
    inf = g.info()
    H, hs, n1, n2 = inf["H"], inf["hs"], inf["n1"], inf["n2"]
    s = np.asarray(spec["strength"])
    order = np.lexsort((np.arange(len(s)), s))
    stream = torch.cuda.current_stream()
    # inputs: per-infoset simplex vectors (library hand order), resident in HBM
    def make(p, n, seed):
        v = synth.simplex_vectors(g.sequences(p)["nact"], H, BATCH, seed=seed + 1000 * rank,
                                  dtype=np.float32)
        out = np.zeros((BATCH, n, hs), dtype=np.float32)
        out[..., :H] = v
        return torch.from_numpy(out).cuda()
    y = make(1, n2, 3)
    x = make(0, n1, 4)
    oy = torch.empty((BATCH, n1, hs), device="cuda", dtype=torch.float32)
    ox = torch.empty((BATCH, n2, hs), device="cuda", dtype=torch.float32)
    g.upload(stream)

    def step():
        kps.matvec_A(g, y, oy, BATCH, stream=stream)
        kps.matvec_AT(g, x, ox, BATCH, stream=stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    # per-launch durations (CUDA events on the launching stream)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
            torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(args.steps):
            a, b, c = evs[i]
            a.record(stream)
            kps.matvec_A(g, y, oy, BATCH, stream=stream)
            b.record(stream)
            kps.matvec_AT(g, x, ox, BATCH, stream=stream)
            c.record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = t_start.elapsed_time(t_end)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ran = [g.kernel(0), g.kernel(1)]
    la = [e[0].elapsed_time(e[1]) for e in evs]
    lt = [e[1].elapsed_time(e[2]) for e in evs]
    # end to end through the host-buffer entry points (pinned host memory)
    e2e = None
    if not args.no_e2e:
        e2e = _e2e(g, y, x, oy, ox, stream, args, world)

    # the batched workload, sharded over every rank
    batched = None
    if not args.no_secondary:
        try:
            batched = measure_batch(args.games, 10, 3, rank, world, dist, solve_iters=50)
        except Exception as exc:   # reported, never silently dropped
            batched = {"error": f"{type(exc).__name__}: {exc}"}
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    _report(args, world, ms, la, lt, H, n1, n2, inf, clk, e2e, spec, ran, batched)
    if dist:
        dist.destroy_process_group()


BATCH_WORKLOAD = ("uneven river endgames in one persistent launch: boards of 3-5 cards (1176/1128/1081 "
                  "hands), 13-209 terminals, one fp32 vector per game and player")


def measure_batch(ngames: int, steps: int, warmup: int, rank: int = 0, world: int = 1, dist=None,
                  solve_iters: int = 0, fixed_shape=None):
    """Batched products over uneven games (one A and one A^T launch per
    step, captured in a CUDA graph), launch shape from the autotuner.  With
    `world` ranks the job is ngames * world games, split into contiguous
    ranges by kps_partition (weights 4 H (n1 + n2) from the specs); each
    rank builds and runs only its own games, the step time is the maximum
    over ranks and nothing on the data path communicates.  With solve_iters
    > 0 every rank then runs the batched FP32 solver on its games for that
    many iterations and the per-game exploitabilities are gathered in game
    order (the one collective)."""
    import torch
    from paper_2112_03804_gb300 import kps, shard, synth
    specs = synth.batch_specs(seed=4, n=ngames * world)
    bounds = kps.partition(shard.spec_weights(specs), world)
    lo, hi = int(bounds[rank]), int(bounds[rank + 1])
    games = [kps.Game(specs[i]) for i in range(lo, hi)]
    b = kps.Batch(games)
    stream = torch.cuda.current_stream()
    off = [b.offsets(p) for p in (0, 1)]
    vec = {}
    for p in (0, 1):
        flat = np.zeros(int(off[p][-1]), dtype=np.float32)
        for j, g in enumerate(games):
            inf = g.info()
            v = synth.simplex_vectors(g.sequences(p)["nact"], inf["H"], 1, seed=11 * (lo + j) + p,
                                      dtype=np.float32)[0]
            w = np.zeros((v.shape[0], inf["hs"]), dtype=np.float32)
            w[:, :inf["H"]] = v
            flat[off[p][j]:off[p][j + 1]] = w.reshape(-1)
        vec[p] = torch.from_numpy(flat).cuda()
    out = {p: torch.empty(int(off[p][-1]), device="cuda") for p in (0, 1)}
    if fixed_shape:
        kern, warps, grid, sched = (int(v) for v in fixed_shape.split(","))
        b.set_shape(kps.F32, warps, grid, sched, kern)
        shape = dict(b.shape(kps.F32), ms_per_pair=None)
    else:
        shape = b.tune(kps.F32, stream)
    # one step = A y and A^T x for every game, captured once as a graph
    b.matvec_A(vec[1], out[0], stream=stream)
    b.matvec_AT(vec[0], out[1], stream=stream)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        b.matvec_A(vec[1], out[0], stream=side)
        b.matvec_AT(vec[0], out[1], stream=side)
    torch.cuda.synchronize()
    for _ in range(max(warmup, 3)):
        graph.replay()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        graph.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # A*y reads n2 rows and writes n1 rows of H values per game, A^T*x reads
    # n1 and writes n2: 2 * 4 * H * (n1 + n2) bytes per game and step
    alg = 0.0
    for g in games:
        inf = g.info()
        alg += 8.0 * inf["H"] * (inf["n1"] + inf["n2"])
    if dist:
        t = torch.tensor([ms, alg], dtype=torch.float64, device="cuda")
        tmax = t.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        ms, alg = float(tmax[0]), float(t[1])
    total = ngames * world
    res = {"workload": BATCH_WORKLOAD, "games": total, "n_gpus": world,
           "matvecs_per_s": 2 * total / (ms / 1e3), "ms_per_step": ms, "alg_bytes_per_step": alg,
           "achieved_gbs": alg / (ms / 1e3) / 1e9,
           "launch_shape": {k: shape[k] for k in ("kernel", "warps", "grid", "schedule")},
           "tuned_ms_per_pair": shape["ms_per_pair"], "cuda_graph": True,
           "sharding": "contiguous game ranges by kps_partition (4 H (n1+n2) per game); no collective on the "
                       "data path; step time = max over ranks",
           "l2": "inputs larger than L2" if alg / world > 2.6e8 else "inputs smaller than L2"}
    if solve_iters > 0:
        s = kps.Solver(b, kps.F32)
        s.step(solve_iters)
        e = torch.zeros(len(games), dtype=torch.float64, device="cuda")
        s.exploitability(e)
        torch.cuda.synchronize()
        local = e.cpu().numpy()
        allv = shard.gather_scalars(local, np.diff(bounds)) if dist else local
        res["solver"] = {"iters": solve_iters, "storage": "f32", "games": int(len(allv)),
                         "expl_pot_mean": float(np.mean(allv)), "expl_pot_max": float(np.max(allv)),
                         "gathered": "per-game exploitabilities, game order" + (
                             " (all_gather over ranks)" if dist else "")}
        s.close()
    return res


def measure_turn(steps: int = 10, warmup: int = 3, seed: int = 2):
    """Products of a turn endgame (end of Sec. 3): the 52-card turn (4-card
    board, 1128 hands), a turn round with one pot-size bet and at most two
    aggressive actions, then 48 river cards and a river round with bets of
    0.5 and 1.0 pot: one batched launch over the turn round and its river
    blocks per product, FP32.  The inputs are smaller than L2, so L2 is
    flushed (a 512 MB write) before every step, outside the timed events."""
    import torch
    from paper_2112_03804_gb300 import kps, synth
    t = kps.Turn(synth.turn_spec(seed=seed))
    inf = t.info()
    off = [t.offsets(p) for p in (0, 1)]
    gen = torch.Generator(device="cuda").manual_seed(9)
    vec = {p: torch.rand(int(off[p][-1]), device="cuda", generator=gen) for p in (0, 1)}
    out = {p: torch.empty(int(off[p][-1]), device="cuda") for p in (0, 1)}
    stream = torch.cuda.current_stream()
    shape = t.tune(kps.F32, stream)
    flush = torch.empty(128 << 20, dtype=torch.float32, device="cuda")
    for _ in range(max(warmup, 3)):
        t.matvec_A(vec[1], out[0], stream=stream)
        t.matvec_AT(vec[0], out[1], stream=stream)
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t.matvec_A(vec[1], out[0], stream=stream)
        t.matvec_AT(vec[0], out[1], stream=stream)
        e1.record(stream)
        times.append((e0, e1))
    torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in times)
    # every game of the layout: one input read and one output written per product
    alg = 8.0 * inf["hs"] * (inf["n1"] + inf["n2"])
    peak, peak_kind = _peaks()
    gbs = alg / (ms / 1e3) / 1e9
    return {"workload": f"turn endgame: {inf['H']} hands, {inf['endings']} turn endings x 48 river cards = "
                        f"{inf['blocks']} river blocks, {inf['n1']}+{inf['n2']} sequences, fp32, one vector",
            "ms_per_step": ms, "turn_matvecs_per_s": 2 / (ms / 1e3), "alg_bytes_per_step": alg,
            "achieved_gbs": gbs, "frac_of_peak": gbs / peak, "peak_source": peak_kind,
            "launch_shape": {k: shape[k] for k in ("kernel", "warps", "grid", "schedule")},
            "l2": "flushed before every step (inputs smaller than L2)"}


def measure_factors(batch: int = BATCH, steps: int = 3, warmup: int = 2):
    """The three routes to A*y on the headline workload (river game, FP32):
    the fused kernel, Technique B's explicit factors with this library's
    sparse kernels, and the same factors with cuSPARSE (SpMM + SpSM), the
    paper's GPU route (Sec. 4).  Times per launch from CUDA events."""
    import torch
    from paper_2112_03804_gb300 import kps
    spec = _workload()
    g = kps.Game(spec)
    inf = g.info()
    H, hs, n1, n2 = inf["H"], inf["hs"], inf["n1"], inf["n2"]
    tb = kps.TechniqueB(g)
    sz = tb.sizes()
    gen = torch.Generator(device="cuda").manual_seed(5)
    y = torch.rand((batch, n2, hs), device="cuda", generator=gen)
    y[..., H:] = 0
    routes = {"fused": lambda o: kps.matvec_A(g, y, o, batch),
              "own_sparse": lambda o: tb.matvec(y, o, batch, backend=0),
              "cusparse": lambda o: tb.matvec(y, o, batch, backend=1)}
    ms, outs = {}, {}
    for name, fn in routes.items():
        o = torch.empty((batch, n1, hs), device="cuda")
        for _ in range(warmup):
            fn(o)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn(o)
        e1.record()
        torch.cuda.synchronize()
        ms[name] = e0.elapsed_time(e1) / steps
        outs[name] = o
    ref = outs["fused"].double()
    scale = float(ref.abs().max())
    diff = {k: float((outs[k].double() - ref).abs().max()) / scale for k in ("own_sparse", "cusparse")}
    total = sz["nnz_Ahat"] + sz["nnz_U"] + sz["nnz_M"] + sz["nnz_V"]
    return {"workload": WORKLOAD + ", A*y", "vectors": batch,
            "factor_nnz": {"Ahat": sz["nnz_Ahat"], "U": sz["nnz_U"], "M": sz["nnz_M"], "V": sz["nnz_V"],
                           "total": total, "explicit_A": inf["nnz_A"]},
            "ms_per_launch": ms, "matvecs_per_s": {k: batch / (v / 1e3) for k, v in ms.items()},
            "fused_speedup": {k: ms[k] / ms["fused"] for k in ("own_sparse", "cusparse")},
            "max_normwise_diff_vs_fused": diff}


def measure_libratus(batch: int = BATCH, steps: int = 5, warmup: int = 3):
    """The large-tree stress shape: the fused products on a 1081-hand river
    game with the Libratus betting menus (247 + 247 sequences, 329
    terminals), FP32, `batch` vectors per launch, inputs resident in HBM."""
    import torch
    from paper_2112_03804_gb300 import kps, synth
    g = kps.Game(synth.libratus_spec(seed=2))
    inf = g.info()
    H, hs, n1, n2 = inf["H"], inf["hs"], inf["n1"], inf["n2"]
    gen = torch.Generator(device="cuda").manual_seed(7)
    y = torch.rand((batch, n2, hs), device="cuda", generator=gen)
    x = torch.rand((batch, n1, hs), device="cuda", generator=gen)
    oa = torch.empty((batch, n1, hs), device="cuda")
    ot = torch.empty((batch, n2, hs), device="cuda")
    ms = {}
    for name, fn, i, o in (("A", kps.matvec_A, y, oa), ("AT", kps.matvec_AT, x, ot)):
        for _ in range(warmup):
            fn(g, i, o, batch)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn(g, i, o, batch)
        e1.record()
        torch.cuda.synchronize()
        ms[name] = e0.elapsed_time(e1) / steps
    alg = 4.0 * H * (n1 + n2) * batch
    peak, peak_kind = _peaks()
    gbs = alg / (statistics.mean(ms.values()) / 1e3) / 1e9
    return {"workload": f"river endgame with the Libratus betting menus, {H} hands, {n1}+{n2} sequences, "
                        f"{inf['T']} terminals, batch {batch}, fp32",
            "ms_per_launch": ms, "matvecs_per_s": 2 * batch / (sum(ms.values()) / 1e3),
            "alg_bytes_per_launch": alg, "achieved_gbs": gbs, "frac_of_peak": gbs / peak, "peak_source": peak_kind}


def measure_solver(target: float = 1e-3, block: int = 10, max_iters: int = 4000):
    """RM+ on the tiny Kronecker game (6 one-card hands) until the FP64
    exploitability of the averages is below `target` of the pot (checked
    every `block` iterations), per storage type; error against the
    FP64-storage run at every checkpoint; Discounted CFR (1.5, 0, 2) in FP32
    and BF16 storage beside it."""
    import torch
    from paper_2112_03804_gb300 import kps, synth
    spec = synth.tiny_spec()
    g = kps.Game(spec)
    b = kps.Batch([g])
    res = {}
    traces = {}
    names = {kps.F64: "f64", kps.F32: "f32", kps.BF16: "bf16", kps.F16: "f16"}
    runs = [(dt, 0) for dt in (kps.F64, kps.F32, kps.BF16, kps.F16)] + [(kps.F32, 1), (kps.BF16, 1)]
    for dt, method in runs:
        s = kps.Solver(b, dt)
        if method == 1:
            s.set_method(1, 1.5, 0.0, 2.0)
        e = torch.zeros(1, dtype=torch.float64, device="cuda")
        s.step(block)          # capture the graph outside the timed run
        s.reset()
        torch.cuda.synchronize()
        tr = []
        it = 0
        t0 = time.perf_counter()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        while it < max_iters:
            s.step(block)
            it += block
            s.exploitability(e)
            v = float(e.item())
            tr.append(v)
            if v < target:
                break
        ev1.record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        key = names[dt] + ("_dcfr" if method else "")
        traces[key] = tr
        res[key] = {"iters_to_target": it if tr[-1] < target else None, "final_expl": tr[-1],
                    "wall_ms": 1e3 * wall, "gpu_ms": ev0.elapsed_time(ev1)}
        s.close()
    ref = traces["f64"]
    for key in ("f32", "bf16", "f16"):
        n = min(len(ref), len(traces[key]))
        res[key]["max_abs_err_vs_f64"] = float(np.max(np.abs(np.array(traces[key][:n]) - np.array(ref[:n]))))
    return {"game": "tiny Kronecker game: 3 ranks x 2 suits, one card each (6 hands), 7+7 sequences",
            "target_expl_pot": target, "check_every": block, "by_storage": res}


def measure_libratus_solve(target: float = 1e-3, block: int = 10, max_iters: int = 5000, seeds=(2, 3, 4, 5)):
    """Time to solve one river endgame with the Libratus betting menus (1081
    hands, 247 + 247 sequences at a 1000-chip pot) to `target` of the pot:
    the paper's GPU claim is stated per endgame (Sec. 5).  DCFR (1.5, 0, 2)
    and RM+, FP32 storage, FP64 exploitability of the averages checked every
    `block` iterations (inside the timed region); one game per solver.  The
    same number of iterations is then timed again without the checks."""
    import torch
    from paper_2112_03804_gb300 import kps, synth
    out = {}
    for method, name in ((1, "dcfr_f32"), (0, "rmplus_f32")):
        rows = []
        for seed in seeds:
            g = kps.Game(synth.libratus_spec(seed=seed))
            b = kps.Batch([g])
            s = kps.Solver(b, kps.F32)
            if method == 1:
                s.set_method(1, 1.5, 0.0, 2.0)
            e = torch.zeros(1, dtype=torch.float64, device="cuda")
            s.step(block)
            s.exploitability(e)
            s.reset()
            torch.cuda.synchronize()
            it, v = 0, float("inf")
            t0 = time.perf_counter()
            while it < max_iters:
                s.step(block)
                it += block
                s.exploitability(e)
                v = float(e.item())
                if v < target:
                    break
            secs = time.perf_counter() - t0
            # the same iterations again without the checks (one graph launch)
            s.reset()
            s.step(it)
            s.reset()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            s.step(it)
            torch.cuda.synchronize()
            rows.append({"seed": seed, "iterations": it, "expl": v, "seconds": secs,
                         "seconds_without_checks": time.perf_counter() - t1})
            s.close()
        out[name] = rows
    return {"workload": "one river endgame with the Libratus betting menus per solve: 1081 hands, 247+247 "
                        "sequences, 329 terminals (synthetic strengths and beliefs)",
            "target_expl_pot": target, "check_every": block, "solves": out}


def measure_warmstart(train_games: int = 20480, per_game: int = 64, heldout: int = 512, epochs: int = 12,
                      kappa: float = 0.02, t0: int = 0, kappa_dcfr: float = 0.02, t0_dcfr: int = 5):
    """Learned warm start: equilibria of `train_games` river endgames (the
    1081-hand generator, solved by the batched FP32 solver to 1e-3 of the
    pot, 4096 per batch), `per_game` sampled (node, hand) queries each, the
    network trained by its own kernels; then iterations and wall time to
    1e-3 of the pot on `heldout` other endgames: FP32 cold start against
    warm starts in FP32 and in BF16 storage (inference included).  The
    warm-start parameters were chosen per method on 256 validation endgames
    (another seed than the held-out ones): RM+ kappa 0.02, t0 0; DCFR kappa
    0.02, t0 5 (grid kappa in {0.02, 0.1, 0.3}, t0 in {0, 5, 20, 50}; t0 > 0
    makes the discounts of the first iterations mild, so that the seeded
    regrets are not halved at once)."""
    import torch
    from paper_2112_03804_gb300 import kps, synth, warmstart as W

    def batch(seed, n):
        r = np.random.default_rng(seed)
        games = [kps.Game(synth.river_spec(seed=int(s))) for s in r.integers(1 << 62, size=n)]
        return kps.Batch(games)

    t_start = time.perf_counter()
    data, solve_s, iters = [], 0.0, []
    for i in range(0, train_games, 4096):
        b = batch(1000 + i, min(4096, train_games - i))
        s, it, ex, sec = W.solve(b, kps.F32, 1e-3, block=25, max_iters=2000)
        solve_s += sec
        iters.append(it)
        data.append(W.sample(b, s, per_game, seed=i))
        del s, b
        torch.cuda.empty_cache()
    D = W.concat(data)
    rows = int(D["X"].shape[0])
    mlp = kps.MLP(seed=1)
    t_train = time.perf_counter()
    hist = W.train(mlp, D, epochs=epochs, rows=8192, lr=1e-3, lr_decay=0.8)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t_train
    del D, data
    torch.cuda.empty_cache()
    hb = batch(5555, heldout)
    res = {}
    for method in (0, 1):
        for name, dt in (("f32", kps.F32), ("bf16", kps.BF16)):
            k_m, t_m = (kappa, t0) if method == 0 else (kappa_dcfr, t0_dcfr)
            r = W.compare(mlp, hb, dt, 1e-3, k_m, t_m, block=25, max_iters=2000, method=method)
            tag = ("dcfr_" if method else "") + name
            res["cold_" + tag] = r["cold"]
            res["warm_" + tag] = r["warm"]
    out = {"train_games": train_games, "train_rows": rows, "train_solve_seconds": solve_s,
           "train_solve_iterations": iters, "train_seconds": train_s, "epochs": epochs,
           "loss_first_last": [hist[0], hist[-1]], "heldout_games": heldout,
           "warm_start": {"rmplus": {"kappa": kappa, "t0": t0}, "dcfr": {"kappa": kappa_dcfr, "t0": t0_dcfr}}}
    out.update(res)
    out["total_seconds"] = time.perf_counter() - t_start
    return out


def measure_predict(ngames: int = 512, steps: int = 5, warmup: int = 3):
    """The fused warm-start predictor (`kps_warm_predict`) over every
    (game, player, node, hand) query of `ngames` river endgames (the
    1081-hand generator, seeds 0..ngames-1) with a freshly initialised
    network; CUDA events around each call (which includes its game- and
    node-part products and a sync)."""
    import torch
    from paper_2112_03804_gb300 import kps, synth, warmstart as W
    b = kps.Batch([kps.Game(synth.river_spec(seed=i)) for i in range(ngames)])
    mlp = kps.MLP(seed=1)
    for _ in range(max(warmup, 1)):
        W.predict(mlp, b)
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        W.predict(mlp, b)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    nq = kps.warm_num_queries(b)
    return {"workload": f"warm-start predictor over {ngames} river endgames (1081 hands, 43+43 sequences)",
            "queries": nq, "ms_per_call": statistics.median(ms), "queries_per_s": nq / (statistics.median(ms) / 1e3)}


def warmstart_summary(train_games: int = 2048, heldout: int = 128):
    """A scaled-down learned warm start for the headline line: the network
    trained on `train_games` solved endgames, then iterations and wall
    seconds to 1e-3 of the pot on `heldout` other endgames, per arm (RM+ and
    DCFR; cold FP32, cold BF16, warm FP32, warm BF16; inference included in
    the warm arms)."""
    r = measure_warmstart(train_games=train_games, heldout=heldout)
    arms = {}
    for k, v in r.items():
        if k.startswith(("cold_", "warm_")) and isinstance(v, dict) and "iterations" in v:
            arms[k] = [v["iterations"], round(v["seconds"], 4)]
    return {"train_games": train_games, "heldout_games": heldout, "loss_first_last": r["loss_first_last"],
            "arms_iterations_seconds": arms, "total_seconds": round(r["total_seconds"], 1)}


def _e2e(g, y, x, oy, ox, stream, args, world):
    import torch
    from paper_2112_03804_gb300 import kps
    mv_per_step = 2 * BATCH
    yh = y.cpu().pin_memory()
    xh = x.cpu().pin_memory()
    oyh = torch.empty(oy.shape, dtype=torch.float32).pin_memory()
    oxh = torch.empty(ox.shape, dtype=torch.float32).pin_memory()
    ne = max(2, min(args.steps, 5))
    kps.matvec_A_host(g, yh.data_ptr(), oyh.data_ptr(), BATCH, kps.F32, stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ne):
        kps.matvec_A_host(g, yh.data_ptr(), oyh.data_ptr(), BATCH, kps.F32, stream)
        kps.matvec_AT_host(g, xh.data_ptr(), oxh.data_ptr(), BATCH, kps.F32, stream)
    e2e_dt = time.perf_counter() - t0
    h2d = int(yh.numel() * 4 + xh.numel() * 4)
    d2h = int(oyh.numel() * 4 + oxh.numel() * 4)
    link = _host_link(yh, y, oyh, oy)
    # the step moves h2d + d2h bytes over the link; copies in both directions
    # overlap, so the bound is the concurrent rate
    bound = mv_per_step / ((h2d + d2h) / (link["both_gbs"] * 1e9))
    return {"value": mv_per_step * ne * world / e2e_dt, "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "host_link": dict(link, bound_matvecs_per_s=bound)}


def _host_link(hin, din, hout, dout, reps: int = 3):
    """Pinned host <-> device copy rates (GB/s) measured with CUDA events:
    host to device alone, device to host alone, and both at once on two
    streams (what the end-to-end step overlaps)."""
    import torch
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def timed(fn):
        best = None
        for _ in range(reps):
            torch.cuda.synchronize()
            t = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t
            best = dt if best is None else min(best, dt)
        return best

    n = hin.numel() * 4
    t_h2d = timed(lambda: din.copy_(hin, non_blocking=True))
    t_d2h = timed(lambda: hout.copy_(dout, non_blocking=True))

    def both():
        with torch.cuda.stream(s1):
            din.copy_(hin, non_blocking=True)
        with torch.cuda.stream(s2):
            hout.copy_(dout, non_blocking=True)

    t_both = timed(both)
    return {"h2d_gbs": n / t_h2d / 1e9, "d2h_gbs": hout.numel() * 4 / t_d2h / 1e9,
            "both_gbs": (n + hout.numel() * 4) / t_both / 1e9, "bytes_per_copy": int(n)}


def _report(args, world, ms, la, lt, H, n1, n2, inf, clk, e2e, spec, ran, batched=None):
    mv_per_step = 2 * BATCH
    value = mv_per_step * args.steps * world / (ms / 1e3)
    peak, peak_kind = _peaks()
    alg_bytes = 4.0 * H * (n1 + n2) * BATCH           # read one input, write one output, per vector
    avg_launch_s = statistics.mean(la + lt) / 1e3
    achieved = alg_bytes / avg_launch_s / 1e9
    kh = _kernel_hash()
    traffic = _traffic(kh) if ran == ["tma", "tma"] else None
    clk_sum = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": BATCH * world, "hands": H,
                   "sequences": [n1, n2], "terminals": inf["T"],
                   "l2": "inputs larger than L2 (191 MB per operand, no flush)",
                   "parallelism": f"dp{world}" if world > 1 else "single"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind,
                     "kernel": KERNEL, "kernel_paths": ran, "alg_bytes_per_launch": alg_bytes,
                     "launch_ms": {"A": statistics.mean(la), "AT": statistics.mean(lt)}},
        "clocks": clk_sum,
        "e2e": e2e,
        "gpu_launches": 2 * args.steps,
    }
    if e2e is None:
        del line["e2e"]
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(spec, args.cpu_seconds)
    if not args.no_secondary:
        # the batched and warm-start figures go last, where a tail of the
        # output keeps them
        for key, fn in (("solver", measure_solver),
                        ("technique_b", measure_factors), ("libratus", measure_libratus),
                        ("libratus_solve", lambda: measure_libratus_solve(seeds=(2, 3))),
                        ("turn", measure_turn), ("batched", lambda: batched),
                        ("warmstart", warmstart_summary)):
            try:
                line[key] = fn()
            except Exception as exc:   # reported, never silently dropped
                line[key] = {"error": f"{type(exc).__name__}: {exc}"}
    print(json.dumps(line), flush=True)


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        import torch
        rank, world, local = _dist()
        torch.cuda.set_device(local)
        dist = None
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl")
        res = measure_batch(args.games, args.steps, args.warmup, rank, world, dist, fixed_shape=args.batch_shape)
        if rank == 0:
            print(json.dumps(res), flush=True)
        if dist:
            dist.destroy_process_group()
    elif args.workload == "predict":
        import torch
        torch.cuda.set_device(_dist()[2])
        print(json.dumps(measure_predict(args.games, args.steps, args.warmup)), flush=True)
    elif args.workload == "warmstart":
        import torch
        torch.cuda.set_device(_dist()[2])
        print(json.dumps(measure_warmstart()), flush=True)
    elif args.workload == "solver":
        import torch
        torch.cuda.set_device(_dist()[2])
        print(json.dumps(measure_solver()), flush=True)
    elif args.workload == "libratus_solve":
        import torch
        torch.cuda.set_device(_dist()[2])
        print(json.dumps(measure_libratus_solve()), flush=True)
    elif args.workload == "libratus":
        import torch
        torch.cuda.set_device(_dist()[2])
        print(json.dumps(measure_libratus()), flush=True)
    elif args.workload == "turn":
        import torch
        torch.cuda.set_device(_dist()[2])
        print(json.dumps(measure_turn(steps=args.steps, warmup=args.warmup)), flush=True)
    elif args.workload == "factors":
        import torch
        torch.cuda.set_device(_dist()[2])
        print(json.dumps(measure_factors(steps=args.steps, warmup=args.warmup)), flush=True)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
