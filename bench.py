"""Benchmark of the per-sample PEPS hot path (PEPS++, arXiv:1806.03761) on GB300.

One step = one variational Monte Carlo iteration over a batch of B chains:
  1. peps_vmc_step (one fused launch per chain): the chain's configuration is
     evaluated -- amplitude, every J1/J2 flip ratio, E(S), Delta and the
     gradient sums (Steps 2, 4, 5; Eqs. ess, delta, gradients) -- and then
     advanced by one Metropolis sweep that reuses the lower environments just
     built (Steps 1-3, Fig. "contraction"),
  2. the deterministic reduction of the per-slot sums,
  3. peps_grad_step: the sign update of the GO step.
The metric is local-energy samples/s = B / device time of the step (chain
states and tensors resident in HBM).  `e2e` is the same metric through the
host-buffer entry point peps_vmc_step_host: every step copies the chain
states in from pinned host memory and the advanced states, the energies and
sum E out (up to E2E_MAX_STEPS steps after the timed ones).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
                    [--batch B] [--workload NAME] [--impl gb300|reference]

Under torchrun (N > 1) every rank runs its own B chains (weak scaling); the
gradient sums are all-reduced (the GO update's one exchange) and every rank
applies the same update.  --impl reference times the FP64 CPU oracle on a
bounded sample of the same workload.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import CONFIGS, make_peps  # noqa: E402

WORKLOAD = "16x16_D6_Dc24"
FP64_MAX_WARMUP, FP64_MAX_STEPS = 1, 3
E2E_MAX_STEPS = 3

# DRAM traffic of one launch of the fused kernel, bytes per chain (ncu
# dram__bytes_read.sum + dram__bytes_write.sum over a smaller launch of the
# same kernel, scaled by the chains it processed; the summaries under
# profiles/ give the command).  Keyed by (workload, precision form); only
# valid for the kernel the capture was taken from.
# DRAM bytes per chain of the fused kernel, from one ncu capture of a 32-chain
# launch, keyed by (workload, form, library variant): a kernel that has
# changed since its capture has no entry, and its line reports null
TRAFFIC_PER_CHAIN = {
    # 8.375 GB read + 46.217 GB written (profiles/peps_vmc_16x16_D6_Dc24_mixed_traffic.md:
    # the tuned variant, three blocks per SM, QR column prefetch, A'^T v one
    # thread per column, pipelined contractions, compensated QR update)
    ("16x16_D6_Dc24", "mixed", "mixed-PEPS_BIDIAG_TPC1-PEPS_MINB3-PEPS_QR_PREFETCH1"):
        (8375110144 + 46216911872) / 32,
    # the earlier variant (two blocks per SM, neither of the last two paths):
    # 8.162 GB read + 44.148 GB written
    ("16x16_D6_Dc24", "mixed", "mixed-PEPS_BIDIAG_TPC1-PEPS_CTR_PIPE0-PEPS_QR_ACC0-PEPS_QR_PREFETCH1"):
        (8162261504 + 44147782144) / 32,
}


def library_tag(ctx):
    """The variant tag of the library a context runs on ('default' for the
    default build)."""
    d = os.path.basename(os.path.dirname(getattr(ctx.lib, "_name", "") or ""))
    return "default" if d in ("", "lib") else d
METRIC = "local-energy samples/s at 16x16 D=6 Dc=24, mixed vs FP64; p50/p99 latency"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "fp32"])
    p.add_argument("--batch", type=int, default=0,
                   help="chains per rank (0: two waves of the persistent kernel's slots)")
    p.add_argument("--workload", default=WORKLOAD, choices=sorted(CONFIGS))
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--slots", type=int, default=0)
    p.add_argument("--dt", type=float, default=1e-3)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--mode", default="vmc",
                   choices=["vmc", "serving", "contraction", "correlations", "multi", "phases"],
                   help="serving: a Poisson stream of evaluation jobs through peps_server_*; "
                        "contraction: tensor-core vs CUDA-core column-step contractions; "
                        "phases: per-phase cycles of the fused VMC kernel")
    p.add_argument("--arrival-s", type=float, default=20.0,
                   help="serving: length of the arrival window per precision form")
    p.add_argument("--rates", default="0.25,0.5,1.0",
                   help="serving: job arrival rates per second (comma-separated sweep)")
    p.add_argument("--no-coverage", action="store_true",
                   help="serving: skip the run with one job of every shape")
    p.add_argument("--no-fp64-compare", action="store_true",
                   help="skip the one-wave FP64 step timed beside the mixed form")
    return p.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if "Active" in r[3 + k]
                          and "Not" not in r[3 + k]})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl"
        dist.init_process_group(backend)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline(cfg, A, n_samples, seed):
    """The FP64 oracle on a bounded sample of the workload on the host cores:
    n_samples configurations through one Metropolis sweep each and a full
    evaluation (E, Delta), timed on the wall clock.  Returns (samples/s,
    cores, oracle-counted flops per sample of the fused VMC step).

    The flops are counted by the oracle's operation counter while it runs:
    the evaluation plus the sweep, less the sweep's own rebuild of the lower
    environments (the fused step reuses the evaluation's) and less the strip
    rebuilds that follow an accepted exchange (an incremental sweep never
    needs them)."""
    import oracle
    from oracle import flops as oflops
    L, Dc = cfg["L"], cfg["Dc"]
    t0 = time.perf_counter()
    with oflops.counting() as cnt:
        out, _, _ = oracle.sample_chains(A, L, Dc, seed, n_samples, 0, 1, 1)
        oracle.evaluate_batch(A, out, L, Dc, want_delta=True)
    dt = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        cores = max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        pass
    counted = cnt.by_class(exclude_tags=("rebuild", "sweep_lower_envs"))
    flops = {k: v / n_samples for k, v in counted.items()}
    return n_samples / dt, cores, flops


def run_reference(args, cfg):
    """--impl reference: the oracle as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    A = make_peps(cfg["L"], cfg["D"], cfg["seed"], cfg["recipe"], cfg.get("eps", 1e-2))
    per_step = 1
    for _ in range(args.warmup):
        cpu_baseline(cfg, A, per_step, 7)
    times = []
    cores = 1
    for k in range(args.steps):
        t0 = time.perf_counter()
        _, cores, _ = cpu_baseline(cfg, A, per_step, 11 + k)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    value = per_step / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "samples/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "L": cfg["L"], "D": cfg["D"], "Dc": cfg["Dc"],
                       "batch_per_step": per_step, "recipe": cfg["recipe"]},
            "cpu_baseline": {"value": value, "unit": "samples/s", "cores": cores, "kind": "oracle",
                             "sample": "%d chain(s) x 1 Metropolis sweep + full evaluation per step" % per_step},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# The serving mix: every lattice side L in {8, 12, 16, 20, 24} with D in {4, 6, 8}
# and Dc = 4 D, 64 to 1024 configurations per request.  A shape's weight is
# inverse to its per-sample cost (about L^3 D^6: L rows of L sites, QR and SVD
# of (Dc D)-sized bond matrices), so every shape class brings the same work
# on average and the large lattices stay rare but present.
SERVING_SHAPES = [(L, D, 4 * D) for L in (8, 12, 16, 20, 24) for D in (4, 6, 8)]
SERVING_SAMPLES = [64, 128, 256, 512, 1024]


def serving_weights():
    w = np.array([1.0 / (L ** 3 * D ** 6) for (L, D, _) in SERVING_SHAPES])
    return w / w.sum()


def serving_stream(seed, rate, window_s):
    """Seeded Poisson arrivals: (arrival time, L, D, Dc, B, tensor seed)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    w = serving_weights()
    while True:
        t += rng.exponential(1.0 / rate)
        if t > window_s:
            return out
        L, D, Dc = SERVING_SHAPES[rng.choice(len(SERVING_SHAPES), p=w)]
        out.append((t, L, D, Dc, int(rng.choice(SERVING_SAMPLES)), int(rng.integers(1 << 30))))


def _serve(P, stream, prec, tensors, warm_shapes):
    """Submit the stream at its arrival times; returns per-job results."""
    srv = P.PepsServer()
    from synth import make_peps as mk, random_sz0_configs
    for (L, D, Dc) in warm_shapes:  # contexts of these shapes pooled
        srv.wait(srv.submit(mk(L, D, 1, "gauss"), random_sz0_configs(L, 8, 1), L, D, Dc, prec))
    t0 = time.perf_counter()
    ids = []
    for (ta, L, D, Dc, B, sd) in stream:
        dt = ta - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        A, S = tensors[sd]
        ids.append((srv.submit(A, S, L, D, Dc, prec), (L, D, Dc, B)))
    outs = [(srv.wait(i), shp) for i, shp in ids]
    srv.close()
    return outs


def _summary(outs):
    lat = np.array([o["latency_s"] for o, _ in outs])
    first = min(o["submit_s"] for o, _ in outs)
    last = max(o["done_s"] for o, _ in outs)
    n = sum(shp[3] for _, shp in outs)
    return {"value": n / (last - first), "unit": "samples/s", "jobs": len(outs), "samples": n,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "makespan_s": last - first, "errors": int(sum(o["status"] != 0 for o, _ in outs)),
            "shapes": sorted({"%dx%d D%d" % (s[0], s[0], s[1]) for _, s in outs})}


def run_serving(args):
    """--mode serving: the request loop under Poisson streams of the serving
    mix at each rate of --rates (mixed form, and FP64 on the same arrivals
    unless --no-fp64-compare), then a coverage run submitting one 64-sample
    job of every shape at once; one JSON line."""
    import torch  # noqa: F401  (CUDA context)

    import paper_1806_03761_gb300 as P
    from synth import make_peps as mk, random_sz0_configs
    rates = [float(x) for x in args.rates.split(",")]
    forms = ["mixed"] if args.no_fp64_compare else ["mixed", "fp64"]
    sweep = []
    for k, rate in enumerate(rates):
        stream = serving_stream(1234 + k, rate, args.arrival_s)
        tensors = {sd: (mk(L, D, sd % 1000, "gauss"), random_sz0_configs(L, B, sd % 997))
                   for (_, L, D, Dc, B, sd) in stream}
        warm = sorted({(L, D, Dc) for (_, L, D, Dc, _, _) in stream})
        row = {"rate_per_s": rate, "jobs": len(stream)}
        for prec in forms:
            row[prec] = _summary(_serve(P, stream, prec, tensors, warm))
        sweep.append(row)
        print("rate %.3g/s: %s" % (rate, json.dumps(row)), file=sys.stderr, flush=True)
    coverage = None
    if not args.no_coverage:
        stream = [(0.0, L, D, Dc, 64, 7000 + q) for q, (L, D, Dc) in enumerate(SERVING_SHAPES)]
        tensors = {sd: (mk(L, D, sd % 1000, "gauss"), random_sz0_configs(L, B, sd % 997))
                   for (_, L, D, Dc, B, sd) in stream}
        outs = _serve(P, stream, "mixed", tensors, [])
        coverage = {"%dx%d D%d Dc%d" % (shp[0], shp[0], shp[1], shp[2]):
                    {"latency_s": o["latency_s"], "status": o["status"]} for o, shp in outs}
    best = max(sweep, key=lambda r: r["mixed"]["value"])
    m = best["mixed"]
    line = {"metric": "serving: local-energy samples/s and p50/p99 request latency, Poisson job mix",
            "value": m["value"], "unit": "samples/s", "n_gpus": 1, "steps": m["jobs"], "warmup": 0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "ff (float-float on FP32)", "data": "synthetic",
            "config": {"workload": "serving mix", "shapes": [list(x) for x in SERVING_SHAPES],
                       "weights": [round(float(x), 6) for x in serving_weights()],
                       "samples_per_job": SERVING_SAMPLES, "rates_per_s": rates,
                       "arrival_window_s": args.arrival_s},
            "p50_s": m["p50_s"], "p99_s": m["p99_s"], "rate_sweep": sweep, "coverage": coverage}
    print(json.dumps(line), flush=True)


# Column-step contractions of the 16x16, D=6, Dc=24 workload as (M, N, K):
# C[M][N] = A[M][K] B[K][N] (strip step G2/G3 and the absorption's X,
# the strip step G1 and the absorption's S1, the strip closing step).
CONTRACTIONS = [(3456, 36, 36), (864, 144, 24), (864, 24, 144)]


def run_contraction(args):
    """--mode contraction: each column-step shape, batch = one contraction per
    slot of the persistent kernel, on the tensor cores (peps_tc_gemm: split +
    MMA, output in float-float and in FP64) and on the CUDA cores
    (peps_cc_gemm: contract() in float-float and in FP64, operands converted
    beforehand, output left in the form); device time per batch (CUDA
    events, mean of --steps after --warmup) and the worst error against the
    FP64 product relative to sum |a||b| on 4 batch elements."""
    import torch

    import paper_1806_03761_gb300 as P
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    batch = args.batch or 2 * sms
    rng = np.random.default_rng(2024)
    stream = torch.cuda.current_stream()
    rows = []
    for (M, N, K) in CONTRACTIONS:
        A = torch.from_numpy(rng.standard_normal((batch, M, K))).cuda()
        Bm = torch.from_numpy(rng.standard_normal((batch, K, N))).cuda()
        c = P.Contraction(M, N, K, batch, slices=7)
        An, Bn = A[:4].cpu().numpy(), Bm[:4].cpu().numpy()
        exact = np.einsum("bmk,bkn->bmn", An, Bn)
        scale = np.einsum("bmk,bkn->bmn", np.abs(An), np.abs(Bn))
        res = {"M": M, "N": N, "K": K, "batch": batch}
        for name, fn in (("tensor_cores_ff_out", lambda: c.tensor_cores(A, Bm, Cf, out="mixed")),
                         ("tensor_cores_fp64_out", lambda: c.tensor_cores(A, Bm, C)),
                         ("cuda_cores_ff", lambda: c.cuda_cores(A, Bm, "mixed", C, convert=False)),
                         ("cuda_cores_fp64", lambda: c.cuda_cores(A, Bm, "fp64", C, convert=False))):
            C = torch.empty(batch, M, N, dtype=torch.float64, device="cuda")
            Cf = torch.empty(batch, M, N, 2, dtype=torch.float32, device="cuda")
            if name.startswith("cuda"):  # operands converted once, outside the timing
                c.cuda_cores(A, Bm, "mixed" if name.endswith("ff") else "fp64", C, convert=True)
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            for _ in range(args.steps):
                fn()
            t1.record(stream)
            torch.cuda.synchronize()
            ms = t0.elapsed_time(t1) / max(args.steps, 1)
            if name.startswith("cuda"):
                c.cuda_cores(A, Bm, "mixed" if name.endswith("ff") else "fp64", C, convert=True)
            else:
                fn()
            torch.cuda.synchronize()
            got = C[:4].cpu().numpy() if name != "tensor_cores_ff_out" else \
                Cf[:4].cpu().numpy().astype(np.float64).sum(axis=-1)
            err = float(np.max(np.abs(got - exact) / scale))
            res[name] = {"ms": ms, "tflops": 2.0 * M * N * K * batch / (ms / 1e3) / 1e12, "err": err}
        res["status"] = int(c.status.item())
        rows.append(res)
    line = {"metric": "column-step contraction time, tensor cores (tcgen05, 7 BF16 slices) vs CUDA cores",
            "unit": "ms per batch", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "data": "synthetic (N(0,1) operands)", "config": {"workload": "16x16_D6_Dc24 column steps",
                                                              "batch": batch}, "shapes": rows}
    print(json.dumps(line), flush=True)


def run_correlations(args):
    """--mode correlations: <S_0 . S_m> for the centre source over one wave of
    configurations of the workload (peps_correlations; items (sample, source)
    one per block), and M^2 = m_s^2(pi, pi) over the bulk of an 8x8 lattice
    with every bulk site a source; device time (CUDA events, mean of --steps
    after --warmup)."""
    import torch

    import paper_1806_03761_gb300 as P
    from synth import make_peps, random_sz0_configs
    stream = torch.cuda.current_stream()
    rows = []
    for (wl, bulk_sources) in ((args.workload, False), ("8x8_D4_Dc16", True)):
        cfg = dict(CONFIGS[wl])
        L, D, Dc = cfg["L"], cfg["D"], cfg["Dc"]
        A = torch.from_numpy(make_peps(L, D, cfg["seed"], cfg["recipe"], cfg.get("eps", 1e-2))).cuda()
        ctx = P.PepsContext(L, D, Dc, precision=args.precision)
        ctx.set_tensors(A)
        if bulk_sources:
            lo, hi = (2, L - 2) if L > 4 else (0, L)
            sources = [i * L + j for i in range(lo, hi) for j in range(lo, hi)]
            B = max(1, ctx.slots // len(sources))
        else:
            sources = [(L // 2) * L + L // 2]
            B = ctx.slots
        spins = torch.from_numpy(random_sz0_configs(L, B, cfg.get("config_seed", 5))).cuda()
        for _ in range(args.warmup):
            r = ctx.correlations(spins, sources)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            r = ctx.correlations(spins, sources)
        t1.record(stream)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / max(args.steps, 1)
        row = {"workload": wl, "samples": B, "sources": len(sources), "ms": ms,
               "items_per_s": B * len(sources) / (ms / 1e3), "status": ctx.sync_status()[0]}
        if bulk_sources:
            row["M2"] = ctx.structure_factor(r["mean"], sources).item()
        else:
            row["centre_row"] = [float(x) for x in r["mean"][0].view(L, L)[L // 2].cpu()]
        rows.append(row)
        ctx.close()
    print(json.dumps({"metric": "spin-correlation items (sample, source) per second", "unit": "items/s",
                      "precision": args.precision, "steps": args.steps, "warmup": args.warmup,
                      "data": "synthetic", "runs": rows}), flush=True)


MULTI_JOBS = [  # (L, D, Dc, B): jobs of the serving mix's smaller shapes
    (16, 6, 24, 64), (12, 6, 24, 128), (16, 4, 16, 256), (12, 4, 16, 256), (8, 6, 24, 256),
    (8, 4, 16, 512), (20, 4, 16, 128), (8, 8, 32, 64)]


def run_multi(args):
    """--mode multi: the local energies of jobs of different shapes (MULTI_JOBS,
    mixed form), three ways: one persistent launch over all their samples
    (peps_local_energy_multi: a work queue of (job, sample) items on a pool
    of two slots per SM), every job's own launches on its own stream at the
    same time, and the jobs one after another; makespan (CUDA events)."""
    import torch

    import paper_1806_03761_gb300 as P
    from synth import make_peps, random_sz0_configs
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ctxs, spins = [], []
    for q, (L, D, Dc, B) in enumerate(MULTI_JOBS):
        c = P.PepsContext(L, D, Dc, precision="mixed", slots=min(B, 2 * sms))
        c.set_tensors(torch.from_numpy(make_peps(L, D, 300 + q)).cuda())
        ctxs.append(c)
        spins.append(torch.from_numpy(random_sz0_configs(L, B, 400 + q)).cuda())
    pool = P.PepsPool([j[:3] for j in MULTI_JOBS], precision="mixed", slots=2 * sms,
                      max_jobs=len(MULTI_JOBS))
    jobs = list(zip(ctxs, spins))
    main = torch.cuda.current_stream()
    streams = [torch.cuda.Stream() for _ in jobs]

    def one_launch():
        pool.local_energy(jobs)

    def concurrent():
        for (c, sp), st in zip(jobs, streams):
            st.wait_stream(main)
            with torch.cuda.stream(st):
                c.local_energy(sp)
        for st in streams:
            main.wait_stream(st)

    def sequential():
        for c, sp in jobs:
            c.local_energy(sp)

    res = {}
    for name, fn in (("one_launch", one_launch), ("concurrent_streams", concurrent),
                     ("sequential", sequential)):
        for _ in range(max(args.warmup, 1)):
            fn()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(main)
        for _ in range(args.steps):
            fn()
        t1.record(main)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / max(args.steps, 1)
        res[name] = {"ms": ms, "samples_per_s": sum(j[3] for j in MULTI_JOBS) / (ms / 1e3)}
    res["pool_status"] = pool.sync_status()[0]
    pool.close()
    for c in ctxs:
        c.close()
    print(json.dumps({"metric": "makespan of a batch of jobs of different shapes (local energies)",
                      "unit": "ms", "jobs": [list(j) for j in MULTI_JOBS], "precision": "mixed",
                      "steps": args.steps, "warmup": args.warmup, "data": "synthetic",
                      "results": res}), flush=True)


def run_phases(args):
    """--mode phases: per-phase clock64 cycles of the fused VMC kernel, from a
    PEPS_PHASES build of the library variant the tuning table names for the
    workload's shape (the same kernel otherwise): one wave of chains, one
    uncounted step, then one counted step; cycles per chain and shares of
    evaluation + sweep.  Not a throughput measurement."""
    import torch

    import paper_1806_03761_gb300 as P
    from paper_1806_03761_gb300 import build as B
    from synth import make_peps
    cfg = dict(CONFIGS[args.workload])
    L, D, Dc = cfg["L"], cfg["D"], cfg["Dc"]
    entry = json.load(open(B.TUNING)).get(P.tuning_key(L, D, Dc, args.precision)) \
        if os.path.exists(B.TUNING) else None
    knobs = dict(entry["choice"]) if entry else {}
    knobs["PEPS_PHASES"] = 1
    A = torch.from_numpy(make_peps(L, D, cfg["seed"], cfg["recipe"], cfg.get("eps", 1e-2))).cuda()
    ctx = P.PepsContext(L, D, Dc, precision=args.precision, variant=knobs)
    ctx.set_tensors(A)
    n = ctx.slots
    state = ctx.sample(0x5EED0000 + cfg["seed"], n, 0, 1, 1).contiguous()
    ctx.vmc_step(0x5EED0000 + cfg["seed"], state, 1)
    torch.cuda.synchronize()
    ctx.phase_cycles()
    ctx.vmc_step(0x5EED0000 + cfg["seed"], state, 2)
    torch.cuda.synchronize()
    ph = ctx.phase_cycles()
    rc, flags = ctx.sync_status()
    total = ph["eval"] + ph["sweep"]
    print(json.dumps({"metric": "fused VMC kernel cycles per chain by phase (clock64, one block)",
                      "workload": args.workload, "precision": args.precision, "chains": n,
                      "library": B.variant_tag(dict(B.DEFAULTS, **knobs), args.precision),
                      "mcycles_per_chain": {k: v / n / 1e6 for k, v in ph.items()},
                      "share_of_step": {k: v / total for k, v in ph.items()},
                      "status": {"rc": rc, "flags": flags}}), flush=True)
    ctx.close()


def main():
    args = parse()
    if args.mode == "phases":
        run_phases(args)
        return
    if args.mode == "multi":
        run_multi(args)
        return
    if args.mode == "contraction":
        run_contraction(args)
        return
    if args.mode == "correlations":
        run_correlations(args)
        return
    cfg = dict(CONFIGS[args.workload])
    if args.impl == "reference":
        run_reference(args, cfg)
        return
    if args.mode == "serving":
        run_serving(args)
        return
    import torch

    import paper_1806_03761_gb300 as P

    rank, world = dist_init()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    L, D, Dc = cfg["L"], cfg["D"], cfg["Dc"]
    N = L * L
    A_host = make_peps(L, D, cfg["seed"], cfg["recipe"], cfg.get("eps", 1e-2))
    A = torch.from_numpy(A_host).cuda()
    ctx = P.PepsContext(L, D, Dc, precision=args.precision, slots=args.slots)
    ctx.set_tensors(A)
    slots = ctx.slots
    variant = library_tag(ctx)
    full_batch = cfg.get("batch", cfg.get("chains", 256))
    B = args.batch or 2 * slots
    seed = 0x5EED0000 + cfg["seed"]
    from paper_1806_03761_gb300.dist import allreduce_sums, weak_scaling_plan
    chain_offset, B, M_total = weak_scaling_plan(rank, world, B)
    stream = torch.cuda.current_stream()
    # chains start from their Fisher-Yates states; every step continues them
    state = ctx.sample(seed, B, 0, 1, 1, chain_offset=chain_offset, first_sweep=1)
    state = state.view(B, N).contiguous()
    sums = ctx.new_sums()
    out = dict(e_loc=torch.empty(B, dtype=torch.float64, device="cuda"),
               log_abs=torch.empty(B, dtype=torch.float64, device="cuda"),
               sign=torch.empty(B, dtype=torch.int8, device="cuda"))
    counters = {"sweep": 2, "step": 0}

    def vmc_step(c, st, sm, o, n_total):
        # 1+2. evaluate every chain and advance it by one sweep (one launch),
        #      then reduce the per-slot sums
        c.vmc_step(seed, st, counters["sweep"], chain_offset=chain_offset, sums=sm, out=o)
        counters["sweep"] += 1
        # 3. GO update (sums all-reduced across ranks first)
        allreduce_sums(sm, world)
        c.grad_step(sm, n_total, args.dt, seed, counters["step"], A)
        counters["step"] += 1

    for _ in range(args.warmup):
        vmc_step(ctx, state, sums, out, M_total)
    torch.cuda.synchronize()
    barrier(world)

    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    barrier(world)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    marks = []
    for _ in range(args.steps):
        k1, k2 = ev(), ev()
        k1.record(stream)
        vmc_step(ctx, state, sums, out, M_total)
        k2.record(stream)
        marks.append((k1, k2))
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    rc, flags = ctx.sync_status()
    step_ms = [a.elapsed_time(b) for a, b in marks]
    dev_ms = max_over_ranks(float(np.sum(step_ms)), world) / max(args.steps, 1)

    # end to end through the host-buffer entry point: every step copies the
    # chain states in from pinned host memory and the advanced states, the
    # energies and sum E back (peps_vmc_step_host), then the GO update
    e2e_steps = max(1, min(args.steps, E2E_MAX_STEPS))
    host_state = torch.empty(B, N, dtype=torch.uint8).pin_memory()
    host_state.copy_(state)
    host_e = torch.empty(B, dtype=torch.float64).pin_memory()
    host_se = torch.empty(1, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    barrier(world)
    e2e_marks = []
    for _ in range(e2e_steps):
        k0, k3 = ev(), ev()
        k0.record(stream)
        ctx.vmc_step_host(seed, host_state, counters["sweep"], sums, host_e, host_se,
                          chain_offset=chain_offset)
        counters["sweep"] += 1
        allreduce_sums(sums, world)
        ctx.grad_step(sums, M_total, args.dt, seed, counters["step"], A)
        counters["step"] += 1
        k3.record(stream)
        stream.synchronize()
        e2e_marks.append((k0, k3))
    e2e_ms = [a.elapsed_time(b) for a, b in e2e_marks]
    e2e_total = max_over_ranks(float(np.sum(e2e_ms)), world) / e2e_steps
    rc2, flags2 = ctx.sync_status()
    rc, flags = rc or rc2, flags | flags2

    # the mixed form against the FP64 GPU path: the same batch of chains and
    # the same step, timed the same way (warm-up and timed steps capped at
    # FP64_MAX_WARMUP / FP64_MAX_STEPS: an FP64 step takes about twice as long)
    fp64 = None
    if args.precision == "mixed" and not args.no_fp64_compare and world == 1:
        c64 = P.PepsContext(L, D, Dc, precision="fp64", slots=args.slots)
        A64 = A.clone()
        c64.set_tensors(A64)
        st64 = state.clone()
        s64 = c64.new_sums()
        o64 = dict(e_loc=torch.empty(B, dtype=torch.float64, device="cuda"),
                   log_abs=torch.empty(B, dtype=torch.float64, device="cuda"),
                   sign=torch.empty(B, dtype=torch.int8, device="cuda"))
        cnt64 = {"sweep": counters["sweep"], "step": counters["step"]}

        def step64():
            c64.vmc_step(seed, st64, cnt64["sweep"], chain_offset=chain_offset, sums=s64, out=o64)
            c64.grad_step(s64, M_total, args.dt, seed, cnt64["step"], A64)
            cnt64["sweep"] += 1
            cnt64["step"] += 1

        w64, k64 = min(args.warmup, FP64_MAX_WARMUP), max(1, min(args.steps, FP64_MAX_STEPS))
        for _ in range(w64):
            step64()
        torch.cuda.synchronize()
        ms64 = []
        for _ in range(k64):
            a64, b64 = ev(), ev()
            a64.record(stream)
            step64()
            b64.record(stream)
            torch.cuda.synchronize()
            ms64.append(a64.elapsed_time(b64))
        rc64, fl64 = c64.sync_status()
        t64 = float(np.mean(ms64))
        fp64 = {"value": B / (t64 / 1e3), "unit": "samples/s", "batch": B,
                "ms_per_step": t64, "steps": k64, "warmup": w64, "slots": c64.slots,
                "p50_ms": float(np.percentile(ms64, 50)), "p99_ms": float(np.percentile(ms64, 99)),
                "status": {"rc": rc64, "flags": fl64}}
        c64.close()

    if rank != 0:
        return
    value = M_total / (dev_ms / 1e3)
    cpu, oflops = None, None
    if not args.no_cpu_baseline and world == 1:
        v, cores, oflops = cpu_baseline(cfg, A_host, 1, 99)
        cpu = {"value": v, "unit": "samples/s", "cores": cores, "kind": "oracle",
               "sample": "1 chain x 1 Metropolis sweep + full evaluation (E, Delta)"}
    # roofline of the dominant kernel, the fused evaluation + sweep kernel (the
    # per-slot reduction and the GO update inside the bracket are < 0.1 % of it).
    # Numerator: the oracle's operation count of one fused step per chain,
    # counted live above (falls back to the kernels' own model without it).
    model_flops = P.flops_per_sample(L, D, Dc, precision=args.precision, what="vmc")
    flops = sum(oflops.values()) if oflops else model_flops
    sec = float(np.mean(step_ms)) / 1e3
    achieved = flops * B / sec / 1e12
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    sm_max = clk.get("sm_max_mhz") or 2070.0
    if args.precision == "fp64":
        peak, unit = sms * 2 * 2 * sm_max * 1e6 / 1e12, "TFLOP/s (FP64 pipe: 2 DFMA/clk/SM)"
    elif args.precision == "mixed":
        # float-float multiply-add = 12 FP32 instructions on 128 lanes per SM
        peak, unit = sms * 128 * 2 * sm_max * 1e6 / 12 / 1e12, "TFLOP/s (FP32 pipe / 12 per ff MAC)"
    else:
        peak, unit = sms * 128 * 2 * sm_max * 1e6 / 1e12, "TFLOP/s (FP32 pipe)"
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak,
            "traffic": (TRAFFIC_PER_CHAIN[(args.workload, args.precision, variant)] * B
                        if (args.workload, args.precision, variant) in TRAFFIC_PER_CHAIN else None),
            "kernel": "peps_vmc_kernel",
            "flops_per_sample": flops,
            "flops_source": "oracle operation counter (1 chain)" if oflops else "kernel model",
            "flops_per_sample_by_class": oflops,
            "flops_per_sample_kernel_model": model_flops,
            "frac_kernel_model": model_flops * B / sec / 1e12 / peak,
            "peak_source": "unit counts x %d SMs (device) x sampled max SM clock" % sms}
    lat = sorted(step_ms)
    h2d, d2h = B * N, B * N + B * 8 + 8
    metric = METRIC if args.workload == WORKLOAD else \
        "local-energy samples/s at %dx%d D=%d Dc=%d (fused VMC step)" % (L, L, D, Dc)
    line = {"metric": metric, "value": value, "unit": "samples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dev_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"mixed": "ff (float-float on FP32)", "fp64": "f64", "fp32": "f32"}[args.precision],
            "data": "synthetic",
            "config": {"workload": args.workload, "L": L, "D": D, "Dc": Dc, "batch_per_gpu": B,
                       "workload_batch": full_batch, "slots": slots,
                       "recipe": cfg["recipe"], "precision": args.precision,
                       "step": "fused evaluate (E, ratios, Delta sums) + 1 Metropolis sweep, slot "
                               "reduction, GO update",
                       "l2": "per-chain working sets (%d slots) exceed L2 (129 MB)" % slots,
                       "library": variant},
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "latency_per": "batch (one step)",
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": M_total / (e2e_total / 1e3), "unit": "samples/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": e2e_total, "steps": e2e_steps,
                    "call": "peps_vmc_step_host (pinned host buffers) + peps_grad_step"},
            "fp64_gpu": fp64,
            "gpu_launches": 3 * (args.steps + e2e_steps), "clocks": clk,
            "status": {"rc": rc, "flags": flags}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
