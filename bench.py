"""Benchmark of the per-sample PEPS hot path (PEPS++, arXiv:1806.03761) on GB300.

One step = one variational Monte Carlo iteration over a batch of B chains:
  1. peps_sample_batch: one Metropolis sweep per chain from its current state
     (Fig. "contraction", Steps 1-3),
  2. peps_evaluate: amplitudes, every J1/J2 flip ratio, E(S), Delta and the
     gradient sums over the batch (Steps 2, 4, 5; Eqs. ess, delta, gradients),
  3. peps_grad_step: the sign update of the GO step.
The metric is local-energy samples/s = B / step time (device-resident inputs).

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
METRIC = "local-energy samples/s at 16x16 D=6 Dc=24, mixed vs FP64; p50/p99 latency"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "fp32"])
    p.add_argument("--batch", type=int, default=0, help="chains per rank (0: the workload's batch)")
    p.add_argument("--workload", default=WORKLOAD, choices=sorted(CONFIGS))
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--slots", type=int, default=0)
    p.add_argument("--dt", type=float, default=1e-3)
    p.add_argument("--no-cpu-baseline", action="store_true")
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
    evaluation (E, Delta), timed on the wall clock."""
    import oracle
    L, Dc = cfg["L"], cfg["Dc"]
    t0 = time.perf_counter()
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
    return n_samples / dt, cores


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
        _, cores = cpu_baseline(cfg, A, per_step, 11 + k)
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


def main():
    args = parse()
    cfg = dict(CONFIGS[args.workload])
    if args.impl == "reference":
        run_reference(args, cfg)
        return
    import torch

    import paper_1806_03761_gb300 as P

    rank, world = dist_init()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    L, D, Dc = cfg["L"], cfg["D"], cfg["Dc"]
    B = args.batch or cfg.get("batch", cfg.get("chains", 256))
    N = L * L
    A_host = make_peps(L, D, cfg["seed"], cfg["recipe"], cfg.get("eps", 1e-2))
    A = torch.from_numpy(A_host).cuda()
    ctx = P.PepsContext(L, D, Dc, precision=args.precision, slots=args.slots)
    ctx.set_tensors(A)
    seed = 0x5EED0000 + cfg["seed"]
    from paper_1806_03761_gb300.dist import allreduce_sums, shard
    chain_offset, B = shard(rank, world, B)
    # chains start from their Fisher-Yates states; every step continues them
    state = ctx.sample(seed, B, 0, 1, 1, chain_offset=chain_offset, first_sweep=1)
    state = state.view(B, N).contiguous()
    sweep = [2]
    sums = ctx.new_sums()
    out = dict(e_loc=torch.empty(B, dtype=torch.float64, device="cuda"),
               log_abs=torch.empty(B, dtype=torch.float64, device="cuda"),
               sign=torch.empty(B, dtype=torch.int8, device="cuda"))
    spins = torch.empty(B, N, dtype=torch.uint8, device="cuda")
    step_no = [0]
    stream = torch.cuda.current_stream()
    ev_eval = []

    def vmc_step(record=False):
        # 1. one Metropolis sweep per chain (continues from `state`)
        P_lib = ctx.lib
        rc = P_lib.peps_sample_batch(ctx.h, seed, B, chain_offset, 0, 1, 1, sweep[0],
                                     P._ptr(spins), P._ptr(state), None, ctx._stream())
        ctx._check(rc)
        sweep[0] += 1
        # 2. energies, ratios and Delta sums
        if record:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        ctx.evaluate(spins, sums=sums, out=out)
        if record:
            e1.record(stream)
            ev_eval.append((e0, e1))
        # 3. GO update (sums all-reduced across ranks first)
        allreduce_sums(sums, world)
        ctx.grad_step(sums, B * world, args.dt, seed, step_no[0], A)
        step_no[0] += 1

    for _ in range(args.warmup):
        vmc_step()
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    barrier(world)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    step_ms = []
    t_start.record(stream)
    for _ in range(args.steps):
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        vmc_step(record=True)
        s1.record(stream)
        step_ms.append((s0, s1))
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    total_ms = max_over_ranks(total_ms, world)
    per_step = [a.elapsed_time(b) for a, b in step_ms]
    eval_ms = [a.elapsed_time(b) for a, b in ev_eval]
    rc, flags = ctx.sync_status()

    # end to end through the public API with host buffers: pinned host chain
    # states in, energies and the energy sum out, every step
    e2e = None
    if args.steps > 0:
        host_state = torch.empty(B, N, dtype=torch.uint8).pin_memory()
        host_state.copy_(state)
        host_e = torch.empty(B, dtype=torch.float64).pin_memory()
        host_se = torch.empty(1, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            state.copy_(host_state, non_blocking=True)
            vmc_step()
            host_e.copy_(out["e_loc"], non_blocking=True)
            host_se.copy_(sums[2], non_blocking=True)
            torch.cuda.synchronize()
            host_state.copy_(state)
        e2e_ms = 1e3 * (time.perf_counter() - t0) / args.steps
        e2e_ms = max_over_ranks(e2e_ms, world)
        e2e = {"value": B * world / (e2e_ms / 1e3), "unit": "samples/s",
               "h2d_bytes_per_step": B * N, "d2h_bytes_per_step": B * 8 + 8}

    if rank != 0:
        return
    ms = total_ms / max(args.steps, 1)
    value = B * world / (ms / 1e3)
    # roofline of the dominant kernel (the evaluation kernel)
    flops = P.flops_per_sample(L, D, Dc, precision=args.precision)
    ev = float(np.mean(eval_ms)) if eval_ms else float("nan")
    achieved = flops * B / (ev / 1e3) / 1e12
    sm_max = clk.get("sm_max_mhz") or 2070.0
    if args.precision == "fp64":
        peak, unit = 152 * 2 * 2 * sm_max * 1e6 / 1e12, "TFLOP/s (FP64 pipe: 2 DFMA/clk/SM)"
    elif args.precision == "mixed":
        # float-float multiply-add = 12 FP32 instructions on 128 lanes per SM
        peak, unit = 152 * 128 * 2 * sm_max * 1e6 / 12 / 1e12, "TFLOP/s (FP32 pipe / 12 per ff MAC)"
    else:
        peak, unit = 152 * 128 * 2 * sm_max * 1e6 / 1e12, "TFLOP/s (FP32 pipe)"
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "traffic": None, "kernel": "peps_eval_kernel",
            "flops_per_sample": flops, "eval_ms": ev}
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        v, cores = cpu_baseline(cfg, A_host, 1, 99)
        cpu = {"value": v, "unit": "samples/s", "cores": cores, "kind": "oracle",
               "sample": "1 chain x 1 Metropolis sweep + full evaluation (E, Delta)"}
    lat = sorted(per_step)
    line = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"mixed": "ff (float-float on FP32)", "fp64": "f64", "fp32": "f32"}[args.precision],
            "data": "synthetic",
            "config": {"workload": args.workload, "L": L, "D": D, "Dc": Dc, "batch_per_gpu": B,
                       "recipe": cfg["recipe"], "precision": args.precision,
                       "step": "1 Metropolis sweep + evaluate (E, ratios, Delta sums) + GO update",
                       "l2": "inputs and per-sample working sets exceed L2 (129 MB)"},
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "local_energy_samples_per_s": B / (ev / 1e3) if eval_ms else None,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": 4 * args.steps, "clocks": clk,
            "status": {"rc": rc, "flags": flags}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
