"""Autotuner of the fused VMC-step kernel's compile-time knobs, per lattice
shape and precision form (the paper tunes its kernels' blocking for the
irregular contraction shapes, Sec. "Implementation on Sunway TaihuLight").

Knobs: PEPS_QR_NB (Householder panel width; it also sets the panel capacity
of the blocked bidiagonalisation), PEPS_BA_FF / PEPS_BA_F64 (outputs per
thread along the A-only digit of a contraction), PEPS_MINB (blocks per SM
the register budget is set for; the default slot count is this many per SM),
PEPS_NT (threads per block), PEPS_BB_FF (outputs per thread along the
B-only digit), and the code paths PEPS_QR_PREFETCH (the next trailing column
of the blocked QR prefetched into L1), PEPS_BIDIAG_TPC (A'^T v of the
bidiagonalisation with one thread per column), PEPS_QR_TALL_PAIR (panels of
897 to 2048 rows held in the registers of two warps per column),
PEPS_CTR_PIPE (contraction operands loaded one reduction step ahead),
PEPS_QR_ACC (the QR's trailing update as compensated accumulations) and
PEPS_BIDIAG_FUSE (two barriers per bidiagonalisation step left out).  Search: the default, then one knob changed
at a time (a coordinate step); every candidate library is built (the C ABI
and the form's fused kernel recompiled, see build.py), then timed in its own
process on one wave of chains of the shape: one warm-up VMC step and --steps
timed steps (CUDA events), samples/s.  The fastest candidate is written to
tuning.json under the shape's key; build() then builds it and PepsContext
loads it for that shape.

    python -m paper_1806_03761_gb300.autotune --L 16 --D 6 --Dc 24 --precision mixed [--write]
"""
import argparse
import json
import os
import subprocess
import sys
import time

from . import build as B

CANDIDATES = [
    {},                                   # the default (pipelined contractions, compensated QR update)
    {"PEPS_QR_PREFETCH": 1},
    {"PEPS_BIDIAG_TPC": 1},
    {"PEPS_QR_PREFETCH": 1, "PEPS_BIDIAG_TPC": 1},
    {"PEPS_QR_PREFETCH": 1, "PEPS_BIDIAG_TPC": 1, "PEPS_QR_TALL_PAIR": 1},
    {"PEPS_QR_NB": 8},
    {"PEPS_QR_NB": 2},
    {"PEPS_BA_FF": 2, "PEPS_BA_F64": 1},
    {"PEPS_MINB": 1, "PEPS_NT": 512},     # one block of 16 warps per SM
    {"PEPS_MINB": 1},                     # one block of 8 warps per SM, 255 registers
    {"PEPS_QR_PREFETCH": 1, "PEPS_BIDIAG_TPC": 1, "PEPS_CTR_PIPE": 0, "PEPS_QR_ACC": 0},
    {"PEPS_QR_PREFETCH": 1, "PEPS_BIDIAG_TPC": 1, "PEPS_BB_FF": 4},
    {"PEPS_QR_PREFETCH": 1, "PEPS_BIDIAG_TPC": 1, "PEPS_MINB": 3},  # 3 blocks per SM, 80 registers
    {"PEPS_QR_PREFETCH": 1, "PEPS_BIDIAG_TPC": 1, "PEPS_QR_TALL_PAIR": 1, "PEPS_MINB": 3},
    {"PEPS_QR_PREFETCH": 1, "PEPS_BIDIAG_TPC": 1, "PEPS_MINB": 3, "PEPS_BA_FF": 2},
    {"PEPS_QR_PREFETCH": 1, "PEPS_BIDIAG_TPC": 1, "PEPS_MINB": 4},  # 4 blocks per SM, 64 registers
    {"PEPS_QR_PREFETCH": 1, "PEPS_BIDIAG_TPC": 1, "PEPS_MINB": 3, "PEPS_BIDIAG_FUSE": 1},
]


def knobs_of(delta):
    k = dict(B.DEFAULTS)
    k.update(delta)
    return k


def time_variant(lib_path, L, D, Dc, precision, chains, steps):
    """Samples/s of the fused VMC step of one library build, in a child
    process (each build is its own CUDA module)."""
    env = dict(os.environ, PEPS_LIB=lib_path)
    cmd = [sys.executable, "-m", "paper_1806_03761_gb300.autotune", "--child", "--L", str(L),
           "--D", str(D), "--Dc", str(Dc), "--precision", precision, "--chains", str(chains),
           "--steps", str(steps)]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env,
                       cwd=os.path.dirname(B.PKG), timeout=3600)
    if r.returncode != 0:
        return None, r.stderr[-2000:]
    for line in r.stdout.splitlines():
        if line.startswith("{"):
            return json.loads(line), ""
    return None, r.stdout[-2000:]


def child(args):
    import numpy as np
    import torch

    import paper_1806_03761_gb300 as P
    from synth import make_peps
    L, D, Dc = args.L, args.D, args.Dc
    A = torch.from_numpy(make_peps(L, D, 1234)).cuda()
    ctx = P.PepsContext(L, D, Dc, precision=args.precision)
    ctx.set_tensors(A)
    n = args.chains or ctx.slots
    state = ctx.sample(99, n, 0, 1, 1).contiguous()
    sums = ctx.new_sums()
    ctx.vmc_step(99, state, 2, sums=sums)  # warm-up
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(args.steps):
        ctx.vmc_step(99, state, 3 + k, sums=sums)
    t1.record(stream)
    torch.cuda.synchronize()
    rc, flags = ctx.sync_status()
    ms = t0.elapsed_time(t1) / args.steps
    print(json.dumps({"samples_per_s": n / (ms / 1e3), "ms_per_step": ms, "chains": n,
                      "slots": ctx.slots, "rc": rc, "flags": flags, "lib": P._lib.LIB_PATH
                      if not os.environ.get("PEPS_LIB") else os.environ["PEPS_LIB"]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, required=True)
    ap.add_argument("--D", type=int, required=True)
    ap.add_argument("--Dc", type=int, required=True)
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--chains", type=int, default=0, help="0: one wave of the candidate's slots")
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--child", action="store_true")
    ap.add_argument("--write", action="store_true", help="record the winner in tuning.json")
    ap.add_argument("--only", default="", help="comma-separated candidate numbers to time (default all)")
    ap.add_argument("--also", default="", help="record the winner also for these shapes, "
                    "'L,D,Dc;L,D,Dc' (shapes with the same per-site bond matrices)")
    args = ap.parse_args()
    if args.child:
        child(args)
        return
    B.build_default()
    import concurrent.futures as cf
    cands = [knobs_of(d) for d in CANDIDATES]
    if args.only:
        cands = [cands[int(q)] for q in args.only.split(",")]
    t0 = time.time()
    with cf.ThreadPoolExecutor(max_workers=len(cands)) as ex:
        libs = list(ex.map(lambda k: B.build_variant(k, args.precision), cands))
    print("built %d candidates in %.0f s" % (len(cands), time.time() - t0), flush=True)
    results = []
    for k, lib in zip(cands, libs):
        res, err = time_variant(lib, args.L, args.D, args.Dc, args.precision, args.chains, args.steps)
        tag = B.variant_tag(k, args.precision)
        if res is None or res.get("rc") != 0:
            print("%-40s failed: %s" % (tag, err.strip().splitlines()[-1:] if err else res), flush=True)
            continue
        print("%-40s %8.3f samples/s  (%d chains on %d slots)" % (tag, res["samples_per_s"],
                                                                  res["chains"], res["slots"]), flush=True)
        results.append((res["samples_per_s"], k, res))
    if not results:
        sys.exit(1)
    best = max(results, key=lambda x: x[0])
    key = "%dx%d_D%d_Dc%d_%s" % (args.L, args.L, args.D, args.Dc, args.precision)
    entry = {"precision": args.precision, "choice": best[1],
             "samples_per_s": {B.variant_tag(k, args.precision): r["samples_per_s"] for _, k, r in results},
             "chains": best[2]["chains"], "steps": args.steps}
    print(json.dumps({key: entry}), flush=True)
    if args.write:
        table = json.load(open(B.TUNING)) if os.path.exists(B.TUNING) else {}
        table[key] = entry
        for shp in filter(None, args.also.split(";")):
            L, D, Dc = (int(x) for x in shp.split(","))
            other = dict(entry, measured_on=key)
            table["%dx%d_D%d_Dc%d_%s" % (L, L, D, Dc, args.precision)] = other
        json.dump(table, open(B.TUNING, "w"), indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
