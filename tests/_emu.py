"""Build the library's kernels and C ABI for the host (tests/host/emu): every
kernel launch `k<<<grid, block, ...>>>(args)` of the CUDA translation units
is rewritten to `emu_launch(grid, block, [=] { k(args); })`, and the units
are compiled with g++ against the emulated runtime header.  Only tests use
it; the product is the CUDA build."""
import concurrent.futures as cf
import os
import re
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1806_03761_gb300", "csrc")
EMU = os.path.join(HERE, "host", "emu")
# the units without tensor-core or static-scratch code
UNITS = ["peps_api.cu", "peps_k_misc.cu"] + [
    "peps_k_%s_%s.cu" % (k, f) for k in ("eval", "sample", "vmc") for f in ("f64", "ff", "f32")] + [
    "peps_k_%s_%s.cu" % (k, f) for k in ("corr", "multi") for f in ("f64", "ff")] + ["peps_server.cu"]

_LAUNCH = re.compile(r"(\b[A-Za-z_]\w*(?:<[^<>;]*>)?)\s*<<<([^>]*)>>>\s*\((.*?)\)\s*;", re.S)


def rewrite(src):
    def sub(m):
        cfg = [x.strip() for x in m.group(2).split(",")]
        return "emu_launch(dim3(%s), dim3(%s), [=]() { %s(%s); });" % (cfg[0], cfg[1], m.group(1),
                                                                   m.group(3))
    return _LAUNCH.sub(sub, src)


def build(outdir, defines=(), sanitize=False, units=None):
    """Compile and link the emulated library into outdir; returns its path.
    sanitize: instrument it with AddressSanitizer (the process that loads it
    needs libasan preloaded)."""
    gxx = shutil.which("g++")
    if not gxx:
        raise RuntimeError("no g++")
    os.makedirs(outdir, exist_ok=True)
    opt = ["-O1", "-g", "-fsanitize=address", "-fno-omit-frame-pointer"] if sanitize else ["-O2"]
    # -U_FORTIFY_SOURCE: the fibers switch stacks with _longjmp, which the
    # fortified longjmp would refuse
    flags = [gxx, "-std=c++20", "-ffp-contract=off", "-fPIC", "-pthread", "-w", "-U_FORTIFY_SOURCE",
             "-I", EMU, "-I", CSRC, "-I", os.path.join(ROOT, "include")] + opt + \
        ["-D%s" % d for d in defines]
    jobs = []
    for u in (units or UNITS):
        dst = os.path.join(outdir, u[:-3] + ".cpp")
        with open(os.path.join(CSRC, u)) as f:
            text = rewrite(f.read())
        with open(dst, "w") as f:
            f.write('#include "cuda_runtime.h"\n' + text)
        jobs.append((dst, dst[:-4] + ".o"))
    jobs.append((os.path.join(EMU, "emu.cpp"), os.path.join(outdir, "emu.o")))
    if units:
        jobs.append((os.path.join(EMU, "launch_stubs.cpp"), os.path.join(outdir, "launch_stubs.o")))

    def cc(j):
        r = subprocess.run(flags + ["-c", j[0], "-o", j[1]], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("g++ failed on %s:\n%s" % (j[0], r.stderr[-4000:]))
        return j[1]
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(cc, jobs))
    lib = os.path.join(outdir, "libpeps_emu.so")
    r = subprocess.run([gxx, "-shared", "-pthread"] + (["-fsanitize=address"] if sanitize else []) +
                       ["-o", lib] + objs, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stderr[-4000:])
    return lib


def _asan_cases(lib_path):
    """Evaluation, sampling and the fused step of both forms at 4x4, D=3,
    Dc=4 on the instrumented library (run in a process with libasan
    preloaded); prints each case's energy error against the oracle."""
    import ctypes
    import sys
    sys.path.insert(0, ROOT)
    import numpy as np
    import oracle
    from paper_1806_03761_gb300 import _lib as B
    from synth import make_peps, random_sz0_configs
    from tests.test_emu_parity import Ctx
    lib = ctypes.CDLL(lib_path)
    for name, (res, args) in B._SIGS.items():
        if hasattr(lib, name):
            fn = getattr(lib, name)
            fn.restype, fn.argtypes = res, args
    for prec in ("fp64", "mixed"):
        c = Ctx(lib, 4, 3, 4, prec, slots=2)
        A = make_peps(4, 3, seed=7)
        c.set_tensors(A)
        sp = random_sz0_configs(4, 2, seed=8)
        r = c.evaluate(sp)
        st, _ = c.sample(99, 2, 1, 1, 1)
        c.vmc_step(99, st.copy(), 3)
        ref = oracle.evaluate_batch(A, sp, 4, 4)
        print(prec, "status", c.status(), "energy error %.2e" % np.max(np.abs(r["e_loc"] - ref["e_loc"])),
              flush=True)
        c.close()


def count_ops(L, D, Dc, chains=1, knobs=(), what="EMU_COUNT_OPS"):
    """FP32 operations per phase of one fused VMC step of the float-float
    form (a build with the phase counters whose clock is the emulation's
    count of FP32 rounding operations and fmaf), per chain, with the
    kernels' own flop count (12 FP32 operations per float-float
    multiply-add, 2 flops)."""
    import ctypes
    import sys
    import tempfile
    sys.path.insert(0, ROOT)
    import numpy as np
    import paper_1806_03761_gb300 as P
    from paper_1806_03761_gb300 import _lib as B
    from synth import make_peps, random_sz0_configs
    from tests.test_emu_parity import Ctx
    path = build(tempfile.mkdtemp(prefix="emu_ops"),
                 defines=[what, "PEPS_PHASES=1"] + list(knobs),
                 units=["peps_api.cu", "peps_k_misc.cu", "peps_k_vmc_ff.cu"])
    lib = ctypes.CDLL(path)
    for name, (res, args) in B._SIGS.items():
        if hasattr(lib, name):
            fn = getattr(lib, name)
            fn.restype, fn.argtypes = res, args
    c = Ctx(lib, L, D, Dc, "mixed", slots=1)
    c.set_tensors(make_peps(L, D, seed=3))
    state = np.ascontiguousarray(random_sz0_configs(L, chains, seed=4))
    n_ph = len(P.PepsContext.PHASES)
    buf = (ctypes.c_uint64 * n_ph)()
    n = ctypes.c_int32(0)
    lib.peps_phase_cycles(c.h, buf, n_ph, ctypes.byref(n))
    c.vmc_step(5, state, 2)
    lib.peps_phase_cycles(c.h, buf, n_ph, ctypes.byref(n))
    assert n.value == n_ph and c.status() == (0, 0)
    c.close()
    ops = {k: buf[i] / chains for i, k in enumerate(P.PepsContext.PHASES)}
    return ops, P.flops_per_sample(L, D, Dc, "mixed", "vmc")


if __name__ == "__main__":
    # python -m tests._emu --asan-check: the emulated kernels under
    # AddressSanitizer (any out-of-bounds access of a buffer aborts the run)
    import sys
    import tempfile
    if sys.argv[1:2] == ["--asan-check"]:
        path = build(tempfile.mkdtemp(prefix="emu_asan"), sanitize=True)
        libasan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True,
                                 text=True).stdout.strip()
        env = dict(os.environ, LD_PRELOAD=libasan, ASAN_OPTIONS="detect_leaks=0")
        r = subprocess.run([sys.executable, "-c", "from tests._emu import _asan_cases; _asan_cases(%r)" % path],
                           cwd=ROOT, env=env)
        sys.exit(r.returncode)
    if sys.argv[1:2] == ["--count-ops"]:
        # python -m tests._emu --count-ops L D Dc [KNOB=value ...]
        L, D, Dc = (int(x) for x in sys.argv[2:5])
        ops, model = count_ops(L, D, Dc, knobs=sys.argv[5:])
        bars, _ = count_ops(L, D, Dc, knobs=sys.argv[5:], what="EMU_COUNT_BARRIERS")
        total = ops["eval"] + ops["sweep"]
        print("%dx%d D=%d Dc=%d, float-float, one fused VMC step per chain %s" % (L, L, D, Dc,
                                                                             " ".join(sys.argv[5:])))
        print("FP32 operations %.4g (%.4g flop-equivalent at 12 per multiply-add); "
              "kernel flop count %.4g; ratio %.3f; block barriers %d" %
              (total, total / 6, model, total / 6 / model, bars["eval"] + bars["sweep"]))
        print("  %-9s %11s %7s %10s %14s" % ("phase", "FP32 ops", "share", "barriers",
                                              "ops/barrier"))
        for k, v in ops.items():
            b = bars[k]
            print("  %-9s %11.4g %6.1f%% %10d %14.4g" % (k, v, 100.0 * v / total, b,
                                                          v / b if b else float("nan")))
