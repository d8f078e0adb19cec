"""Build libpeps.so (the C ABI of include/peps.h) for sm_103a with nvcc.

Every translation unit in csrc/ is compiled in parallel and the objects are
linked into paper_1806_03761_gb300/lib/libpeps.so.  A unit is rebuilt when
it or any header in csrc/ or include/ is newer than its object.

Tuned variants (paper_1806_03761_gb300/tuning.json, written by the
autotuner): a variant sets compile-time knobs of the kernels (PEPS_QR_NB,
PEPS_BA_FF, PEPS_BA_F64, PEPS_BB_FF, PEPS_MINB, PEPS_NT, and the code paths
PEPS_QR_PREFETCH, PEPS_BIDIAG_TPC, PEPS_QR_TALL_PAIR, PEPS_CTR_PIPE and
PEPS_QR_ACC).  It recompiles the units those
knobs reach for one precision form -- the C ABI and the form's fused
VMC-step kernel -- and links them with the default objects of every other
unit (device code is compiled per unit, without relocatable device code, so
the units share no device functions) into lib/<tag>/libpeps.so.

    python -m paper_1806_03761_gb300.build [--verbose]
"""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libpeps.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
         "-I" + os.path.join(ROOT, "include")]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA 13 toolkit is required to build libpeps.so")
    return exe


def _headers_mtime():
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
    hs += glob.glob(os.path.join(ROOT, "include", "*.h"))
    return max(os.path.getmtime(h) for h in hs)


def _compile(src, obj, verbose, extra=()):
    cmd = [nvcc()] + ARCH + FLAGS + list(extra) + (["-Xptxas", "-v"] if verbose else []) + \
        ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed on %s:\n%s%s" % (src, r.stdout, r.stderr))
    return (src, r.stderr if verbose else "")


DEFAULTS = {"PEPS_QR_NB": 4, "PEPS_BA_FF": 4, "PEPS_BA_F64": 2, "PEPS_MINB": 2, "PEPS_NT": 256,
            "PEPS_QR_PREFETCH": 0, "PEPS_BIDIAG_TPC": 0, "PEPS_QR_TALL_PAIR": 0,
            "PEPS_BB_FF": 2, "PEPS_CTR_PIPE": 1, "PEPS_QR_ACC": 1,
            "PEPS_PHASES": 0, "PEPS_BIDIAG_FUSE": 0}
FORMS = {"fp64": "f64", "mixed": "ff", "fp32": "f32"}
TUNING = os.path.join(PKG, "tuning.json")


def variant_tag(knobs, precision):
    """Directory name of a variant: the form and every knob that differs from
    the default, e.g. 'mixed-PEPS_QR_NB8'; 'default' when none differs."""
    diff = sorted((k, v) for k, v in knobs.items() if DEFAULTS.get(k) != v)
    if not diff:
        return "default"
    return precision + "-" + "-".join("%s%d" % (k, v) for k, v in diff)


def variant_path(knobs, precision):
    tag = variant_tag(knobs, precision)
    return LIB if tag == "default" else os.path.join(LIBDIR, tag, "libpeps.so")


def build_variant(knobs, precision, verbose=False):
    """Build the library of one tuned variant (the default objects must exist:
    call build() first); returns its path."""
    tag = variant_tag(knobs, precision)
    if tag == "default":
        return LIB
    out_dir = os.path.join(BUILD, tag)
    lib_dir = os.path.join(LIBDIR, tag)
    os.makedirs(out_dir, exist_ok=True)
    os.makedirs(lib_dir, exist_ok=True)
    flags = ["-D%s=%d" % (k, v) for k, v in sorted(knobs.items())]
    units = ["peps_api.cu", "peps_k_vmc_%s.cu" % FORMS[precision]]
    hmt = _headers_mtime()
    jobs = []
    for u in units:
        src = os.path.join(CSRC, u)
        obj = os.path.join(out_dir, u[:-3] + ".o")
        if not os.path.exists(obj) or os.path.getmtime(obj) < max(hmt, os.path.getmtime(src)):
            jobs.append((src, obj))
    with cf.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        list(ex.map(lambda j: _compile(j[0], j[1], verbose, flags), jobs))
    objs = [os.path.join(out_dir, u[:-3] + ".o") for u in units]
    for o in sorted(glob.glob(os.path.join(BUILD, "*.o"))):
        if os.path.basename(o)[:-2] + ".cu" not in units:
            objs.append(o)
    lib = os.path.join(lib_dir, "libpeps.so")
    cmd = [nvcc()] + ARCH + ["-shared", "-o", lib] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    return lib


def tuned_variants():
    """[(knobs, precision)] of the tuning table's choices."""
    import json
    if not os.path.exists(TUNING):
        return []
    table = json.load(open(TUNING))
    return [(dict(v["choice"]), v["precision"]) for v in table.values()]


def build(verbose=False, force=False):
    """Compile and link libpeps.so and the tuned variants; returns its path."""
    lib = build_default(verbose, force)
    todo = {}
    for knobs, prec in tuned_variants():
        todo.setdefault(variant_tag(knobs, prec), (knobs, prec))
    if todo:
        with cf.ThreadPoolExecutor(max_workers=len(todo)) as ex:
            list(ex.map(lambda kp: build_variant(kp[0], kp[1], verbose), todo.values()))
    return lib


def build_default(verbose=False, force=False):
    """Compile and link libpeps.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hmt = _headers_mtime()
    jobs = []
    objs = []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(hmt, os.path.getmtime(s)):
            jobs.append((s, o))
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
            for src, log in ex.map(lambda j: _compile(j[0], j[1], verbose), jobs):
                if verbose and log:
                    sys.stderr.write("== %s\n%s" % (os.path.basename(src), log))
    if jobs or not os.path.exists(LIB):
        cmd = [nvcc()] + ARCH + ["-shared", "-o", LIB] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    return LIB


if __name__ == "__main__":
    print(build(verbose="--verbose" in sys.argv, force="--force" in sys.argv))
