"""ctypes declarations of libpeps.so (include/peps.h).

Argument marshalling only: every computation happens in the library's CUDA
kernels.  Loading fails loudly when the library has not been built."""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libpeps.so")

PEPS_OK = 0
PEPS_EINVAL = -1
PEPS_ENOMEM = -2
PEPS_ECUDA = -3
PEPS_ENUMERIC = -4
PEPS_ETIMEOUT = -5
PEPS_ESCRATCH = -6
PEPS_FP64 = 0
PEPS_MIXED = 1
PEPS_FP32 = 2

ERRNAMES = {0: "PEPS_OK", -1: "PEPS_EINVAL", -2: "PEPS_ENOMEM", -3: "PEPS_ECUDA",
            -4: "PEPS_ENUMERIC", -5: "PEPS_ETIMEOUT", -6: "PEPS_ESCRATCH"}

# every entry point include/peps.h declares
EXPORTS = ("peps_create", "peps_destroy", "peps_last_error", "peps_workspace_bytes", "peps_slots",
           "peps_set_tensors", "peps_amplitudes", "peps_local_energy", "peps_logderiv",
           "peps_evaluate", "peps_grad_step", "peps_sample_batch", "peps_sync_status",
           "peps_flops_per_sample", "peps_amplitudes_noalloc", "peps_vmc_step",
           "peps_server_create", "peps_server_submit", "peps_server_wait", "peps_server_destroy",
           "peps_correlations", "peps_structure_factor", "peps_tc_workspace_bytes", "peps_tc_gemm",
           "peps_cc_workspace_bytes", "peps_cc_gemm", "peps_pool_create", "peps_pool_destroy",
           "peps_pool_slots", "peps_local_energy_multi", "peps_pool_sync_status",
           "peps_vmc_step_dc", "peps_grad_step_dc", "peps_counters_advance", "peps_vmc_step_host",
           "peps_phase_cycles")


class PepsShape(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("D", ctypes.c_int32), ("Dc", ctypes.c_int32),
                ("J1", ctypes.c_double), ("J2", ctypes.c_double),
                ("precision", ctypes.c_int32)]




class PepsJob(ctypes.Structure):
    _fields_ = [("shape", PepsShape), ("A", ctypes.c_void_p), ("spins", ctypes.c_void_p),
                ("B", ctypes.c_int64), ("e_loc", ctypes.c_void_p), ("log_abs", ctypes.c_void_p),
                ("sign", ctypes.c_void_p)]


class PepsMultiJob(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("spins", ctypes.c_void_p), ("B", ctypes.c_int64),
                ("e_loc", ctypes.c_void_p), ("log_abs", ctypes.c_void_p), ("sign", ctypes.c_void_p),
                ("ratios", ctypes.c_void_p), ("n_flips", ctypes.c_void_p)]


class PepsJobStats(ctypes.Structure):
    _fields_ = [("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double),
                ("done_s", ctypes.c_double), ("footprint_bytes", ctypes.c_int64),
                ("status", ctypes.c_int32), ("flags", ctypes.c_int32)]


_lib = None

P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64
U64 = ctypes.c_uint64
F64 = ctypes.c_double

_SIGS = {
    "peps_create": (I32, [ctypes.POINTER(PepsShape), I32, ctypes.POINTER(P)]),
    "peps_destroy": (I32, [P]),
    "peps_last_error": (ctypes.c_char_p, [P]),
    "peps_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(PepsShape), I32]),
    "peps_slots": (I32, [P, ctypes.POINTER(I32)]),
    "peps_phase_cycles": (I32, [P, ctypes.POINTER(ctypes.c_uint64), I32, ctypes.POINTER(I32)]),
    "peps_set_tensors": (I32, [P, P, P]),
    "peps_amplitudes": (I32, [P, P, I64, P, P, P]),
    "peps_local_energy": (I32, [P, P, I64, P, P, P, P, P, P]),
    "peps_logderiv": (I32, [P, P, I64, P, P, P, P, P, I32, P]),
    "peps_evaluate": (I32, [P, P, I64, P, P, P, P, P, P, P, P, P, I32, P]),
    "peps_grad_step": (I32, [P, P, P, P, I64, F64, U64, U64, P, P]),
    "peps_sample_batch": (I32, [P, U64, I64, I64, I32, I32, I32, U64, P, P, P, P]),
    "peps_sync_status": (I32, [P, P, ctypes.POINTER(I32)]),
    "peps_flops_per_sample": (F64, [ctypes.POINTER(PepsShape), I32]),
    "peps_amplitudes_noalloc": (I32, [ctypes.POINTER(PepsShape), P, P, I64, P, P, P]),
    "peps_vmc_step": (I32, [P, U64, I64, I64, U64, P, P, P, P, P, P, P, I32, P, P]),
    "peps_server_create": (I32, [ctypes.c_size_t, I32, ctypes.POINTER(P)]),
    "peps_server_submit": (I32, [P, ctypes.POINTER(PepsJob), ctypes.POINTER(I64)]),
    "peps_server_wait": (I32, [P, I64, F64, ctypes.POINTER(PepsJobStats)]),
    "peps_server_destroy": (I32, [P]),
    "peps_correlations": (I32, [P, P, I64, I32, P, P, P, P]),
    "peps_structure_factor": (I32, [P, P, I32, P, F64, F64, P, P]),
    "peps_tc_workspace_bytes": (ctypes.c_size_t, [I32, I32, I32, I64, I32, I32]),
    "peps_tc_gemm": (I32, [P, P, P, I32, I32, I32, I64, I32, I32, I32, P, ctypes.c_size_t, P, P]),
    "peps_cc_workspace_bytes": (ctypes.c_size_t, [I32, I32, I32, I32, I64, I32]),
    "peps_cc_gemm": (I32, [I32, P, P, P, I32, I32, I32, I64, I32, P, ctypes.c_size_t, I32, P]),
    "peps_pool_create": (I32, [I32, I32, ctypes.POINTER(PepsShape), I32, I32, ctypes.POINTER(P)]),
    "peps_pool_destroy": (I32, [P]),
    "peps_pool_slots": (I32, [P, ctypes.POINTER(I32)]),
    "peps_local_energy_multi": (I32, [P, ctypes.POINTER(PepsMultiJob), I32, P]),
    "peps_pool_sync_status": (I32, [P, P, ctypes.POINTER(I32)]),
    "peps_vmc_step_dc": (I32, [P, U64, I64, I64, P, P, P, P, P, P, P, P, I32, P, P]),
    "peps_grad_step_dc": (I32, [P, P, P, P, I64, F64, U64, P, P, P]),
    "peps_counters_advance": (I32, [P, I32, ctypes.c_uint32, P]),
    "peps_vmc_step_host": (I32, [P, U64, I64, I64, U64, P, P, P, P, P, P, P, P, P]),
}


_variants = {}


def load_path(path):
    """Load a library built at `path` (a tuned variant) once and declare its
    signatures."""
    if path not in _variants:
        if not os.path.exists(path):
            raise RuntimeError("library variant not built: %s" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _variants[path] = lib
    return _variants[path]


def load(path=None):
    """Load libpeps.so (once) and declare its signatures.  The environment
    variable PEPS_LIB names another build of the library to load instead
    (the autotuner's timing runs use it)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("PEPS_LIB") or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(
            "libpeps.so not found at %s: build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` "
            "(there is no CPU fallback)" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
