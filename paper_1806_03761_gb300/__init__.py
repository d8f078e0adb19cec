"""GB300 (sm_103a) per-sample PEPS contraction: the data-parallel hot path of
PEPS++ (He et al., arXiv:1806.03761) behind the C ABI of ``include/peps.h``.

This module is a thin binding: it allocates outputs with PyTorch on the
current CUDA device, passes raw pointers and the current stream to
``libpeps.so`` and returns the tensors.  Every step of the contraction runs in
the library's CUDA kernels; there is no CPU path.
"""
import ctypes

from . import _lib
from ._lib import PEPS_FP32, PEPS_FP64, PEPS_MIXED, PepsShape  # noqa: F401

__all__ = ["PepsContext", "PepsError", "bond_count", "PEPS_FP64", "PEPS_MIXED", "PEPS_FP32",
           "workspace_bytes", "flops_per_sample"]


class PepsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (_lib.ERRNAMES.get(code, code), msg))
        self.code = code


def bond_count(L):
    """Number of J1 + J2 bonds of the open L x L lattice."""
    return 2 * L * (L - 1) + 2 * (L - 1) ** 2


_PREC = {"fp64": PEPS_FP64, "mixed": PEPS_MIXED, "fp32": PEPS_FP32}


def _shape(L, D, Dc, J1, J2, precision):
    prec = _PREC.get(precision, precision)
    return PepsShape(int(L), int(D), int(Dc), float(J1), float(J2), int(prec))


def workspace_bytes(L, D, Dc, precision="fp64", slots=0, J1=1.0, J2=0.5):
    s = _shape(L, D, Dc, J1, J2, precision)
    return int(_lib.load().peps_workspace_bytes(ctypes.byref(s), int(slots)))


def flops_per_sample(L, D, Dc, precision="fp64", what="evaluate"):
    """Algorithmic flops per chain (host call): what = "evaluate", "sweep"
    or "vmc" (evaluation + sweep in one peps_vmc_step)."""
    s = _shape(L, D, Dc, 1.0, 0.5, precision)
    w = {"evaluate": 0, "sweep": 1, "vmc": 2}[what]
    return float(_lib.load().peps_flops_per_sample(ctypes.byref(s), w))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _lib_for(L, D, Dc, precision):
    """The library a context of this shape uses: the tuned variant named by
    tuning.json for (L, D, Dc, form) when it has been built, else the
    default build (always the default under PEPS_LIB)."""
    import json
    import os
    from . import build as B
    if os.environ.get("PEPS_LIB") or not os.path.exists(B.TUNING):
        return _lib.load()
    entry = json.load(open(B.TUNING)).get(tuning_key(L, D, Dc, precision))
    if entry:
        path = B.variant_path(entry["choice"], precision)
        if path != B.LIB and os.path.exists(path):
            return _lib.load_path(path)
    return _lib.load()


def tuning_key(L, D, Dc, precision):
    return "%dx%d_D%d_Dc%d_%s" % (L, L, D, Dc, precision)


class PepsContext:
    """One library context: shape, precision form and device workspace."""

    def __init__(self, L, D, Dc, J1=1.0, J2=0.5, precision="fp64", slots=0, variant=None):
        """variant: compile-time knobs of the fused VMC kernel ({"PEPS_QR_NB":
        8, ...}, see build.py); that build is made if missing (two
        translation units) and used by this context.  Default: the tuned
        variant of tuning.json for this shape, else the default build."""
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (there is no CPU path)")
        self.torch = torch
        if variant:
            from . import build as B
            knobs = dict(B.DEFAULTS)
            knobs.update(variant)
            self.lib = _lib.load_path(B.build_variant(knobs, precision))
        else:
            self.lib = _lib_for(int(L), int(D), int(Dc), precision)
        self.L, self.D, self.Dc = int(L), int(D), int(Dc)
        self.N = self.L * self.L
        self.D4 = self.D ** 4
        self.nbonds = bond_count(self.L)
        self.precision = precision
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._shape = _shape(L, D, Dc, J1, J2, precision)
        h = ctypes.c_void_p()
        rc = self.lib.peps_create(ctypes.byref(self._shape), int(slots), ctypes.byref(h))
        if rc != 0:
            raise PepsError(rc, "peps_create failed")
        self.h = h
        n = ctypes.c_int32(0)
        self._check(self.lib.peps_slots(self.h, ctypes.byref(n)))
        self.slots = n.value  # samples processed concurrently (one wave)

    def close(self):
        if getattr(self, "h", None):
            self.lib.peps_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- helpers -------------------------------------------------------------
    def _stream(self):
        return ctypes.c_void_p(self.torch.cuda.current_stream().cuda_stream)

    def _check(self, rc):
        if rc != 0:
            raise PepsError(rc, self.lib.peps_last_error(self.h).decode())

    def _spins(self, spins):
        t = self.torch
        assert spins.dtype == t.uint8 and spins.is_cuda and spins.is_contiguous()
        assert spins.dim() == 2 and spins.shape[1] == self.N
        return spins

    def _empty(self, *shape, dtype=None):
        return self.torch.empty(*shape, dtype=dtype or self.torch.float64, device=self.device)

    # -- entry points --------------------------------------------------------
    def set_tensors(self, A):
        t = self.torch
        assert A.dtype == t.float64 and A.is_cuda and A.is_contiguous()
        assert A.numel() == self.N * 2 * self.D4
        self._check(self.lib.peps_set_tensors(self.h, _ptr(A), self._stream()))

    def amplitudes(self, spins):
        s = self._spins(spins)
        B = s.shape[0]
        la, sg = self._empty(B), self._empty(B, dtype=self.torch.int8)
        self._check(self.lib.peps_amplitudes(self.h, _ptr(s), B, _ptr(la), _ptr(sg), self._stream()))
        return la, sg

    def local_energy(self, spins, ratios=False, n_flips=False):
        s = self._spins(spins)
        B = s.shape[0]
        e, la = self._empty(B), self._empty(B)
        sg = self._empty(B, dtype=self.torch.int8)
        r = self._empty(B, self.nbonds) if ratios else None
        nf = self._empty(B, dtype=self.torch.int32) if n_flips else None
        self._check(self.lib.peps_local_energy(self.h, _ptr(s), B, _ptr(e), _ptr(la), _ptr(sg),
                                               _ptr(r), _ptr(nf), self._stream()))
        return dict(e_loc=e, log_abs=la, sign=sg, ratios=r, n_flips=nf)

    def new_sums(self):
        return (self.torch.zeros(self.N, 2, self.D4, dtype=self.torch.float64, device=self.device),
                self.torch.zeros(self.N, 2, self.D4, dtype=self.torch.float64, device=self.device),
                self.torch.zeros(1, dtype=self.torch.float64, device=self.device))

    def logderiv(self, spins, e_loc, delta=False, sums=None, accumulate=False):
        s = self._spins(spins)
        B = s.shape[0]
        sums = sums or self.new_sums()
        d = self._empty(B, self.N, self.D4) if delta else None
        self._check(self.lib.peps_logderiv(self.h, _ptr(s), B, _ptr(e_loc), _ptr(d),
                                           _ptr(sums[0]), _ptr(sums[1]), _ptr(sums[2]),
                                           int(bool(accumulate)), self._stream()))
        return dict(delta=d, sum_delta=sums[0], sum_delta_e=sums[1], sum_e=sums[2])

    def evaluate(self, spins, ratios=False, n_flips=False, delta=False, sums=None,
                 accumulate=False, out=None):
        """Local energy and log-derivative sums in one pass (peps_evaluate)."""
        s = self._spins(spins)
        B = s.shape[0]
        sums = sums or self.new_sums()
        if out is None:
            out = dict(e_loc=self._empty(B), log_abs=self._empty(B),
                       sign=self._empty(B, dtype=self.torch.int8))
        r = self._empty(B, self.nbonds) if ratios else None
        nf = self._empty(B, dtype=self.torch.int32) if n_flips else None
        d = self._empty(B, self.N, self.D4) if delta else None
        self._check(self.lib.peps_evaluate(
            self.h, _ptr(s), B, _ptr(out["e_loc"]), _ptr(out["log_abs"]), _ptr(out["sign"]),
            _ptr(r), _ptr(nf), _ptr(d), _ptr(sums[0]), _ptr(sums[1]), _ptr(sums[2]),
            int(bool(accumulate)), self._stream()))
        res = dict(out)
        res.update(ratios=r, n_flips=nf, delta=d, sum_delta=sums[0], sum_delta_e=sums[1],
                   sum_e=sums[2])
        return res

    def grad_step(self, sums, M, dt, seed, step, A):
        self._check(self.lib.peps_grad_step(self.h, _ptr(sums[0]), _ptr(sums[1]), _ptr(sums[2]),
                                            int(M), float(dt), int(seed), int(step), _ptr(A),
                                            self._stream()))
        return A

    def sample(self, seed, n_chains, n_burn, n_thin, samples_per_chain, chain_offset=0,
               first_sweep=1, state=None, accepted=False):
        t = self.torch
        out = self._empty(n_chains * samples_per_chain, self.N, dtype=t.uint8)
        acc = self._empty(n_chains, dtype=t.int64) if accepted else None
        if state is not None:
            assert state.dtype == t.uint8 and state.is_cuda and state.shape == (n_chains, self.N)
        self._check(self.lib.peps_sample_batch(self.h, int(seed), int(n_chains), int(chain_offset),
                                               int(n_burn), int(n_thin), int(samples_per_chain),
                                               int(first_sweep), _ptr(out), _ptr(state), _ptr(acc),
                                               self._stream()))
        return (out, acc) if accepted else out

    def vmc_step(self, seed, state, sweep, chain_offset=0, sums=None, accumulate=False,
                 out=None, accepted=False):
        """Evaluate the chains' configurations and advance each by one
        Metropolis sweep, in one launch (peps_vmc_step); `state` is updated."""
        t = self.torch
        assert state.dtype == t.uint8 and state.is_cuda and state.is_contiguous()
        n = state.shape[0]
        sums = sums or self.new_sums()
        if out is None:
            out = dict(e_loc=self._empty(n), log_abs=self._empty(n), sign=self._empty(n, dtype=t.int8))
        acc = self._empty(n, dtype=t.int64) if accepted else None
        self._check(self.lib.peps_vmc_step(
            self.h, int(seed), n, int(chain_offset), int(sweep), _ptr(state), _ptr(out["e_loc"]),
            _ptr(out["log_abs"]), _ptr(out["sign"]), _ptr(sums[0]), _ptr(sums[1]), _ptr(sums[2]),
            int(bool(accumulate)), _ptr(acc), self._stream()))
        res = dict(out)
        res.update(sum_delta=sums[0], sum_delta_e=sums[1], sum_e=sums[2], accepted=acc)
        return res

    def correlations(self, spins, sources, mean=True):
        """Local values of S_src . S_m (peps_correlations): returns
        dict(ss=float64[B][n_src][N], mean=float64[n_src][N] or None)."""
        import numpy as np
        t = self.torch
        s = self._spins(spins)
        B = s.shape[0]
        src = np.ascontiguousarray(np.asarray(sources, dtype=np.int32).reshape(-1))
        ss = self._empty(B, src.size, self.N)
        mn = self._empty(src.size, self.N) if mean else None
        self._check(self.lib.peps_correlations(self.h, _ptr(s), B, int(src.size),
                                               src.ctypes.data_as(ctypes.c_void_p), _ptr(ss),
                                               _ptr(mn), self._stream()))
        return dict(ss=ss, mean=mn)

    def structure_factor(self, mean, sources, k=(3.141592653589793, 3.141592653589793)):
        """m_s^2(k) over the bulk from the batch means (peps_structure_factor);
        a one-element float64 device tensor."""
        import numpy as np
        src = np.ascontiguousarray(np.asarray(sources, dtype=np.int32).reshape(-1))
        out = self._empty(1)
        self._check(self.lib.peps_structure_factor(self.h, _ptr(mean), int(src.size),
                                                   src.ctypes.data_as(ctypes.c_void_p),
                                                   float(k[0]), float(k[1]), _ptr(out),
                                                   self._stream()))
        return out

    def vmc_step_host(self, seed, state, sweep, sums, e_loc, sum_e=None, chain_offset=0):
        """peps_vmc_step_host: `state` (uint8 [n, N]), `e_loc` (float64 [n]) and
        `sum_e` (float64 [1], optional) are HOST tensors (pinned for
        asynchronous copies); `sums` the device gradient sums.  Returns when
        the results are in host memory."""
        n = state.shape[0]
        assert not state.is_cuda and not e_loc.is_cuda and state.is_contiguous()
        self._check(self.lib.peps_vmc_step_host(
            self.h, int(seed), n, int(chain_offset), int(sweep), _ptr(state), _ptr(e_loc), None, None,
            _ptr(sum_e), _ptr(sums[0]), _ptr(sums[1]), _ptr(sums[2]), self._stream()))
        return e_loc

    # -- device-resident counters (CUDA-graph capture) -------------------------
    def new_counters(self, sweep, step):
        """uint32[2] device counters: the next sweep number and GO step number."""
        return self.torch.tensor([sweep, step], dtype=self.torch.int32, device=self.device)

    def vmc_step_dc(self, seed, state, counters, chain_offset=0, sums=None, out=None):
        """peps_vmc_step with the sweep number read from counters[0] at run time."""
        t = self.torch
        n = state.shape[0]
        sums = sums or self.new_sums()
        if out is None:
            out = dict(e_loc=self._empty(n), log_abs=self._empty(n), sign=self._empty(n, dtype=t.int8))
        self._check(self.lib.peps_vmc_step_dc(
            self.h, int(seed), n, int(chain_offset), _ptr(counters), _ptr(state), _ptr(out["e_loc"]),
            _ptr(out["log_abs"]), _ptr(out["sign"]), _ptr(sums[0]), _ptr(sums[1]), _ptr(sums[2]), 0,
            None, self._stream()))
        res = dict(out)
        res.update(sum_delta=sums[0], sum_delta_e=sums[1], sum_e=sums[2])
        return res

    def grad_step_dc(self, sums, M, dt, seed, counters, A):
        """peps_grad_step with the GO step number read from counters[1]."""
        self._check(self.lib.peps_grad_step_dc(self.h, _ptr(sums[0]), _ptr(sums[1]), _ptr(sums[2]),
                                               int(M), float(dt), int(seed), _ptr(counters), _ptr(A),
                                               self._stream()))
        return A

    def advance_counters(self, counters, inc=1):
        rc = self.lib.peps_counters_advance(_ptr(counters), int(counters.numel()), int(inc),
                                            self._stream())
        if rc != 0:
            raise PepsError(rc, "peps_counters_advance failed")

    def sync_status(self):
        f = ctypes.c_int32(0)
        rc = self.lib.peps_sync_status(self.h, self._stream(), ctypes.byref(f))
        if rc not in (0, _lib.PEPS_ENUMERIC):
            self._check(rc)
        return rc, f.value

    PHASES = ("eval", "sweep", "compress", "qr", "svd_qr", "svd", "strip1", "ratio_h", "btens",
              "strip2", "ratio_2", "sweep_h", "sweep_r2", "sweep_v")

    def phase_cycles(self):
        """Per-phase clock64 cycles of the fused VMC kernel summed over blocks
        since the last call (peps_phase_cycles), as {phase: cycles}; empty
        unless this context's library was built with PEPS_PHASES=1."""
        buf = (ctypes.c_uint64 * len(self.PHASES))()
        n = ctypes.c_int32(0)
        self._check(self.lib.peps_phase_cycles(self.h, buf, len(self.PHASES), ctypes.byref(n)))
        return {self.PHASES[i]: int(buf[i]) for i in range(min(n.value, len(self.PHASES)))}


class PepsServer:
    """Serving loop with continuous batching (peps_server_*): evaluation jobs
    of any shape are admitted under an HBM budget and their waves overlap on
    the device.  submit() returns a job id; wait() returns the job's
    energies, log|W|, signs and timings (host numpy arrays)."""

    def __init__(self, hbm_budget_bytes=0, slots_per_job=0):
        import numpy as np
        self.np = np
        self.lib = _lib.load()
        h = ctypes.c_void_p()
        rc = self.lib.peps_server_create(int(hbm_budget_bytes), int(slots_per_job), ctypes.byref(h))
        if rc != 0:
            raise PepsError(rc, "peps_server_create failed")
        self.h = h
        self._jobs = {}

    def submit(self, A, spins, L, D, Dc, precision="mixed", J1=1.0, J2=0.5):
        np = self.np
        A = np.ascontiguousarray(A, dtype=np.float64)
        spins = np.ascontiguousarray(spins, dtype=np.uint8).reshape(-1, L * L)
        B = spins.shape[0]
        out = dict(e_loc=np.empty(B), log_abs=np.empty(B), sign=np.empty(B, dtype=np.int8))
        job = _lib.PepsJob(_shape(L, D, Dc, J1, J2, precision), A.ctypes.data, spins.ctypes.data, B,
                           out["e_loc"].ctypes.data, out["log_abs"].ctypes.data,
                           out["sign"].ctypes.data)
        jid = ctypes.c_int64(0)
        rc = self.lib.peps_server_submit(self.h, ctypes.byref(job), ctypes.byref(jid))
        if rc != 0:
            raise PepsError(rc, "peps_server_submit failed")
        self._jobs[jid.value] = (A, spins, out)  # the buffers live until wait()
        return jid.value

    def wait(self, job_id, timeout=0.0):
        st = _lib.PepsJobStats()
        rc = self.lib.peps_server_wait(self.h, int(job_id), float(timeout), ctypes.byref(st))
        if rc == _lib.PEPS_ETIMEOUT:
            raise TimeoutError("job %d still running" % job_id)
        if job_id not in self._jobs:
            raise PepsError(rc, "unknown job id %d (or already waited for)" % job_id)
        _, _, out = self._jobs.pop(job_id)
        res = dict(out)
        res.update(status=rc, flags=st.flags, submit_s=st.submit_s, admit_s=st.admit_s,
                   done_s=st.done_s, latency_s=st.done_s - st.submit_s,
                   footprint_bytes=st.footprint_bytes)
        return res

    def close(self):
        if getattr(self, "h", None):
            self.lib.peps_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PepsPool:
    """Jobs of different shapes in one persistent launch (peps_local_energy_multi):
    a slot pool sized for the largest of `shapes` ((L, D, Dc) tuples), one
    precision form.  local_energy(jobs) takes [(PepsContext, spins), ...] and
    returns one dict per job (e_loc, log_abs, sign, ratios, n_flips)."""

    def __init__(self, shapes, precision="mixed", slots=0, max_jobs=64, J1=1.0, J2=0.5):
        import torch
        self.torch = torch
        self.lib = _lib.load()
        arr = (PepsShape * len(shapes))(*[_shape(L, D, Dc, J1, J2, precision) for (L, D, Dc) in shapes])
        h = ctypes.c_void_p()
        rc = self.lib.peps_pool_create(_PREC[precision], int(slots), arr, len(shapes), int(max_jobs),
                                       ctypes.byref(h))
        if rc != 0:
            raise PepsError(rc, "peps_pool_create failed")
        self.h = h
        n = ctypes.c_int32(0)
        self.lib.peps_pool_slots(self.h, ctypes.byref(n))
        self.slots = n.value

    def local_energy(self, jobs, ratios=False, n_flips=False):
        t = self.torch
        outs, arr = [], (_lib.PepsMultiJob * len(jobs))()
        for q, (ctx, spins) in enumerate(jobs):
            s = ctx._spins(spins)
            B = s.shape[0]
            o = dict(e_loc=ctx._empty(B), log_abs=ctx._empty(B), sign=ctx._empty(B, dtype=t.int8),
                     ratios=ctx._empty(B, ctx.nbonds) if ratios else None,
                     n_flips=ctx._empty(B, dtype=t.int32) if n_flips else None)
            outs.append(o)
            arr[q] = _lib.PepsMultiJob(ctx.h, s.data_ptr(), B, o["e_loc"].data_ptr(),
                                       o["log_abs"].data_ptr(), o["sign"].data_ptr(),
                                       o["ratios"].data_ptr() if ratios else None,
                                       o["n_flips"].data_ptr() if n_flips else None)
        stream = ctypes.c_void_p(t.cuda.current_stream().cuda_stream)
        rc = self.lib.peps_local_energy_multi(self.h, arr, len(jobs), stream)
        if rc != 0:
            raise PepsError(rc, "peps_local_energy_multi failed")
        return outs

    def sync_status(self):
        f = ctypes.c_int32(0)
        rc = self.lib.peps_pool_sync_status(self.h, ctypes.c_void_p(
            self.torch.cuda.current_stream().cuda_stream), ctypes.byref(f))
        return rc, f.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.peps_pool_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Contraction:
    """Batched C_b = A_b B_b (float64 device tensors [batch, M, K] and
    [batch or 1, K, N]) on the tensor cores (tcgen05, error-free BF16 slices:
    peps_tc_gemm) or on the CUDA cores (contract(): peps_cc_gemm), with the
    workspace held between calls so that repeated calls time the kernels."""

    def __init__(self, M, N, K, batch, b_shared=False, slices=7):
        import torch
        self.torch = torch
        self.lib = _lib.load()
        self.M, self.N, self.K, self.batch = int(M), int(N), int(K), int(batch)
        self.b_shared = int(bool(b_shared))
        self.slices = int(slices)
        nb = self.lib.peps_tc_workspace_bytes(self.M, self.N, self.K, self.batch, self.slices,
                                              self.b_shared)
        if nb == 0:
            raise PepsError(_lib.PEPS_EINVAL, "shape not supported by peps_tc_gemm")
        self.ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        self.status = torch.zeros(1, dtype=torch.int32, device="cuda")
        self._cc = {}

    def _stream(self):
        return ctypes.c_void_p(self.torch.cuda.current_stream().cuda_stream)

    def tensor_cores(self, A, B, C=None, out="fp64"):
        """out = "fp64": C float64 [batch, M, N]; out = "mixed": C as
        float-float pairs, a float32 tensor [batch, M, N, 2] (hi, lo)."""
        t = self.torch
        if C is None:
            C = (t.empty(self.batch, self.M, self.N, dtype=t.float64, device="cuda") if out == "fp64"
                 else t.empty(self.batch, self.M, self.N, 2, dtype=t.float32, device="cuda"))
        rc = self.lib.peps_tc_gemm(_ptr(A), _ptr(B), _ptr(C), self.M, self.N, self.K, self.batch,
                                   self.b_shared, self.slices, _PREC[out], _ptr(self.ws),
                                   self.ws.numel(), _ptr(self.status), self._stream())
        if rc != 0:
            raise PepsError(rc, "peps_tc_gemm failed")
        return C

    def cuda_cores(self, A, B, precision="mixed", C=None, convert=True):
        t = self.torch
        prec = _PREC[precision]
        if precision not in self._cc:
            nb = self.lib.peps_cc_workspace_bytes(prec, self.M, self.N, self.K, self.batch, self.b_shared)
            self._cc[precision] = t.empty(nb, dtype=t.uint8, device="cuda")
        w = self._cc[precision]
        C = C if C is not None else t.empty(self.batch, self.M, self.N, dtype=t.float64, device="cuda")
        rc = self.lib.peps_cc_gemm(prec, _ptr(A), _ptr(B), _ptr(C), self.M, self.N, self.K, self.batch,
                                   self.b_shared, _ptr(w), w.numel(), int(bool(convert)), self._stream())
        if rc != 0:
            raise PepsError(rc, "peps_cc_gemm failed")
        return C
