"""The library's kernels and C ABI built for the host (tests/_emu.py: the
CUDA translation units compiled with g++ against an emulated runtime, the
threads of a block run as fibers) against the oracle on small lattices: the
evaluation (E, log|W|, sign, every ratio, flip counts, Delta sums) in both
forms, the fused VMC step against evaluation then sweep, and bit-exact
Metropolis chains and GO update.  The kernel source is the GPU build's;
these tests check its logic without a GPU (FP32 operations are IEEE, with
no fused multiply-add contraction, so roundings may differ from the GPU's
at the last bit)."""
import ctypes

import numpy as np
import pytest

import oracle
from synth import make_peps, random_sz0_configs

from . import _emu

TOL = {"fp64": 1e-10, "mixed": 1e-4}


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    from paper_1806_03761_gb300 import _lib as B
    try:
        path = _emu.build(str(tmp_path_factory.mktemp("emu")))
    except RuntimeError as e:
        pytest.skip(str(e))
    L = ctypes.CDLL(path)
    for name, (res, args) in B._SIGS.items():
        if hasattr(L, name):
            fn = getattr(L, name)
            fn.restype, fn.argtypes = res, args
    return L


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class Ctx:
    """A context of the emulated library; numpy arrays stand for device
    buffers (the emulated device memory is host memory)."""

    def __init__(self, lib, L, D, Dc, prec, slots=0):
        from paper_1806_03761_gb300 import _lib as B
        self.lib, self.L, self.D, self.N = lib, L, D, L * L
        self.nb = 2 * L * (L - 1) + 2 * (L - 1) ** 2
        code = {"fp64": B.PEPS_FP64, "mixed": B.PEPS_MIXED}[prec]
        self.shape = B.PepsShape(L, D, Dc, 1.0, 0.5, code)
        self.h = ctypes.c_void_p()
        assert lib.peps_create(ctypes.byref(self.shape), slots, ctypes.byref(self.h)) == 0

    def set_tensors(self, A):
        self.A = np.ascontiguousarray(A)
        assert self.lib.peps_set_tensors(self.h, _p(self.A), None) == 0

    def status(self):
        f = ctypes.c_int32(0)
        rc = self.lib.peps_sync_status(self.h, None, ctypes.byref(f))
        return rc, f.value

    def sums(self):
        n = self.N * 2 * self.D ** 4
        return np.zeros(n), np.zeros(n), np.zeros(1)

    def evaluate(self, spins):
        B = len(spins)
        sp = np.ascontiguousarray(spins, np.uint8)
        r = dict(e_loc=np.zeros(B), log_abs=np.zeros(B), sign=np.zeros(B, np.int8),
                 ratios=np.zeros((B, self.nb)), n_flips=np.zeros(B, np.int32))
        sd, sde, se = self.sums()
        assert self.lib.peps_evaluate(self.h, _p(sp), B, _p(r["e_loc"]), _p(r["log_abs"]),
                                      _p(r["sign"]), _p(r["ratios"]), _p(r["n_flips"]), None,
                                      _p(sd), _p(sde), _p(se), 0, None) == 0
        r.update(sum_delta=sd, sum_delta_e=sde, sum_e=se)
        return r

    def vmc_step(self, seed, state, sweep):
        B = len(state)
        assert state.shape == (B, self.N) and state.dtype == np.uint8
        r = dict(e_loc=np.zeros(B), log_abs=np.zeros(B), sign=np.zeros(B, np.int8),
                 accepted=np.zeros(B, np.int64))
        sd, sde, se = self.sums()
        assert self.lib.peps_vmc_step(self.h, seed, B, 0, sweep, _p(state), _p(r["e_loc"]),
                                      _p(r["log_abs"]), _p(r["sign"]), _p(sd), _p(sde), _p(se), 0,
                                      _p(r["accepted"]), None) == 0
        r.update(sum_delta=sd, sum_delta_e=sde, sum_e=se)
        return r

    def sample(self, seed, n, n_burn, n_thin, spc, first_sweep=1, state=None):
        assert state is None or state.shape == (n, self.N)
        out = np.zeros((n * spc, self.N), np.uint8)
        acc = np.zeros(n, np.int64)
        assert self.lib.peps_sample_batch(self.h, seed, n, 0, n_burn, n_thin, spc, first_sweep,
                                          _p(out), _p(state), _p(acc), None) == 0
        return out, acc

    def close(self):
        self.lib.peps_destroy(self.h)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("L,D,Dc", [(3, 2, 8), (4, 3, 4), (6, 4, 8)])
def test_evaluation_matches_the_oracle(lib, prec, L, D, Dc):
    A = make_peps(L, D, seed=40 + L)
    spins = random_sz0_configs(L, 3, seed=41 + L)
    c = Ctx(lib, L, D, Dc, prec, slots=2)
    c.set_tensors(A)
    r = c.evaluate(spins)
    assert c.status() == (0, 0)
    c.close()
    ref = oracle.evaluate_batch(A, spins, L, Dc, want_delta=True)
    tol = TOL[prec]
    assert np.array_equal(r["sign"], ref["sign"].astype(np.int8))
    assert np.array_equal(r["n_flips"], ref["n_flips"])
    assert np.max(np.abs(r["log_abs"] - ref["log_abs"])) <= tol
    assert np.max(np.abs(r["e_loc"] - ref["e_loc"]) / np.maximum(1, np.abs(ref["e_loc"]))) <= tol
    for b in range(len(spins)):
        rr = ref["ratios"][b]
        m = rr != 0
        assert np.array_equal(r["ratios"][b] == 0, ~m)
        floor = tol * np.sqrt(np.mean(rr[m] ** 2))
        assert np.all(np.abs(r["ratios"][b][m] - rr[m]) <= tol * np.maximum(np.abs(rr[m]), floor / tol))
    N, D4 = L * L, D ** 4
    sd, sde = np.zeros((N, 2, D4)), np.zeros((N, 2, D4))
    for b in range(len(spins)):
        for m in range(N):
            dv = ref["delta"][b, m, spins[b][m]].reshape(-1)
            sd[m, spins[b][m]] += dv
            sde[m, spins[b][m]] += dv * ref["e_loc"][b]
    assert np.max(np.abs(r["sum_delta"].reshape(sd.shape) - sd)) <= tol * np.abs(sd).max()
    assert np.max(np.abs(r["sum_delta_e"].reshape(sde.shape) - sde)) <= tol * np.abs(sde).max()
    assert abs(r["sum_e"][0] - ref["e_loc"].sum()) <= tol * max(1, abs(ref["e_loc"].sum()))


@pytest.mark.parametrize("prec,L,D,Dc", [("fp64", 4, 3, 4), ("mixed", 4, 3, 4), ("fp64", 6, 4, 8)])
def test_sampler_bit_exact(lib, prec, L, D, Dc):
    """Metropolis chains (Fisher-Yates starts, exchange moves, Philox draws)
    equal the oracle's configurations and acceptance counts bit for bit, and
    resume from their final states (6x6 D=4 Dc=8: multi-panel QR and
    blocked bidiagonalisation in every compression)."""
    A = make_peps(L, D, seed=1)
    c = Ctx(lib, L, D, Dc, prec, slots=2)
    c.set_tensors(A)
    out, acc = c.sample(12345678901, 3, 1, 1, 1)
    ref, fin, racc = oracle.sample_chains(A, L, Dc, 12345678901, 3, 1, 1, 1)
    assert np.array_equal(out, ref) and np.array_equal(acc, racc)
    assert racc.sum() > 0
    state = fin.copy()
    out2, _ = c.sample(12345678901, 3, 0, 1, 1, first_sweep=10, state=state)
    ref2, fin2, _ = oracle.sample_chains(A, L, Dc, 12345678901, 3, 0, 1, 1, init=fin, first_sweep=10)
    assert np.array_equal(out2, ref2) and np.array_equal(state, fin2)
    assert c.status() == (0, 0)
    c.close()


def test_vmc_step_is_evaluation_then_sweep(lib):
    """The fused step (evaluation, then one sweep reusing the lower
    environments) equals peps_evaluate on the chains' states followed by one
    sweep of peps_sample_batch, bit for bit."""
    L, D, Dc = 4, 2, 4
    A = make_peps(L, D, seed=51)
    c = Ctx(lib, L, D, Dc, "fp64", slots=2)
    c.set_tensors(A)
    state0, _ = c.sample(77, 2, 1, 1, 1)
    ev = c.evaluate(state0)
    after = state0.copy()
    c.sample(77, len(after), 0, 1, 1, first_sweep=5, state=after)
    state = state0.copy()
    r = c.vmc_step(77, state, 5)
    for k in ("e_loc", "log_abs", "sign", "sum_delta", "sum_delta_e", "sum_e"):
        assert np.array_equal(r[k], ev[k]), k
    assert np.array_equal(state, after)
    c.close()


def test_grad_step_bit_exact(lib):
    """The GO update (Eq. gradients, the sign step with Philox step lengths)
    equals the oracle's, element by element."""
    L, D = 4, 2
    A = make_peps(L, D, seed=11)
    rng = np.random.default_rng(12)
    sd = rng.standard_normal((L * L, 2, D ** 4))
    sde = rng.standard_normal((L * L, 2, D ** 4))
    sd[0, 0, :3] = sde[0, 0, :3] = 0.0  # g = 0 exactly: unchanged
    se = np.array([rng.standard_normal()])
    M, dt, seed, step = 37, 0.05, 0xDEADBEEF12345, 9
    c = Ctx(lib, L, D, 4, "fp64")
    c.set_tensors(A)
    Ad = A.copy()
    assert lib.peps_grad_step(c.h, _p(sd), _p(sde), _p(se), M, dt, seed, step, _p(Ad), None) == 0
    g = oracle.gradient(sd, sde, se[0], M)
    assert np.array_equal(Ad, oracle.go_step(A, g.reshape(A.shape), dt, seed, step))
    c.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_correlations_match_the_oracle(lib, prec):
    """The correlation kernel: S_a . S_m for every target, sources at the
    centre and a corner, against the oracle's local estimator (the exchange
    ratio relative, with a floor of tol * RMS of the sample's ratios)."""
    from oracle import correlations as oc
    L, D, Dc = 4, 3, 4
    A = make_peps(L, D, seed=61)
    spins = random_sz0_configs(L, 2, seed=62)
    sources = np.array([oc.centre_site(L), 0], np.int32)
    c = Ctx(lib, L, D, Dc, prec, slots=2)
    c.set_tensors(A)
    ss = np.zeros((2, len(sources), L * L))
    mean = np.zeros((len(sources), L * L))
    assert lib.peps_correlations(c.h, _p(np.ascontiguousarray(spins)), 2, len(sources), _p(sources),
                                 _p(ss), _p(mean), None) == 0
    assert c.status() == (0, 0)
    c.close()
    tol = TOL[prec]
    for b, s in enumerate(spins):
        for q, a in enumerate(sources):
            ref = oc.local_correlations(A, s, L, Dc, int(a))
            ex_ref, ex_got = ref - np.where(s == s[a], 0.25, -0.25), ss[b, q] - np.where(s == s[a], 0.25, -0.25)
            ex_ref[a] = ex_got[a] = 0.0
            floor = tol * max(np.sqrt(np.mean(ex_ref ** 2)), 1e-300)
            assert np.all(np.abs(ex_got - ex_ref) <= np.maximum(tol * np.abs(ex_ref), floor)), (b, q)
            assert ss[b, q, a] == 0.75
    assert np.allclose(mean, ss.mean(axis=0), rtol=0, atol=1e-15)


def test_multi_shape_launch_equals_each_context(lib):
    """Jobs of three shapes in one persistent launch (the pool's work queue)
    give each context's own local energies bit for bit."""
    from paper_1806_03761_gb300 import _lib as B
    shapes = [(3, 2, 4), (4, 2, 4), (4, 3, 4)]
    ctxs, jobs, outs, refs, keep = [], [], [], [], []
    arr = (B.PepsShape * len(shapes))()
    for k, (L, D, Dc) in enumerate(shapes):
        arr[k] = B.PepsShape(L, D, Dc, 1.0, 0.5, B.PEPS_MIXED)
        c = Ctx(lib, L, D, Dc, "mixed", slots=2)
        c.set_tensors(make_peps(L, D, seed=70 + k))
        sp = np.ascontiguousarray(random_sz0_configs(L, 2, seed=80 + k))
        refs.append(c.evaluate(sp)["e_loc"])
        e = np.zeros(2)
        keep.append(sp)
        outs.append(e)
        jobs.append(B.PepsMultiJob(c.h.value, _p(sp).value, 2, _p(e).value, None, None, None, None))
        ctxs.append(c)
    pool = ctypes.c_void_p()
    assert lib.peps_pool_create(B.PEPS_MIXED, 3, arr, len(shapes), 8, ctypes.byref(pool)) == 0
    jarr = (B.PepsMultiJob * len(jobs))(*jobs)
    assert lib.peps_local_energy_multi(pool, jarr, len(jobs), None) == 0
    f = ctypes.c_int32(0)
    assert lib.peps_pool_sync_status(pool, None, ctypes.byref(f)) == 0 and f.value == 0
    lib.peps_pool_destroy(pool)
    for e, ref in zip(outs, refs):
        assert np.array_equal(e, ref)
    for c in ctxs:
        c.close()


# ---------------------------------------------------------------------------
# the serving loop (peps_server_*: host C++ worker and reaper threads) on the
# emulated device: every stream operation completes when issued
# ---------------------------------------------------------------------------
SERVE_JOBS = [(4, 2, 4, "fp64", 2, 11), (4, 3, 4, "mixed", 2, 12), (3, 2, 8, "fp64", 2, 13)]


class Server:
    def __init__(self, lib, budget=0, slots=2):
        self.lib, self.h, self.keep = lib, ctypes.c_void_p(), {}
        assert lib.peps_server_create(budget, slots, ctypes.byref(self.h)) == 0

    def submit(self, L, D, Dc, prec, B, seed):
        from paper_1806_03761_gb300 import _lib as Bl
        A = np.ascontiguousarray(make_peps(L, D, seed))
        S = np.ascontiguousarray(random_sz0_configs(L, B, seed + 100))
        out = dict(e_loc=np.zeros(B), log_abs=np.zeros(B), sign=np.zeros(B, np.int8))
        code = {"fp64": Bl.PEPS_FP64, "mixed": Bl.PEPS_MIXED}[prec]
        job = Bl.PepsJob(Bl.PepsShape(L, D, Dc, 1.0, 0.5, code), _p(A).value, _p(S).value, B,
                         _p(out["e_loc"]).value, _p(out["log_abs"]).value, _p(out["sign"]).value)
        jid = ctypes.c_int64(0)
        rc = self.lib.peps_server_submit(self.h, ctypes.byref(job), ctypes.byref(jid))
        if rc != 0:
            return rc
        self.keep[jid.value] = (A, S, out)
        return jid.value

    def wait(self, jid):
        from paper_1806_03761_gb300 import _lib as Bl
        st = Bl.PepsJobStats()
        rc = self.lib.peps_server_wait(self.h, jid, 0.0, ctypes.byref(st))
        A, S, out = self.keep.pop(jid)
        return dict(out, A=A, S=S, status=rc, admit_s=st.admit_s, done_s=st.done_s,
                    footprint=st.footprint_bytes)

    def close(self):
        self.lib.peps_server_destroy(self.h)


def test_server_mix_equals_alone_and_the_oracle(lib):
    srv = Server(lib)
    alone = [srv.wait(srv.submit(*j)) for j in SERVE_JOBS]
    ids = [srv.submit(*j) for j in SERVE_JOBS]
    mixed = [srv.wait(i) for i in ids]
    srv.close()
    for job, a, m in zip(SERVE_JOBS, alone, mixed):
        assert a["status"] == 0 and m["status"] == 0
        for k in ("e_loc", "log_abs", "sign"):
            assert np.array_equal(a[k], m[k]), (job, k)
        L, D, Dc, prec = job[:4]
        ref = oracle.evaluate_batch(m["A"], m["S"], L, Dc)
        assert np.array_equal(m["sign"], ref["sign"].astype(np.int8))
        assert np.max(np.abs(m["e_loc"] - ref["e_loc"]) / np.maximum(1, np.abs(ref["e_loc"]))) <= TOL[prec]


def test_server_budget_gates_admission_and_refuses(lib):
    from paper_1806_03761_gb300 import _lib as Bl
    job = SERVE_JOBS[0]
    probe = Server(lib)
    fp = probe.wait(probe.submit(*job))["footprint"]
    probe.close()
    assert fp > 0
    srv = Server(lib, budget=int(1.5 * fp))  # one such job at a time
    res = [srv.wait(i) for i in [srv.submit(*job) for _ in range(3)]]
    assert srv.submit(4, 2, 200, "fp64", 2, 1) == Bl.PEPS_EINVAL   # Dc * D > 256
    srv.close()
    for k in range(1, 3):
        assert res[k]["admit_s"] >= res[k - 1]["done_s"] - 1e-6
        assert np.array_equal(res[k]["e_loc"], res[0]["e_loc"])
    small = Server(lib, budget=fp // 2)
    assert small.submit(*job) == Bl.PEPS_ENOMEM  # alone larger than the budget
    small.close()


def test_server_eviction_under_a_tight_budget(lib):
    jobs = [SERVE_JOBS[0], SERVE_JOBS[2], SERVE_JOBS[0], SERVE_JOBS[2]]
    probe = Server(lib)
    alone = [probe.wait(probe.submit(*j)) for j in jobs]
    probe.close()
    srv = Server(lib, budget=int(1.2 * max(a["footprint"] for a in alone)))
    res = [srv.wait(i) for i in [srv.submit(*j) for j in jobs]]
    srv.close()
    for a, r in zip(alone, res):
        assert r["status"] == 0 and np.array_equal(a["e_loc"], r["e_loc"])


def test_tuned_variants_match_the_oracle(tmp_path_factory):
    """Every library variant the tuning table selects, built for the host
    with its knobs (the QR column prefetch, A'^T v one thread per column,
    three blocks' register budget, the two-warp tall panels with their
    named barriers): the evaluation matches the oracle, at 5x5 D=8 Dc=16
    (1024-row QR panels: the tall path) for a variant with the tall-panel
    pairing, else at 6x6 D=4 Dc=8."""
    import json
    from paper_1806_03761_gb300 import _lib as Bl
    from paper_1806_03761_gb300 import build as B
    table = json.load(open(B.TUNING))
    seen = set()
    for key, entry in sorted(table.items()):
        knobs, prec = entry["choice"], entry["precision"]
        tag = B.variant_tag(dict(B.DEFAULTS, **knobs), prec)
        if tag in seen:
            continue
        seen.add(tag)
        path = _emu.build(str(tmp_path_factory.mktemp("emu_variant")),
                          defines=["%s=%d" % kv for kv in sorted(knobs.items())])
        vlib = ctypes.CDLL(path)
        for name, (res, args) in Bl._SIGS.items():
            if hasattr(vlib, name):
                fn = getattr(vlib, name)
                fn.restype, fn.argtypes = res, args
        tall = bool(knobs.get("PEPS_QR_TALL_PAIR"))
        L, D, Dc = (5, 8, 16) if tall else (6, 4, 8)
        A = make_peps(L, D, seed=6)
        spins = random_sz0_configs(L, 1 if tall else 2, seed=7)
        c = Ctx(vlib, L, D, Dc, prec, slots=2)
        c.set_tensors(A)
        r = c.evaluate(spins)
        assert c.status() == (0, 0), tag
        c.close()
        ref = oracle.evaluate_batch(A, spins, L, Dc)
        assert np.array_equal(r["sign"], ref["sign"].astype(np.int8)), tag
        assert np.max(np.abs(r["log_abs"] - ref["log_abs"])) <= TOL[prec], tag
        assert np.max(np.abs(r["e_loc"] - ref["e_loc"]) / np.maximum(1, np.abs(ref["e_loc"]))) <= TOL[prec], tag
    assert seen


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_no_data_race_between_barriers(lib, prec):
    """Race check: the emulation resumes a block's threads in ascending,
    descending and pseudo-random orders between barriers; a read of another
    thread's write not separated from it by a barrier (__syncthreads,
    __syncwarp, a shuffle, a named barrier) would see a different value in
    some order.  Evaluation, the fused VMC step, sampling and correlations
    give the same bits in every order."""
    from oracle import correlations as oc
    L, D, Dc = 4, 3, 4
    A = make_peps(L, D, seed=90)
    spins = np.ascontiguousarray(random_sz0_configs(L, 3, seed=91))
    src = np.array([oc.centre_site(L), 3], np.int32)
    lib.emu_set_schedule.argtypes = [ctypes.c_int, ctypes.c_ulonglong]
    runs = []
    try:
        for order, seed in ((0, 1), (1, 1), (2, 7)):
            lib.emu_set_schedule(order, seed)
            c = Ctx(lib, L, D, Dc, prec, slots=2)
            c.set_tensors(A)
            ev = c.evaluate(spins)
            state = spins.copy()
            v = c.vmc_step(5, state, 2)
            out, acc = c.sample(9, 2, 1, 1, 1)
            ss = np.zeros((3, 2, L * L))
            assert lib.peps_correlations(c.h, _p(spins), 3, 2, _p(src), _p(ss), None, None) == 0
            assert c.status() == (0, 0)
            c.close()
            runs.append([ev[k] for k in sorted(ev)] + [v[k] for k in sorted(v)] + [state, out, acc, ss])
    finally:
        lib.emu_set_schedule(0, 1)
    for r in runs[1:]:
        for a, b in zip(runs[0], r):
            assert np.array_equal(a, b)


def test_the_race_check_sees_a_planted_race(tmp_path):
    """The schedule orders of the race check expose a read of another
    thread's write with no barrier between them (a planted race), and agree
    once the barrier is there."""
    import os
    import subprocess
    out_so = str(tmp_path / "planted.so")
    subprocess.run(["g++", "-std=c++20", "-O1", "-fPIC", "-shared", "-pthread", "-U_FORTIFY_SOURCE",
                    "-I", _emu.EMU, os.path.join(_emu.EMU, "planted_race.cpp"),
                    os.path.join(_emu.EMU, "emu.cpp"), "-o", out_so], check=True)
    p = ctypes.CDLL(out_so)
    p.emu_set_schedule.argtypes = [ctypes.c_int, ctypes.c_ulonglong]
    res = {}
    for barrier in (0, 1):
        for order in (0, 1):
            p.emu_set_schedule(order, 1)
            o = np.zeros(64, np.int32)
            p.planted_race(_p(o), barrier)
            res[barrier, order] = o
    assert not np.array_equal(res[0, 0], res[0, 1])
    assert np.array_equal(res[1, 0], res[1, 1])
    assert np.array_equal(res[1, 0], (np.arange(64) + 1) % 64 + 1)


def test_bidiag_without_the_two_barriers_is_bit_identical(tmp_path_factory):
    """PEPS_BIDIAG_FUSE leaves out two barriers per bidiagonalisation step
    where each thread reads only what it wrote itself: the fused step's
    outputs equal those of the build with the barriers bit for bit, in every
    resume order of the race check (both forms, 6x6 D=4 Dc=8; by hand also
    4x4 D=6 Dc=24 and the 1024-row panels of 5x5 D=8 Dc=16)."""
    from paper_1806_03761_gb300 import _lib as Bl

    def load(defs):
        lib = ctypes.CDLL(_emu.build(str(tmp_path_factory.mktemp("fuse")), defines=defs))
        for name, (res, args) in Bl._SIGS.items():
            if hasattr(lib, name):
                fn = getattr(lib, name)
                fn.restype, fn.argtypes = res, args
        lib.emu_set_schedule.argtypes = [ctypes.c_int, ctypes.c_ulonglong]
        return lib

    base = load(["PEPS_BIDIAG_TPC=1"])
    fuse = load(["PEPS_BIDIAG_TPC=1", "PEPS_BIDIAG_FUSE=1"])

    def run(lib, L, D, Dc, prec, order):
        lib.emu_set_schedule(order, 3)
        try:
            c = Ctx(lib, L, D, Dc, prec, slots=1)
            c.set_tensors(make_peps(L, D, seed=L + D))
            state = np.ascontiguousarray(random_sz0_configs(L, 1, seed=5))
            v = c.vmc_step(3, state, 1)
            assert c.status() == (0, 0)
            c.close()
        finally:
            lib.emu_set_schedule(0, 1)
        return [v[k] for k in sorted(v)] + [state]

    for (L, D, Dc, prec) in [(6, 4, 8, "mixed"), (6, 4, 8, "fp64")]:
        ref = run(base, L, D, Dc, prec, 0)
        for order in ((0, 2) if prec == "mixed" else (0,)):
            got = run(fuse, L, D, Dc, prec, order)
            for a, b in zip(ref, got):
                assert np.array_equal(a, b), (L, D, Dc, prec, order)


def test_abi_argument_checks(lib):
    """The C ABI refuses invalid arguments with PEPS_EINVAL and a message
    (peps_last_error), and accepts the empty batch: shapes out of range,
    NULL buffers, calls before peps_set_tensors, bad counts and ranges."""
    from paper_1806_03761_gb300 import _lib as Bl
    E = Bl.PEPS_EINVAL
    h = ctypes.c_void_p()
    for (L, D, Dc, prec) in [(1, 2, 4, 0), (33, 2, 4, 0), (4, 0, 4, 0), (4, 9, 4, 0), (4, 2, 0, 0),
                             (4, 8, 33, 0), (4, 2, 4, 7)]:
        sh = Bl.PepsShape(L, D, Dc, 1.0, 0.5, prec)
        assert lib.peps_create(ctypes.byref(sh), 0, ctypes.byref(h)) == E, (L, D, Dc, prec)
    sh = Bl.PepsShape(4, 2, 4, float("nan"), 0.5, Bl.PEPS_FP64)
    assert lib.peps_create(ctypes.byref(sh), 0, ctypes.byref(h)) == E
    sh = Bl.PepsShape(4, 2, 4, 1.0, 0.5, Bl.PEPS_FP64)
    assert lib.peps_create(ctypes.byref(sh), -1, ctypes.byref(h)) == E
    assert lib.peps_workspace_bytes(ctypes.byref(sh), 3) > 0
    c = Ctx(lib, 4, 2, 4, "fp64", slots=2)
    L, N = 4, 16
    sp = np.ascontiguousarray(random_sz0_configs(L, 2, seed=1))
    e = np.zeros(2)
    out = np.zeros((2, N), np.uint8)
    # before peps_set_tensors
    assert lib.peps_sample_batch(c.h, 1, 2, 0, 0, 1, 1, 1, _p(out), None, None, None) == E
    assert b"set_tensors" in lib.peps_last_error(c.h)
    c.set_tensors(make_peps(L, 2, seed=2))
    assert lib.peps_sample_batch(c.h, 1, 2, 0, 0, 0, 1, 1, _p(out), None, None, None) == E  # n_thin
    assert lib.peps_sample_batch(c.h, 1, 2, 1 << 32, 0, 1, 1, 1, _p(out), None, None, None) == E
    assert lib.peps_sample_batch(c.h, 1, 2, 0, 0, 1, 1, 1, None, None, None, None) == E
    assert lib.peps_sample_batch(c.h, 1, 0, 0, 0, 1, 1, 1, None, None, None, None) == 0  # empty
    assert lib.peps_vmc_step(c.h, 1, 0, 0, 1, _p(out), _p(e), None, None, None, None, None, 0,
                             None, None) == E
    assert lib.peps_vmc_step(c.h, 1, 2, 0, 1, None, _p(e), None, None, None, None, None, 0,
                             None, None) == E
    assert lib.peps_local_energy(c.h, _p(sp), 2, None, None, None, None, None, None) == E
    sd = np.zeros(N * 2 * 16)
    se = np.zeros(1)
    A = np.ascontiguousarray(make_peps(L, 2, seed=2))
    assert lib.peps_grad_step(c.h, _p(sd), _p(sd), _p(se), 0, 0.1, 1, 1, _p(A), None) == E  # M
    assert lib.peps_grad_step(c.h, _p(sd), _p(sd), _p(se), 4, float("inf"), 1, 1, _p(A), None) == E
    assert lib.peps_grad_step(c.h, _p(sd), _p(sd), _p(se), 4, 0.1, 1, 1 << 32, _p(A), None) == E
    assert lib.peps_grad_step(c.h, None, _p(sd), _p(se), 4, 0.1, 1, 1, _p(A), None) == E
    ss = np.zeros((2, 1, N))
    bad = np.array([N], np.int32)
    assert lib.peps_correlations(c.h, _p(sp), 2, 1, _p(bad), _p(ss), None, None) == E
    assert b"source" in lib.peps_last_error(c.h)
    assert lib.peps_correlations(c.h, _p(sp), 2, 0, _p(bad), _p(ss), None, None) == E
    assert lib.peps_correlations(c.h, _p(sp), -1, 1, _p(np.array([0], np.int32)), _p(ss), None,
                                 None) == E
    assert c.status() == (0, 0)
    c.close()
    sh32 = Bl.PepsShape(4, 2, 4, 1.0, 0.5, Bl.PEPS_FP32)
    h32 = ctypes.c_void_p()
    assert lib.peps_create(ctypes.byref(sh32), 1, ctypes.byref(h32)) == 0
    A32 = np.ascontiguousarray(make_peps(4, 2, seed=2))
    assert lib.peps_set_tensors(h32, _p(A32), None) == 0
    assert lib.peps_correlations(h32, _p(sp), 2, 1, _p(np.array([0], np.int32)), _p(ss), None,
                                 None) == E  # FP32 form
    lib.peps_destroy(h32)


def test_counter_and_host_buffer_steps_equal_the_direct_step(lib):
    """Two VMC steps with the sweep and GO step numbers in device counters
    (peps_vmc_step_dc, peps_grad_step_dc, peps_counters_advance: the calls a
    CUDA graph replays) and through the host-buffer entry point
    (peps_vmc_step_host) equal the direct calls bit for bit: chain states,
    energies, gradient sums and the updated tensors."""
    from paper_1806_03761_gb300 import _lib as Bl
    lib.peps_counters_advance.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32,
                                          ctypes.c_void_p]
    L, D, Dc, n = 4, 2, 4, 3
    A0 = make_peps(L, D, seed=33)
    start = np.ascontiguousarray(random_sz0_configs(L, n, seed=34))
    runs = {}
    for mode in ("direct", "counters", "host"):
        c = Ctx(lib, L, D, Dc, "mixed", slots=2)
        A = np.ascontiguousarray(A0.copy())
        c.set_tensors(A)
        state = start.copy()
        cnt = np.array([7, 3], np.uint32)
        rec = []
        for step in range(2):
            e = np.zeros(n)
            sd, sde, se = c.sums()
            if mode == "direct":
                assert lib.peps_vmc_step(c.h, 11, n, 0, 7 + step, _p(state), _p(e), None, None, _p(sd),
                                         _p(sde), _p(se), 0, None, None) == 0
                assert lib.peps_grad_step(c.h, _p(sd), _p(sde), _p(se), n, 0.05, 11, 3 + step, _p(A),
                                          None) == 0
            elif mode == "counters":
                assert lib.peps_vmc_step_dc(c.h, 11, n, 0, _p(cnt), _p(state), _p(e), None, None, _p(sd),
                                            _p(sde), _p(se), 0, None, None) == 0
                assert lib.peps_grad_step_dc(c.h, _p(sd), _p(sde), _p(se), n, 0.05, 11, _p(cnt), _p(A),
                                             None) == 0
                assert lib.peps_counters_advance(_p(cnt), 2, 1, None) == 0
            else:
                assert lib.peps_vmc_step_host(c.h, 11, n, 0, 7 + step, _p(state), _p(e), None, None, None,
                                              _p(sd), _p(sde), _p(se), None) == 0
                assert lib.peps_grad_step(c.h, _p(sd), _p(sde), _p(se), n, 0.05, 11, 3 + step, _p(A),
                                          None) == 0
            rec += [state.copy(), e, sd, sde, se, A.copy()]
        assert c.status() == (0, 0)
        c.close()
        runs[mode] = rec
    for mode in ("counters", "host"):
        for a, b in zip(runs["direct"], runs[mode]):
            assert np.array_equal(a, b), mode


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_amplitudes_and_logderiv_entry_points(lib, prec):
    """peps_amplitudes (row-0 strip against Dn_1) and peps_logderiv (Delta of
    every site on its s_m slice, the sums with given energies, accumulate)
    against the oracle and against peps_evaluate."""
    L, D, Dc = 4, 3, 4
    A = make_peps(L, D, seed=101)
    spins = np.ascontiguousarray(random_sz0_configs(L, 3, seed=102))
    N, D4, B = L * L, D ** 4, 3
    tol = TOL[prec]
    c = Ctx(lib, L, D, Dc, prec, slots=2)
    c.set_tensors(A)
    la, sg = np.zeros(B), np.zeros(B, np.int8)
    assert lib.peps_amplitudes(c.h, _p(spins), B, _p(la), _p(sg), None) == 0
    ref = oracle.evaluate_batch(A, spins, L, Dc, want_delta=True)
    assert np.array_equal(sg, ref["sign"].astype(np.int8))
    assert np.max(np.abs(la - ref["log_abs"])) <= tol
    e = np.ascontiguousarray(ref["e_loc"])
    delta = np.zeros((B, N, D4))
    sd, sde, se = c.sums()
    assert lib.peps_logderiv(c.h, _p(spins), B, _p(e), _p(delta), _p(sd), _p(sde), _p(se), 0,
                             None) == 0
    for b in range(B):
        for m in range(N):
            want = ref["delta"][b, m, spins[b][m]].reshape(-1)
            assert np.max(np.abs(delta[b, m] - want)) <= tol * max(1.0, np.abs(want).max())
    # accumulate = 1 adds a second pass to the sums
    sd2, sde2, se2 = sd.copy(), sde.copy(), se.copy()
    assert lib.peps_logderiv(c.h, _p(spins), B, _p(e), None, _p(sd2), _p(sde2), _p(se2), 1,
                             None) == 0
    assert np.allclose(sd2, 2 * sd, rtol=1e-12, atol=0) and np.allclose(sde2, 2 * sde, rtol=1e-12, atol=0)
    assert se2[0] == 2 * se[0] and abs(se[0] - e.sum()) <= 1e-12 * max(1, abs(e.sum()))
    ev = c.evaluate(spins)
    assert np.array_equal(ev["log_abs"], la) and np.array_equal(ev["sign"], sg)
    assert c.status() == (0, 0)
    c.close()
