"""Serving loop with continuous batching (peps_server_*): each job's result is
the same alone and in a mix of jobs of other shapes and precision forms, the
HBM budget gates admission, and oversized or invalid jobs are refused."""
import numpy as np
import pytest

from synth import make_peps, random_sz0_configs

JOBS = [  # (L, D, Dc, precision, B, tensor seed, recipe)
    (4, 2, 4, "fp64", 40, 11, "gauss"),
    (6, 2, 4, "mixed", 24, 12, "gauss"),
    (5, 3, 6, "fp64", 16, 13, "gauss"),
    (8, 2, 4, "mixed", 70, 14, "neel"),
    (6, 3, 9, "fp32", 8, 15, "gauss"),
]


def _inputs(job):
    L, D, Dc, prec, B, seed, recipe = job
    return make_peps(L, D, seed, recipe), random_sz0_configs(L, B, seed + 100)


@pytest.fixture(scope="module")
def server_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_1806_03761_gb300 as P
    return P


@pytest.mark.gpu
def test_mix_equals_alone_equals_context(server_mod):
    P = server_mod
    import torch
    srv = P.PepsServer(slots_per_job=32)  # several waves for the larger jobs
    inputs = [_inputs(j) for j in JOBS]
    alone = []
    for job, (A, S) in zip(JOBS, inputs):
        L, D, Dc, prec = job[:4]
        alone.append(srv.wait(srv.submit(A, S, L, D, Dc, prec)))
    ids = [srv.submit(A, S, j[0], j[1], j[2], j[3]) for j, (A, S) in zip(JOBS, inputs)]
    mixed = [srv.wait(i) for i in ids]
    srv.close()
    for job, (A, S), a, m in zip(JOBS, inputs, alone, mixed):
        assert a["status"] == 0 and m["status"] == 0, job
        # the same per-sample code alone and in the mix: bit-identical
        assert np.array_equal(a["e_loc"], m["e_loc"]), job
        assert np.array_equal(a["log_abs"], m["log_abs"]), job
        assert np.array_equal(a["sign"], m["sign"]), job
        L, D, Dc, prec = job[:4]
        ctx = P.PepsContext(L, D, Dc, precision=prec, slots=32)
        ctx.set_tensors(torch.from_numpy(A).cuda())
        r = ctx.local_energy(torch.from_numpy(S).cuda())
        assert np.array_equal(r["e_loc"].cpu().numpy(), m["e_loc"]), job
        assert np.array_equal(r["sign"].cpu().numpy(), m["sign"]), job
        ctx.close()


@pytest.mark.gpu
def test_mix_matches_oracle(server_mod):
    import oracle
    P = server_mod
    srv = P.PepsServer()
    picks = [JOBS[0], JOBS[1], JOBS[3]]
    inputs = [_inputs(j) for j in picks]
    ids = [srv.submit(A, S, j[0], j[1], j[2], j[3]) for j, (A, S) in zip(picks, inputs)]
    res = [srv.wait(i) for i in ids]
    srv.close()
    for job, (A, S), r in zip(picks, inputs, res):
        L, D, Dc, prec = job[:4]
        tol = 1e-10 if prec == "fp64" else 1e-4
        for b in range(3):
            o = oracle.evaluate(A, S[b], L, Dc)
            assert r["sign"][b] == o["sign"]
            assert abs(r["log_abs"][b] - o["log_abs"]) <= tol
            assert abs(r["e_loc"][b] - o["e_loc"]) <= tol * max(1.0, abs(o["e_loc"]))


@pytest.mark.gpu
def test_budget_gates_admission(server_mod):
    P = server_mod
    job = JOBS[3]
    A, S = _inputs(job)
    L, D, Dc, prec = job[:4]
    probe = P.PepsServer(slots_per_job=32)
    fp = probe.wait(probe.submit(A, S, L, D, Dc, prec))["footprint_bytes"]
    probe.close()
    # room for one such job at a time: the second waits for the first
    srv = P.PepsServer(hbm_budget_bytes=int(1.5 * fp), slots_per_job=32)
    ids = [srv.submit(A, S, L, D, Dc, prec) for _ in range(3)]
    res = [srv.wait(i) for i in ids]
    srv.close()
    for k in range(1, 3):
        assert res[k]["admit_s"] >= res[k - 1]["done_s"] - 1e-6
        assert np.array_equal(res[k]["e_loc"], res[0]["e_loc"])
    with pytest.raises(P.PepsError):  # alone larger than the budget
        small = P.PepsServer(hbm_budget_bytes=fp // 2, slots_per_job=32)
        try:
            small.submit(A, S, L, D, Dc, prec)
        finally:
            small.close()


@pytest.mark.gpu
def test_invalid_jobs_refused(server_mod):
    P = server_mod
    srv = P.PepsServer()
    A, S = _inputs(JOBS[0])
    with pytest.raises(P.PepsError):
        srv.submit(A, S, 4, 2, 200, "fp64")  # Dc * D > 256
    with pytest.raises(P.PepsError):
        srv.submit(A, S[:0], 4, 2, 4, "fp64")  # empty batch
    srv.close()


@pytest.mark.gpu
def test_a_job_arriving_later_overlaps_a_running_one(server_mod):
    """Continuous batching: under an ample budget a short job submitted while
    a long one runs is admitted and finished before the long one is done,
    and its result is the one it has alone."""
    P = server_mod
    long_job = (8, 4, 16, "mixed", 64, 21, "neel")  # 16 waves of 4 slots
    short_job = (4, 2, 4, "fp64", 4, 22, "gauss")   # one wave
    (Al, Sl), (As, Ss) = _inputs(long_job), _inputs(short_job)
    srv = P.PepsServer(slots_per_job=4)
    alone = srv.wait(srv.submit(As, Ss, *short_job[:4]))
    i_long = srv.submit(Al, Sl, *long_job[:4])
    i_short = srv.submit(As, Ss, *short_job[:4])
    r_short = srv.wait(i_short)
    r_long = srv.wait(i_long)
    srv.close()
    assert r_long["status"] == 0 and r_short["status"] == 0
    assert r_short["admit_s"] < r_long["done_s"]
    assert r_short["done_s"] < r_long["done_s"]
    assert np.array_equal(r_short["e_loc"], alone["e_loc"])
    assert np.array_equal(r_short["sign"], alone["sign"])


@pytest.mark.gpu
def test_eviction_under_a_tight_budget_keeps_results(server_mod):
    """Idle contexts are evicted (freed off the worker thread) when a new
    shape needs their memory; every job still returns its alone result."""
    P = server_mod
    jobs = [JOBS[0], JOBS[2], JOBS[0], JOBS[2]]
    inputs = [_inputs(j) for j in jobs]
    probe = P.PepsServer(slots_per_job=8)
    alone = [probe.wait(probe.submit(A, S, *j[:4])) for j, (A, S) in zip(jobs, inputs)]
    fps = [a["footprint_bytes"] for a in alone]
    probe.close()
    # room for one job's context and buffers at a time: every shape change
    # evicts the other shape's idle context
    srv = P.PepsServer(hbm_budget_bytes=int(1.2 * max(fps)), slots_per_job=8)
    ids = [srv.submit(A, S, *j[:4]) for j, (A, S) in zip(jobs, inputs)]
    res = [srv.wait(i) for i in ids]
    srv.close()
    for a, r in zip(alone, res):
        assert r["status"] == 0
        assert np.array_equal(a["e_loc"], r["e_loc"])
