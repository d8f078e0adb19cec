"""The N>1 host path with two gloo ranks on CPU: chain sharding, the
all-reduce of the gradient accumulators, and the identical GO update on every
rank, against the single-process result (oracle arithmetic, tiny lattice)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

L, D, DC, CHAINS, SEED = 2, 2, 4, 3, 77


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_sums(rank, world):
    import oracle
    from paper_1806_03761_gb300.dist import weak_scaling_plan
    from synth import make_peps
    A = make_peps(L, D, seed=5)
    off, n, _ = weak_scaling_plan(rank, world, CHAINS)
    out, _, _ = oracle.sample_chains(A, L, DC, SEED, n, 2, 1, 1, chain_offset=off)
    r = oracle.evaluate_batch(A, out, L, DC, want_delta=True)
    sd = np.zeros((L * L, 2, D ** 4))
    sde = np.zeros_like(sd)
    for b in range(n):
        for m in range(L * L):
            dv = r["delta"][b, m, out[b][m]].reshape(-1)
            sd[m, out[b][m]] += dv
            sde[m, out[b][m]] += dv * r["e_loc"][b]
    return A, [torch.from_numpy(sd), torch.from_numpy(sde), torch.tensor([r["e_loc"].sum()])]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1806_03761_gb300.dist import allreduce_sums, weak_scaling_plan
    A, sums = _rank_sums(rank, world)
    allreduce_sums(sums, world)
    _, _, M = weak_scaling_plan(rank, world, CHAINS)
    g = oracle.gradient(sums[0].numpy(), sums[1].numpy(), float(sums[2][0]), M)
    An = oracle.go_step(A, g.reshape(A.shape), 0.01, SEED, 3)
    q.put((rank, An, sums[2].item()))
    dist.destroy_process_group()


def test_two_rank_allreduce_matches_single_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda x: x[0])
    assert np.array_equal(res[0][1], res[1][1])  # identical update on both ranks
    # single process over all 2*CHAINS chains gives the same sums and update
    import oracle
    A, s0 = _rank_sums(0, 2)
    _, s1 = _rank_sums(1, 2)
    tot = [a + b for a, b in zip(s0, s1)]
    assert abs(tot[2].item() - res[0][2]) < 1e-12 * max(1, abs(tot[2].item()))
    g = oracle.gradient(tot[0].numpy(), tot[1].numpy(), float(tot[2][0]), 2 * CHAINS)
    An = oracle.go_step(A, g.reshape(A.shape), 0.01, SEED, 3)
    assert np.array_equal(An, res[0][1])


def test_shard_bounds():
    from paper_1806_03761_gb300.dist import shard
    assert shard(0, 4, 10) == (0, 10) and shard(3, 4, 10) == (30, 10)
    with pytest.raises(ValueError):
        shard(4, 4, 10)


def test_weak_scaling_plan_keeps_the_per_rank_batch():
    """The bench's layout for world = 1, 2, 8: every rank runs B chains, the
    ranks' chain ranges are disjoint and together cover 0 .. B*world-1, and the
    gradient mean divides by M = B * world (the chains actually summed)."""
    from paper_1806_03761_gb300.dist import weak_scaling_plan
    B = 608
    for world in (1, 2, 8):
        seen = []
        for rank in range(world):
            off, n, M = weak_scaling_plan(rank, world, B)
            assert n == B and M == B * world
            seen.extend(range(off, off + n))
        assert sorted(seen) == list(range(B * world))
