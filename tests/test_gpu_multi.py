"""Jobs of different shapes in one persistent launch (peps_local_energy_multi):
every job's energies, amplitudes, flip ratios and flip counts are bit-identical
to its own peps_local_energy (the same per-sample code), with a pool of fewer
slots than items (blocks take items from the queue one after another) and in
both precision forms."""
import numpy as np
import pytest

from synth import make_peps, random_sz0_configs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

JOBS = [(4, 2, 4, 7), (6, 3, 4, 5), (8, 4, 16, 4), (5, 2, 3, 9), (6, 2, 8, 3)]  # L, D, Dc, B


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_mixed_shapes_in_one_launch_equal_their_own_launches(prec):
    from paper_1806_03761_gb300 import PepsContext, PepsPool
    ctxs, spins = [], []
    for q, (L, D, Dc, B) in enumerate(JOBS):
        c = PepsContext(L, D, Dc, precision=prec, slots=2)
        c.set_tensors(torch.from_numpy(make_peps(L, D, seed=80 + q, kind="neel" if L == 8 else "gauss")).cuda())
        ctxs.append(c)
        spins.append(torch.from_numpy(random_sz0_configs(L, B, seed=90 + q)).cuda())
    pool = PepsPool([j[:3] for j in JOBS], precision=prec, slots=6, max_jobs=8)
    assert pool.slots == 6 and sum(j[3] for j in JOBS) > 6
    outs = pool.local_energy(list(zip(ctxs, spins)), ratios=True, n_flips=True)
    rc, flags = pool.sync_status()
    assert rc == 0, flags
    for c, s, o in zip(ctxs, spins, outs):
        ref = c.local_energy(s, ratios=True, n_flips=True)
        torch.cuda.synchronize()
        for k in ("e_loc", "log_abs", "sign", "ratios", "n_flips"):
            assert torch.equal(o[k], ref[k]), k
        c.close()
    pool.close()


def test_pool_refuses_a_shape_it_was_not_sized_for():
    from paper_1806_03761_gb300 import PepsContext, PepsError, PepsPool
    pool = PepsPool([(4, 2, 4)], precision="fp64", slots=2, max_jobs=2)
    c = PepsContext(8, 4, 16, precision="fp64", slots=1)
    c.set_tensors(torch.from_numpy(make_peps(8, 4, seed=1)).cuda())
    with pytest.raises(PepsError):
        pool.local_energy([(c, torch.from_numpy(random_sz0_configs(8, 2, seed=1)).cuda())])
    c.close()
    pool.close()
