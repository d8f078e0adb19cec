"""Per-phase cycle counters of the fused VMC kernel (peps_phase_cycles): a
library built with PEPS_PHASES=1 reports every phase, nested phases within
their parents; the default build reports none.  The step's results do not
depend on the counters (the same outputs bit for bit)."""
import numpy as np
import pytest

from synth import make_peps, random_sz0_configs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _step(ctx, A, spins):
    ctx.set_tensors(torch.from_numpy(A).cuda())
    st = torch.from_numpy(spins.copy()).cuda()
    r = ctx.vmc_step(5, st, 3)
    assert ctx.sync_status()[0] == 0
    return r["e_loc"].cpu().numpy(), st.cpu().numpy()


def test_phase_counters():
    from paper_1806_03761_gb300 import PepsContext
    L, D, Dc = 6, 4, 16
    A = make_peps(L, D, seed=91)
    spins = random_sz0_configs(L, 4, seed=92)
    plain = PepsContext(L, D, Dc, precision="mixed", slots=2)
    e0, s0 = _step(plain, A, spins)
    assert plain.phase_cycles() == {}
    plain.close()
    traced = PepsContext(L, D, Dc, precision="mixed", slots=2, variant={"PEPS_PHASES": 1})
    e1, s1 = _step(traced, A, spins)
    ph = traced.phase_cycles()
    assert np.array_equal(e0, e1) and np.array_equal(s0, s1)
    assert set(ph) == set(PepsContext.PHASES)
    for k in ("eval", "sweep", "compress", "qr", "svd", "strip1", "strip2", "sweep_h", "sweep_r2",
              "sweep_v"):
        assert ph[k] > 0, k
    assert ph["compress"] >= ph["qr"] + ph["svd_qr"] + ph["svd"]
    assert ph["eval"] + ph["sweep"] >= ph["compress"]
    assert ph["eval"] >= ph["strip1"] + ph["ratio_h"] + ph["btens"] + ph["strip2"] + ph["ratio_2"]
    assert ph["sweep"] >= ph["sweep_h"] + ph["sweep_r2"] + ph["sweep_v"]
    assert traced.phase_cycles()["eval"] == 0  # read clears
    traced.close()
