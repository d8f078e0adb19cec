"""Host logic of the GO loop on the CPU: the step-length schedule, the energy
criterion and the checkpoint round trip, with a stand-in for the library
context (deterministic arithmetic in torch on the CPU, no device)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1806_03761_gb300.go import GOLoop  # noqa: E402


class FakeContext:
    """Mimics the PepsContext calls GOLoop makes: sample, vmc_step,
    new_sums, grad_step, set_tensors.  Energies depend on A, the step's sweep
    number and the chain states, so any counter mix-up changes the history."""

    def __init__(self, L=3, D=2, Dc=2, precision="fp64"):
        self.L, self.D, self.Dc, self.precision = L, D, Dc, precision
        self.N = L * L
        self.calls = []

    def set_tensors(self, A):
        self.A = A

    def new_sums(self):
        return (torch.zeros(self.N * 2 * self.D ** 4, dtype=torch.float64),
                torch.zeros_like(torch.zeros(self.N * 2 * self.D ** 4, dtype=torch.float64)),
                torch.zeros(1, dtype=torch.float64))

    def sample(self, seed, n_chains, n_burn, n_thin, spc, chain_offset=0, first_sweep=1):
        g = torch.Generator().manual_seed(seed + n_burn)
        return (torch.rand(n_chains * spc, self.N, generator=g) < 0.5).to(torch.uint8)

    def vmc_step(self, seed, state, sweep, chain_offset=0, sums=None, accumulate=False):
        self.calls.append(("vmc", sweep, accumulate))
        e = float(self.A.sum()) * 1e-3 - 0.01 * sweep + state.double().mean()
        if not accumulate:
            for x in sums:
                x.zero_()
        sums[0].add_(1.0)
        sums[1].add_(e)
        sums[2].add_(e * state.shape[0])
        state.copy_(1 - state)  # the "sweep"
        return {}

    def grad_step(self, sums, M, dt, seed, step, A):
        self.calls.append(("grad", step, dt, M))
        A.sub_(dt)


def _loop(ctx, **kw):
    A = torch.ones(ctx.N, 2, ctx.D, ctx.D, ctx.D, ctx.D, dtype=torch.float64)
    args = dict(seed=5, n_chains=4, samples_per_step=3, n_burn=2, dt0=1e-2, decay=0.5, tol=0.0)
    args.update(kw)
    return GOLoop(ctx, A, **args)


def test_schedule_counters_and_criterion():
    ctx = FakeContext()
    loop = _loop(ctx)
    loop.run(3)
    grads = [c for c in ctx.calls if c[0] == "grad"]
    assert [c[1] for c in grads] == [0, 1, 2]
    assert [c[2] for c in grads] == [1e-2, 5e-3, 2.5e-3]  # dt0 * decay**n
    assert all(c[3] == 4 * 3 for c in grads)  # M = chains x samples per step
    vmc = [c for c in ctx.calls if c[0] == "vmc"]
    assert [c[1] for c in vmc] == list(range(3, 3 + 9))  # sweeps after the burn-in
    assert [c[2] for c in vmc[:3]] == [False, True, True]
    assert len(loop.energies) == 3 and not loop.converged()
    # the criterion: two steps with equal energies stop the loop
    loop2 = _loop(FakeContext(), tol=1.0)
    loop2.run(10)
    assert len(loop2.energies) == 2


def test_checkpoint_round_trip(tmp_path):
    ref = _loop(FakeContext())
    ref.run(4)
    part = _loop(FakeContext())
    ck = str(tmp_path / "go.npz")
    part.run(2, checkpoint=ck)
    back = GOLoop.load(ck, ctx=FakeContext(), device="cpu")
    assert (back.step, back.sweep, back.seed, back.n_chains, back.spc) == (2, part.sweep, 5, 4, 3)
    assert (back.dt0, back.decay, back.tol) == (1e-2, 0.5, 0.0)
    back.run(2)
    assert back.energies == ref.energies
    assert torch.equal(back.A, ref.A) and torch.equal(back.state, ref.state)
    with pytest.raises(ValueError):  # a context of another shape
        GOLoop.load(ck, ctx=FakeContext(L=4), device="cpu")
    assert not (tmp_path / "go.npz.tmp").exists()
    np.load(ck)  # a complete archive
