"""The GO main loop (Step B): it follows the oracle's loop step for step
(FP64: chains bit-exact, energies and tensors to rounding), and a loop saved
and restored from a checkpoint continues bit-identically."""
import numpy as np
import pytest

from synth import make_peps

torch = pytest.importorskip("torch")


def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_1806_03761_gb300 as P
    from paper_1806_03761_gb300.go import GOLoop
    return P, GOLoop


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_resume_is_bit_identical(tmp_path, prec):
    P, GOLoop = _gpu()
    L, D, Dc = 4, 2, 4
    A0 = make_peps(L, D, 21, "gauss")
    kw = dict(seed=77, n_chains=24, samples_per_step=2, n_burn=3, dt0=2e-3, decay=0.9)
    ref = GOLoop(P.PepsContext(L, D, Dc, precision=prec, slots=16), torch.from_numpy(A0.copy()).cuda(), **kw)
    ref.run(4)
    part = GOLoop(P.PepsContext(L, D, Dc, precision=prec, slots=16), torch.from_numpy(A0.copy()).cuda(), **kw)
    ck = str(tmp_path / "go.npz")
    part.run(2, checkpoint=ck)
    del part
    resumed = GOLoop.load(ck, slots=16)
    assert resumed.step == 2
    resumed.run(2)
    assert resumed.energies == ref.energies
    assert torch.equal(resumed.A, ref.A)
    assert torch.equal(resumed.state, ref.state)
    assert not np.array_equal(ref.A.cpu().numpy(), A0)  # the tensors did move


@pytest.mark.gpu
def test_loop_follows_the_oracle():
    import oracle
    P, GOLoop = _gpu()
    L, D, Dc, n, seed, nb = 4, 2, 16, 6, 91, 2
    dt0, decay = 3e-3, 0.8
    A0 = make_peps(L, D, 22, "gauss")
    loop = GOLoop(P.PepsContext(L, D, Dc, precision="fp64"), torch.from_numpy(A0.copy()).cuda(),
                  seed, n, samples_per_step=1, n_burn=nb, dt0=dt0, decay=decay)
    loop.run(2)
    # the same loop written with the oracle's pieces
    N, D4 = L * L, D ** 4
    A = A0.copy()
    state = oracle.sample_chains(A, L, Dc, seed, n, nb - 1, 1, 1)[0]
    sweep = nb + 1
    energies = []
    for step in range(2):
        ev = oracle.evaluate_batch(A, state, L, Dc, want_delta=True)
        sd = np.zeros((N, 2, D4))
        sde = np.zeros((N, 2, D4))
        for b in range(n):
            for m in range(N):
                dv = ev["delta"][b, m, state[b][m]].reshape(-1)
                sd[m, state[b][m]] += dv
                sde[m, state[b][m]] += dv * ev["e_loc"][b]
        se = float(np.sum(ev["e_loc"]))
        energies.append(se / n / N)
        state = oracle.sample_chains(A, L, Dc, seed, n, 0, 1, 1, init=state, first_sweep=sweep)[1]
        sweep += 1
        g = oracle.gradient(sd, sde, se, n)
        A = oracle.go_step(A, g.reshape(A.shape), dt0 * decay ** step, seed, step)
    assert np.array_equal(loop.state.cpu().numpy(), state)
    assert np.allclose(loop.energies, energies, rtol=1e-10, atol=1e-12)
    diff = loop.A.cpu().numpy() != A
    # a differing element needs a gradient sign decided by rounding
    gmax = np.abs(g).max()
    assert not np.any(diff & (np.abs(g.reshape(A.shape)) > 1e-8 * gmax))
