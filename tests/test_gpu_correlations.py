"""GPU parity of the spin correlations (peps_correlations, peps_structure_factor)
against the FP64 oracle (oracle/correlations.py), element by element: the
S^z S^z part and the 3/4 at the source exactly, the exchange part W(S')/W(S)
relative with a floor of tol * RMS of the sample's exchange ratios (FP64
1e-10, mixed 1e-4), the batch means and m_s^2(k) relative to their scale."""
import numpy as np
import pytest

import oracle
from oracle import correlations as oc
from synth import make_peps, random_sz0_configs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _ctx(L, D, Dc, prec, A, slots=0):
    from paper_1806_03761_gb300 import PepsContext
    ctx = PepsContext(L, D, Dc, precision=prec, slots=slots)
    ctx.set_tensors(torch.from_numpy(A).cuda())
    return ctx


def _check(ss, spins, A, L, Dc, sources, tol):
    worst = 0.0
    for b, s in enumerate(spins):
        for q, a in enumerate(sources):
            ref = oc.local_correlations(A, s, L, Dc, a)
            got = ss[b, q]
            sig = 1.0 - 2.0 * s.astype(np.float64)
            zz = sig[a] * sig / 4.0
            zz[a] = 0.75
            ex_ref, ex_got = 2 * (ref - zz), 2 * (got - zz)
            anti = (s != s[a])
            anti[a] = False
            # parallel pairs and the source: exactly the diagonal part
            assert np.array_equal(got[~anti], ref[~anti]), (b, q)
            if anti.any():
                floor = tol * np.sqrt(np.mean(ex_ref[anti] ** 2))
                err = np.max(np.abs(ex_got[anti] - ex_ref[anti]) /
                             np.maximum(np.abs(ex_ref[anti]), floor / tol))
                worst = max(worst, err)
    return worst


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("L,D,Dc,kind,B", [(4, 2, 4, "gauss", 3), (6, 3, 4, "gauss", 3),
                                           (8, 4, 16, "neel", 2)])
def test_correlations_match_the_oracle(prec, L, D, Dc, kind, B):
    A = make_peps(L, D, seed=60 + L, kind=kind)
    spins = random_sz0_configs(L, B, seed=61 + L)
    sources = [oc.centre_site(L), 0, L - 1, L * L - 1, L + 1]  # centre, corners, inside
    ctx = _ctx(L, D, Dc, prec, A, slots=5)  # 5 slots over B * 5 items
    r = ctx.correlations(torch.from_numpy(spins).cuda(), sources)
    rc, flags = ctx.sync_status()
    assert rc == 0, flags
    ss = r["ss"].cpu().numpy()
    err = _check(ss, spins, A, L, Dc, sources, TOL[prec])
    print(prec, L, D, Dc, "worst exchange-ratio error %.2e" % err)
    assert err <= TOL[prec]
    mean = r["mean"].cpu().numpy()
    assert np.max(np.abs(mean - ss.mean(axis=0))) <= 1e-14
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_structure_factor_over_the_bulk(prec):
    L, D, Dc = 6, 3, 4
    A = make_peps(L, D, seed=70)
    spins = random_sz0_configs(L, 4, seed=71)
    bulk = oc.bulk_sites(L)
    ctx = _ctx(L, D, Dc, prec, A)
    r = ctx.correlations(torch.from_numpy(spins).cuda(), bulk)
    ref_C = np.mean([[oc.local_correlations(A, s, L, Dc, a) for a in bulk] for s in spins], axis=0)
    for k in ((np.pi, np.pi), (0.0, 0.0), (np.pi, 0.0)):
        m2 = ctx.structure_factor(r["mean"], bulk, k).item()
        want = oc.structure_factor(ref_C, L, bulk, k)
        assert abs(m2 - want) <= TOL[prec] * max(1.0, abs(want)), (k, m2, want)
    assert ctx.sync_status()[0] == 0
    ctx.close()


def test_correlation_arguments_are_checked():
    from paper_1806_03761_gb300 import PepsError
    L, D, Dc = 4, 2, 4
    A = make_peps(L, D, seed=1)
    ctx = _ctx(L, D, Dc, "fp64", A)
    sp = torch.from_numpy(random_sz0_configs(L, 1, seed=2)).cuda()
    with pytest.raises(PepsError):
        ctx.correlations(sp, [16])          # source outside the lattice
    with pytest.raises(PepsError):
        ctx.correlations(sp, [])            # no source
    r = ctx.correlations(sp, [5])
    with pytest.raises(PepsError):
        ctx.structure_factor(r["mean"], [5])  # the bulk (all 16 sites at L = 4) is not covered
    ctx.close()
    c32 = _ctx(L, D, Dc, "fp32", A)
    with pytest.raises(PepsError):
        c32.correlations(sp, [5])
    c32.close()
