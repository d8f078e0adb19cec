"""GPU parity on the 64-configuration subset of the 16x16, D=6, Dc=24 workload
against the FP64 oracle's stored results (tests/golden/oracle_16x16_D6_Dc24.npz,
written by tests/golden/make_golden_16x16.py, which calls only the oracle and
the seeded generators), in both precision forms, element by element: sign,
flip count and the zero pattern of the ratios exactly; log|W|, E(S), every
flip ratio and a seeded sample of 4096 entries of the Delta sums within the
bounds below.  Each quantity's worst error and its ratio to its bound are
printed.

Bounds.  The amplitude of a 16x16 Gaussian PEPS carries heavy cancellation
(W(S) is about 1e-6 of the norms of the tensors it is contracted from), so two
backward-stable FP64 evaluations differ by about kappa * u, above the plain
1e-10 tolerance on some configurations.  The golden file stores each result's
sensitivity s: its largest change over 8 seeded relative perturbations of A
by one unit roundoff u = 2^-52.  A perturbation in a random direction moves
a result by |N(0, sigma)|, and the largest of 8 draws is about 1.9 sigma;
the rounding errors of one evaluation act like a perturbation of about
sqrt(K) u, K the length of its longest reduction (K_max = Dc D D = 864, the
columns of the QR sweep), and two evaluations (GPU and oracle) add in
quadrature, so at 4 sigma the difference stays below
sqrt(2) * 4 / 1.9 * sqrt(K_max) * s ~= 3 sqrt(K_max) s = 88 s.  Hence
    FP64:  bound = max(1e-10, 3 sqrt(K_max) s)
    mixed: bound = max(1e-4,  3 sqrt(K_max) s * 16)
the float-float form's rounding unit being 2^-48 = 16 u."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden", "oracle_16x16_D6_Dc24.npz")
TOL = {"fp64": 1e-10, "mixed": 1e-4}
UNIT = {"fp64": 1.0, "mixed": 16.0}


@pytest.fixture(scope="module")
def gold():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    g = np.load(GOLD)
    return {k: g[k] for k in g.files}


def _factor(g):
    kmax = int(g["Dc"]) * int(g["D"]) ** 2
    return 3.0 * np.sqrt(kmax)


def check_against_gold(g, res, prec, first=None):
    """res: numpy arrays of the GPU results on the golden configurations
    (the first `first` of them, default all).  Returns {quantity: (worst
    error, worst error / bound)}."""
    B = g["spins"].shape[0] if first is None else first
    c = _factor(g) * UNIT[prec]
    tol = TOL[prec]
    assert np.array_equal(res["sign"][:B], g["sign"][:B])
    out = {}

    def record(name, err, bound):
        w, r = out.get(name, (0.0, 0.0))
        out[name] = (max(w, float(err)), max(r, float(err / bound)))

    for b in range(B):
        bl = max(tol, c * g["sens_log_abs"][b])
        record("log_abs", abs(res["log_abs"][b] - g["log_abs"][b]), bl)
        be = max(tol, c * g["sens_e_loc"][b])
        record("e_loc", abs(res["e_loc"][b] - g["e_loc"][b]) / max(1.0, abs(g["e_loc"][b])), be)
        if "ratios" in res:
            rr = g["ratios"][b]
            assert np.array_equal(res["ratios"][b] == 0, rr == 0), b
            m = rr != 0
            floor = tol * np.sqrt(np.mean(rr[m] ** 2))
            er = np.max(np.abs(res["ratios"][b][m] - rr[m]) / np.maximum(np.abs(rr[m]), floor))
            record("ratios", er, max(tol, c * g["sens_ratios"][b]))
    return out


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_64_configurations_16x16_D6_Dc24_against_the_oracle(gold, prec):
    from paper_1806_03761_gb300 import PepsContext
    from synth import make_peps
    g = gold
    L, D, Dc = int(g["L"]), int(g["D"]), int(g["Dc"])
    A = make_peps(L, D, int(g["tensor_seed"]))
    ctx = PepsContext(L, D, Dc, precision=prec)
    ctx.set_tensors(torch.from_numpy(A).cuda())
    sp = torch.from_numpy(np.ascontiguousarray(g["spins"])).cuda()
    r = ctx.evaluate(sp, ratios=True, n_flips=True)
    rc, flags = ctx.sync_status()
    assert rc == 0, flags
    res = {k: r[k].cpu().numpy() for k in ("e_loc", "log_abs", "sign", "ratios", "n_flips")}
    assert np.array_equal(res["n_flips"], g["n_flips"])
    errs = check_against_gold(g, res, prec)
    # the Delta sums (Eq. gradients) on the stored sample of entries
    c = _factor(g) * UNIT[prec]
    bs = max(TOL[prec], c * float(g["sens_sums"]))
    idx = g["sum_index"]
    sd = r["sum_delta"].cpu().numpy().reshape(-1)[idx]
    sde = r["sum_delta_e"].cpu().numpy().reshape(-1)[idx]
    e_sd = np.max(np.abs(sd - g["sum_delta"])) / float(g["sum_delta_absmax"])
    e_sde = np.max(np.abs(sde - g["sum_delta_e"])) / float(g["sum_delta_e_absmax"])
    e_se = abs(r["sum_e"].item() - float(g["sum_e"])) / max(1.0, abs(float(g["sum_e"])))
    errs["sum_delta"] = (e_sd, e_sd / bs)
    errs["sum_delta_e"] = (e_sde, e_sde / bs)
    errs["sum_e"] = (e_se, e_se / max(TOL[prec], c * float(np.max(g["sens_e_loc"]))))
    print(prec, {k: "%.2e (%.2f of bound)" % v for k, v in errs.items()})
    ctx.close()
    for k, (e, ratio) in errs.items():
        assert ratio <= 1.0, (k, e, ratio)
