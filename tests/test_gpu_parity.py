"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle,
element by element, on seeded synthetic inputs.

Tolerances: FP64 form 1e-10, mixed (float-float) form 1e-4 -- relative on
E(S), on W(S) as |dlog|W|| with equal signs, on every flip ratio (with an
absolute floor of tol * RMS of the sample's ratios) and on the Delta sums
(relative to their largest entry).  Integer outputs (signs, flip counts,
sampled spins) must match exactly.  The 16x16, D=6, Dc=24 workload, whose
amplitudes are ill-conditioned, is compared with the oracle's stored results
under a conditioning-aware bound in test_gpu_golden.py."""
import numpy as np
import pytest

import oracle
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


def ctx_for(L, D, Dc, prec, slots=0, J2=0.5):
    from paper_1806_03761_gb300 import PepsContext
    return PepsContext(L, D, Dc, J1=1.0, J2=J2, precision=prec, slots=slots)


def check_eval(A, spins, L, D, Dc, prec, slots=0, delta=True):
    tol = TOL[prec]
    ctx = ctx_for(L, D, Dc, prec, slots)
    ctx.set_tensors(torch.from_numpy(A).cuda())
    sp = torch.from_numpy(np.ascontiguousarray(spins)).cuda()
    res = ctx.evaluate(sp, ratios=True, n_flips=True, delta=delta)
    rc, flags = ctx.sync_status()
    assert rc == 0, flags
    ref = oracle.evaluate_batch(A, spins, L, Dc, want_delta=delta)
    la = res["log_abs"].cpu().numpy()
    sg = res["sign"].cpu().numpy()
    e = res["e_loc"].cpu().numpy()
    r = res["ratios"].cpu().numpy()
    nf = res["n_flips"].cpu().numpy()
    assert np.array_equal(sg, ref["sign"].astype(np.int8))
    assert np.array_equal(nf, ref["n_flips"])
    err = dict(log_abs=np.max(np.abs(la - ref["log_abs"])),
               e_loc=np.max(np.abs(e - ref["e_loc"]) / np.maximum(1.0, np.abs(ref["e_loc"]))))
    for b in range(len(spins)):
        rr = ref["ratios"][b]
        assert np.array_equal(r[b] == 0, rr == 0)
        m = rr != 0
        if m.any():
            floor = tol * np.sqrt(np.mean(rr[m] ** 2))
            err["ratios"] = max(err.get("ratios", 0.0),
                                np.max(np.abs(r[b][m] - rr[m]) / np.maximum(np.abs(rr[m]), floor / tol)))
    if delta:
        N, D4 = L * L, D ** 4
        sd = np.zeros((N, 2, D4))
        sde = np.zeros((N, 2, D4))
        for b in range(len(spins)):
            for mm in range(N):
                dv = ref["delta"][b, mm, spins[b][mm]].reshape(-1)
                sd[mm, spins[b][mm]] += dv
                sde[mm, spins[b][mm]] += dv * ref["e_loc"][b]
        gd = res["sum_delta"].cpu().numpy()
        gde = res["sum_delta_e"].cpu().numpy()
        err["sum_delta"] = np.max(np.abs(gd - sd)) / np.abs(sd).max()
        err["sum_delta_e"] = np.max(np.abs(gde - sde)) / np.abs(sde).max()
        err["sum_e"] = abs(res["sum_e"].item() - ref["e_loc"].sum()) / max(1, abs(ref["e_loc"].sum()))
        dg = res["delta"].cpu().numpy()
        dr = np.stack([ref["delta"][b, np.arange(N), spins[b]].reshape(N, -1) for b in range(len(spins))])
        err["delta"] = np.max(np.abs(dg - dr)) / np.abs(dr).max()
    bound = {k: tol for k in err}
    print(prec, L, D, Dc, {k: "%.2e" % v for k, v in err.items()})
    for k, v in err.items():
        assert v <= bound[k], (k, v, bound[k])
    ctx.close()
    return err


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_parity_4x4_D2_Dc16_exact_regime(prec):
    A = make_peps(4, 2, seed=1)
    spins = random_sz0_configs(4, 40, seed=2)
    check_eval(A, spins, 4, 2, 16, prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_parity_6x6_D3_Dc4_truncated_ragged_batch(prec):
    A = make_peps(6, 3, seed=3)
    spins = random_sz0_configs(6, 7, seed=4)
    check_eval(A, spins, 6, 3, 4, prec, slots=3)  # 7 samples over 3 slots


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_parity_8x8_D4_Dc16_neel(prec):
    A = make_peps(8, 4, seed=2, kind="neel", eps=1e-2)
    spins = random_sz0_configs(8, 10, seed=3)
    check_eval(A, spins, 8, 4, 16, prec)


def test_full_wave_16x16_in_the_bench_launch():
    # the bench's launch configuration: one wave of 304 chains on the default
    # slots, both forms; every output compared across forms (a property at
    # any size) and the first 64 against the oracle's stored results (the
    # golden configurations are the workload's first 64)
    from tests.test_gpu_golden import GOLD, check_against_gold
    L, D, Dc, B = 16, 6, 24, 304
    A = make_peps(L, D, seed=4)
    spins = random_sz0_configs(L, B, seed=5)
    g = dict(np.load(GOLD))
    assert np.array_equal(g["spins"], spins[:64])
    sp = torch.from_numpy(spins).cuda()
    res = {}
    for prec in ("fp64", "mixed"):
        ctx = ctx_for(L, D, Dc, prec)
        assert ctx.slots >= B
        ctx.set_tensors(torch.from_numpy(A).cuda())
        r = ctx.local_energy(sp)
        rc, flags = ctx.sync_status()
        assert rc == 0, flags
        res[prec] = {k: r[k].cpu().numpy() for k in ("e_loc", "log_abs", "sign")}
        ctx.close()
    e64, emx = res["fp64"]["e_loc"], res["mixed"]["e_loc"]
    assert np.array_equal(res["fp64"]["sign"], res["mixed"]["sign"])
    de = np.abs(emx - e64) / np.maximum(1.0, np.abs(e64))
    dl = np.abs(res["mixed"]["log_abs"] - res["fp64"]["log_abs"])
    # every chain: within the mixed form's conditioning bound at the largest
    # sensitivity the oracle measured on the workload's subset (the chains
    # beyond the first 64 have no sensitivity of their own); most within 1e-4
    c = 3.0 * np.sqrt(Dc * D * D) * 16.0
    be = max(TOL["mixed"], c * float(np.max(g["sens_e_loc"])))
    bl = max(TOL["mixed"], c * float(np.max(g["sens_log_abs"])))
    print("mixed vs fp64 over the wave: E max %.2e (bound %.2e) median %.2e, %d above 1e-4; "
          "log|W| max %.2e (bound %.2e)" % (de.max(), be, np.median(de), int((de > 1e-4).sum()),
                                          dl.max(), bl))
    assert de.max() <= be and dl.max() <= bl
    assert np.mean(de <= TOL["mixed"]) >= 0.99
    for prec in ("fp64", "mixed"):
        errs = check_against_gold(g, res[prec], prec, first=64)
        print(prec, "first 64 vs oracle:", {k: "%.2e (%.2f of bound)" % v for k, v in errs.items()})
        for k, (e, ratio) in errs.items():
            assert ratio <= 1.0, (prec, k, e, ratio)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_parity_6x6_D8_Dc32_tall_panels(prec):
    # D*Dc = 256: the QR sweep's panels reach 2048 x 256 (the tall blocked
    # path) and the SVDs 256 x 256
    A = make_peps(6, 8, seed=6)
    spins = random_sz0_configs(6, 2, seed=7)
    check_eval(A, spins, 6, 8, 32, prec, delta=False)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_amplitudes_and_logderiv_entry_points(prec):
    L, D, Dc = 5, 2, 4
    tol = TOL[prec]
    A = make_peps(L, D, seed=9)
    spins = random_sz0_configs(L, 9, seed=10)
    ctx = ctx_for(L, D, Dc, prec)
    ctx.set_tensors(torch.from_numpy(A).cuda())
    sp = torch.from_numpy(spins).cuda()
    la, sg = ctx.amplitudes(sp)
    ref = oracle.evaluate_batch(A, spins, L, Dc, want_delta=True)
    assert np.array_equal(sg.cpu().numpy(), ref["sign"].astype(np.int8))
    assert np.max(np.abs(la.cpu().numpy() - ref["log_abs"])) < tol
    le = ctx.local_energy(sp, ratios=True)
    assert np.allclose(le["e_loc"].cpu().numpy(), ref["e_loc"], rtol=tol, atol=tol)
    # logderiv with given energies, then accumulate a second batch
    e_in = torch.from_numpy(ref["e_loc"]).cuda()
    r1 = ctx.logderiv(sp, e_in, delta=True)
    sums = (r1["sum_delta"].clone(), r1["sum_delta_e"].clone(), r1["sum_e"].clone())
    ctx.logderiv(sp, e_in, sums=sums, accumulate=True)
    N = L * L
    sd = np.zeros((N, 2, D ** 4))
    for b in range(len(spins)):
        for m in range(N):
            sd[m, spins[b][m]] += ref["delta"][b, m, spins[b][m]].reshape(-1)
    got = sums[0].cpu().numpy()
    assert np.max(np.abs(got - 2 * sd)) <= tol * np.abs(sd).max() * 2
    assert abs(sums[2].item() - 2 * ref["e_loc"].sum()) <= tol * max(1, abs(ref["e_loc"].sum()))
    assert ctx.sync_status()[0] == 0
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_grad_step_bit_exact(prec):
    L, D = 4, 2
    A = make_peps(L, D, seed=11)
    rng = np.random.default_rng(12)
    sd = rng.standard_normal((L * L, 2, D ** 4))
    sde = rng.standard_normal((L * L, 2, D ** 4))
    sd[0, 0, :3] = 0.0
    sde[0, 0, :3] = 0.0  # g = 0 exactly: element unchanged
    se = np.array([rng.standard_normal()])
    M, dt, seed, step = 37, 0.05, 0xDEADBEEF12345, 9
    ctx = ctx_for(L, D, 4, prec)
    Ad = torch.from_numpy(A.copy()).cuda()
    ctx.set_tensors(Ad)
    ctx.grad_step((torch.from_numpy(sd).cuda(), torch.from_numpy(sde).cuda(), torch.from_numpy(se).cuda()),
                  M, dt, seed, step, Ad)
    g = oracle.gradient(sd, sde, se[0], M)
    ref = oracle.go_step(A, g.reshape(A.shape), dt, seed, step)
    assert np.array_equal(Ad.cpu().numpy(), ref)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("L,D,Dc", [(4, 2, 16), (4, 3, 4)])
def test_sampler_bit_exact(prec, L, D, Dc):
    A = make_peps(L, D, seed=1)
    ctx = ctx_for(L, D, Dc, prec, slots=2)
    ctx.set_tensors(torch.from_numpy(A).cuda())
    out, acc = ctx.sample(seed=12345678901, n_chains=3, n_burn=3, n_thin=2, samples_per_chain=3,
                          accepted=True)
    ref, fin, racc = oracle.sample_chains(A, L, Dc, 12345678901, 3, 3, 2, 3)
    assert np.array_equal(out.cpu().numpy(), ref)
    assert np.array_equal(acc.cpu().numpy(), racc)
    # resume from the final states: the next sweeps continue the chains
    state = torch.from_numpy(fin.copy()).cuda()
    out2 = ctx.sample(seed=12345678901, n_chains=3, n_burn=0, n_thin=1, samples_per_chain=2,
                      first_sweep=10, state=state)
    ref2, fin2, _ = oracle.sample_chains(A, L, Dc, 12345678901, 3, 0, 1, 2, init=fin, first_sweep=10)
    assert np.array_equal(out2.cpu().numpy(), ref2)
    assert np.array_equal(state.cpu().numpy(), fin2)
    ctx.close()


@pytest.mark.parametrize("kind", ["neel", "gauss"])
def test_sampler_bit_exact_8x8_fp64(kind):
    """FP64 form, 8x8, D=4, Dc=16 (multi-panel QR and blocked
    bidiagonalisation in every compression): two sweeps of three chains give
    the oracle's configurations and acceptance counts bit for bit."""
    L, D, Dc = 8, 4, 16
    A = make_peps(L, D, seed=2, kind=kind)
    ctx = ctx_for(L, D, Dc, "fp64", slots=3)
    ctx.set_tensors(torch.from_numpy(A).cuda())
    seed = 0x5EED0002
    out, acc = ctx.sample(seed=seed, n_chains=3, n_burn=1, n_thin=1, samples_per_chain=1,
                          accepted=True)
    ref, fin, racc = oracle.sample_chains(A, L, Dc, seed, 3, 1, 1, 1)
    assert np.array_equal(out.cpu().numpy(), ref)
    assert np.array_equal(acc.cpu().numpy(), racc)
    assert racc.sum() > 0  # some exchanges were accepted
    assert ctx.sync_status()[0] == 0
    ctx.close()


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
def test_empty_batch_and_invalid_arguments():
    from paper_1806_03761_gb300 import PepsError
    ctx = ctx_for(4, 2, 4, "fp64")
    ctx.set_tensors(torch.from_numpy(make_peps(4, 2, seed=1)).cuda())
    sp = torch.zeros(0, 16, dtype=torch.uint8, device="cuda")
    res = ctx.evaluate(sp)
    assert res["e_loc"].numel() == 0 and float(res["sum_delta"].abs().max()) == 0.0
    with pytest.raises(PepsError):
        ctx.sample(seed=1, n_chains=2, n_burn=1, n_thin=0, samples_per_chain=1)
    with pytest.raises(PepsError):
        ctx.grad_step(ctx.new_sums(), 0, 0.1, 1, 1, torch.zeros(16, 2, 16, dtype=torch.float64, device="cuda"))
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_minimal_lattice_and_product_state(prec):
    # L = 2 (smallest lattice) and D = 1 (product state, closed forms)
    check_eval(make_peps(2, 2, seed=5), random_sz0_configs(2, 6, seed=6), 2, 2, 4, prec)
    L = 5
    rng = np.random.default_rng(3)
    a = rng.uniform(0.5, 2.0, (L * L, 2)) * rng.choice([-1, 1], (L * L, 2))
    check_eval(a.reshape(L * L, 2, 1, 1, 1, 1), random_sz0_configs(L, 4, seed=7), L, 1, 2, prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_unbalanced_configs_and_largest_bond(prec):
    # S^z != 0 configurations (all up: no flips) and D*Dc at its maximum 256
    L, D, Dc = 3, 8, 32
    A = make_peps(L, D, seed=13)
    spins = np.zeros((3, 9), np.uint8)
    spins[1, :4] = 1
    spins[2] = random_sz0_configs(3, 1, seed=1)[0]
    check_eval(A, spins, L, D, Dc, prec, delta=False)


def test_zero_amplitude_is_flagged():
    L, D, Dc = 3, 2, 4
    A = make_peps(L, D, seed=14)
    A[4, 0] = 0.0  # the centre site's spin-up slice vanishes
    spins = np.array([[0, 1, 0, 1, 0, 1, 0, 1, 0]], np.uint8)
    ctx = ctx_for(L, D, Dc, "fp64")
    ctx.set_tensors(torch.from_numpy(A).cuda())
    la, sg = ctx.amplitudes(torch.from_numpy(spins).cuda())
    rc, flags = ctx.sync_status()
    assert sg.item() == 0 and rc != 0 and flags & 2
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_vmc_step_equals_evaluate_then_sweep(prec):
    """peps_vmc_step = peps_evaluate on the chain states, then one sweep of
    peps_sample_batch (same outputs, same new states, bit for bit)."""
    L, D, Dc = 5, 2, 4
    A = torch.from_numpy(make_peps(L, D, seed=17)).cuda()
    ctx = ctx_for(L, D, Dc, prec, slots=3)
    ctx.set_tensors(A)
    seed, n = 424242, 7
    state0 = ctx.sample(seed, n, 2, 1, 1)  # a few sweeps from the Fisher-Yates starts
    state = state0.clone()
    fused = ctx.vmc_step(seed, state, sweep=9, accepted=True)
    ref_eval = ctx.evaluate(state0.clone())
    st = state0.clone()
    ctx.sample(seed, n, 0, 1, 1, first_sweep=9, state=st)
    torch.cuda.synchronize()
    assert torch.equal(state, st)
    for k in ("e_loc", "log_abs", "sign", "sum_delta", "sum_delta_e", "sum_e"):
        assert torch.equal(fused[k], ref_eval[k]), k
    # and against the oracle
    import oracle as orc
    ref, fin, acc = orc.sample_chains(A.cpu().numpy(), L, Dc, seed, n, 0, 1, 1,
                                      init=state0.cpu().numpy(), first_sweep=9)
    assert np.array_equal(state.cpu().numpy(), fin)
    assert np.array_equal(fused["accepted"].cpu().numpy(), acc)
    assert ctx.sync_status()[0] == 0
    ctx.close()


def test_tall_panel_pair_variant_matches_the_oracle():
    """The fused VMC kernel built with the two-warp tall-panel QR
    (PEPS_QR_TALL_PAIR; 6x6, D=8, Dc=32: panels of 2048 x 256): its
    evaluation of the chains' configurations matches the oracle."""
    L, D, Dc = 6, 8, 32
    A = make_peps(L, D, seed=6)
    spins = random_sz0_configs(L, 2, seed=7)
    from paper_1806_03761_gb300 import PepsContext
    c = PepsContext(L, D, Dc, precision="mixed", slots=2,
                    variant={"PEPS_QR_TALL_PAIR": 1, "PEPS_QR_PREFETCH": 1, "PEPS_BIDIAG_TPC": 1})
    c.set_tensors(torch.from_numpy(A).cuda())
    st = torch.from_numpy(spins.copy()).cuda()
    r = c.vmc_step(5, st, 3)
    assert c.sync_status()[0] == 0
    ref = oracle.evaluate_batch(A, spins, L, Dc)
    e = r["e_loc"].cpu().numpy()
    assert np.array_equal(r["sign"].cpu().numpy(), ref["sign"].astype(np.int8))
    assert np.max(np.abs(r["log_abs"].cpu().numpy() - ref["log_abs"])) <= TOL["mixed"]
    assert np.max(np.abs(e - ref["e_loc"]) / np.maximum(1.0, np.abs(ref["e_loc"]))) <= TOL["mixed"]
    c.close()


def _vmc_outputs(ctx, A, spins):
    ctx.set_tensors(torch.from_numpy(A).cuda())
    st = torch.from_numpy(spins.copy()).cuda()
    r = ctx.vmc_step(5, st, 3)
    assert ctx.sync_status()[0] == 0
    out = {k: v.cpu().numpy().copy() for k, v in r.items() if hasattr(v, "cpu")}
    out["state"] = st.cpu().numpy().copy()
    return out


@pytest.mark.parametrize("prec,base", [
    ("fp64", {}),
    ("mixed", {"PEPS_QR_PREFETCH": 1, "PEPS_BIDIAG_TPC": 1}),
])
def test_pipelined_contraction_is_bit_identical(prec, base):
    """PEPS_CTR_PIPE (the default) loads the next reduction step's operands
    ahead of the multiply-adds: every product and sum is the same, so the
    fused step's outputs equal those of a build without it bit for bit (8x8,
    D=4, Dc=16: every contraction shape of the strips and the absorption;
    FP64 also without PEPS_QR_ACC, the same fused multiply-adds in FP64)."""
    from paper_1806_03761_gb300 import PepsContext
    L, D, Dc = 8, 4, 16
    A = make_peps(L, D, seed=81)
    spins = random_sz0_configs(L, 6, seed=82)
    got = _vmc_outputs(PepsContext(L, D, Dc, precision=prec, slots=3, variant=base or None), A, spins)
    knobs = dict(base, PEPS_CTR_PIPE=0)
    if prec == "fp64":
        knobs["PEPS_QR_ACC"] = 0
    ref = _vmc_outputs(PepsContext(L, D, Dc, precision=prec, slots=3, variant=knobs), A, spins)
    assert set(ref) == set(got)
    for k in ref:
        assert np.array_equal(ref[k], got[k]), k


def test_compensated_qr_update_matches_the_oracle():
    """PEPS_QR_ACC in the float-float form (the trailing update of the
    blocked QR as one compensated accumulation per element, the warp
    reductions on the accumulators), with the pipelined contractions and the
    wider register block: the fused step's evaluation matches the oracle at
    8x8, D=4, Dc=16 (QR panels of 256 rows) and 6x6, D=6, Dc=24 (864)."""
    from paper_1806_03761_gb300 import PepsContext
    knobs = {"PEPS_QR_PREFETCH": 1, "PEPS_BIDIAG_TPC": 1, "PEPS_CTR_PIPE": 1, "PEPS_QR_ACC": 1,
             "PEPS_BB_FF": 4}
    for (L, D, Dc, seed) in [(8, 4, 16, 83), (6, 6, 24, 85)]:
        A = make_peps(L, D, seed=seed)
        spins = random_sz0_configs(L, 3, seed=seed + 1)
        c = PepsContext(L, D, Dc, precision="mixed", slots=3, variant=knobs)
        r = _vmc_outputs(c, A, spins)
        c.close()
        ref = oracle.evaluate_batch(A, spins, L, Dc)
        assert np.array_equal(r["sign"], ref["sign"].astype(np.int8))
        assert np.max(np.abs(r["log_abs"] - ref["log_abs"])) <= TOL["mixed"]
        assert np.max(np.abs(r["e_loc"] - ref["e_loc"]) /
                      np.maximum(1.0, np.abs(ref["e_loc"]))) <= TOL["mixed"]


def test_compensated_tall_pair_update_matches_the_oracle():
    """PEPS_QR_ACC with the two-warp tall-panel QR (6x6, D=8, Dc=32: panels
    of 2048 x 256), float-float: the fused step's evaluation matches the
    oracle."""
    from paper_1806_03761_gb300 import PepsContext
    L, D, Dc = 6, 8, 32
    A = make_peps(L, D, seed=6)
    spins = random_sz0_configs(L, 2, seed=7)
    knobs = {"PEPS_QR_TALL_PAIR": 1, "PEPS_QR_PREFETCH": 1, "PEPS_BIDIAG_TPC": 1,
             "PEPS_CTR_PIPE": 1, "PEPS_QR_ACC": 1}
    c = PepsContext(L, D, Dc, precision="mixed", slots=2, variant=knobs)
    r = _vmc_outputs(c, A, spins)
    c.close()
    ref = oracle.evaluate_batch(A, spins, L, Dc)
    assert np.array_equal(r["sign"], ref["sign"].astype(np.int8))
    assert np.max(np.abs(r["log_abs"] - ref["log_abs"])) <= TOL["mixed"]
    assert np.max(np.abs(r["e_loc"] - ref["e_loc"]) /
                  np.maximum(1.0, np.abs(ref["e_loc"]))) <= TOL["mixed"]


def test_tuned_variants_match_the_oracle():
    """Every library variant the tuning table selects (the code paths and
    launch shape a shape's contexts run on) evaluates the chains'
    configurations as the oracle does: 6x6 D=8 Dc=32 (2048 x 256 QR panels)
    for a variant with the two-warp tall panels, else 6x6 D=6 Dc=24
    (864 x 144 panels, the 16x16 workload's site shapes)."""
    import json
    from paper_1806_03761_gb300 import PepsContext
    from paper_1806_03761_gb300 import build as B
    table = json.load(open(B.TUNING))
    seen = set()
    for key, entry in sorted(table.items()):
        prec, knobs = entry["precision"], entry["choice"]
        tag = B.variant_tag(dict(B.DEFAULTS, **knobs), prec)
        if tag in seen:
            continue
        seen.add(tag)
        L, D, Dc = (6, 8, 32) if knobs.get("PEPS_QR_TALL_PAIR") else (6, 6, 24)
        A = make_peps(L, D, seed=95)
        spins = random_sz0_configs(L, 2, seed=96)
        c = PepsContext(L, D, Dc, precision=prec, slots=2, variant=knobs)
        r = _vmc_outputs(c, A, spins)
        c.close()
        ref = oracle.evaluate_batch(A, spins, L, Dc)
        assert np.array_equal(r["sign"], ref["sign"].astype(np.int8)), tag
        assert np.max(np.abs(r["log_abs"] - ref["log_abs"])) <= TOL[prec], tag
        assert np.max(np.abs(r["e_loc"] - ref["e_loc"]) /
                      np.maximum(1.0, np.abs(ref["e_loc"]))) <= TOL[prec], tag
    assert seen
