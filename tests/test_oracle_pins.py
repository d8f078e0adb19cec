"""Pins of the FP64 oracle against things other than itself: published
Philox known-answer vectors, brute-force contraction, exact transfer-matrix
amplitudes, exact diagonalisation, closed forms, finite differences and
invariants of the method (PEPS++, arXiv:1806.03761)."""
import os

import numpy as np
import pytest

import oracle
from oracle import peps as op
from synth import make_peps, random_sz0_configs

from . import _exact as ex

HERE = os.path.dirname(os.path.abspath(__file__))


# --------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al., SC'11): published known-answer vectors
# --------------------------------------------------------------------------
def test_philox_known_answers():
    n = 0
    for line in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        assert oracle.philox4x32_10(w[0:4], w[4:6]) == tuple(w[6:10])
        n += 1
    assert n == 3


def test_uniform_conversions():
    assert oracle.uniform53(0, 0) == 0.0
    assert oracle.uniform53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert oracle.uniform_open53(0, 0) == 2.0 ** -53
    assert oracle.uniform_open53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53


# --------------------------------------------------------------------------
# Lattice bookkeeping (Sec. "Experiment Setup")
# --------------------------------------------------------------------------
@pytest.mark.parametrize("L", [2, 3, 4, 7])
def test_bond_list(L):
    b = op.bond_list(L)
    assert len(b) == 2 * L * (L - 1) + 2 * (L - 1) ** 2
    ref = {(min(a, c), max(a, c)): J for a, c, J in ex.pairs(L, "J1", "J2")}
    got = {(min(m1, m2), max(m1, m2)): ("J1" if k in "hv" else "J2") for k, m1, m2 in b}
    assert got == ref


# --------------------------------------------------------------------------
# Exact contraction (Eq. PEPS): brute force and transfer matrices
# --------------------------------------------------------------------------
@pytest.mark.parametrize("L,D,chi", [(2, 3, 3), (3, 2, 2), (3, 3, 3), (3, 2, 8)])
def test_amplitude_matches_brute_force(L, D, chi):
    A = make_peps(L, D, seed=11 + L + D)
    rng = np.random.default_rng(5)
    for _ in range(6):
        s = rng.integers(0, 2, L * L).astype(np.uint8)
        la, sg = oracle.amplitude(A, s, L, chi)
        w = ex.brute_amplitude(A, s, L)
        assert sg == np.sign(w)
        assert abs(la - np.log(abs(w))) < 1e-12


def test_amplitude_4x4_all_configs_transfer_matrix():
    L, D = 4, 2
    A = make_peps(L, D, seed=21)
    psi = ex.all_amplitudes(A, L)
    rng = np.random.default_rng(7)
    for x in rng.choice(1 << 16, 25, replace=False):
        s = np.array([(x >> m) & 1 for m in range(16)], np.uint8)
        la, sg = oracle.amplitude(A, s, L, 4)
        assert sg == np.sign(psi[x])
        assert abs(la - np.log(abs(psi[x]))) < 1e-12
    # and the transfer matrix agrees with brute force
    s = np.array([(12345 >> m) & 1 for m in range(16)], np.uint8)
    assert abs(ex.brute_amplitude(A, s, L) / psi[12345] - 1) < 1e-12


# --------------------------------------------------------------------------
# Local energy (Eq. ess) against exact psi and an independent H
# --------------------------------------------------------------------------
@pytest.mark.parametrize("J2", [0.0, 0.5, 1.0])
def test_h_normalisation_2x2(J2):
    # 2x2 open square = 4-site ring (+ both diagonals for J2): ground
    # energies -2 (J2 = 0) and -3/2 (J2 = J1, complete graph: S_tot^2/2 - 3/2)
    H = ex.dense_H(2, 1.0, J2)
    e0 = np.linalg.eigvalsh(H)[0]
    if J2 == 0.0:
        assert abs(e0 + 2.0) < 1e-12
    elif J2 == 1.0:
        assert abs(e0 + 1.5) < 1e-12
    psi = np.random.default_rng(0).standard_normal(16)
    assert np.allclose(H @ psi, ex.apply_H(psi, 2, 1.0, J2))


def test_local_energy_exact_4x4():
    L, D = 4, 2
    A = make_peps(L, D, seed=31)
    psi = ex.all_amplitudes(A, L)
    Hpsi = ex.apply_H(psi, L, 1.0, 0.5)
    cfgs = random_sz0_configs(L, 12, seed=8)
    for s in cfgs:
        r = oracle.evaluate(A, s, L, 4)
        x = ex.config_index(s)
        e_exact = Hpsi[x] / psi[x]
        assert abs(r["e_loc"] - e_exact) < 1e-10 * max(1.0, abs(e_exact))
        # every flip ratio against the exact amplitudes
        for b, (kind, m1, m2) in enumerate(op.bond_list(L)):
            if s[m1] == s[m2]:
                assert r["ratios"][b] == 0.0
                continue
            y = x ^ ((1 << m1) | (1 << m2))
            assert abs(r["ratios"][b] - psi[y] / psi[x]) < 1e-10 * max(1.0, abs(psi[y] / psi[x]))
        assert r["n_flips"] == sum(int(s[m1] != s[m2]) for _, m1, m2 in op.bond_list(L))


def test_ed_identity_3x3():
    """sum_S W^2 E(S) / sum_S W^2 = <psi|H|psi>/<psi|psi> (Eq. energy-MC)."""
    L, D, J2 = 3, 2, 0.5
    A = make_peps(L, D, seed=41)
    H = ex.dense_H(L, 1.0, J2)
    psi = np.array([ex.brute_amplitude(A, [(x >> m) & 1 for m in range(9)], L)
                    for x in range(512)])
    e_exact = psi @ H @ psi / (psi @ psi)
    num = den = 0.0
    for x in range(512):
        s = np.array([(x >> m) & 1 for m in range(9)], np.uint8)
        r = oracle.evaluate(A, s, L, 2, J2=J2)
        w2 = np.exp(2 * r["log_abs"])
        num += w2 * r["e_loc"]
        den += w2
    assert abs(num / den - e_exact) < 1e-11


# --------------------------------------------------------------------------
# D = 1 product states: closed forms
# --------------------------------------------------------------------------
@pytest.mark.parametrize("L,chi", [(4, 1), (5, 1), (5, 3)])
def test_product_state_closed_form(L, chi):
    rng = np.random.default_rng(L)
    a = rng.uniform(0.5, 2.0, (L * L, 2)) * rng.choice([-1, 1], (L * L, 2))
    A = a.reshape(L * L, 2, 1, 1, 1, 1)
    s = random_sz0_configs(L, 1, seed=3)[0]
    r = oracle.evaluate(A, s, L, chi, want_delta=True)
    w = np.prod([a[m, s[m]] for m in range(L * L)])
    assert abs(r["log_abs"] - np.log(abs(w))) < 1e-12 and r["sign"] == np.sign(w)
    e = 0.0
    for b, (kind, m1, m2) in enumerate(op.bond_list(L)):
        J = 1.0 if kind in "hv" else 0.5
        sg = (1 - 2 * int(s[m1])) * (1 - 2 * int(s[m2]))
        e += J * sg / 4
        if s[m1] != s[m2]:
            ratio = a[m1, s[m2]] * a[m2, s[m1]] / (a[m1, s[m1]] * a[m2, s[m2]])
            assert abs(r["ratios"][b] - ratio) < 1e-12 * abs(ratio)
            e += J * 0.5 * ratio
    assert abs(r["e_loc"] - e) < 1e-12 * max(1, abs(e))
    for m in range(L * L):
        assert abs(r["delta"][m, s[m], 0, 0, 0, 0] - 1.0 / a[m, s[m]]) < 1e-12
        assert r["delta"][m, 1 - s[m]].max() == 0.0


# --------------------------------------------------------------------------
# Truncation (Fig. 1(c)): invariance once D_c reaches the exact bond
# --------------------------------------------------------------------------
@pytest.mark.parametrize("L,D,chis", [(4, 2, (4, 8, 16)), (6, 2, (8, 16))])
def test_truncation_invariance(L, D, chis):
    A = make_peps(L, D, seed=51)
    s = random_sz0_configs(L, 1, seed=9)[0]
    rs = [oracle.evaluate(A, s, L, c) for c in chis]
    for r in rs[1:]:
        assert abs(r["log_abs"] - rs[0]["log_abs"]) < 1e-10
        assert abs(r["e_loc"] - rs[0]["e_loc"]) < 1e-10 * max(1, abs(rs[0]["e_loc"]))
        assert np.allclose(r["ratios"], rs[0]["ratios"], rtol=1e-10, atol=1e-12)


def test_truncation_changes_result_below_exact_bond():
    L, D = 6, 2
    A = make_peps(L, D, seed=51)
    s = random_sz0_configs(L, 1, seed=9)[0]
    exact = oracle.evaluate(A, s, L, 8)["log_abs"]
    trunc = oracle.evaluate(A, s, L, 2)["log_abs"]
    assert abs(exact - trunc) > 1e-8


def test_compress_keeps_chi_largest_singular_values():
    """A truncated two-site MPS keeps exactly the chi largest singular values
    of its bond matrix (LAPACK SVD of the contracted pair)."""
    rng = np.random.default_rng(3)
    M0 = rng.standard_normal((1, 5, 7))
    M1 = rng.standard_normal((7, 6, 1))
    env = op.BMPS([M0, M1])
    out = op.compress(env, 3)
    full = np.einsum("apb,bqc->pq", M0, M1)
    U, S, Vt = np.linalg.svd(full)
    best = (U[:, :3] * S[:3]) @ Vt[:3]
    got = np.einsum("apb,bqc->pq", *out.sites) * np.exp(out.logscale)
    assert np.allclose(got, best, atol=1e-12 * S[0])


def _tt_svd_right_to_left(psi, chi):
    """Sequential truncated SVDs of a full tensor from its last index to its
    first (the tensor-train SVD of Oseledets, 2011, run right to left),
    keeping chi singular values at every bond; returns the truncated
    tensor.  Written on the full vector, independent of any MPS."""
    dims = psi.shape
    L = len(dims)
    cur = psi.reshape(-1, dims[-1])
    right = np.eye(dims[-1]).reshape(dims[-1], dims[-1])  # rows: kept basis of the right part
    for j in range(L - 1, 0, -1):
        U, S, Vt = np.linalg.svd(cur, full_matrices=False)
        k = min(chi, S.size)
        right = Vt[:k] @ right                       # k x (p_j ... p_{L-1})
        right = right.reshape(k, -1)
        cur = (U[:, :k] * S[:k]).reshape(-1, dims[j - 1] * k)
        right = np.kron(np.eye(dims[j - 1]), right).reshape(dims[j - 1] * k, -1)
    return (cur @ right).reshape(dims)


def test_compress_is_the_sequential_truncated_svd_of_the_state():
    """A truncated five-site MPS (bonds up to 9, chi = 3) represents the
    tensor that sequential truncated SVDs of the exact state vector give,
    bond by bond from the right (numpy SVD of the full 3^5 tensor): the QR
    sweep makes the left part an isometry, so every SVD of the sweep sees
    the full reshaped state."""
    rng = np.random.default_rng(11)
    bonds = [1, 3, 9, 9, 3, 1]
    sites = [rng.standard_normal((bonds[j], 3, bonds[j + 1])) for j in range(5)]
    psi = sites[0]
    for M in sites[1:]:
        psi = np.tensordot(psi, M, axes=([-1], [0]))
    psi = psi.reshape((3,) * 5)
    want = _tt_svd_right_to_left(psi, 3)
    out = op.compress(op.BMPS([x.copy() for x in sites]), 3)
    got = out.sites[0]
    for M in out.sites[1:]:
        got = np.tensordot(got, M, axes=([-1], [0]))
    got = got.reshape((3,) * 5) * np.exp(out.logscale)
    assert max(M.shape[2] for M in out.sites) == 3
    assert np.linalg.norm(psi - want) > 1e-3 * np.linalg.norm(psi)  # truncation is active
    assert np.allclose(got, want, atol=1e-11 * np.abs(want).max())


# --------------------------------------------------------------------------
# Log-derivatives (Eq. delta) and the gradient (Eq. gradients)
# --------------------------------------------------------------------------
def test_delta_finite_difference():
    L, D = 3, 2
    A = make_peps(L, D, seed=61)
    s = np.array([0, 1, 0, 1, 1, 0, 0, 1, 1], np.uint8)
    r = oracle.evaluate(A, s, L, 8, want_delta=True)
    w0 = ex.brute_amplitude(A, s, L)
    rng = np.random.default_rng(1)
    h = 1e-6
    for _ in range(12):
        m = rng.integers(0, 9)
        idx = (m, s[m]) + tuple(rng.integers(0, D, 4))
        Ap, Am = A.copy(), A.copy()
        Ap[idx] += h
        Am[idx] -= h
        fd = (ex.brute_amplitude(Ap, s, L) - ex.brute_amplitude(Am, s, L)) / (2 * h * w0)
        assert abs(r["delta"][idx] - fd) < 1e-7 * max(1, abs(fd))


@pytest.mark.parametrize("L,D,chi", [(4, 3, 4), (6, 3, 4)])
def test_linearity_sum_T_delta_is_one(L, D, chi):
    """sum_{lrud} A^{s_m} Delta^{s_m} = 1 per site, also under truncation:
    B_m is the strip contracted without site m, W_i the strip itself."""
    A = make_peps(L, D, seed=71)
    s = random_sz0_configs(L, 1, seed=4)[0]
    r = oracle.evaluate(A, s, L, chi, want_delta=True, want_energy=False)
    for m in range(L * L):
        v = np.sum(A[m, s[m]] * r["delta"][m, s[m]])
        assert abs(v - 1.0) < 1e-10


def test_gradient_matches_finite_difference_3x3():
    """Exact-weight version of Eq. gradients against central differences of
    E(A) = <psi|H|psi>/<psi|psi>, both over all 2^9 configurations."""
    L, D, J2 = 3, 2, 0.5
    A = make_peps(L, D, seed=81)
    H = ex.dense_H(L, 1.0, J2)
    confs = [np.array([(x >> m) & 1 for m in range(9)], np.uint8) for x in range(512)]
    res = [oracle.evaluate(A, s, L, 8, J2=J2, want_delta=True) for s in confs]
    w2 = np.array([np.exp(2 * r["log_abs"]) for r in res])
    p = w2 / w2.sum()
    E = np.array([r["e_loc"] for r in res])
    sd = sum(pi * r["delta"] for pi, r in zip(p, res))
    sde = sum(pi * r["delta"] * e for pi, r, e in zip(p, res, E))
    g = oracle.gradient(sd, sde, float(p @ E), 1.0)

    def energy(Ax):
        psi = np.array([ex.brute_amplitude(Ax, s, L) for s in confs])
        return psi @ H @ psi / (psi @ psi)

    rng = np.random.default_rng(2)
    h = 1e-5
    for _ in range(5):
        idx = (rng.integers(0, 9), rng.integers(0, 2)) + tuple(rng.integers(0, D, 4))
        Ap, Am = A.copy(), A.copy()
        Ap[idx] += h
        Am[idx] -= h
        fd = (energy(Ap) - energy(Am)) / (2 * h)
        assert abs(g[idx] - fd) < 1e-6 * max(1.0, abs(fd))


def test_go_step_sign_update():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((4, 2, 1, 1, 1, 1))
    g = rng.standard_normal(A.shape)
    g.reshape(-1)[3] = 0.0
    dt = 0.1
    An = oracle.go_step(A, g, dt, seed=123, step=7)
    d = (An - A).reshape(-1)
    gf = g.reshape(-1)
    assert d[3] == 0.0
    for k in range(d.size):
        if gf[k] != 0:
            assert np.sign(d[k]) == -np.sign(gf[k]) and 0 < abs(d[k]) < dt


def test_go_step_lengths_are_uniform_and_fresh_per_step():
    """The step lengths p of the GO update (after Eq. delta) are i.i.d.
    uniform on (0, 1): over 20000 elements their mean, quartiles and
    lag-1 correlation match U(0,1) within 5 sigma, and another step number
    draws other lengths."""
    n = 20000
    A = np.zeros((n, 1, 1, 1, 1, 1))
    g = np.ones_like(A)
    dt = 1.0
    p = -(oracle.go_step(A, g, dt, seed=99, step=3) - A).reshape(-1)
    assert p.min() > 0.0 and p.max() < 1.0
    sig = np.sqrt(1.0 / 12.0 / n)
    assert abs(p.mean() - 0.5) < 5 * sig
    for q in (0.25, 0.5, 0.75):
        assert abs(np.mean(p < q) - q) < 5 * np.sqrt(q * (1 - q) / n)
    c = np.corrcoef(p[:-1], p[1:])[0, 1]
    assert abs(c) < 5 / np.sqrt(n)
    p2 = -(oracle.go_step(A, g, dt, seed=99, step=4) - A).reshape(-1)
    assert abs(np.corrcoef(p, p2)[0, 1]) < 5 / np.sqrt(n)


# --------------------------------------------------------------------------
# Metropolis sampling (Fig. "contraction", Steps 1-3; Eq. energy-MC)
# --------------------------------------------------------------------------
def test_init_config_is_sz0_permutation():
    for c in range(5):
        s = oracle.init_config(4, 99, c)
        assert s.sum() == 8 and s.dtype == np.uint8
    assert not np.array_equal(oracle.init_config(4, 99, 0), oracle.init_config(4, 99, 1))


def test_init_config_is_uniform_over_the_sz0_sector():
    """Fig. "contraction", Step 1 (a random start): the Fisher-Yates start
    draws every S^z = 0 configuration with equal probability.  On the 2x2
    lattice each of the C(4,2) = 6 configurations has probability 1/6 over
    12000 chains, within 5 sigma (a shuffle that drew j from [0, k) instead
    of [0, k] -- Sattolo's cycles -- never returns the start and fails); on
    the 3x3 lattice every site is up with probability 4/9 over 6000 chains."""
    from collections import Counter
    n = 12000
    cnt = Counter(tuple(oracle.init_config(2, 2024, c)) for c in range(n))
    assert len(cnt) == 6
    sig = np.sqrt((1 / 6) * (5 / 6) / n)
    for k, v in cnt.items():
        assert sum(k) == 2
        assert abs(v / n - 1 / 6) < 5 * sig, (k, v)
    n3 = 6000
    S = np.array([oracle.init_config(3, 77, c) for c in range(n3)])
    assert np.all(S.sum(axis=1) == 5)  # floor(9/2) = 4 up (s = 0), 5 down
    up = np.mean(S == 0, axis=0)
    assert np.all(np.abs(up - 4 / 9) < 5 * np.sqrt((4 / 9) * (5 / 9) / n3))


def test_burn_in_and_thinning_record_the_stated_sweeps():
    """sample_chains records the configuration after sweep t when t > n_burn
    and (t - n_burn) % n_thin == 0: with n_burn = 2, n_thin = 3 and two
    samples per chain that is after sweeps 5 and 8 (of 8), checked against
    the chain advanced by hand, sweep by sweep."""
    L, D, chi, seed = 3, 2, 4, 31337
    A = make_peps(L, D, seed=8)
    out, final, acc = oracle.sample_chains(A, L, chi, seed, 2, 2, 3, 2, first_sweep=11)
    for c in range(2):
        s = oracle.init_config(L, seed, c)
        seen, a = {}, 0
        for t in range(1, 9):
            a += oracle.metropolis_sweep(A, s, L, chi, seed, c, 10 + t)
            seen[t] = s.copy()
        assert np.array_equal(out[2 * c], seen[5]) and np.array_equal(out[2 * c + 1], seen[8])
        assert np.array_equal(final[c], seen[8]) and acc[c] == a
    # the recorded sweeps differ from their neighbours for some chain (the
    # rule is not vacuous on this input)
    assert any(not np.array_equal(out[2 * c], out[2 * c + 1]) for c in range(2))


def test_sampler_stationary_distribution_2x2():
    """Long chains on 2x2 visit the six S^z = 0 states with frequency
    W(S)^2 / Z (W by brute force)."""
    L, D = 2, 2
    A = make_peps(L, D, seed=91)
    out, final, acc = oracle.sample_chains(A, L, 4, seed=5, n_chains=4, n_burn=5,
                                           n_thin=1, samples_per_chain=1500)
    assert (out.sum(axis=1) == 2).all()
    idx = np.array([ex.config_index(s) for s in out])
    states = sorted(set(x for x in range(16) if bin(x).count("1") == 2))
    w2 = np.array([ex.brute_amplitude(A, [(x >> m) & 1 for m in range(4)], L) ** 2 for x in states])
    p = w2 / w2.sum()
    f = np.array([(idx == x).mean() for x in states])
    # 6000 correlated draws: allow 5 sigma of a binomial with a factor 2
    sig = np.sqrt(p * (1 - p) / out.shape[0]) * 2
    assert (np.abs(f - p) < 5 * sig + 1e-3).all()


@pytest.mark.slow
def test_mc_energy_4x4_within_error_bars():
    """The MC estimate of Eq. energy-MC lies within 4 binned sigma of the
    exact energy of the S^z = 0 projected state."""
    L, D = 4, 2
    A = make_peps(L, D, seed=1)
    psi = ex.all_amplitudes(A, L)
    sz0 = np.array([bin(x).count("1") == 8 for x in range(1 << 16)])
    pp = np.where(sz0, psi, 0.0)
    e_exact = pp @ ex.apply_H(pp, L, 1.0, 0.5) / (pp @ pp)
    out, _, _ = oracle.sample_chains(A, L, 16, seed=3, n_chains=4, n_burn=10,
                                     n_thin=1, samples_per_chain=40)
    E = np.array([oracle.evaluate(A, s, L, 16)["e_loc"] for s in out])
    means = E.reshape(4, -1).mean(axis=1)
    sig = means.std(ddof=1) / np.sqrt(4)
    assert abs(E.mean() - e_exact) < 4 * sig + 1e-9
