"""Pins of the oracle's spin correlations (oracle/correlations.py): the
Monte Carlo identity against exact diagonalisation-style dense operators,
the D = 1 closed form, invariance under truncation in the exact regime, and
the structure factor of a classical Neel product state."""
import numpy as np
import pytest

import oracle
from oracle import correlations as oc
from synth import make_peps, neel_config

from . import _exact as ex


def _configs(N):
    return [np.array([(x >> m) & 1 for m in range(N)], np.uint8) for x in range(1 << N)]


@pytest.mark.parametrize("D,chi,a", [(2, 2, 4), (2, 2, 0), (3, 3, 5)])
def test_mc_identity_against_dense_operators_3x3(D, chi, a):
    """sum_S W^2 (S_a . S_m)(S) / sum_S W^2 = <psi|S_a . S_m|psi>/<psi|psi>
    for every m (exact regime: chi >= D^floor(L/2)); m runs over the source's
    row, the rows next to it and the row two away, so every branch of the
    exchange ratio is exercised."""
    L = 3
    N = L * L
    A = make_peps(L, D, seed=50 + D)
    psi = np.array([ex.brute_amplitude(A, s, L) for s in _configs(N)])
    nrm = psi @ psi
    num = np.zeros(N)
    den = 0.0
    for s in _configs(N):
        la, sg = oracle.amplitude(A, s, L, chi)
        w2 = np.exp(2 * la)
        num += w2 * oc.local_correlations(A, s, L, chi, a)
        den += w2
    for m in range(N):
        exact = psi @ ex.dense_SS(L, a, m) @ psi / nrm
        assert abs(num[m] / den - exact) < 1e-11, (m, num[m] / den, exact)


@pytest.mark.parametrize("L,chi", [(4, 1), (5, 2)])
def test_product_state_exchange_ratio_closed_form(L, chi):
    """D = 1: W = prod_m a_m[s_m], so exchanging a and m gives
    a_a[s_m] a_m[s_a] / (a_a[s_a] a_m[s_m]) at any distance."""
    rng = np.random.default_rng(7)
    N = L * L
    a_ = rng.uniform(0.5, 2.0, (N, 2)) * rng.choice([-1, 1], (N, 2))
    A = a_.reshape(N, 2, 1, 1, 1, 1)
    s = rng.permutation(np.array([0] * (N // 2) + [1] * (N - N // 2), np.uint8))
    for a in (0, oc.centre_site(L), N - 1):
        r = oc.exchange_ratios(A, s, L, chi, a)
        for m in range(N):
            if m == a or s[m] == s[a]:
                assert r[m] == 0.0
            else:
                want = a_[a, s[m]] * a_[m, s[a]] / (a_[a, s[a]] * a_[m, s[m]])
                assert abs(r[m] - want) < 1e-12 * abs(want)


def test_exact_regime_does_not_depend_on_chi():
    L, D = 4, 2
    A = make_peps(L, D, seed=9)
    s = np.array([0, 1, 1, 0, 1, 0, 0, 1, 0, 0, 1, 1, 1, 1, 0, 0], np.uint8)
    a = oc.centre_site(L)
    r4 = oc.local_correlations(A, s, L, 4, a)
    r8 = oc.local_correlations(A, s, L, 8, a)
    assert np.allclose(r4, r8, rtol=1e-11, atol=1e-13)


def test_structure_factor_of_the_neel_configuration():
    """A single Neel configuration of a D = 1 Neel product state: every
    exchange ratio vanishes (the state has weight on one configuration), so
    <S_a . S_m> = (-1)^{a+m}/4 off the diagonal and 3/4 on it; m_s^2(pi, pi)
    over the n bulk sites is then (n (n - 1)/4 + 3n/4) / n^2 = 1/4 + 1/(2n)."""
    L = 6
    N = L * L
    s = neel_config(L)
    A = np.zeros((N, 2, 1, 1, 1, 1))
    for m in range(N):
        A[m, s[m]] = 1.0
    bulk = oc.bulk_sites(L)
    C = np.array([oc.local_correlations(A, s, L, 2, q) for q in bulk])
    n = len(bulk)
    assert abs(oc.structure_factor(C, L, bulk, (np.pi, np.pi)) - (0.25 + 0.5 / n)) < 1e-14
    # k = 0: the staggered signs cancel except on the diagonal
    k0 = oc.structure_factor(C, L, bulk, (0.0, 0.0))
    assert abs(k0 - (0.75 * n + 0.25 * sum((-1) ** ((a // L + a % L + m // L + m % L) % 2)
                                           for a in bulk for m in bulk if m != a)) / n ** 2) < 1e-14
