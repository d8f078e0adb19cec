"""Spin-spin correlations <S_a . S_m> and the structure factor m_s^2(k) of the
sampled PEPS (PEPS++, Sec. "Experiment Setup" and the results that follow it:
m_s^2(k) = (1/N^2) sum_{m m'} <S_m . S_m'> e^{i k (r_m - r_m')} over the
central (L-4) x (L-4) bulk, M^2 = m_s^2(pi, pi), and the map <S_0 . S_m> with
S_0 at the centre).  TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Monte Carlo estimator.  With configurations S drawn from W(S)^2,
<S_a . S_m> is the mean of the local value
    (S_a . S_m)(S) = sigma_a sigma_m / 4 + [s_a != s_m] (1/2) W(S')/W(S),
S' = S with s_a and s_m exchanged (S_a . S_m = S^z S^z + (S^+S^- + S^-S^+)/2;
the exchange part maps S to S' with matrix element 1/2), and 3/4 for m = a.

Reading taken where the paper is silent (it only says the correlations cost
about as much as the energy): the ratio W(S')/W(S) is taken on the one-row
strip of the target's row i(m), each configuration with its own
environments,
    W(S')/W(S) = W_{i(m)}(S') / W_{i(m)}(S),
W_i(X) the strip of row i of X between U_{i-1}(X) and Dn_{i+1}(X) (Fig.
"contraction", Step 4).  For a pair in one row this is the window ratio of
the horizontal J1 bonds; when D_c reaches the exact bond dimension every
strip is exact and so is the ratio.  S' and the configuration with only s_a
flipped agree outside row i(m), so U_{i-1}(S') and Dn_{i+1}(S') are the
environments of S with s_a flipped (equal to those of S on the side of row
i(m) that does not hold a).
"""
import numpy as np

from .peps import Strip1, lower_envs, site_tensor, upper_envs

__all__ = ["exchange_ratios", "local_correlations", "bulk_sites", "structure_factor",
           "centre_site"]


def centre_site(L):
    """The site S_0 of the correlation map: (L // 2, L // 2)."""
    return (L // 2) * L + L // 2


def bulk_sites(L):
    """The central (L-4) x (L-4) sites (all sites when L <= 4)."""
    lo, hi = (2, L - 2) if L > 4 else (0, L)
    return [i * L + j for i in range(lo, hi) for j in range(lo, hi)]


def _strip_log_value(strip):
    """(log|W_i|, sign) of a one-row strip."""
    return strip.log_value()


def exchange_ratios(A, spins, L, chi, a):
    """r[m] = W(S^{a<->m})/W(S) for every site m with s_m != s_a, 0 elsewhere
    (and at m = a), each on the one-row strip of row i(m)."""
    spins = np.asarray(spins)
    N = L * L
    sf = spins.copy()
    sf[a] = 1 - sf[a]
    up, dn = upper_envs(A, spins, L, chi), lower_envs(A, spins, L, chi)
    upf, dnf = upper_envs(A, sf, L, chi), lower_envs(A, sf, L, chi)
    r = np.zeros(N)
    for i in range(L):
        targets = [i * L + j for j in range(L)
                   if i * L + j != a and spins[i * L + j] != spins[a]]
        if not targets:
            continue
        la0, sg0 = Strip1(A, spins, L, i, up[i - 1], dn[i + 1]).log_value()
        st = Strip1(A, sf, L, i, upf[i - 1], dnf[i + 1])
        base = upf[i - 1].logscale + dnf[i + 1].logscale
        for m in targets:
            j = m - i * L
            # S' = sf with s_m set to s_a (the exchange): column j replaced
            T = site_tensor(A, sf, L, i, j, spins[a])
            v = st.window(j, [T])
            if v == 0.0:
                continue
            lw = np.log(abs(v)) + st.cL[j] + st.cR[j + 1] + base
            r[m] = np.sign(v) * sg0 * np.exp(lw - la0)
    return r


def local_correlations(A, spins, L, chi, a):
    """(S_a . S_m)(S) for every site m (float64[N]): the local values whose
    mean over configurations drawn from W^2 is <S_a . S_m>."""
    spins = np.asarray(spins)
    sigma = 1.0 - 2.0 * spins.astype(np.float64)
    out = sigma[a] * sigma / 4.0 + 0.5 * exchange_ratios(A, spins, L, chi, a)
    out[a] = 0.75
    return out


def structure_factor(C, L, sources, k):
    """m_s^2(k) = (1/n^2) sum_{a, m in the bulk} C[a][m] cos(k . (r_a - r_m)),
    C[q][m] = <S_{sources[q]} . S_m> (float64[len(sources)][N]); every bulk
    site must be among the sources."""
    bulk = bulk_sites(L)
    pos = {s: q for q, s in enumerate(sources)}
    kx, ky = k
    tot = 0.0
    for a in bulk:
        ia, ja = divmod(a, L)
        for m in bulk:
            im, jm = divmod(m, L)
            tot += C[pos[a]][m] * np.cos(kx * (ia - im) + ky * (ja - jm))
    return tot / len(bulk) ** 2
