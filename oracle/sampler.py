"""Metropolis sampling of spin configurations with weight W(S)^2 (PEPS++,
Sec. "Thread-level parallelism", Fig. "contraction", Steps 1-3, and
Eq. energy-MC).  TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Readings taken where the paper is silent (it only says a configuration is
created at random and accepted or rejected):
  * moves are nearest-neighbour exchanges of antiparallel spins, so the
    S^z = 0 sector of the start configuration is kept;
  * a chain starts from a Fisher-Yates shuffle of floor(N/2) up spins and
    N - floor(N/2) down spins: for k = N-1 .. 1 the word
    x = Philox(key=seed, ctr=(k, 0, chain, 0)) picks j = x mod (k + 1)
    (x is the 64-bit word out[1]:out[0]) and entries k and j are swapped;
  * one sweep rebuilds the lower environments, then visits the rows
    top-down: in row i the horizontal bonds (i,j)-(i,j+1), j = 0..L-2, with
    the one-row strip between U_{i-1} and Dn_{i+1}; then the vertical bonds
    (i,j)-(i+1,j), j = 0..L-1, with the two-row strip between U_{i-1} and
    Dn_{i+2}; then row i is absorbed into U;
  * a proposal on an antiparallel bond b (canonical bond index) in sweep t
    of chain c draws u = (x >> 11) 2^-53 from Philox(seed, (b, t, c, 1)) and
    is accepted iff u < (W(S')/W(S))^2, the ratio taken on the current strip;
  * a chain records its configuration after sweep t when t > n_burn and
    (t - n_burn) mod n_thin == 0.
"""
import numpy as np

from .peps import (BMPS, Strip1, Strip2, absorb, compress, lower_envs, row,
                   site_tensor)
from .flops import tagged
from .philox import philox4x32_10, uniform53

__all__ = ["init_config", "metropolis_sweep", "sample_chains"]


def _word64(w):
    return (int(w[1]) << 32) | int(w[0])


def init_config(L, seed, chain):
    N = L * L
    s = np.ones(N, np.uint8)
    s[: N // 2] = 0
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for k in range(N - 1, 0, -1):
        j = _word64(philox4x32_10((k, 0, chain, 0), key)) % (k + 1)
        s[k], s[j] = s[j], s[k]
    return s


def metropolis_sweep(A, spins, L, chi, seed, chain, sweep):
    """One sweep over all nearest-neighbour bonds; updates ``spins`` in place
    and returns the number of accepted exchanges."""
    key = (seed & 0xFFFFFFFF, seed >> 32)
    with tagged("sweep_lower_envs"):
        dn = lower_envs(A, spins, L, chi)
    up = BMPS.trivial(L)
    acc = 0

    def t(i, j, s):
        return site_tensor(A, spins, L, i, j, s)

    for i in range(L):
        strip = Strip1(A, spins, L, i, up, dn[i + 1])
        for j in range(L - 1):
            m1, m2 = i * L + j, i * L + j + 1
            if spins[m1] == spins[m2]:
                continue
            b = i * (L - 1) + j
            r = strip.ratio(j, [t(i, j, spins[m2]), t(i, j + 1, spins[m1])])
            w = philox4x32_10((b, sweep, chain, 1), key)
            if uniform53(w[0], w[1]) < r * r:
                spins[m1], spins[m2] = spins[m2], spins[m1]
                acc += 1
                with tagged("rebuild"):
                    strip = Strip1(A, spins, L, i, up, dn[i + 1])
        if i < L - 1:
            strip2 = Strip2(A, spins, L, i, up, dn[i + 2])
            for j in range(L):
                m1, m2 = i * L + j, (i + 1) * L + j
                if spins[m1] == spins[m2]:
                    continue
                b = L * (L - 1) + i * L + j
                r = strip2.ratio(j, [(t(i, j, spins[m2]), t(i + 1, j, spins[m1]))])
                w = philox4x32_10((b, sweep, chain, 1), key)
                if uniform53(w[0], w[1]) < r * r:
                    spins[m1], spins[m2] = spins[m2], spins[m1]
                    acc += 1
                    with tagged("rebuild"):
                        strip2 = Strip2(A, spins, L, i, up, dn[i + 2])
            up = compress(absorb(up, row(A, spins, L, i), True), chi)
    return acc


def sample_chains(A, L, chi, seed, n_chains, n_burn, n_thin, samples_per_chain,
                  chain_offset=0, init=None, first_sweep=1):
    """Run chains chain_offset .. chain_offset+n_chains-1.

    Returns (samples uint8[n_chains * samples_per_chain, N] chain-major,
    final uint8[n_chains, N], accepted int[n_chains]).  ``init`` (optional
    uint8[n_chains, N]) replaces the Fisher-Yates start; sweeps are numbered
    first_sweep, first_sweep+1, ... (the burn-in/thinning rule counts sweeps
    of this call from 1)."""
    N = L * L
    out = np.empty((n_chains * samples_per_chain, N), np.uint8)
    final = np.empty((n_chains, N), np.uint8)
    accepted = np.zeros(n_chains, np.int64)
    total = n_burn + samples_per_chain * n_thin
    for c in range(n_chains):
        chain = chain_offset + c
        s = init_config(L, seed, chain) if init is None else np.array(init[c], np.uint8)
        k = 0
        for t in range(1, total + 1):
            accepted[c] += metropolis_sweep(A, s, L, chi, seed, chain,
                                            first_sweep + t - 1)
            if t > n_burn and (t - n_burn) % n_thin == 0:
                out[c * samples_per_chain + k] = s
                k += 1
        final[c] = s
    return out, final, accepted
