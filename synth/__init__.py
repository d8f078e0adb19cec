"""Seeded synthetic inputs for the per-sample PEPS contraction.

This module only builds input data: site tensors and spin configurations.
It holds none of the method's arithmetic, so both the CPU oracle and the
CUDA path can be fed from it without sharing any computation.

Conventions (the paper's Eq. PEPS, Sec. "PEPS++ Algorithm"):
  * square L x L lattice, site m = i*L + j, row i = 0 at the top;
  * site tensors A[m][s][l][r][u][d] (float64, C order), physical index s
    first, then the four virtual legs left/right/up/down of dimension D;
  * spins uint8[B][N] with s = 0 for spin up (sigma = +1) and s = 1 for down.

Workload recipes (stand-ins for the SU-initialised PEPS the paper reads from
a file, which is not available):
  * "gauss":  A ~ N(0, 1) / D                      (i.i.d. entries)
  * "neel":   A = P_neel + eps * G, G ~ N(0, 1) / D^2, where P_neel is the
              Neel product state: P(s, 0, 0, 0, 0) = [s == (i + j) mod 2]
              (eps = 1e-2 for the 8x8 workload).
"""
import numpy as np

__all__ = ["make_peps", "random_sz0_configs", "neel_config", "near_neel_configs",
           "CONFIGS", "workload"]


def make_peps(L, D, seed, kind="gauss", eps=1e-2):
    """Return A as float64[L*L, 2, D, D, D, D] drawn from numpy PCG64(seed)."""
    rng = np.random.default_rng(seed)
    N = L * L
    G = rng.standard_normal((N, 2, D, D, D, D))
    if kind == "gauss":
        return np.ascontiguousarray(G / D)
    if kind == "neel":
        A = eps * G / (D * D)
        for m in range(N):
            i, j = divmod(m, L)
            A[m, (i + j) % 2, 0, 0, 0, 0] += 1.0
        return np.ascontiguousarray(A)
    raise ValueError(f"unknown PEPS recipe {kind!r}")


def random_sz0_configs(L, B, seed):
    """B spin configurations with floor(N/2) up spins, each a uniform random
    permutation (numpy PCG64(seed)); uint8[B, N]."""
    rng = np.random.default_rng(seed)
    N = L * L
    base = np.ones(N, np.uint8)
    base[: N // 2] = 0
    out = np.empty((B, N), np.uint8)
    for b in range(B):
        out[b] = rng.permutation(base)
    return out


def neel_config(L):
    """The Neel configuration s_m = (i + j) mod 2 as uint8[N]."""
    return np.array([(m // L + m % L) % 2 for m in range(L * L)], np.uint8)


def near_neel_configs(L, B, seed, n_moves):
    """B configurations obtained from the Neel configuration by n_moves
    random exchanges of antiparallel nearest-neighbour pairs (numpy
    PCG64(seed)); S^z = 0 is kept.  Typical configurations of a Neel-like
    state's W^2 distribution lie this close to the Neel configuration."""
    rng = np.random.default_rng(seed)
    N = L * L
    pairs = [(i * L + j, i * L + j + 1) for i in range(L) for j in range(L - 1)]
    pairs += [(i * L + j, (i + 1) * L + j) for i in range(L - 1) for j in range(L)]
    pairs = np.array(pairs)
    out = np.empty((B, N), np.uint8)
    for b in range(B):
        s = neel_config(L).copy()
        done = 0
        while done < n_moves:
            a, c = pairs[rng.integers(len(pairs))]
            if s[a] != s[c]:
                s[a], s[c] = s[c], s[a]
                done += 1
        out[b] = s
    return out


# The workloads: shapes, truncation, recipe, seeds and batch sizes.
CONFIGS = {
    "4x4_D2_Dc16": dict(L=4, D=2, Dc=16, recipe="gauss", seed=1, chains=16,
                        samples_per_chain=16, n_burn=20, n_thin=1, dt=1e-2),
    "8x8_D4_Dc16": dict(L=8, D=4, Dc=16, recipe="neel", eps=1e-2, seed=2,
                        config_seed=3, batch=4096),
    "16x16_D6_Dc24": dict(L=16, D=6, Dc=24, recipe="gauss", seed=4,
                          config_seed=5, batch=8192),
    "24x24_D8_Dc32": dict(L=24, D=8, Dc=32, recipe="gauss", seed=6,
                          config_seed=7, batch=1024),
    # a smaller lattice with the 16x16 workload's bond dimensions (the same
    # QR and SVD shapes per site): profiling captures
    "12x12_D6_Dc24": dict(L=12, D=6, Dc=24, recipe="gauss", seed=8,
                          config_seed=9, batch=304),
    # a smaller lattice with the 24x24 workload's bond dimensions (QR panels
    # of 2048 x 256, 256 x 256 SVDs): tuning and profiling
    "12x12_D8_Dc32": dict(L=12, D=8, Dc=32, recipe="gauss", seed=10,
                          config_seed=11, batch=304),
}


def workload(name):
    """(A, cfg) for a named workload."""
    cfg = dict(CONFIGS[name])
    A = make_peps(cfg["L"], cfg["D"], cfg["seed"], cfg["recipe"],
                  cfg.get("eps", 1e-2))
    return A, cfg
