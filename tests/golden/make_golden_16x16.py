"""Write tests/golden/oracle_16x16_D6_Dc24.npz: the FP64 oracle's results on
the 64-configuration subset of the 16x16, D=6, Dc=24 workload (site tensors
A ~ N(0,1)/D from seed 4; the first 64 of its seeded S^z = 0 configurations,
seed 5), with each result's sensitivity to one unit roundoff of the input.

Only the oracle and the seeded input generators are called.  Stored per
configuration b:
  spins[b], log_abs[b], sign[b], e_loc[b], n_flips[b], ratios[b, n_bonds];
and over the 64 configurations: sum_e, the largest |entry| of
sum_delta / sum_delta_e (the Delta sums of Eq. gradients), and a seeded
sample of 4096 of their entries on the configurations' support
(flat indices into [N][2][D^4]).
Sensitivity: the oracle rerun on A * (1 + 2^-52 xi_k), xi_k ~ N(0, 1)
(seeds 1000 + k, k < 8); per configuration the largest change over the 8
perturbations of log|W|, of E(S) (relative to max(1, |E|)) and of the
ratios (relative, with a floor of 1e-10 * their RMS), and over the batch the
largest relative change of the sampled Delta sums.

    python tests/golden/make_golden_16x16.py [--workers 8]
"""
import argparse
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))

L, D, DC, B, NPERT = 16, 6, 24, 64, 8
U = 2.0 ** -52


def _one(args):
    """(b, k): evaluate configuration b on the tensors perturbed by draw k
    (k = -1: unperturbed).  Returns the per-sample results and Delta."""
    b, k = args
    import numpy as np
    import oracle
    from synth import make_peps, random_sz0_configs
    A = make_peps(L, D, 4)
    if k >= 0:
        xi = np.random.default_rng(1000 + k).standard_normal(A.shape)
        A = A * (1.0 + U * xi)
    s = random_sz0_configs(L, B, 5)[b]
    r = oracle.evaluate(A, s, L, DC, want_delta=True)
    N = L * L
    d = r["delta"][np.arange(N), s].reshape(N, -1)  # the s_m slices
    return b, k, r["log_abs"], r["sign"], r["e_loc"], r["n_flips"], r["ratios"], d


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    sys.path.insert(0, ROOT)
    import multiprocessing as mp
    import numpy as np
    from synth import random_sz0_configs
    spins = random_sz0_configs(L, B, 5)
    N, D4 = L * L, D ** 4
    jobs = [(b, k) for k in range(-1, NPERT) for b in range(B)]
    res = {}
    with mp.get_context("spawn").Pool(args.workers) as pool:
        for out in pool.imap_unordered(_one, jobs):
            res[(out[0], out[1])] = out[2:]
            print("done", out[0], out[1], len(res), "/", len(jobs), flush=True)

    def sums(k):
        sd = np.zeros((N, 2, D4))
        sde = np.zeros((N, 2, D4))
        for b in range(B):
            la, sg, e, nf, rat, d = res[(b, k)]
            sd[np.arange(N), spins[b]] += d
            sde[np.arange(N), spins[b]] += d * e
        return sd.reshape(-1), sde.reshape(-1)

    base = [res[(b, -1)] for b in range(B)]
    log_abs = np.array([x[0] for x in base])
    sign = np.array([x[1] for x in base], np.int8)
    e_loc = np.array([x[2] for x in base])
    n_flips = np.array([x[3] for x in base], np.int32)
    ratios = np.stack([x[4] for x in base])
    sd, sde = sums(-1)
    support = np.flatnonzero(sd)
    pick = np.sort(np.random.default_rng(77).choice(support, size=4096, replace=False))
    sens_la = np.zeros(B)
    sens_e = np.zeros(B)
    sens_r = np.zeros(B)
    sens_sums = 0.0
    for k in range(NPERT):
        for b in range(B):
            la, sg, e, nf, rat, d = res[(b, k)]
            assert sg == sign[b] and nf == n_flips[b]
            sens_la[b] = max(sens_la[b], abs(la - log_abs[b]))
            sens_e[b] = max(sens_e[b], abs(e - e_loc[b]) / max(1.0, abs(e_loc[b])))
            m = ratios[b] != 0
            floor = 1e-10 * np.sqrt(np.mean(ratios[b][m] ** 2))
            sens_r[b] = max(sens_r[b], np.max(np.abs(rat[m] - ratios[b][m]) /
                                              np.maximum(np.abs(ratios[b][m]), floor)))
        psd, psde = sums(k)
        sens_sums = max(sens_sums,
                        np.max(np.abs(psd[pick] - sd[pick])) / np.abs(sd).max(),
                        np.max(np.abs(psde[pick] - sde[pick])) / np.abs(sde).max())
    out = os.path.join(HERE, "oracle_16x16_D6_Dc24.npz")
    np.savez_compressed(
        out, L=L, D=D, Dc=DC, tensor_seed=4, config_seed=5, spins=spins,
        log_abs=log_abs, sign=sign, e_loc=e_loc, n_flips=n_flips, ratios=ratios,
        sum_e=e_loc.sum(), sum_delta_absmax=np.abs(sd).max(),
        sum_delta_e_absmax=np.abs(sde).max(), sum_index=pick,
        sum_delta=sd[pick], sum_delta_e=sde[pick],
        sens_log_abs=sens_la, sens_e_loc=sens_e, sens_ratios=sens_r, sens_sums=sens_sums,
        n_perturbations=NPERT, unit_roundoff=U)
    print("wrote", out)


if __name__ == "__main__":
    main()
