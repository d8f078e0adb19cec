"""FP64 oracle: single-layer PEPS contraction, local energy, log-derivatives,
gradient and gradient-optimisation step (PEPS++, arXiv:1806.03761).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Notation follows the paper's Eq. PEPS and Sec. "PEPS++ Algorithm": an L x L
open-boundary square lattice, site m = i*L + j (row i = 0 on top), site tensors
A_m(l, r, u, d, s) stored as ``A[m, s, l, r, u, d]`` with bond dimension D and
physical dimension d = 2.  For a spin configuration S the single-layer network
has tensors T_m = A_m^{s_m}; W(S) is its full contraction.

Readings taken where the paper is silent:
  * open boundary: the outward legs of boundary tensors keep index 0 only,
    i.e. they are legs of dimension 1 (Sec. "Introduction" states OBC only);
  * s = 0 is spin up, sigma = +1, S^z = +1/2;
  * truncation to D_c (Fig. 1(c), Sec. "PEPS++ Algorithm"): after absorbing a
    row, a left-to-right Householder QR sweep and a right-to-left SVD sweep
    that keeps the min(D_c, m, n) largest singular values of each m x n bond
    matrix; every site tensor is then scaled to unit max-abs and the log of
    the scale is accumulated;
  * ratios and log-derivatives use the strip-local amplitude W_i(S) of the
    strip they are computed on; the reported amplitude is the row-0 strip;
  * the off-diagonal matrix element of an exchange is +J/2 (no sign rotation).
"""
import numpy as np

from . import flops as _f

__all__ = [
    "bond_list", "site_tensor", "BMPS", "compress", "upper_envs", "lower_envs",
    "Strip1", "Strip2", "evaluate", "evaluate_batch", "gradient", "go_step",
    "amplitude",
]


# ----------------------------------------------------------------------------
# Lattice and Hamiltonian (Sec. "Experiment Setup": the J1-J2 Hamiltonian)
# ----------------------------------------------------------------------------
def bond_list(L):
    """All J1 (nearest-neighbour) and J2 (next-nearest) pairs of the open
    L x L lattice, in canonical order: horizontal J1 (i,j)-(i,j+1) row-major,
    vertical J1 (i,j)-(i+1,j), diagonal J2 (i,j)-(i+1,j+1), anti-diagonal J2
    (i,j+1)-(i+1,j).  Returns a list of (kind, m1, m2) with kind in
    {"h", "v", "d", "a"}."""
    out = []
    for i in range(L):
        for j in range(L - 1):
            out.append(("h", i * L + j, i * L + j + 1))
    for i in range(L - 1):
        for j in range(L):
            out.append(("v", i * L + j, (i + 1) * L + j))
    for i in range(L - 1):
        for j in range(L - 1):
            out.append(("d", i * L + j, (i + 1) * L + j + 1))
    for i in range(L - 1):
        for j in range(L - 1):
            out.append(("a", i * L + j + 1, (i + 1) * L + j))
    return out


def site_tensor(A, spins, L, i, j, s=None):
    """T_m = A_m^{s_m} (Eq. PEPS) with the outward boundary legs cut to
    index 0.  Axes (l, r, u, d).  ``s`` overrides the spin of the site."""
    D = A.shape[2]
    m = i * L + j
    sm = spins[m] if s is None else s
    T = A[m, int(sm)]
    return T[: 1 if j == 0 else D, : 1 if j == L - 1 else D,
             : 1 if i == 0 else D, : 1 if i == L - 1 else D]


# ----------------------------------------------------------------------------
# Boundary MPS with truncation D_c (Fig. 1(b,c); Sec. "PEPS++ Algorithm")
# ----------------------------------------------------------------------------
class BMPS:
    """A boundary MPS: site tensors M_j[a, p, b] (left bond, physical leg,
    right bond) and a scalar log-scale, so that the represented tensor is
    exp(logscale) * prod_j M_j."""

    def __init__(self, sites, logscale=0.0):
        self.sites = sites
        self.logscale = float(logscale)

    @staticmethod
    def trivial(L):
        return BMPS([np.ones((1, 1, 1)) for _ in range(L)], 0.0)


def absorb(env, Trow, from_above):
    """Absorb a row of the single-layer network into a boundary MPS.

    from_above: env is an upper environment whose physical legs are the up
    legs of this row; the result's physical legs are the row's down legs.
    Otherwise env is a lower environment and the result carries up legs.
    The new bond is (old bond, PEPS bond), of dimension D_c * D."""
    out = []
    for M, T in zip(env.sites, Trow):
        a, _, b = M.shape
        l, r, u, d = T.shape
        if from_above:
            N = _f.einsum("aub,lrud->aldbr", M, T).reshape(a * l, d, b * r)
        else:
            N = _f.einsum("adb,lrud->alubr", M, T).reshape(a * l, u, b * r)
        out.append(N)
    return BMPS(out, env.logscale)


def compress(env, chi):
    """Truncate the bond dimension to chi: a left-to-right QR sweep brings the
    MPS to left-canonical form, then a right-to-left SVD sweep keeps the
    min(chi, m, n) largest singular values at each bond (Fig. 1(c)).  QR and
    SVD are LAPACK's (numpy.linalg), called through the operation counter of
    ``oracle.flops``."""
    sites = [x.copy() for x in env.sites]
    L = len(sites)
    for j in range(L - 1):
        a, p, b = sites[j].shape
        Q, R = _f.qr(sites[j].reshape(a * p, b))
        k = Q.shape[1]
        sites[j] = Q.reshape(a, p, k)
        sites[j + 1] = _f.einsum("kb,bpc->kpc", R, sites[j + 1])
    for j in range(L - 1, 0, -1):
        a, p, b = sites[j].shape
        U, S, Vt = _f.svd(sites[j].reshape(a, p * b), keep=min(chi, a, p * b))
        k = min(chi, S.shape[0])
        sites[j] = Vt[:k].reshape(k, p, b)
        sites[j - 1] = _f.einsum("apb,bk->apk", sites[j - 1], U[:, :k] * S[:k])
    logscale = env.logscale
    for j in range(L):
        s = np.abs(sites[j]).max()
        if s > 0.0:
            sites[j] = sites[j] / s
            logscale += np.log(s)
    return BMPS(sites, logscale)


def row(A, spins, L, i):
    return [site_tensor(A, spins, L, i, j) for j in range(L)]


def upper_envs(A, spins, L, chi):
    """U_i, i = 0 .. L-2: rows 0..i contracted from the top and truncated.
    Returns a dict i -> BMPS (with U_{-1} the trivial MPS)."""
    env = BMPS.trivial(L)
    out = {-1: env}
    for i in range(0, L - 1):
        env = compress(absorb(env, row(A, spins, L, i), True), chi)
        out[i] = env
    return out


def lower_envs(A, spins, L, chi):
    """Dn_i, i = L-1 .. 1: rows i..L-1 contracted from the bottom and
    truncated.  Returns a dict i -> BMPS (with Dn_L the trivial MPS)."""
    env = BMPS.trivial(L)
    out = {L: env}
    for i in range(L - 1, 0, -1):
        env = compress(absorb(env, row(A, spins, L, i), False), chi)
        out[i] = env
    return out


# Column steps of the strips, written as pairwise tensordot contractions.
def _left1(L, U, T, Dn):
    """L'[B,r,D] = sum L[x,y,z] U[x,u,B] T[y,r,u,d] Dn[z,d,D]."""
    t = _f.tensordot(L, U, axes=([0], [0]))          # y z u B
    t = _f.tensordot(t, T, axes=([0, 2], [0, 2]))    # z B r d
    return _f.tensordot(t, Dn, axes=([0, 3], [0, 1]))  # B r D


def _right1(U, T, Dn, R):
    """R'[x,y,z] = sum U[x,u,B] T[y,r,u,d] Dn[z,d,D] R[B,r,D]."""
    t = _f.tensordot(Dn, R, axes=([2], [2]))         # z d B r
    t = _f.tensordot(T, t, axes=([1, 3], [3, 1]))    # y u z B
    return _f.tensordot(U, t, axes=([1, 2], [1, 3])).transpose(0, 1, 2)  # x y z


def _left2(L, U, T1, T2, Dn):
    """L'[B,r,s,D] = sum L[w,x,y,z] U[w,u,B] T1[x,r,u,m] T2[y,s,m,d] Dn[z,d,D]."""
    t = _f.tensordot(L, U, axes=([0], [0]))          # x y z u B
    t = _f.tensordot(t, T1, axes=([0, 3], [0, 2]))   # y z B r m
    t = _f.tensordot(t, T2, axes=([0, 4], [0, 2]))   # z B r s d
    return _f.tensordot(t, Dn, axes=([0, 4], [0, 1]))  # B r s D


def _right2(U, T1, T2, Dn, R):
    """R'[w,x,y,z] = sum U[w,u,B] T1[x,r,u,m] T2[y,s,m,d] Dn[z,d,D] R[B,r,s,D]."""
    t = _f.tensordot(Dn, R, axes=([2], [3]))         # z d B r s
    t = _f.tensordot(T2, t, axes=([1, 3], [4, 1]))   # y m z B r
    t = _f.tensordot(T1, t, axes=([1, 3], [4, 1]))   # x u y z B
    return _f.tensordot(U, t, axes=([1, 2], [1, 4]))  # w x y z


def _unit(x):
    """Scale to unit max-abs; returns (scaled, log of the scale)."""
    s = np.abs(x).max()
    if s == 0.0:
        return x, 0.0
    return x / s, float(np.log(s))


# ----------------------------------------------------------------------------
# Strips: the left/right auxiliary tensors of Fig. "contraction", Step 4
# ----------------------------------------------------------------------------
class Strip1:
    """One row i between U_{i-1} (above) and Dn_{i+1} (below), with left and
    right auxiliary tensors over its columns."""

    def __init__(self, A, spins, L, i, up, dn):
        self.A, self.spins, self.L, self.i = A, spins, L, i
        self.up, self.dn = up, dn
        self.T = row(A, spins, L, i)
        self.Lenv = [np.ones((1, 1, 1))]
        self.cL = [0.0]
        for j in range(L):
            x = _left1(self.Lenv[j], up.sites[j], self.T[j], dn.sites[j])
            x, c = _unit(x)
            self.Lenv.append(x)
            self.cL.append(self.cL[-1] + c)
        self.Renv = [None] * (L + 1)
        self.cR = [0.0] * (L + 1)
        self.Renv[L] = np.ones((1, 1, 1))
        for j in range(L - 1, -1, -1):
            x = _right1(up.sites[j], self.T[j], dn.sites[j], self.Renv[j + 1])
            x, c = _unit(x)
            self.Renv[j] = x
            self.cR[j] = self.cR[j + 1] + c

    def log_value(self):
        """(log|W_i|, sign W_i) of the whole strip."""
        v = float(self.Lenv[self.L].reshape(()))
        return (np.log(abs(v)) + self.cL[self.L] + self.up.logscale
                + self.dn.logscale), np.sign(v)

    def window(self, j, Ts):
        """Contract L_j, the columns j..j+len(Ts)-1 with tensors Ts, R_{j+k}."""
        x = self.Lenv[j]
        for k, T in enumerate(Ts):
            x = _left1(x, self.up.sites[j + k], T, self.dn.sites[j + k])
        return float(_f.einsum("xyz,xyz->", x, self.Renv[j + len(Ts)]))

    def ratio(self, j, new_T):
        """W_i(S')/W_i(S) where S' replaces the tensors of columns j, j+1...
        by ``new_T`` (same envs, Eq. ess)."""
        old = self.T[j: j + len(new_T)]
        return self.window(j, new_T) / self.window(j, old)

    def B(self, j):
        """B^{s_m}(S) of Eq. delta for site (i, j), scaled so that dividing by
        ``scaled_value`` gives Delta: returns (B_scaled, W_scaled)."""
        # B = L_j U_j Dn_j R_{j+1} with the site tensor left out
        lu = _f.tensordot(self.Lenv[j], self.up.sites[j], axes=([0], [0]))   # y z u B
        rd = _f.tensordot(self.Renv[j + 1], self.dn.sites[j], axes=([2], [2]))  # B r z d
        Bt = _f.tensordot(lu, rd, axes=([1, 3], [2, 0]))                     # y u r d
        Bt = Bt.transpose(0, 2, 1, 3)                                        # y r u d
        v = float(self.Lenv[self.L].reshape(()))
        # Bt carries exp(-(cL[j]+cR[j+1])), v carries exp(-cL[L])
        factor = np.exp(self.cL[j] + self.cR[j + 1] - self.cL[self.L])
        return Bt * factor / v


class Strip2:
    """Two rows i, i+1 between U_{i-1} and Dn_{i+2}, with left and right
    auxiliary tensors; used for vertical J1 and for J2 pairs."""

    def __init__(self, A, spins, L, i, up, dn):
        self.A, self.spins, self.L, self.i = A, spins, L, i
        self.up, self.dn = up, dn
        self.T1 = row(A, spins, L, i)
        self.T2 = row(A, spins, L, i + 1)
        self.Lenv = [np.ones((1, 1, 1, 1))]
        for j in range(L):
            x = self._step_left(self.Lenv[j], j, self.T1[j], self.T2[j])
            self.Lenv.append(_unit(x)[0])
        self.Renv = [None] * (L + 1)
        self.Renv[L] = np.ones((1, 1, 1, 1))
        for j in range(L - 1, -1, -1):
            x = _right2(self.up.sites[j], self.T1[j], self.T2[j],
                        self.dn.sites[j], self.Renv[j + 1])
            self.Renv[j] = _unit(x)[0]

    def _step_left(self, x, j, T1, T2):
        return _left2(x, self.up.sites[j], T1, T2, self.dn.sites[j])

    def window(self, j, cols):
        x = self.Lenv[j]
        for k, (T1, T2) in enumerate(cols):
            x = self._step_left(x, j + k, T1, T2)
        return float(_f.einsum("wxyz,wxyz->", x, self.Renv[j + len(cols)]))

    def ratio(self, j, new_cols):
        old = [(self.T1[j + k], self.T2[j + k]) for k in range(len(new_cols))]
        return self.window(j, new_cols) / self.window(j, old)


# ----------------------------------------------------------------------------
# Per-sample evaluation: amplitude, ratios, E(S), Delta (Eqs. ess, delta)
# ----------------------------------------------------------------------------
def evaluate(A, spins, L, chi, J1=1.0, J2=0.5, want_energy=True,
             want_delta=False):
    """Everything the sampling step needs for one configuration.

    Returns a dict with
      log_abs, sign : the amplitude W(S) from the row-0 strip,
      ratios        : float64[n_bonds], W(S')/W(S) for antiparallel pairs
                      (0 for parallel pairs), in bond_list order,
      n_flips       : number of antiparallel pairs,
      e_loc         : E(S) of Eq. ess (total, not per site),
      delta         : float64[N, 2, D, D, D, D], Delta^{s_m}(S) of Eq. delta
                      (zero outside the s_m slice and outside the open
                      boundary's index-0 legs).
    """
    spins = np.asarray(spins)
    N = L * L
    D = A.shape[2]
    up = upper_envs(A, spins, L, chi)
    dn = lower_envs(A, spins, L, chi)
    out = {}
    s1 = [Strip1(A, spins, L, i, up[i - 1], dn[i + 1]) for i in range(L)]
    la, sg = s1[0].log_value()
    out["log_abs"], out["sign"] = la, sg
    if want_energy:
        bonds = bond_list(L)
        sigma = 1.0 - 2.0 * spins.astype(np.float64)
        ratios = np.zeros(len(bonds))
        e = 0.0
        nf = 0
        s2 = [Strip2(A, spins, L, i, up[i - 1], dn[i + 2]) for i in range(L - 1)]
        for b, (kind, m1, m2) in enumerate(bonds):
            J = J1 if kind in ("h", "v") else J2
            e += J * sigma[m1] * sigma[m2] / 4.0
            if spins[m1] == spins[m2]:
                continue
            nf += 1
            i1, j1 = divmod(m1, L)
            i2, j2 = divmod(m2, L)
            t = lambda i, j, s: site_tensor(A, spins, L, i, j, s)
            s_a, s_b = spins[m1], spins[m2]
            if kind == "h":
                r = s1[i1].ratio(j1, [t(i1, j1, s_b), t(i1, j2, s_a)])
            elif kind == "v":
                r = s2[i1].ratio(j1, [(t(i1, j1, s_b), t(i2, j2, s_a))])
            elif kind == "d":
                r = s2[i1].ratio(j1, [(t(i1, j1, s_b), t(i1 + 1, j1, spins[(i1 + 1) * L + j1])),
                                      (t(i1, j1 + 1, spins[i1 * L + j1 + 1]), t(i2, j2, s_a))])
            else:  # "a": (i, j+1)-(i+1, j)
                jj = j2  # left column of the pair
                r = s2[i1].ratio(jj, [(t(i1, jj, spins[i1 * L + jj]), t(i2, jj, s_a)),
                                      (t(i1, j1, s_b), t(i1 + 1, j1, spins[(i1 + 1) * L + j1]))])
            ratios[b] = r
            e += J * 0.5 * r
        out["ratios"] = ratios
        out["n_flips"] = nf
        out["e_loc"] = e
    if want_delta:
        delta = np.zeros((N, 2, D, D, D, D))
        for i in range(L):
            for j in range(L):
                m = i * L + j
                Bt = s1[i].B(j)
                l, r, u, d = Bt.shape
                delta[m, int(spins[m]), :l, :r, :u, :d] = Bt
        out["delta"] = delta
    return out


def evaluate_batch(A, spins_batch, L, chi, J1=1.0, J2=0.5, want_energy=True,
                   want_delta=False):
    """``evaluate`` over a batch; returns stacked arrays."""
    res = [evaluate(A, s, L, chi, J1, J2, want_energy, want_delta)
           for s in spins_batch]
    out = {k: np.array([r[k] for r in res]) for k in res[0]}
    return out


def amplitude(A, spins, L, chi):
    """(log|W(S)|, sign W(S)) from the row-0 strip against Dn_1."""
    r = evaluate(A, spins, L, chi, want_energy=False)
    return r["log_abs"], r["sign"]


# ----------------------------------------------------------------------------
# Gradient and GO update (Eq. gradients; the sign update after Eq. delta)
# ----------------------------------------------------------------------------
def gradient(sum_delta, sum_delta_e, sum_e, M):
    """dE/dA = 2 <Delta E> - 2 <Delta> <E> with MC means over M samples."""
    return 2.0 * (sum_delta_e / M) - 2.0 * (sum_delta / M) * (sum_e / M)


def go_step(A, g, dt, seed, step):
    """A(n+1) = A(n) - p * dt * sign(g) with p in (0,1) drawn per element from
    Philox4x32-10 (key = seed, counter = (e mod 2^32, e >> 32, step, 2)),
    p = ((x >> 12) + 0.5) * 2^-52 from the first two output words x.
    sign(0) = 0."""
    from .philox import philox4x32_10, uniform_open53
    flat = A.reshape(-1)
    gf = g.reshape(-1)
    out = flat.copy()
    for e in range(flat.shape[0]):
        w = philox4x32_10((e & 0xFFFFFFFF, e >> 32, step & 0xFFFFFFFF, 2),
                          (seed & 0xFFFFFFFF, seed >> 32))
        p = uniform_open53(w[0], w[1])
        out[e] = flat[e] - p * dt * np.sign(gf[e])
    return out.reshape(A.shape)
