"""Exact references for tiny lattices, written independently of ``oracle/``:
brute-force contraction of the whole single-layer network, an exact row
transfer-matrix amplitude for every configuration, and the J1-J2
Hamiltonian built from spin operators.  Used only to pin the oracle."""
import itertools

import numpy as np


def brute_amplitude(A, spins, L):
    """W(S) = Tr(prod_m A_m^{s_m}) (Eq. PEPS) by one einsum over the whole
    network; outward boundary legs are fixed to index 0."""
    D = A.shape[2]
    ops = []
    # label every virtual bond: horizontal (i,j)-(i,j+1) and vertical (i,j)-(i+1,j)
    h = {}
    v = {}
    nxt = [0]

    def lab():
        nxt[0] += 1
        return nxt[0] - 1

    for i in range(L):
        for j in range(L - 1):
            h[i, j] = lab()
    for i in range(L - 1):
        for j in range(L):
            v[i, j] = lab()
    for i in range(L):
        for j in range(L):
            T = A[i * L + j, int(spins[i * L + j])]
            idx = [slice(None)] * 4
            labels = []
            legs = [(j > 0, h.get((i, j - 1))), (j < L - 1, h.get((i, j))),
                    (i > 0, v.get((i - 1, j))), (i < L - 1, v.get((i, j)))]
            for k, (inner, b) in enumerate(legs):
                if inner:
                    labels.append(b)
                else:
                    idx[k] = 0
            ops += [T[tuple(idx)], labels]
    return float(np.einsum(*ops, [], optimize=True)) if D > 0 else 0.0


def all_amplitudes(A, L):
    """psi[x] for every configuration x (bit m of x is s_m, site m = i*L+j),
    by multiplying exact row transfer matrices over D^L vertical bond
    states."""
    D = A.shape[2]
    N = L * L
    patterns = list(itertools.product([0, 1], repeat=L))  # s_{i,0..L-1}

    def row_transfer(i, pat):
        # X[u_0..u_{L-1}, d_0..d_{L-1}] for row i with spins pat
        X = None
        for j in range(L):
            T = A[i * L + j, pat[j]]
            if j == 0:
                T = T[0:1]
            if j == L - 1:
                T = T[:, 0:1]
            if i == 0:
                T = T[:, :, 0:1]
            if i == L - 1:
                T = T[:, :, :, 0:1]
            if X is None:
                X = T[0]  # (r, u, d)
                X = np.transpose(X, (1, 2, 0))  # (u0, d0, r)
                X = X.reshape(X.shape[0], X.shape[1], X.shape[2])
                us, ds = [X.shape[0]], [X.shape[1]]
                X = X.reshape(-1, X.shape[-1])  # ((u0,d0), r)
            else:
                # X[(U,Dd), l] T[l, r, u, d] -> [(U,Dd), r, u, d]
                Y = np.einsum("xl,lrud->xrud", X, T)
                us.append(T.shape[2])
                ds.append(T.shape[3])
                Y = np.transpose(Y, (0, 2, 3, 1))
                X = Y.reshape(-1, Y.shape[-1])
        X = X[:, 0]
        # X is indexed by (u0,d0,u1,d1,...); regroup to (u..., d...)
        X = X.reshape([x for pair in zip(us, ds) for x in pair])
        perm = list(range(0, 2 * L, 2)) + list(range(1, 2 * L, 2))
        X = np.transpose(X, perm)
        return X.reshape(int(np.prod(us)), int(np.prod(ds)))

    # vec[pattern-prefix index, bond state]
    vecs = None
    for i in range(L):
        mats = [row_transfer(i, p) for p in patterns]
        if vecs is None:
            vecs = np.stack([m[0] for m in mats])  # u dim is 1 on top
        else:
            vecs = np.einsum("pu,qud->pqd", vecs, np.stack(mats)).reshape(-1, mats[0].shape[1])
    psi_rows = vecs[:, 0]  # bottom d dim is 1
    # psi_rows index = sum_i pat_i * 2^(L*(L-1-i)), pat as binary s_{i,0} most significant
    psi = np.zeros(1 << N)
    for idx in range(1 << N):
        x = 0
        rem = idx
        for i in range(L - 1, -1, -1):
            p = rem % (1 << L)
            rem //= 1 << L
            for j in range(L):
                bit = (p >> (L - 1 - j)) & 1
                x |= bit << (i * L + j)
        psi[x] = psi_rows[idx]
    return psi


def config_index(spins):
    return int(sum(int(s) << m for m, s in enumerate(spins)))


def pairs(L, J1, J2):
    out = []
    for i in range(L):
        for j in range(L):
            m = i * L + j
            if j + 1 < L:
                out.append((m, m + 1, J1))
            if i + 1 < L:
                out.append((m, m + L, J1))
            if i + 1 < L and j + 1 < L:
                out.append((m, m + L + 1, J2))
            if i + 1 < L and j > 0:
                out.append((m, m + L - 1, J2))
    return out


def apply_H(psi, L, J1, J2):
    """(H psi) for H = J1 sum_NN S_i.S_j + J2 sum_NNN S_i.S_j, written with
    S.S = S^z S^z + (S^+ S^- + S^- S^+)/2 on bit strings (bit 1 = down)."""
    N = L * L
    x = np.arange(1 << N)
    out = np.zeros_like(psi)
    for a, b, J in pairs(L, J1, J2):
        sa = (x >> a) & 1
        sb = (x >> b) & 1
        same = sa == sb
        out += J * np.where(same, 0.25, -0.25) * psi
        flipped = x ^ ((1 << a) | (1 << b))
        out[flipped[~same]] += J * 0.5 * psi[x[~same]]
    return out


def dense_H(L, J1, J2):
    """Dense H from Kronecker products of spin-1/2 matrices (bit m <-> site m,
    |0> = up)."""
    N = L * L
    sx = np.array([[0, 0.5], [0.5, 0]])
    sy = np.array([[0, -0.5j], [0.5j, 0]])
    sz = np.array([[0.5, 0], [0, -0.5]])
    dim = 1 << N

    def op(o, m):
        # site m is bit m: kron order puts the highest site first
        mats = [np.eye(2)] * N
        mats[N - 1 - m] = o
        r = np.array([[1.0]])
        for M in mats:
            r = np.kron(r, M)
        return r

    H = np.zeros((dim, dim), complex)
    for a, b, J in pairs(L, J1, J2):
        for o in (sx, sy, sz):
            H += J * op(o, a) @ op(o, b)
    assert np.allclose(H.imag, 0)
    return H.real


def dense_SS(L, a, b):
    """S_a . S_b as a dense matrix (Kronecker products of the spin-1/2
    matrices; bit m <-> site m, |0> = up).  a == b gives 3/4 times 1."""
    N = L * L
    sx = np.array([[0, 0.5], [0.5, 0]])
    sy = np.array([[0, -0.5j], [0.5j, 0]])
    sz = np.array([[0.5, 0], [0, -0.5]])

    def op(o, m):
        mats = [np.eye(2)] * N
        mats[N - 1 - m] = o
        r = np.array([[1.0]])
        for M in mats:
            r = np.kron(r, M)
        return r

    S = sum(op(o, a) @ op(o, b) for o in (sx, sy, sz))
    assert np.allclose(S.imag, 0)
    return S.real
