// peps_mps.cuh -- boundary-MPS absorption and truncation, and the one- and
// two-row strips with their left/right auxiliary tensors (PEPS++,
// arXiv:1806.03761: Fig. 1(b,c), Sec. "PEPS++ Algorithm", Fig. "contraction"
// Step 4, Eqs. ess and delta).
//
// Layouts (row-major):
//   MPS site         M[a][p][b]       (left bond, physical leg, right bond)
//   site tensor      A[m][s][l][r][u][d], spin slice T = A[m][s_m]
//   one-row env      L[a_u][l][a_d]   (upper bond, PEPS bond, lower bond)
//   two-row env      L2[a_u][l1][l2][a_d]
// Open-boundary legs are the index-0 slice of T: their extent is 1.
#pragma once
#include "peps_core.cuh"

// Scratch of one sample (one thread block), in the form's scalar type R.
template <class R>
struct Work {
  R* dn;      // lower environments Dn_1..Dn_{L-1} and the trivial one at L
  R* up;      // upper environments: [0] trivial, [1],[2] rolling
  R* rst;     // R factors of the QR sweep, L matrices of (Dc D)^2
  R* b0;      // three temporaries of Dc^2 D^3
  R* b1;
  R* b2;
  R* y;       // Y_j of the SVD sweep
  R* xj;      // X_j of the SVD sweep
  R* vt;      // V^T of the kept singular vectors
  R* c0;      // carried right factor C_j (two buffers)
  R* c1;
  R* l1;      // one-row strip envs, L+1 each
  R* r1;
  R* l2;      // two-row strip envs, L+1 each
  R* r2;
  double* scl;    // log-scales of the strip envs: 4 (L+1)
  double* delta;  // staged Delta of one sample: N D^4
  R* alpha;       // singular-value scratch (d, e, tau of the bidiagonal)
  R* inv;         // inverse-iteration scratch
  R* dnf;         // lower / upper environments of a configuration with one
  R* upf;         // spin flipped (spin correlations)
  // shared memory
  double* red;
  R* redR;
  R* wsh;
  R* qrv;  // PEPS_QR_NB * PEPS_QR_ROWS: the blocked QR's panel (null: unblocked)
  double* rot;
  int* flags;
};

struct EnvDims {
  const int16_t* a;
  const int16_t* b;
  int p;  // physical extent (1 for the trivial environment)
};

__device__ __forceinline__ EnvDims env_dims(const PepsPlan& P, const PepsStep* steps, int step) {
  // step < 0: the trivial environment (all extents 1)
  EnvDims e;
  if (step < 0) {
    e.a = nullptr;
    e.b = nullptr;
    e.p = 1;
  } else {
    e.a = steps[step].oa;
    e.b = steps[step].ob;
    e.p = P.D;
  }
  return e;
}
__device__ __forceinline__ int ed_a(const EnvDims& e, int j) { return e.a ? e.a[j] : 1; }
__device__ __forceinline__ int ed_b(const EnvDims& e, int j) { return e.b ? e.b[j] : 1; }

// ---------------------------------------------------------------------------
// Absorb row `row` into the environment Min (dims of `st`'s input) and
// truncate to Dc (dims of `st`'s output), writing Mout.  above: Min is an
// upper environment (its physical legs meet the row's up legs); else a lower
// one.  The absorbed tensor N_j[(a,l)][q][(b,r)] = sum_p M_j[a][p][b]
// T_j[l][r][p][q] is never formed: the QR sweep works on
// X_j = R_{j-1} N_j (rows (x,q), columns (b,r)) and the SVD sweep on
// R_{j-1} Y_j with Y_j = N_j C_{j+1}; this is the left-canonical QR sweep
// followed by the right-to-left SVD truncation, with the orthogonal factors
// of the QR sweep never formed.  Returns the new log-scale.
// ---------------------------------------------------------------------------
template <class R>
__device__ double compress_row(const PepsPlan& P, const PepsStep& st, bool above,
                               int row, const R* As, const uint8_t* sp,
                               const R* Min, double log_in, R* Mout,
                               const Work<R>& w) {
  const int L = P.L, D = P.D, D2 = P.D2, D3 = P.D3, D4 = P.D4;
  const int Q = D;
  const int sP = above ? D : 1, sQ = above ? 1 : D;  // strides of p, q in T
  const int64_t SC = P.site_cap, MC = P.mat_cap;
  double logs = log_in;
  PEPS_TIC(t_comp);
  // R_{-1} = [1]
  if (threadIdx.x == 0) w.rst[0] = Arith<R>::one();
  __syncthreads();
  // ---- left-to-right QR sweep: R_j from X_j = R_{j-1} N_j --------------
  int rprev = 1;
  for (int j = 0; j < L - 1; ++j) {
    const int a = st.ia[j], p = st.ip[j], b = st.ib[j];
    const int Dl = (j == 0) ? 1 : D, Dr = (j == L - 1) ? 1 : D;
    const int Aj = a * Dl, Bj = b * Dr;
    const R* Rp = w.rst + (int64_t)j * MC;           // rprev x Aj
    const R* Mj = Min + (int64_t)j * SC;
    const int m = row * L + j;
    const R* T = As + ((int64_t)m * 2 + sp[m]) * D4;
    // S1[x][l][p'][b'] = sum_a R[x][a*Dl + l] M[a][p'][b']
    Ctr c = ctr_init();
    c.e[0] = rprev; c.e[1] = Dl; c.e[2] = p; c.e[3] = b;
    c.sa[0] = Aj; c.sa[1] = 1;
    c.sb[2] = b; c.sb[3] = 1;
    c.sc[0] = Dl * p * b; c.sc[1] = p * b; c.sc[2] = b; c.sc[3] = 1;
    c.k1 = a; c.ka1 = Dl; c.kb1 = p * b;
    contract<R>(c, Rp, Mj, w.b0);
    // X[(x,q)][(b',r)] = sum_{l,p'} S1[x][l][p'][b'] T[l][r][p'][q], stored
    // column-major (column (b',r), row (x,q)) for the Householder sweep
    const int mrow = rprev * Q;
    c = ctr_init();
    c.e[0] = rprev; c.e[1] = Q; c.e[2] = b; c.e[3] = Dr;
    c.sa[0] = Dl * p * b; c.sa[2] = 1;
    c.sb[1] = sQ; c.sb[3] = D2;
    c.sc[0] = Q; c.sc[1] = 1; c.sc[2] = Dr * mrow; c.sc[3] = mrow;
    c.k1 = Dl; c.ka1 = p * b; c.kb1 = D3;
    c.k2 = p; c.ka2 = b; c.kb2 = sP;
    contract<R>(c, w.b0, T, w.b1);
    PEPS_TIC(t_qr);
    householder_r<R>(w.b1, mrow, Bj, w.rst + (int64_t)(j + 1) * MC, w.wsh, w.qrv);
    PEPS_TOC(t_qr, PH_QR);
    rprev = st.r[j];
    // only the row space of R_j matters: keep it at unit scale so that the
    // float-float form stays inside the FP32 exponent range
    normalize_pow2<R>(w.rst + (int64_t)(j + 1) * MC, rprev * Bj, w.red);
  }
  // ---- right-to-left SVD sweep -----------------------------------------
  R* Cn = w.c0;
  R* Cx = w.c1;
  if (threadIdx.x == 0) Cn[0] = Arith<R>::one();
  __syncthreads();
  int cn = 1;
  for (int j = L - 1; j >= 0; --j) {
    const int a = st.ia[j], p = st.ip[j], b = st.ib[j];
    const int Dl = (j == 0) ? 1 : D, Dr = (j == L - 1) ? 1 : D;
    const int Aj = a * Dl;
    const R* Mj = Min + (int64_t)j * SC;
    const int m = row * L + j;
    const R* T = As + ((int64_t)m * 2 + sp[m]) * D4;
    // S2[a][p'][r][c] = sum_b M[a][p'][b] C[b*Dr + r][c]
    Ctr c = ctr_init();
    c.e[0] = a; c.e[1] = p; c.e[2] = Dr; c.e[3] = cn;
    c.sa[0] = p * b; c.sa[1] = b;
    c.sb[2] = cn; c.sb[3] = 1;
    c.sc[0] = p * Dr * cn; c.sc[1] = Dr * cn; c.sc[2] = cn; c.sc[3] = 1;
    c.k1 = b; c.ka1 = 1; c.kb1 = Dr * cn;
    contract<R>(c, Mj, Cn, w.b0);
    // Y[(a,l)][(q,c)] = sum_{p',r} S2[a][p'][r][c] T[l][r][p'][q]
    R* Y = (j == 0) ? w.b1 : w.y;
    c = ctr_init();
    c.e[0] = a; c.e[1] = Dl; c.e[2] = Q; c.e[3] = cn;
    c.sa[0] = p * Dr * cn; c.sa[3] = 1;
    c.sb[1] = D3; c.sb[2] = sQ;
    c.sc[0] = Dl * Q * cn; c.sc[1] = Q * cn; c.sc[2] = cn; c.sc[3] = 1;
    c.k1 = p; c.ka1 = Dr * cn; c.kb1 = sP;
    c.k2 = Dr; c.ka2 = cn; c.kb2 = D2;
    contract<R>(c, w.b0, T, Y);
    const int n = Q * cn;
    if (j == 0) {
      // site 0: Y_0 (1 x Q x c_1) is the truncated site, carrying the norm
      R* out = Mout;
      for (int o = threadIdx.x; o < n; o += blockDim.x) out[o] = Y[o];
      __syncthreads();
      logs += normalize_pow2<R>(out, n, w.red);
      break;
    }
    // X_j = R_{j-1} Y_j : rr x n (column-major when a QR reduces it first)
    const int rr = (j >= 1) ? st.r[j - 1] : 1;
    c = ctr_init();
    c.e[0] = rr; c.e[1] = n;
    c.sa[0] = Aj; c.sb[1] = 1;
    if (rr > n) { c.sc[0] = 1; c.sc[1] = rr; } else { c.sc[0] = n; c.sc[1] = 1; }
    c.k1 = Aj; c.ka1 = 1; c.kb1 = n;
    contract<R>(c, w.rst + (int64_t)j * MC, Y, w.xj);
    const int kk = st.oa[j];
    R* V = Mout + (int64_t)j * SC;  // V^T (kk x n) is the truncated site j
    normalize_pow2<R>(w.xj, rr * n, w.red);
    float* fsh = reinterpret_cast<float*>(w.rot);
    if (rr > n) {
      PEPS_TIC(t_q2);
      householder_r<R>(w.xj, rr, n, w.b2, w.wsh, w.qrv);
      PEPS_TOC(t_q2, PH_SVD_QR);
      PEPS_TIC(t_svd);
      svd_topk_rows<R>(w.b2, n, n, kk, V, w.alpha, w.inv, fsh, w.wsh, w.red, w.qrv);
      PEPS_TOC(t_svd, PH_SVD);
    } else {
      PEPS_TIC(t_svd);
      svd_topk_rows<R>(w.xj, rr, n, kk, V, w.alpha, w.inv, fsh, w.wsh, w.red, w.qrv);
      PEPS_TOC(t_svd, PH_SVD);
    }
    // C_j[(a,l)][k] = sum_{(q,c)} Y[(a,l)][(q,c)] V^T[k][(q,c)]
    c = ctr_init();
    c.e[0] = Aj; c.e[1] = kk;
    c.sa[0] = n; c.sb[1] = n; c.sc[0] = kk; c.sc[1] = 1;
    c.k1 = n; c.ka1 = 1; c.kb1 = 1;
    contract<R>(c, Y, V, Cx);
    logs += normalize_pow2<R>(Cx, Aj * kk, w.red);
    R* tmp = Cn; Cn = Cx; Cx = tmp;
    cn = kk;
  }
  PEPS_TOC(t_comp, PH_COMPRESS);
  return logs;
}

// ---------------------------------------------------------------------------
// One-row strip: column step  Lnew[b_u][r][b_d] = sum L[a_u][l][a_d]
// U[a_u][u][b_u] T[l][r][u][d] Dn[a_d][d][b_d], in three contractions.
// ---------------------------------------------------------------------------
struct Col1 {
  int au, pu, bu;  // upper site dims
  int ad, pd, bd;  // lower site dims
  int Dl, Dr;
};

template <class R>
__device__ void strip1_left_step(const PepsPlan& P, const Col1& k, const R* Lj,
                                 const R* U, const R* T, const R* Dn, R* Lout,
                                 const Work<R>& w) {
  const int D = P.D, D2 = P.D2, D3 = P.D3;
  // E1[l][a_d][u][b_u] = sum_{a_u} L[a_u][l][a_d] U[a_u][u][b_u]
  Ctr c = ctr_init();
  c.e[0] = k.Dl; c.e[1] = k.ad; c.e[2] = k.pu; c.e[3] = k.bu;
  c.sa[0] = k.ad; c.sa[1] = 1;
  c.sb[2] = k.bu; c.sb[3] = 1;
  c.sc[0] = k.ad * k.pu * k.bu; c.sc[1] = k.pu * k.bu; c.sc[2] = k.bu; c.sc[3] = 1;
  c.k1 = k.au; c.ka1 = k.Dl * k.ad; c.kb1 = k.pu * k.bu;
  contract<R>(c, Lj, U, w.b0);
  // E2[a_d][b_u][r][d] = sum_{l,u} E1[l][a_d][u][b_u] T[l][r][u][d]
  c = ctr_init();
  c.e[0] = k.ad; c.e[1] = k.bu; c.e[2] = k.Dr; c.e[3] = k.pd;
  c.sa[0] = k.pu * k.bu; c.sa[1] = 1;
  c.sb[2] = D2; c.sb[3] = 1;
  c.sc[0] = k.bu * k.Dr * k.pd; c.sc[1] = k.Dr * k.pd; c.sc[2] = k.pd; c.sc[3] = 1;
  c.k1 = k.Dl; c.ka1 = k.ad * k.pu * k.bu; c.kb1 = D3;
  c.k2 = k.pu; c.ka2 = k.bu; c.kb2 = D;
  contract<R>(c, w.b0, T, w.b1);
  // Lnew[b_u][r][b_d] = sum_{a_d,d} E2[a_d][b_u][r][d] Dn[a_d][d][b_d]
  c = ctr_init();
  c.e[0] = k.bu; c.e[1] = k.Dr; c.e[2] = k.bd;
  c.sa[0] = k.Dr * k.pd; c.sa[1] = k.pd;
  c.sb[2] = 1;
  c.sc[0] = k.Dr * k.bd; c.sc[1] = k.bd; c.sc[2] = 1;
  c.k1 = k.ad; c.ka1 = k.bu * k.Dr * k.pd; c.kb1 = k.pd * k.bd;
  c.k2 = k.pd; c.ka2 = 1; c.kb2 = k.bd;
  contract<R>(c, w.b1, Dn, Lout);
}

// F1[b_u][r][a_d][d] = sum_{b_d} Rj1[b_u][r][b_d] Dn[a_d][d][b_d]
template <class R>
__device__ void strip1_f1(const Col1& k, const R* Rj1, const R* Dn, R* F1) {
  Ctr c = ctr_init();
  c.e[0] = k.bu; c.e[1] = k.Dr; c.e[2] = k.ad; c.e[3] = k.pd;
  c.sa[0] = k.Dr * k.bd; c.sa[1] = k.bd;
  c.sb[2] = k.pd * k.bd; c.sb[3] = k.bd;
  c.sc[0] = k.Dr * k.ad * k.pd; c.sc[1] = k.ad * k.pd; c.sc[2] = k.pd; c.sc[3] = 1;
  c.k1 = k.bd; c.ka1 = 1; c.kb1 = 1;
  contract<R>(c, Rj1, Dn, F1);
}

template <class R>
__device__ void strip1_right_step(const PepsPlan& P, const Col1& k, const R* Rj1,
                                  const R* U, const R* T, const R* Dn, R* Rout,
                                  const Work<R>& w) {
  const int D = P.D, D2 = P.D2, D3 = P.D3;
  strip1_f1<R>(k, Rj1, Dn, w.b0);
  // F2[b_u][u][l][a_d] = sum_{r,d} F1[b_u][r][a_d][d] T[l][r][u][d]
  Ctr c = ctr_init();
  c.e[0] = k.bu; c.e[1] = k.pu; c.e[2] = k.Dl; c.e[3] = k.ad;
  c.sa[0] = k.Dr * k.ad * k.pd; c.sa[3] = k.pd;
  c.sb[1] = D; c.sb[2] = D3;
  c.sc[0] = k.pu * k.Dl * k.ad; c.sc[1] = k.Dl * k.ad; c.sc[2] = k.ad; c.sc[3] = 1;
  c.k1 = k.Dr; c.ka1 = k.ad * k.pd; c.kb1 = D2;
  c.k2 = k.pd; c.ka2 = 1; c.kb2 = 1;
  contract<R>(c, w.b0, T, w.b1);
  // Rnew[a_u][l][a_d] = sum_{u,b_u} U[a_u][u][b_u] F2[b_u][u][l][a_d]
  c = ctr_init();
  c.e[0] = k.au; c.e[1] = k.Dl * k.ad;
  c.sa[0] = k.pu * k.bu; c.sb[1] = 1;
  c.sc[0] = k.Dl * k.ad; c.sc[1] = 1;
  c.k1 = k.pu; c.ka1 = k.bu; c.kb1 = k.Dl * k.ad;
  c.k2 = k.bu; c.ka2 = 1; c.kb2 = k.pu * k.Dl * k.ad;
  contract<R>(c, U, w.b1, Rout);
}

// B[l][r][u][d] of Eq. delta for the site of this column, written with the
// full D^4 layout (entries outside the open-boundary extents untouched):
// B = sum_{a_d,b_u} E1[l][a_d][u][b_u] F1[b_u][r][a_d][d].
template <class R>
__device__ void strip1_btensor(const PepsPlan& P, const Col1& k, const R* Lj,
                               const R* U, const R* Rj1, const R* Dn, R* Bout,
                               const Work<R>& w) {
  const int D = P.D, D2 = P.D2, D3 = P.D3;
  Ctr c = ctr_init();
  c.e[0] = k.Dl; c.e[1] = k.ad; c.e[2] = k.pu; c.e[3] = k.bu;
  c.sa[0] = k.ad; c.sa[1] = 1;
  c.sb[2] = k.bu; c.sb[3] = 1;
  c.sc[0] = k.ad * k.pu * k.bu; c.sc[1] = k.pu * k.bu; c.sc[2] = k.bu; c.sc[3] = 1;
  c.k1 = k.au; c.ka1 = k.Dl * k.ad; c.kb1 = k.pu * k.bu;
  contract<R>(c, Lj, U, w.b0);   // E1
  strip1_f1<R>(k, Rj1, Dn, w.b1);  // F1
  c = ctr_init();
  c.e[0] = k.Dl; c.e[1] = k.Dr; c.e[2] = k.pu; c.e[3] = k.pd;
  c.sa[0] = k.ad * k.pu * k.bu; c.sa[2] = k.bu;
  c.sb[1] = k.ad * k.pd; c.sb[3] = 1;
  c.sc[0] = D3; c.sc[1] = D2; c.sc[2] = D; c.sc[3] = 1;
  c.k1 = k.ad; c.ka1 = k.pu * k.bu; c.kb1 = k.pd;
  c.k2 = k.bu; c.ka2 = 1; c.kb2 = k.Dr * k.ad * k.pd;
  contract<R>(c, w.b0, w.b1, Bout);
}

// Dot product of two equally laid out tensors (block-wide), as double.
template <class R>
__device__ double dot_blk(const R* x, const R* y, int n, const Work<R>& w) {
  typename Arith<R>::acc_t a;
  Arith<R>::acc_init(a);
  for (int i = threadIdx.x; i < n; i += blockDim.x) Arith<R>::mac(a, x[i], y[i]);
  return Arith<R>::to(block_sum<R>(Arith<R>::acc_get(a), w.redR));
}

// ---------------------------------------------------------------------------
// Two-row strip column step:
// L2new[b_u][r1][r2][b_d] = sum L2[a_u][l1][l2][a_d] U[a_u][u1][b_u]
//     T1[l1][r1][u1][m] T2[l2][r2][m][d2] Dn[a_d][d2][b_d]
// ---------------------------------------------------------------------------
template <class R>
__device__ void strip2_left_step(const PepsPlan& P, const Col1& k, const R* L2,
                                 const R* U, const R* T1, const R* T2,
                                 const R* Dn, R* Lout, const Work<R>& w) {
  const int D = P.D, D2 = P.D2, D3 = P.D3;
  const int Dl = k.Dl, Dr = k.Dr;
  // G1[(l1 l2)][a_d][u1][b_u] = sum_{a_u} L2[a_u][(l1 l2)][a_d] U[a_u][u1][b_u]
  Ctr c = ctr_init();
  c.e[0] = Dl * Dl; c.e[1] = k.ad; c.e[2] = k.pu; c.e[3] = k.bu;
  c.sa[0] = k.ad; c.sa[1] = 1;
  c.sb[2] = k.bu; c.sb[3] = 1;
  c.sc[0] = k.ad * k.pu * k.bu; c.sc[1] = k.pu * k.bu; c.sc[2] = k.bu; c.sc[3] = 1;
  c.k1 = k.au; c.ka1 = Dl * Dl * k.ad; c.kb1 = k.pu * k.bu;
  contract<R>(c, L2, U, w.b0);
  // G2[l2][a_d][b_u][r1][m] = sum_{l1,u1} G1[l1][l2][a_d][u1][b_u] T1[l1][r1][u1][m]
  c = ctr_init();
  c.e[0] = Dl; c.e[1] = k.ad; c.e[2] = k.bu; c.e[3] = Dr; c.e[4] = D;
  c.sa[0] = k.ad * k.pu * k.bu; c.sa[1] = k.pu * k.bu; c.sa[2] = 1;
  c.sb[3] = D2; c.sb[4] = 1;
  c.sc[0] = k.ad * k.bu * Dr * D; c.sc[1] = k.bu * Dr * D; c.sc[2] = Dr * D; c.sc[3] = D; c.sc[4] = 1;
  c.k1 = Dl; c.ka1 = Dl * k.ad * k.pu * k.bu; c.kb1 = D3;
  c.k2 = k.pu; c.ka2 = k.bu; c.kb2 = D;
  contract<R>(c, w.b0, T1, w.b1);
  // G3[a_d][b_u][r1][r2][d2] = sum_{l2,m} G2[l2][a_d][b_u][r1][m] T2[l2][r2][m][d2]
  c = ctr_init();
  c.e[0] = k.ad; c.e[1] = k.bu; c.e[2] = Dr; c.e[3] = Dr; c.e[4] = k.pd;
  c.sa[0] = k.bu * Dr * D; c.sa[1] = Dr * D; c.sa[2] = D;
  c.sb[3] = D2; c.sb[4] = 1;
  c.sc[0] = k.bu * Dr * Dr * k.pd; c.sc[1] = Dr * Dr * k.pd; c.sc[2] = Dr * k.pd; c.sc[3] = k.pd; c.sc[4] = 1;
  c.k1 = Dl; c.ka1 = k.ad * k.bu * Dr * D; c.kb1 = D3;
  c.k2 = D; c.ka2 = 1; c.kb2 = D;
  contract<R>(c, w.b1, T2, w.b0);
  // L2new[b_u][r1][r2][b_d] = sum_{a_d,d2} G3[a_d][b_u][r1][r2][d2] Dn[a_d][d2][b_d]
  c = ctr_init();
  c.e[0] = k.bu; c.e[1] = Dr * Dr; c.e[2] = k.bd;
  c.sa[0] = Dr * Dr * k.pd; c.sa[1] = k.pd;
  c.sb[2] = 1;
  c.sc[0] = Dr * Dr * k.bd; c.sc[1] = k.bd; c.sc[2] = 1;
  c.k1 = k.ad; c.ka1 = k.bu * Dr * Dr * k.pd; c.kb1 = k.pd * k.bd;
  c.k2 = k.pd; c.ka2 = 1; c.kb2 = k.bd;
  contract<R>(c, w.b0, Dn, Lout);
}

template <class R>
__device__ void strip2_right_step(const PepsPlan& P, const Col1& k, const R* R2n,
                                  const R* U, const R* T1, const R* T2,
                                  const R* Dn, R* Rout, const Work<R>& w) {
  const int D = P.D, D2 = P.D2, D3 = P.D3;
  const int Dl = k.Dl, Dr = k.Dr;
  // H1[b_u][r1][r2][a_d][d2] = sum_{b_d} R2n[b_u][r1][r2][b_d] Dn[a_d][d2][b_d]
  Ctr c = ctr_init();
  c.e[0] = k.bu; c.e[1] = Dr * Dr; c.e[2] = k.ad; c.e[3] = k.pd;
  c.sa[0] = Dr * Dr * k.bd; c.sa[1] = k.bd;
  c.sb[2] = k.pd * k.bd; c.sb[3] = k.bd;
  c.sc[0] = Dr * Dr * k.ad * k.pd; c.sc[1] = k.ad * k.pd; c.sc[2] = k.pd; c.sc[3] = 1;
  c.k1 = k.bd; c.ka1 = 1; c.kb1 = 1;
  contract<R>(c, R2n, Dn, w.b0);
  // H2[b_u][r1][m][l2][a_d] = sum_{r2,d2} H1[b_u][r1][r2][a_d][d2] T2[l2][r2][m][d2]
  c = ctr_init();
  c.e[0] = k.bu; c.e[1] = Dr; c.e[2] = D; c.e[3] = Dl; c.e[4] = k.ad;
  c.sa[0] = Dr * Dr * k.ad * k.pd; c.sa[1] = Dr * k.ad * k.pd; c.sa[4] = k.pd;
  c.sb[2] = D; c.sb[3] = D3;
  c.sc[0] = Dr * D * Dl * k.ad; c.sc[1] = D * Dl * k.ad; c.sc[2] = Dl * k.ad; c.sc[3] = k.ad; c.sc[4] = 1;
  c.k1 = Dr; c.ka1 = k.ad * k.pd; c.kb1 = D2;
  c.k2 = k.pd; c.ka2 = 1; c.kb2 = 1;
  contract<R>(c, w.b0, T2, w.b1);
  // H3[b_u][u1][l1][l2][a_d] = sum_{r1,m} H2[b_u][r1][m][l2][a_d] T1[l1][r1][u1][m]
  c = ctr_init();
  c.e[0] = k.bu; c.e[1] = k.pu; c.e[2] = Dl; c.e[3] = Dl * k.ad;
  c.sa[0] = Dr * D * Dl * k.ad; c.sa[3] = 1;
  c.sb[1] = D; c.sb[2] = D3;
  c.sc[0] = k.pu * Dl * Dl * k.ad; c.sc[1] = Dl * Dl * k.ad; c.sc[2] = Dl * k.ad; c.sc[3] = 1;
  c.k1 = Dr; c.ka1 = D * Dl * k.ad; c.kb1 = D2;
  c.k2 = D; c.ka2 = Dl * k.ad; c.kb2 = 1;
  contract<R>(c, w.b1, T1, w.b0);
  // R2new[a_u][(l1 l2 a_d)] = sum_{u1,b_u} U[a_u][u1][b_u] H3[b_u][u1][(l1 l2 a_d)]
  const int x = Dl * Dl * k.ad;
  c = ctr_init();
  c.e[0] = k.au; c.e[1] = x;
  c.sa[0] = k.pu * k.bu; c.sb[1] = 1;
  c.sc[0] = x; c.sc[1] = 1;
  c.k1 = k.pu; c.ka1 = k.bu; c.kb1 = x;
  c.k2 = k.bu; c.ka2 = 1; c.kb2 = k.pu * x;
  contract<R>(c, U, w.b0, Rout);
}
