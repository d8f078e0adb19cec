// peps_core.cuh -- thread-block building blocks of the per-sample PEPS
// contraction (PEPS++, arXiv:1806.03761): strided tensor contractions,
// Householder QR, one-sided Jacobi SVD, boundary-MPS absorption with
// truncation, and the one- and two-row strips.
//
// Every routine is executed by all threads of one thread block on the
// workspace of one sample; it ends with __syncthreads() so its result can be
// read by every thread.  Scalars are of the form's type R (double or ff).
#pragma once
#include "peps_arith.cuh"
#include "peps_plan.h"

#define PEPS_NT 256          // threads per block
#define PEPS_JACOBI_MAXSWEEP 40

// ---------------------------------------------------------------------------
// Block-wide reductions through shared memory.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_max(double v, double* red) {
  const int t = threadIdx.x, nt = blockDim.x;
  red[t] = v;
  __syncthreads();
  for (int s = nt >> 1; s > 0; s >>= 1) {
    if (t < s) red[t] = fmax(red[t], red[t + s]);
    __syncthreads();
  }
  double r = red[0];
  __syncthreads();
  return r;
}

template <class R>
__device__ __forceinline__ R block_sum(R v, R* red) {
  const int t = threadIdx.x, nt = blockDim.x;
  red[t] = v;
  __syncthreads();
  for (int s = nt >> 1; s > 0; s >>= 1) {
    if (t < s) red[t] = red[t] + red[t + s];
    __syncthreads();
  }
  R r = red[0];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// Strided contraction C[o] = sum_{k1,k2} A[a(o)+k1*ka1+k2*ka2] B[b(o)+...].
// The output index o runs over five digits (e[4] fastest); each digit has
// a stride in A, B and C (0 where the operand does not carry it).
// ---------------------------------------------------------------------------
struct Ctr {
  int e[5];
  int sa[5], sb[5], sc[5];
  int k1, k2, ka1, ka2, kb1, kb2;
};

__device__ __forceinline__ Ctr ctr_init() {
  Ctr d;
  for (int i = 0; i < 5; ++i) { d.e[i] = 1; d.sa[i] = d.sb[i] = d.sc[i] = 0; }
  d.k1 = d.k2 = 1;
  d.ka1 = d.ka2 = d.kb1 = d.kb2 = 0;
  return d;
}

template <class R>
__device__ void contract(const Ctr& d, const R* __restrict__ A,
                         const R* __restrict__ B, R* __restrict__ C) {
  typedef Arith<R> M;
  const int tot = d.e[0] * d.e[1] * d.e[2] * d.e[3] * d.e[4];
  for (int o = threadIdx.x; o < tot; o += blockDim.x) {
    int t = o;
    int i4 = t % d.e[4]; t /= d.e[4];
    int i3 = t % d.e[3]; t /= d.e[3];
    int i2 = t % d.e[2]; t /= d.e[2];
    int i1 = t % d.e[1];
    int i0 = t / d.e[1];
    int oa = i0 * d.sa[0] + i1 * d.sa[1] + i2 * d.sa[2] + i3 * d.sa[3] + i4 * d.sa[4];
    int ob = i0 * d.sb[0] + i1 * d.sb[1] + i2 * d.sb[2] + i3 * d.sb[3] + i4 * d.sb[4];
    int oc = i0 * d.sc[0] + i1 * d.sc[1] + i2 * d.sc[2] + i3 * d.sc[3] + i4 * d.sc[4];
    typename M::acc_t acc;
    M::acc_init(acc);
    for (int k1 = 0; k1 < d.k1; ++k1) {
      const R* pa = A + oa + k1 * d.ka1;
      const R* pb = B + ob + k1 * d.kb1;
      for (int k2 = 0; k2 < d.k2; ++k2) M::mac(acc, pa[k2 * d.ka2], pb[k2 * d.kb2]);
    }
    C[oc] = M::acc_get(acc);
  }
  __syncthreads();
}

// Scale x[0..n) by a power of two so that max|x| lies in [1/2, 1); returns
// the natural log of the factor removed (0 for an all-zero x).
template <class R>
__device__ double normalize_pow2(R* x, int n, double* red) {
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(Arith<R>::to(x[i])));
  m = block_max(m, red);
  if (!(m > 0.0) || !isfinite(m)) return 0.0;
  int e;
  frexp(m, &e);  // m = f 2^e, f in [1/2, 1)
  double s = ldexp(1.0, -e);
  R rs = Arith<R>::from(s);
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = x[i] * rs;
  __syncthreads();
  return (double)e * 0.69314718055994530942;
}

// ---------------------------------------------------------------------------
// Householder QR, R factor only (LAPACK-style reflectors H = I - tau v v^T,
// v_k = 1).  X is m x n row-major (ld n), overwritten; R = the first
// min(m,n) rows of the upper triangle are written to Rout (ld n), zeros
// below the diagonal.  wbuf: n scalars of scratch (shared or global).
// ---------------------------------------------------------------------------
template <class R>
__device__ void householder_r(R* X, int m, int n, R* Rout, R* wbuf, R* redR,
                              double* sh) {
  typedef Arith<R> M;
  const int t = threadIdx.x, nt = blockDim.x;
  const int kmax = m < n ? m : n;
  for (int k = 0; k < kmax; ++k) {
    // squared norm of the column below the diagonal
    typename M::acc_t a;
    M::acc_init(a);
    for (int i = k + 1 + t; i < m; i += nt) M::mac(a, X[i * n + k], X[i * n + k]);
    R xn2 = block_sum<R>(M::acc_get(a), redR);
    if (t == 0) {
      R alpha = X[k * n + k];
      double x2 = M::to(xn2);
      if (!(x2 > 0.0)) {
        sh[0] = 0.0;  // tau = 0: H = I
      } else {
        R nrm = M::sqrt_(alpha * alpha + xn2);
        R beta = M::to(alpha) >= 0.0 ? -nrm : nrm;
        R tau = (beta - alpha) / beta;
        R scl = M::one() / (alpha - beta);
        X[k * n + k] = beta;
        sh[0] = 1.0;
        redR[0] = tau;
        redR[1] = scl;
      }
    }
    __syncthreads();
    if (sh[0] != 0.0) {
      R tau = redR[0], scl = redR[1];
      for (int i = k + 1 + t; i < m; i += nt) X[i * n + k] = X[i * n + k] * scl;
      __syncthreads();
      // w_c = tau * (X[k][c] + sum_{i>k} v_i X[i][c]),  c > k
      for (int c = k + 1 + t; c < n; c += nt) {
        typename M::acc_t s;
        M::acc_init(s);
        M::mac(s, M::one(), X[k * n + c]);
        for (int i = k + 1; i < m; ++i) M::mac(s, X[i * n + k], X[i * n + c]);
        wbuf[c] = tau * M::acc_get(s);
      }
      __syncthreads();
      const int w = n - k - 1;
      const int tot = (m - k) * w;
      for (int o = t; o < tot; o += nt) {
        int i = k + o / w, c = k + 1 + o % w;
        R v = (i == k) ? M::one() : X[i * n + k];
        X[i * n + c] = X[i * n + c] - v * wbuf[c];
      }
    }
    __syncthreads();
  }
  for (int o = t; o < kmax * n; o += nt) {
    int i = o / n, c = o % n;
    Rout[o] = (c >= i) ? X[i * n + c] : M::zero();
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// One-sided (Hestenes) Jacobi on the ROWS of X (rr x n, rr <= n, ld n):
// rotations of row pairs until all rows are mutually orthogonal; the rows
// are then sigma_i v_i^T with v_i the right singular vectors of X.  Writes
// the kk rows of largest norm, normalised, to VT (kk x n) in decreasing
// order (zero rows for zero singular values).  Pairs are visited in the
// round-robin (circle) order, rr/2 disjoint pairs at a time.  Rows whose
// squared norm is below eps^2 times the largest are left alone (their
// singular values are below rounding level and they take no part in the
// kept subspace beyond it).
// alpha: rr doubles of scratch.  Returns the number of sweeps used.
// ---------------------------------------------------------------------------
template <class R>
__device__ int jacobi_rows(R* X, int rr, int n, int kk, R* VT, double* alpha,
                           R* part, double* rot, int* shi, double* red,
                           int* flags) {
  typedef Arith<R> M;
  const int t = threadIdx.x, nt = blockDim.x;
  const int rp = rr + (rr & 1);
  const int npair = rp / 2;
  const double tol = (double)n * M::eps();
  // exact squared row norms
  for (int p = 0; p < rr; ++p) {
    typename M::acc_t a;
    M::acc_init(a);
    for (int e = t; e < n; e += nt) M::mac(a, X[p * n + e], X[p * n + e]);
    R s = block_sum<R>(M::acc_get(a), part);
    if (t == 0) alpha[p] = M::to(s);
  }
  __syncthreads();
  int sweep = 0;
  for (; sweep < PEPS_JACOBI_MAXSWEEP && rr > 1; ++sweep) {
    double amax = 0.0;
    for (int p = t; p < rr; p += nt) amax = fmax(amax, alpha[p]);
    const double thr = block_max(amax, red) * M::eps() * M::eps();
    if (t == 0) shi[0] = 0;
    __syncthreads();
    for (int rd = 0; rd < rp - 1; ++rd) {
      // team of tm threads per pair computes gamma = x_p . x_q
      int tm = nt / npair;
      if (tm < 1) tm = 1;
      for (int base = 0; base < npair; base += nt / tm) {
        int pr = base + t / tm, mb = t % tm;
        typename M::acc_t a;
        M::acc_init(a);
        if (pr < npair && t / tm < nt / tm) {
          int pp = (pr == 0) ? 0 : ((pr - 1 + rd) % (rp - 1)) + 1;
          int qpos = rp - 1 - pr;
          int qq = (qpos == 0) ? 0 : ((qpos - 1 + rd) % (rp - 1)) + 1;
          if (pp < rr && qq < rr)
            for (int e = mb; e < n; e += tm) M::mac(a, X[pp * n + e], X[qq * n + e]);
        }
        if (t / tm < nt / tm) part[t] = M::acc_get(a);
        __syncthreads();
        if (t < nt / tm && base + t < npair) {
          R g = M::zero();
          for (int u = 0; u < tm; ++u) g = g + part[t * tm + u];
          int pr2 = base + t;
          int pp = (pr2 == 0) ? 0 : ((pr2 - 1 + rd) % (rp - 1)) + 1;
          int qpos = rp - 1 - pr2;
          int qq = (qpos == 0) ? 0 : ((qpos - 1 + rd) % (rp - 1)) + 1;
          double c = 1.0, s = 0.0;
          if (pp < rr && qq < rr) {
            double gam = M::to(g), ap = alpha[pp], aq = alpha[qq];
            if (ap > thr && aq > thr && fabs(gam) > tol * sqrt(ap * aq)) {
              double zeta = (aq - ap) / (2.0 * gam);
              double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
              c = 1.0 / sqrt(1.0 + tt * tt);
              s = c * tt;
              alpha[pp] = ap - tt * gam;
              alpha[qq] = aq + tt * gam;
              shi[0] = 1;
            }
          }
          rot[2 * pr2] = c;
          rot[2 * pr2 + 1] = s;
        }
        __syncthreads();
      }
      // apply the rotations: x_p <- c x_p - s x_q, x_q <- s x_p + c x_q
      const int tot = npair * n;
      for (int o = t; o < tot; o += nt) {
        int pr = o / n, e = o % n;
        double s = rot[2 * pr + 1];
        if (s == 0.0) continue;
        int pp = (pr == 0) ? 0 : ((pr - 1 + rd) % (rp - 1)) + 1;
        int qpos = rp - 1 - pr;
        int qq = (qpos == 0) ? 0 : ((qpos - 1 + rd) % (rp - 1)) + 1;
        R c = M::from(rot[2 * pr]), sr = M::from(s);
        R xp = X[pp * n + e], xq = X[qq * n + e];
        X[pp * n + e] = c * xp - sr * xq;
        X[qq * n + e] = sr * xp + c * xq;
      }
      __syncthreads();
    }
    int any = shi[0];
    // refresh the norms exactly
    for (int p = 0; p < rr; ++p) {
      typename M::acc_t a;
      M::acc_init(a);
      for (int e = t; e < n; e += nt) M::mac(a, X[p * n + e], X[p * n + e]);
      R s = block_sum<R>(M::acc_get(a), part);
      if (t == 0) alpha[p] = M::to(s);
    }
    __syncthreads();
    if (!any) break;
  }
  if (sweep >= PEPS_JACOBI_MAXSWEEP && t == 0) atomicOr(flags, 4);
  // rank rows by norm (ties by index) and write the kk largest, normalised
  for (int p = t; p < rr; p += nt) {
    int rank = 0;
    for (int q = 0; q < rr; ++q)
      rank += (alpha[q] > alpha[p]) || (alpha[q] == alpha[p] && q < p);
    shi[1 + p] = rank;
  }
  __syncthreads();
  for (int o = t; o < kk * n; o += nt) VT[o] = M::zero();
  __syncthreads();
  for (int o = t; o < rr * n; o += nt) {
    int p = o / n, e = o % n;
    int rank = shi[1 + p];
    if (rank < kk && alpha[p] > 0.0)
      VT[rank * n + e] = X[p * n + e] * M::from(1.0 / sqrt(alpha[p]));
  }
  __syncthreads();
  return sweep;
}
