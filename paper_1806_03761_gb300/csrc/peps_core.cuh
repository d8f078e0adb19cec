// peps_core.cuh -- thread-block building blocks of the per-sample PEPS
// contraction (PEPS++, arXiv:1806.03761): reductions, strided tensor
// contractions, Householder QR and the truncated SVD of the bond matrices.
//
// Every routine is executed by all threads of one thread block on the
// workspace of one sample; it ends with __syncthreads() so its result can be
// read by every thread.  Scalars are of the form's type R (double or ff).
#pragma once
#include "peps_arith.cuh"
#include "peps_plan.h"
#include "peps_trace.cuh"

#ifndef PEPS_NT
#define PEPS_NT 256          // threads per block
#endif
#ifndef PEPS_WARP
#define PEPS_WARP 32         // lanes per warp
#endif

// ---------------------------------------------------------------------------
// Warp- and block-wide reductions (warp shuffles, one shared slot per warp).
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ R warp_sum(R v) {
  for (int o = PEPS_WARP / 2; o > 0; o >>= 1) v = v + shfl_xor_r(v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = PEPS_WARP / 2; o > 0; o >>= 1) v = fmax(v, shfl_xor_r(v, o));
  return v;
}

__device__ __forceinline__ double block_max(double v, double* red) {
  const int t = threadIdx.x, lane = t % PEPS_WARP, wid = t / PEPS_WARP,
            nw = (blockDim.x + PEPS_WARP - 1) / PEPS_WARP;
  v = warp_max(v);
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double x = lane < nw ? red[lane] : 0.0;
    x = warp_max(x);
    if (lane == 0) red[PEPS_NT / PEPS_WARP] = x;
  }
  __syncthreads();
  double r = red[PEPS_NT / PEPS_WARP];
  __syncthreads();
  return r;
}

template <class R>
__device__ __forceinline__ R block_sum(R v, R* red) {
  const int t = threadIdx.x, lane = t % PEPS_WARP, wid = t / PEPS_WARP,
            nw = (blockDim.x + PEPS_WARP - 1) / PEPS_WARP;
  v = warp_sum<R>(v);
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    R x = lane < nw ? red[lane] : Arith<R>::zero();
    x = warp_sum<R>(x);
    if (lane == 0) red[PEPS_NT / PEPS_WARP] = x;
  }
  __syncthreads();
  R r = red[PEPS_NT / PEPS_WARP];
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

// The operands are scratch rewritten within the same kernel, so they are
// read through the coherent path (no __restrict__ / read-only cache).
//
// Register blocking: when the output has a digit carried only by A (dA) and
// one carried only by B (dB), each thread computes a BA x BB block of outputs
// over those digits, so that every loaded element of A feeds BB and every
// loaded element of B BA multiply-adds (the summation order of each output
// is unchanged).  Otherwise each thread computes two
// outputs adjacent in the fastest digit (shared loads where an operand does
// not carry it).
// Outputs per thread along the A-only digit: PEPS_BA_FF (default 4) for the
// FP32-word forms, PEPS_BA_F64 (default 2) for FP64, whose accumulators take
// twice the registers (measured slower at 4); the autotuner varies them.
#ifndef PEPS_BA_FF
#define PEPS_BA_FF 4
#endif
#ifndef PEPS_BA_F64
#define PEPS_BA_F64 2
#endif
// Outputs per thread along the B-only digit: PEPS_BB_FF (default 2) for the
// FP32-word forms, 2 for FP64.
#ifndef PEPS_BB_FF
#define PEPS_BB_FF 2
#endif
// PEPS_CTR_PIPE=1 (default): the operands of reduction step t + 1 are loaded
// before the multiply-adds of step t, so that their latency overlaps the
// arithmetic (the same products summed in the same order: bit-identical to
// PEPS_CTR_PIPE=0).
#ifndef PEPS_CTR_PIPE
#define PEPS_CTR_PIPE 1
#endif
template <class R> struct ContractBlock {
  static constexpr int BA = PEPS_BA_FF, BB = PEPS_BB_FF;
};
template <> struct ContractBlock<double> { static constexpr int BA = PEPS_BA_F64, BB = 2; };

template <class R>
__device__ void contract(const Ctr& d, const R* A, const R* B, R* C) {
  typedef Arith<R> M;
  int dA = -1, dB = -1;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    if (d.e[i] > 1 && d.sa[i] != 0 && d.sb[i] == 0) dA = i;
    if (d.e[i] > 1 && d.sb[i] != 0 && d.sa[i] == 0) dB = i;
  }
  if (dA >= 0 && dB >= 0) {
    // BA x BB outputs per thread over (dA, dB)
    constexpr int BA = ContractBlock<R>::BA, BB = ContractBlock<R>::BB;
    int eb[5];
    int tot = 1;
    int sA = 0, sB = 0, cA = 0, cB = 0, nA = 1, nB = 1;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      eb[i] = (i == dA) ? (d.e[i] + BA - 1) / BA : (i == dB) ? (d.e[i] + BB - 1) / BB : d.e[i];
      tot *= eb[i];
      if (i == dA) { sA = d.sa[i]; cA = d.sc[i]; nA = d.e[i]; }
      if (i == dB) { sB = d.sb[i]; cB = d.sc[i]; nB = d.e[i]; }
    }
    for (int o = threadIdx.x; o < tot; o += blockDim.x) {
      int t = o;
      int oa = 0, ob = 0, oc = 0, xA = 0, xB = 0;
#pragma unroll
      for (int i = 4; i >= 0; --i) {
        int q = t % eb[i];
        t /= eb[i];
        if (i == dA) { q *= BA; xA = q; }
        if (i == dB) { q *= BB; xB = q; }
        oa += q * d.sa[i];
        ob += q * d.sb[i];
        oc += q * d.sc[i];
      }
      // rows beyond the extent repeat the last valid one (computed, not stored)
      int da[BA], db[BB];
#pragma unroll
      for (int x = 0; x < BA; ++x) da[x] = (xA + x < nA ? x : nA - 1 - xA) * sA;
#pragma unroll
      for (int y = 0; y < BB; ++y) db[y] = (xB + y < nB ? y : nB - 1 - xB) * sB;
      typename M::acc_t c[BA][BB];
#pragma unroll
      for (int x = 0; x < BA; ++x)
#pragma unroll
        for (int y = 0; y < BB; ++y) M::acc_init(c[x][y]);
#if PEPS_CTR_PIPE
      // reduction steps t = k1 * k2-extent + k2 in order; offsets of step t
      // in fa/fb, the next step's operands loaded ahead (the last step
      // reloads its own, in range)
      const int K2 = d.k2, KT = d.k1 * d.k2;
      if (KT > 0) {
        int fa = oa, fb = ob, k2 = 0;
        R av[BA], bv[BB];
#pragma unroll
        for (int x = 0; x < BA; ++x) av[x] = A[fa + da[x]];
#pragma unroll
        for (int y = 0; y < BB; ++y) bv[y] = B[fb + db[y]];
        for (int t = 0; t < KT; ++t) {
          int ga = fa + d.ka2, gb = fb + d.kb2;
          if (++k2 == K2) {
            k2 = 0;
            ga += d.ka1 - K2 * d.ka2;
            gb += d.kb1 - K2 * d.kb2;
          }
          if (t + 1 == KT) { ga = fa; gb = fb; }
          R an[BA], bn[BB];
#pragma unroll
          for (int x = 0; x < BA; ++x) an[x] = A[ga + da[x]];
#pragma unroll
          for (int y = 0; y < BB; ++y) bn[y] = B[gb + db[y]];
#pragma unroll
          for (int x = 0; x < BA; ++x)
#pragma unroll
            for (int y = 0; y < BB; ++y) M::mac(c[x][y], av[x], bv[y]);
#pragma unroll
          for (int x = 0; x < BA; ++x) av[x] = an[x];
#pragma unroll
          for (int y = 0; y < BB; ++y) bv[y] = bn[y];
          fa = ga;
          fb = gb;
        }
      }
#else
      for (int k1 = 0; k1 < d.k1; ++k1) {
        const R* pa = A + oa + k1 * d.ka1;
        const R* pb = B + ob + k1 * d.kb1;
        for (int k2 = 0; k2 < d.k2; ++k2) {
          R av[BA], bv[BB];
#pragma unroll
          for (int x = 0; x < BA; ++x) av[x] = pa[k2 * d.ka2 + da[x]];
#pragma unroll
          for (int y = 0; y < BB; ++y) bv[y] = pb[k2 * d.kb2 + db[y]];
#pragma unroll
          for (int x = 0; x < BA; ++x)
#pragma unroll
            for (int y = 0; y < BB; ++y) M::mac(c[x][y], av[x], bv[y]);
        }
      }
#endif
#pragma unroll
      for (int x = 0; x < BA; ++x)
#pragma unroll
        for (int y = 0; y < BB; ++y)
          if (xA + x < nA && xB + y < nB) C[oc + x * cA + y * cB] = M::acc_get(c[x][y]);
    }
    __syncthreads();
    return;
  }
  const int e4 = d.e[4];
  const int h4 = (e4 + 1) >> 1;
  const int tot = d.e[0] * d.e[1] * d.e[2] * d.e[3] * h4;
  const int sa4 = d.sa[4], sb4 = d.sb[4], sc4 = d.sc[4];
  for (int o = threadIdx.x; o < tot; o += blockDim.x) {
    int t = o;
    const int i4 = 2 * (t % h4); t /= h4;
    const int i3 = t % d.e[3]; t /= d.e[3];
    const int i2 = t % d.e[2]; t /= d.e[2];
    const int i1 = t % d.e[1];
    const int i0 = t / d.e[1];
    const bool two = i4 + 1 < e4;
    const int oa = i0 * d.sa[0] + i1 * d.sa[1] + i2 * d.sa[2] + i3 * d.sa[3] + i4 * sa4;
    const int ob = i0 * d.sb[0] + i1 * d.sb[1] + i2 * d.sb[2] + i3 * d.sb[3] + i4 * sb4;
    const int oc = i0 * d.sc[0] + i1 * d.sc[1] + i2 * d.sc[2] + i3 * d.sc[3] + i4 * sc4;
    const int da = two ? sa4 : 0, db = two ? sb4 : 0;
    typename M::acc_t acc0, acc1;
    M::acc_init(acc0);
    M::acc_init(acc1);
#if PEPS_CTR_PIPE
    const int K2 = d.k2, KT = d.k1 * d.k2;
    if (KT > 0) {
      int fa = oa, fb = ob, k2 = 0;
      R a0 = A[fa], b0 = B[fb];
      R a1 = da ? A[fa + da] : a0;
      R b1 = db ? B[fb + db] : b0;
      for (int t = 0; t < KT; ++t) {
        int ga = fa + d.ka2, gb = fb + d.kb2;
        if (++k2 == K2) {
          k2 = 0;
          ga += d.ka1 - K2 * d.ka2;
          gb += d.kb1 - K2 * d.kb2;
        }
        if (t + 1 == KT) { ga = fa; gb = fb; }
        const R na0 = A[ga], nb0 = B[gb];
        const R na1 = da ? A[ga + da] : na0;
        const R nb1 = db ? B[gb + db] : nb0;
        M::mac(acc0, a0, b0);
        M::mac(acc1, a1, b1);
        a0 = na0; b0 = nb0; a1 = na1; b1 = nb1;
        fa = ga;
        fb = gb;
      }
    }
#else
    for (int k1 = 0; k1 < d.k1; ++k1) {
      const R* pa = A + oa + k1 * d.ka1;
      const R* pb = B + ob + k1 * d.kb1;
      for (int k2 = 0; k2 < d.k2; ++k2) {
        const R a0 = pa[k2 * d.ka2], b0 = pb[k2 * d.kb2];
        const R a1 = da ? pa[k2 * d.ka2 + da] : a0;
        const R b1 = db ? pb[k2 * d.kb2 + db] : b0;
        M::mac(acc0, a0, b0);
        M::mac(acc1, a1, b1);
      }
    }
#endif
    C[oc] = M::acc_get(acc0);
    if (two) C[oc + sc4] = M::acc_get(acc1);
  }
  __syncthreads();
}

// Scale x[0..n) by a power of two so that max|x| lies in [1/2, 1); returns
// the natural log of the factor removed (0 for an all-zero x).
template <class R>
__device__ double normalize_pow2(R* x, int n, double* red) {
  // the leading part decides the power of two (no FP64 work per element)
  decltype(Arith<R>::hi(R())) mh = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) mh = fmax(mh, fabs(Arith<R>::hi(x[i])));
  double m = block_max((double)mh, red);
  if (!(m > 0.0) || !isfinite(m)) return 0.0;
  int e;
  frexp(m, &e);  // m = f 2^e, f in [1/2, 1)
  double s = ldexp(1.0, -e);
  R rs = Arith<R>::from(s);
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = x[i] * rs;
  __syncthreads();
  return (double)e * 0.69314718055994530942;
}

// Apply H = I - tau w w^T (w = e_k + the stored tail xk[k+1..m-1]) to the
// columns c0..c1-1 of the column-major X (ld m), two columns per warp.
template <class R>
__device__ __forceinline__ void reflect_columns(R* X, int m, int k, int c0, int c1,
                                                const R* xk, R tau) {
  typedef Arith<R> M;
  const int lane = threadIdx.x % PEPS_WARP, wid = threadIdx.x / PEPS_WARP;
  const int nw = (blockDim.x + PEPS_WARP - 1) / PEPS_WARP;
  for (int c = c0 + 2 * wid; c < c1; c += 2 * nw) {
    const bool two = c + 1 < c1;
    R* xa = X + (int64_t)c * m;
    R* xb = two ? xa + m : xa;
    typename M::acc_t a, b;
    M::acc_init(a);
    M::acc_init(b);
    if (lane == 0) {
      M::mac(a, M::one(), xa[k]);
      M::mac(b, M::one(), xb[k]);
    }
    for (int i = k + 1 + lane; i < m; i += PEPS_WARP) {
      const R v = xk[i];
      M::mac(a, v, xa[i]);
      M::mac(b, v, xb[i]);
    }
    const R wa = tau * warp_sum<R>(M::acc_get(a));
    const R wb = tau * warp_sum<R>(M::acc_get(b));
    if (lane == 0) {
      xa[k] = xa[k] - wa;
      if (two) xb[k] = xb[k] - wb;
    }
    for (int i = k + 1 + lane; i < m; i += PEPS_WARP) {
      const R v = xk[i];
      xa[i] = Arith<R>::sub_mul(xa[i], v, wa);
      if (two) xb[i] = Arith<R>::sub_mul(xb[i], v, wb);
    }
  }
}

// ---------------------------------------------------------------------------
// Householder QR, R factor only (LAPACK-style reflectors H = I - tau v v^T,
// v_k = 1).  X is m x n COLUMN-major (X[c*m + i]), overwritten: R on and
// above the diagonal, the reflector tails below.  The first min(m,n) rows of
// R are written row-major to Rout (ld n), zeros below the diagonal.
//
// Unblocked form: warp 0 forms each reflector, which is then applied to the
// columns on its right, two columns per warp (every trailing column is read
// twice and written once per reflector).  sh: >= 2 scalars of shared memory.
// ---------------------------------------------------------------------------
template <class R>
__device__ void householder_r_unblocked(R* X, int m, int n, R* Rout, R* sh) {
  typedef Arith<R> M;
  const int t = threadIdx.x, lane = t % PEPS_WARP, wid = t / PEPS_WARP;
  const int kmax = m < n ? m : n;
  for (int k = 0; k < kmax; ++k) {
    R* xk = X + (int64_t)k * m;
    if (wid == 0) {
      typename M::acc_t a;
      M::acc_init(a);
      for (int i = k + 1 + lane; i < m; i += PEPS_WARP) M::mac(a, xk[i], xk[i]);
      R xn2 = warp_sum<R>(M::acc_get(a));
      if (lane == 0) {
        R alpha = xk[k];
        if (!(M::hi(xn2) > 0)) {
          sh[0] = M::zero();  // tau = 0: H = I
        } else {
          R nrm = M::sqrt_(alpha * alpha + xn2);
          R beta = M::hi(alpha) >= 0 ? -nrm : nrm;
          sh[0] = (beta - alpha) / beta;
          sh[1] = M::one() / (alpha - beta);
          xk[k] = beta;
        }
      }
      __syncwarp();
      R tau = sh[0], scl = sh[1];
      if (M::hi(tau) != 0)
        for (int i = k + 1 + lane; i < m; i += PEPS_WARP) xk[i] = xk[i] * scl;
    }
    __syncthreads();
    const R tau = sh[0];
    if (M::hi(tau) != 0) reflect_columns<R>(X, m, k, k + 1, n, xk, tau);
    __syncthreads();
  }
  for (int o = t; o < kmax * n; o += blockDim.x) {
    int i = o / n, c = o % n;
    Rout[o] = (c >= i) ? X[(int64_t)c * m + i] : M::zero();
  }
  __syncthreads();
}

// Panel width and row capacity of the blocked form.
#ifndef PEPS_QR_NB
#define PEPS_QR_NB 4
#endif
// Autotuned code paths (0 / 1): prefetch a warp's next trailing column of the
// blocked QR into L1; form A'^T v of the bidiagonalisation with one thread
// per column instead of one warp per column.
#ifndef PEPS_QR_PREFETCH
#define PEPS_QR_PREFETCH 0
#endif
#ifndef PEPS_BIDIAG_TPC
#define PEPS_BIDIAG_TPC 0
#endif
// PEPS_BIDIAG_FUSE=1: the bidiagonalisation leaves out two of its barriers
// per step where each thread reads only what it wrote itself (the column
// corrections of Y before the row of the current matrix; the row corrections
// of W before the next step's column); the same operations in the same
// order (bit-identical to PEPS_BIDIAG_FUSE=0).
#ifndef PEPS_BIDIAG_FUSE
#define PEPS_BIDIAG_FUSE 0
#endif
// Tall panels (more than PEPS_QR_ROWS rows, up to 2048): the trailing column
// in the registers of two warps (qr_trailing_pair) instead of two streaming
// passes of one warp.
#ifndef PEPS_QR_TALL_PAIR
#define PEPS_QR_TALL_PAIR 0
#endif
#define PEPS_QR_ROWS 896

// The factorisations' two inline-PTX statements, as macros that a host build
// of the kernels may define otherwise: an L1 prefetch of a global address,
// and the named barrier of warp pair p (barrier 1 + p, 64 threads).
#ifndef PEPS_PREFETCH_L1
#define PEPS_PREFETCH_L1(ptr) asm volatile("prefetch.global.L1 [%0];" ::"l"(ptr))
#endif
#ifndef PEPS_PAIR_SYNC
#define PEPS_PAIR_SYNC(p) asm volatile("bar.sync %0, 64;" ::"r"(1 + (p)) : "memory")
#endif

// PEPS_QR_ACC=1 (default): the trailing update's warp reductions merge the
// lanes' compensated accumulators directly, and x - V w' is one compensated
// accumulation per element (float-float: fewer FP32 operations at the same
// error bound, a few 2^-48 of |x| + |V w'|; FP64 and FP32: bit-identical to
// PEPS_QR_ACC=0).
#ifndef PEPS_QR_ACC
#define PEPS_QR_ACC 1
#endif

// Apply the panel's reflectors (explicit vectors v_s, zero above row s and
// one at row s, in vsh with stride PEPS_QR_ROWS) to the trailing columns
// c0..n-1 of X, rows k0..k0+mr-1, in the compact WY form
// H_{nb-1} .. H_0 x = x - V T^T V^T x  (T: nb x nb upper triangular, in tt
// with tt[r * PEPS_QR_NB + s] = T[r][s]).  One warp per column: the column is
// held in registers (CAP rows per lane), its nb dot products with the
// reflectors are formed together, and it is written back once.
template <class R, int CAP>
__device__ __forceinline__ void qr_trailing(R* X, int m, int n, int k0, int mr, int c0, int nb,
                                            const R* vsh, const R* tt) {
  typedef Arith<R> M;
  const int lane = threadIdx.x % PEPS_WARP, wid = threadIdx.x / PEPS_WARP;
  const int nw = (blockDim.x + PEPS_WARP - 1) / PEPS_WARP;
  for (int c = c0 + wid; c < n; c += nw) {
    R* x = X + (int64_t)c * m + k0;
    R xr[CAP];
#pragma unroll
    for (int q = 0; q < CAP; ++q) {
      const int i = lane + q * PEPS_WARP;
      xr[q] = i < mr ? x[i] : M::zero();
    }
#if PEPS_QR_PREFETCH
    // the warp's next column into L1 while this one is updated
    if (c + nw < n) {
      const R* xn = x + (int64_t)nw * m;
      for (int i = lane * (128 / (int)sizeof(R)); i < mr; i += PEPS_WARP * (128 / (int)sizeof(R)))
        PEPS_PREFETCH_L1(xn + i);
    }
#endif
    // w = V^T x
    typename M::acc_t a[PEPS_QR_NB];
#pragma unroll
    for (int s = 0; s < PEPS_QR_NB; ++s) M::acc_init(a[s]);
#pragma unroll
    for (int q = 0; q < CAP; ++q) {
      const int i = lane + q * PEPS_WARP;
      if (i < mr) {
#pragma unroll
        for (int s = 0; s < PEPS_QR_NB; ++s)
          if (s < nb) M::mac(a[s], vsh[s * PEPS_QR_ROWS + i], xr[q]);
      }
    }
    R wv[PEPS_QR_NB];
#if PEPS_QR_ACC
    // the lanes' accumulators merged as accumulators (FP64: the same sums)
#pragma unroll
    for (int o = PEPS_WARP / 2; o > 0; o >>= 1) {
#pragma unroll
      for (int s = 0; s < PEPS_QR_NB; ++s) M::acc_shfl_add(a[s], o);
    }
#pragma unroll
    for (int s = 0; s < PEPS_QR_NB; ++s) wv[s] = M::acc_get(a[s]);
#else
#pragma unroll
    for (int s = 0; s < PEPS_QR_NB; ++s) wv[s] = M::acc_get(a[s]);
#pragma unroll
    for (int o = PEPS_WARP / 2; o > 0; o >>= 1) {
#pragma unroll
      for (int s = 0; s < PEPS_QR_NB; ++s) wv[s] = wv[s] + shfl_xor_r(wv[s], o);
    }
#endif
    // w' = T^T w
    R wt[PEPS_QR_NB];
#pragma unroll
    for (int s = 0; s < PEPS_QR_NB; ++s) {
      typename M::acc_t b;
      M::acc_init(b);
#pragma unroll
      for (int r = 0; r <= s; ++r)
        if (s < nb) M::mac(b, tt[r * PEPS_QR_NB + s], wv[r]);
      wt[s] = M::acc_get(b);
    }
    // x -= V w'
#if PEPS_QR_ACC
    // x - sum_s v_s w'_s in one compensated accumulation started at x (FP64:
    // the same fused multiply-adds as the chain of x - v w below)
#pragma unroll
    for (int s = 0; s < PEPS_QR_NB; ++s) wt[s] = -wt[s];
#pragma unroll
    for (int q = 0; q < CAP; ++q) {
      const int i = lane + q * PEPS_WARP;
      if (i < mr) {
        typename M::acc_t u;
        M::acc_set(u, xr[q]);
#pragma unroll
        for (int s = 0; s < PEPS_QR_NB; ++s)
          if (s < nb) M::mac(u, vsh[s * PEPS_QR_ROWS + i], wt[s]);
        x[i] = M::acc_get(u);
      }
    }
#else
#pragma unroll
    for (int q = 0; q < CAP; ++q) {
      const int i = lane + q * PEPS_WARP;
      if (i < mr) {
        R v = xr[q];
#pragma unroll
        for (int s = 0; s < PEPS_QR_NB; ++s)
          if (s < nb) v = M::sub_mul(v, vsh[s * PEPS_QR_ROWS + i], wt[s]);
        x[i] = v;
      }
    }
#endif
  }
}

// Trailing update of the tall blocked QR with two warps per column: the
// column's rows k0..m-1 are split between the pair (CAP rows per lane each)
// and held in registers; each warp forms its half of the nb dot products
// V^T x and reduces it within the warp; the halves are added through shared
// memory (xch, 2 NB scalars per pair) under the pair's named barrier, in the
// same order in both warps; then each warp updates its half and writes it
// back once: one read and one write of the column per panel.  Both warps of a
// pair run the same columns, and every iteration meets the barrier twice.
template <class R, int CAP>
__device__ __forceinline__ void qr_trailing_pair(R* X, int m, int n, int k0, int nb, int c0,
                                                 const R* tt, R* xch) {
  typedef Arith<R> M;
  const int lane = threadIdx.x % PEPS_WARP, wid = threadIdx.x / PEPS_WARP;
  const int nw = blockDim.x / PEPS_WARP;
  const int pair = wid >> 1, half = wid & 1, npairs = nw >> 1;
  const int mr = m - k0;
  const int hrows = (mr + 1) >> 1;
  const int r0 = k0 + half * hrows;                 // first row of this half
  const int rcount = half ? mr - hrows : hrows;     // its rows
  R* mine = xch + (pair * 2 + half) * PEPS_QR_NB;
  const R* lo = xch + (pair * 2) * PEPS_QR_NB;
  const R* hi = lo + PEPS_QR_NB;
  for (int c = c0 + pair; c < n; c += npairs) {
    R* x = X + (int64_t)c * m + r0;
    R xr[CAP];
    typename M::acc_t a[PEPS_QR_NB];
#pragma unroll
    for (int s = 0; s < PEPS_QR_NB; ++s) M::acc_init(a[s]);
#pragma unroll
    for (int q = 0; q < CAP; ++q) {
      const int ii = lane + q * PEPS_WARP;
      xr[q] = ii < rcount ? x[ii] : M::zero();
      if (ii < rcount) {
        const int i = r0 + ii;
#pragma unroll
        for (int s = 0; s < PEPS_QR_NB; ++s)
          if (s < nb && i >= k0 + s) {
            const R v = i == k0 + s ? M::one() : X[(int64_t)(k0 + s) * m + i];
            M::mac(a[s], v, xr[q]);
          }
      }
    }
    R wv[PEPS_QR_NB];
#if PEPS_QR_ACC
#pragma unroll
    for (int o = PEPS_WARP / 2; o > 0; o >>= 1) {
#pragma unroll
      for (int s = 0; s < PEPS_QR_NB; ++s) M::acc_shfl_add(a[s], o);
    }
#pragma unroll
    for (int s = 0; s < PEPS_QR_NB; ++s) wv[s] = M::acc_get(a[s]);
#else
#pragma unroll
    for (int s = 0; s < PEPS_QR_NB; ++s) wv[s] = M::acc_get(a[s]);
#pragma unroll
    for (int o = PEPS_WARP / 2; o > 0; o >>= 1) {
#pragma unroll
      for (int s = 0; s < PEPS_QR_NB; ++s) wv[s] = wv[s] + shfl_xor_r(wv[s], o);
    }
#endif
    if (lane == 0) {
#pragma unroll
      for (int s = 0; s < PEPS_QR_NB; ++s) mine[s] = wv[s];
    }
    PEPS_PAIR_SYNC(pair);
    R tot[PEPS_QR_NB];
#pragma unroll
    for (int s = 0; s < PEPS_QR_NB; ++s) tot[s] = lo[s] + hi[s];
    PEPS_PAIR_SYNC(pair);
    R wt[PEPS_QR_NB];
#pragma unroll
    for (int s = 0; s < PEPS_QR_NB; ++s) {
      typename M::acc_t b;
      M::acc_init(b);
#pragma unroll
      for (int r = 0; r <= s; ++r)
        if (s < nb) M::mac(b, tt[r * PEPS_QR_NB + s], tot[r]);
      wt[s] = M::acc_get(b);
    }
#if PEPS_QR_ACC
#pragma unroll
    for (int s = 0; s < PEPS_QR_NB; ++s) wt[s] = -wt[s];
#pragma unroll
    for (int q = 0; q < CAP; ++q) {
      const int ii = lane + q * PEPS_WARP;
      if (ii < rcount) {
        const int i = r0 + ii;
        typename M::acc_t u;
        M::acc_set(u, xr[q]);
#pragma unroll
        for (int s = 0; s < PEPS_QR_NB; ++s)
          if (s < nb && i >= k0 + s) {
            const R w = i == k0 + s ? M::one() : X[(int64_t)(k0 + s) * m + i];
            M::mac(u, w, wt[s]);
          }
        x[ii] = M::acc_get(u);
      }
    }
#else
#pragma unroll
    for (int q = 0; q < CAP; ++q) {
      const int ii = lane + q * PEPS_WARP;
      if (ii < rcount) {
        const int i = r0 + ii;
        R v = xr[q];
#pragma unroll
        for (int s = 0; s < PEPS_QR_NB; ++s)
          if (s < nb && i >= k0 + s) {
            const R w = i == k0 + s ? M::one() : X[(int64_t)(k0 + s) * m + i];
            v = M::sub_mul(v, w, wt[s]);
          }
        x[ii] = v;
      }
    }
#endif
  }
}

// ---------------------------------------------------------------------------
// Blocked form for panels taller than the register/shared-memory capacity
// (m > PEPS_QR_ROWS): the panel of PEPS_QR_NB columns is factored in place
// (unblocked), and the trailing columns are updated in the compact WY form
// x -= V T^T V^T x in two streaming passes per panel (the dot products, then
// the update), the reflectors read from the panel columns (L1-resident,
// shared by the warps): three accesses of a trailing element per panel
// instead of three per reflector; with PEPS_QR_TALL_PAIR, up to 2048 rows
// the column stays in the registers of two warps instead (qr_trailing_pair):
// one read and one write.
// sh: >= 2 PEPS_QR_NB + 2 PEPS_QR_NB^2 + (warps) PEPS_QR_NB scalars of
// shared memory.
// ---------------------------------------------------------------------------
template <class R>
#if PEPS_QR_TALL_PAIR
__device__ __noinline__
#else
__device__
#endif
void householder_r_tall(R* X, int m, int n, R* Rout, R* sh) {
  typedef Arith<R> M;
  const int t = threadIdx.x, lane = t % PEPS_WARP, wid = t / PEPS_WARP;
  const int nw = (blockDim.x + PEPS_WARP - 1) / PEPS_WARP;
  const int kmax = m < n ? m : n;
  R* tau = sh;
  R* tt = sh + 2 * PEPS_QR_NB;
  R* g = tt + PEPS_QR_NB * PEPS_QR_NB;
  for (int k0 = 0; k0 < kmax; k0 += PEPS_QR_NB) {
    const int nb = kmax - k0 < PEPS_QR_NB ? kmax - k0 : PEPS_QR_NB;
    // 1. the panel, unblocked, in place
    for (int s = 0; s < nb; ++s) {
      const int k = k0 + s;
      R* xk = X + (int64_t)k * m;
      if (wid == 0) {
        typename M::acc_t a;
        M::acc_init(a);
        for (int i = k + 1 + lane; i < m; i += PEPS_WARP) M::mac(a, xk[i], xk[i]);
        R xn2 = warp_sum<R>(M::acc_get(a));
        if (lane == 0) {
          R alpha = xk[k];
          if (!(M::hi(xn2) > 0)) {
            tau[s] = M::zero();
          } else {
            R nrm = M::sqrt_(alpha * alpha + xn2);
            R beta = M::hi(alpha) >= 0 ? -nrm : nrm;
            tau[s] = (beta - alpha) / beta;
            tau[PEPS_QR_NB] = M::one() / (alpha - beta);
            xk[k] = beta;
          }
        }
        __syncwarp();
        const R scl = tau[PEPS_QR_NB];
        if (M::hi(tau[s]) != 0)
          for (int i = k + 1 + lane; i < m; i += PEPS_WARP) xk[i] = xk[i] * scl;
        else
          for (int i = k + 1 + lane; i < m; i += PEPS_WARP) xk[i] = M::zero();
      }
      __syncthreads();
      if (M::hi(tau[s]) != 0) reflect_columns<R>(X, m, k, k + 1, k0 + nb, xk, tau[s]);
      __syncthreads();
    }
    if (k0 + nb >= n) continue;
    // 2. T of the compact WY form (v_r: one at row k0+r, the stored tail
    //    below, zeros above)
    for (int q = wid; q < nb * nb; q += nw) {
      const int r = q / nb, c = q % nb;
      if (r < c) {
        const R* vr = X + (int64_t)(k0 + r) * m;
        const R* vc = X + (int64_t)(k0 + c) * m;
        typename M::acc_t a;
        M::acc_init(a);
        if (lane == 0) M::mac(a, vr[k0 + c], M::one());
        for (int i = k0 + c + 1 + lane; i < m; i += PEPS_WARP) M::mac(a, vr[i], vc[i]);
        const R gv = warp_sum<R>(M::acc_get(a));
        if (lane == 0) g[q] = gv;
      }
    }
    __syncthreads();
    if (t == 0) {
      for (int c = 0; c < PEPS_QR_NB; ++c)
        for (int r = 0; r < PEPS_QR_NB; ++r) tt[r * PEPS_QR_NB + c] = M::zero();
      for (int c = 0; c < nb; ++c) {
        tt[c * PEPS_QR_NB + c] = tau[c];
        for (int r = 0; r < c; ++r) {
          typename M::acc_t a;
          M::acc_init(a);
          for (int q = r; q < c; ++q) M::mac(a, tt[r * PEPS_QR_NB + q], g[q * nb + c]);
          tt[r * PEPS_QR_NB + c] = -(tau[c] * M::acc_get(a));
        }
      }
    }
    __syncthreads();
    // 3. the trailing columns: two warps per column held in registers while
    //    the rows fit (up to 2048), else one warp per column in two passes
#if PEPS_QR_TALL_PAIR
    if (nw >= 2 && (nw & 1) == 0 && m - k0 <= 2 * PEPS_WARP * 32) {
      qr_trailing_pair<R, 32>(X, m, n, k0, nb, k0 + nb, tt, g + PEPS_QR_NB * PEPS_QR_NB);
      __syncthreads();
      continue;
    }
#endif
    for (int c = k0 + nb + wid; c < n; c += nw) {
      R* x = X + (int64_t)c * m;
      typename M::acc_t a[PEPS_QR_NB];
#pragma unroll
      for (int s = 0; s < PEPS_QR_NB; ++s) M::acc_init(a[s]);
      for (int i = k0 + lane; i < m; i += PEPS_WARP) {
        const R xi = x[i];
#pragma unroll
        for (int s = 0; s < PEPS_QR_NB; ++s) {
          if (s < nb && i >= k0 + s) {
            const R v = i == k0 + s ? M::one() : X[(int64_t)(k0 + s) * m + i];
            M::mac(a[s], v, xi);
          }
        }
      }
      R wv[PEPS_QR_NB];
#pragma unroll
      for (int s = 0; s < PEPS_QR_NB; ++s) wv[s] = M::acc_get(a[s]);
#pragma unroll
      for (int o = PEPS_WARP / 2; o > 0; o >>= 1) {
#pragma unroll
        for (int s = 0; s < PEPS_QR_NB; ++s) wv[s] = wv[s] + shfl_xor_r(wv[s], o);
      }
      R wt[PEPS_QR_NB];
#pragma unroll
      for (int s = 0; s < PEPS_QR_NB; ++s) {
        typename M::acc_t b;
        M::acc_init(b);
#pragma unroll
        for (int r = 0; r <= s; ++r)
          if (s < nb) M::mac(b, tt[r * PEPS_QR_NB + s], wv[r]);
        wt[s] = M::acc_get(b);
      }
      for (int i = k0 + lane; i < m; i += PEPS_WARP) {
        R xi = x[i];
#pragma unroll
        for (int s = 0; s < PEPS_QR_NB; ++s) {
          if (s < nb && i >= k0 + s) {
            const R v = i == k0 + s ? M::one() : X[(int64_t)(k0 + s) * m + i];
            xi = M::sub_mul(xi, v, wt[s]);
          }
        }
        x[i] = xi;
      }
    }
    __syncthreads();
  }
  for (int o = t; o < kmax * n; o += blockDim.x) {
    int i = o / n, c = o % n;
    Rout[o] = (c >= i) ? X[(int64_t)c * m + i] : M::zero();
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Blocked form of householder_r (the same reflectors, applied in the same
// order to every column): panels of PEPS_QR_NB columns are factored in
// shared memory, then applied to the trailing columns held in registers, so
// that a trailing column is read and written once per panel instead of three
// times per reflector.  vsh: PEPS_QR_NB * PEPS_QR_ROWS scalars of shared
// memory; sh: >= 2 * PEPS_QR_NB + 2 * PEPS_QR_NB^2 scalars.  Panels taller
// than PEPS_QR_ROWS take householder_r_tall; a null vsh the unblocked form.
// ---------------------------------------------------------------------------
template <class R>
__device__ __noinline__ void householder_r(R* X, int m, int n, R* Rout, R* sh, R* vsh) {
  typedef Arith<R> M;
  if (vsh == nullptr) {
    householder_r_unblocked<R>(X, m, n, Rout, sh);
    return;
  }
  if (m > PEPS_QR_ROWS) {
    householder_r_tall<R>(X, m, n, Rout, sh);
    return;
  }
  const int t = threadIdx.x, lane = t % PEPS_WARP, wid = t / PEPS_WARP;
  const int nw = (blockDim.x + PEPS_WARP - 1) / PEPS_WARP;
  const int kmax = m < n ? m : n;
  R* tau = sh;
  for (int k0 = 0; k0 < kmax; k0 += PEPS_QR_NB) {
    const int nb = kmax - k0 < PEPS_QR_NB ? kmax - k0 : PEPS_QR_NB;
    const int mr = m - k0;
    // 1. the panel (rows k0.., columns k0..k0+nb-1) into shared memory
    for (int o = t; o < nb * mr; o += blockDim.x) {
      const int r = o / mr, i = o - r * mr;
      vsh[r * PEPS_QR_ROWS + i] = X[(int64_t)(k0 + r) * m + k0 + i];
    }
    __syncthreads();
    // 2. unblocked factorisation of the panel (its diagonal is at row s of
    //    column s)
    for (int s = 0; s < nb; ++s) {
      R* v = vsh + s * PEPS_QR_ROWS;
      if (wid == 0) {
        typename M::acc_t a;
        M::acc_init(a);
        for (int i = s + 1 + lane; i < mr; i += PEPS_WARP) M::mac(a, v[i], v[i]);
        R xn2 = warp_sum<R>(M::acc_get(a));
        if (lane == 0) {
          R alpha = v[s];
          if (!(M::hi(xn2) > 0)) {
            tau[s] = M::zero();
            tau[PEPS_QR_NB] = M::zero();
          } else {
            R nrm = M::sqrt_(alpha * alpha + xn2);
            R beta = M::hi(alpha) >= 0 ? -nrm : nrm;
            tau[s] = (beta - alpha) / beta;
            tau[PEPS_QR_NB] = M::one() / (alpha - beta);
            v[s] = beta;
          }
        }
        __syncwarp();
        const R scl = tau[PEPS_QR_NB];
        if (M::hi(tau[s]) != 0)
          for (int i = s + 1 + lane; i < mr; i += PEPS_WARP) v[i] = v[i] * scl;
      }
      __syncthreads();
      const R ts = tau[s];
      if (M::hi(ts) != 0) {
        for (int c = s + 1 + wid; c < nb; c += nw) {
          R* x = vsh + c * PEPS_QR_ROWS;
          typename M::acc_t a;
          M::acc_init(a);
          if (lane == 0) M::mac(a, M::one(), x[s]);
          for (int i = s + 1 + lane; i < mr; i += PEPS_WARP) M::mac(a, v[i], x[i]);
          const R wv = ts * warp_sum<R>(M::acc_get(a));
          if (lane == 0) x[s] = x[s] - wv;
          for (int i = s + 1 + lane; i < mr; i += PEPS_WARP) x[i] = M::sub_mul(x[i], v[i], wv);
        }
      }
      __syncthreads();
    }
    // 3. R entries and reflector tails back to X; explicit reflectors
    //    (zero above the diagonal, one on it) left in shared memory
    for (int o = t; o < nb * mr; o += blockDim.x) {
      const int r = o / mr, i = o - r * mr;
      R* p = vsh + r * PEPS_QR_ROWS + i;
      X[(int64_t)(k0 + r) * m + k0 + i] = *p;
      if (i <= r) *p = (i == r) ? M::one() : M::zero();
    }
    __syncthreads();
    // 4. T of the compact WY form: T[s][s] = tau_s,
    //    T[0:s, s] = -tau_s T[0:s, 0:s] (V[:, 0:s]^T v_s)
    if (k0 + nb < n) {
      R* tt = tau + 2 * PEPS_QR_NB;  // PEPS_QR_NB^2 scalars
      R* g = tt + PEPS_QR_NB * PEPS_QR_NB;  // v_r . v_s, r < s
      for (int q = wid; q < nb * nb; q += nw) {
        const int r = q / nb, c = q % nb;
        if (r < c) {
          typename M::acc_t a;
          M::acc_init(a);
          for (int i = c + lane; i < mr; i += PEPS_WARP)
            M::mac(a, vsh[r * PEPS_QR_ROWS + i], vsh[c * PEPS_QR_ROWS + i]);
          const R gv = warp_sum<R>(M::acc_get(a));
          if (lane == 0) g[q] = gv;
        }
      }
      __syncthreads();
      if (t == 0) {
        for (int c = 0; c < PEPS_QR_NB; ++c)
          for (int r = 0; r < PEPS_QR_NB; ++r) tt[r * PEPS_QR_NB + c] = M::zero();
        for (int c = 0; c < nb; ++c) {
          tt[c * PEPS_QR_NB + c] = tau[c];
          for (int r = 0; r < c; ++r) {
            typename M::acc_t a;
            M::acc_init(a);
            for (int q = r; q < c; ++q) M::mac(a, tt[r * PEPS_QR_NB + q], g[q * nb + c]);
            tt[r * PEPS_QR_NB + c] = -(tau[c] * M::acc_get(a));
          }
        }
      }
      __syncthreads();
      // 5. the trailing columns
      if (mr <= 8 * PEPS_WARP)
        qr_trailing<R, (8 * PEPS_WARP + PEPS_WARP - 1) / PEPS_WARP>(X, m, n, k0, mr, k0 + nb, nb, vsh, tt);
      else
        qr_trailing<R, (PEPS_QR_ROWS + PEPS_WARP - 1) / PEPS_WARP>(X, m, n, k0, mr, k0 + nb, nb, vsh, tt);
    }
    __syncthreads();
  }
  for (int o = t; o < kmax * n; o += blockDim.x) {
    int i = o / n, c = o % n;
    Rout[o] = (c >= i) ? X[(int64_t)c * m + i] : M::zero();
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Blocked Golub-Kahan bidiagonalisation of A (m x p column-major, ld m,
// m >= p): A = Q B P^T with B upper bidiagonal (d, e).  The left reflectors
// (tau, tails below the diagonal of A's columns, v_k = 1) are kept for the
// back-transformation; the right ones are dropped.  Panels of nb steps: within
// a panel the trailing matrix is left as stored and the reflectors' effect is
// carried by four thin matrices (the panel's left vectors V, right vectors U
// and the products W = tau_p A' u, Y = tau_q A'^T v), so that A' = A - V Y^T
// - W U^T; each step reads the trailing matrix twice (A^T v and A u), and the
// panel's rank-2nb update is written once at its end (the blocking of Dongarra,
// Sorensen and Hammarling, 1989).
// pan: (2m + 2p) nb scalars of shared memory; sc: >= 2 nb + 8 scalars of
// shared memory.
// ---------------------------------------------------------------------------
template <class R>
__device__ void bidiag_blocked(R* A, int m, int p, int nb, R* d, R* e, R* tau, R* pan, R* sc) {
  typedef Arith<R> M;
  const int t = threadIdx.x, nt = blockDim.x;
  const int lane = t % PEPS_WARP, wid = t / PEPS_WARP, nw = (nt + PEPS_WARP - 1) / PEPS_WARP;
  R* Vp = pan;               // Vp[l*m + i]
  R* Wp = Vp + nb * m;       // Wp[l*m + i]
  R* Up = Wp + nb * m;       // Up[l*p + c]
  R* Yp = Up + nb * p;       // Yp[l*p + c]
  R* cf = sc + 8;            // 2 nb + 1 correction coefficients
  for (int i0 = 0; i0 < p; i0 += nb) {
    const int nbp = p - i0 < nb ? p - i0 : nb;
    for (int j = 0; j < nbp; ++j) {
      const int k = i0 + j;
      R* v = Vp + j * m;
      R* u = Up + j * p;
      // (a) column k of the current matrix, rows k..m-1, into Vp[:, j]
      for (int i = t; i < m; i += nt) {
        R x = M::zero();
        if (i >= k) {
          typename M::acc_t a;
          M::acc_init(a);
          M::mac(a, M::one(), A[(int64_t)k * m + i]);
          for (int l = 0; l < j; ++l) {
            M::mac(a, Vp[l * m + i], -Yp[l * p + k]);
            M::mac(a, Wp[l * m + i], -Up[l * p + k]);
          }
          x = M::acc_get(a);
        }
        v[i] = x;
      }
      __syncthreads();
      // (b) the left reflector: d_k, tau_k, v (v_k = 1), tail kept in A
      if (wid == 0) {
        typename M::acc_t a;
        M::acc_init(a);
        for (int i = k + 1 + lane; i < m; i += PEPS_WARP) M::mac(a, v[i], v[i]);
        const R xn2 = warp_sum<R>(M::acc_get(a));
        if (lane == 0) {
          const R alpha = v[k];
          if (!(M::hi(xn2) > 0)) {
            tau[k] = M::zero();
            d[k] = alpha;
            sc[0] = M::zero();
          } else {
            const R nrm = M::sqrt_(alpha * alpha + xn2);
            const R beta = M::hi(alpha) >= 0 ? -nrm : nrm;
            tau[k] = (beta - alpha) / beta;
            sc[0] = M::one() / (alpha - beta);
            d[k] = beta;
          }
        }
        __syncwarp();
        const R tq = tau[k], scl = sc[0];
        for (int i = k + 1 + lane; i < m; i += PEPS_WARP) {
          const R x = M::hi(tq) != 0 ? v[i] * scl : M::zero();
          v[i] = x;
          A[(int64_t)k * m + i] = x;
        }
        if (lane == 0) v[k] = M::one();
      }
      __syncthreads();
      const R tq = tau[k];
      const int nc = p - k - 1;  // trailing columns k+1..p-1
      if (nc <= 0) break;        // the last column: no row reflector
      // (c) Y[:, j] = tau_q (A'^T v) over columns k+1..p-1, with
      //     A'^T v = A^T v - Y (V^T v) - U (W^T v)
      if (M::hi(tq) != 0) {
#if PEPS_BIDIAG_TPC
        // one thread per column: a sequential dot product (two accumulators),
        // v read from shared memory by all threads at once
        for (int q = t; q < nc + 2 * j; q += nt) {
          const int l = q - nc;  // l < j: V^T v, else W^T v
          const R* col = q < nc ? A + (int64_t)(k + 1 + q) * m : (l < j ? Vp + l * m : Wp + (l - j) * m);
          typename M::acc_t a0, a1;
          M::acc_init(a0);
          M::acc_init(a1);
          int i = k;
          for (; i + 1 < m; i += 2) {
            M::mac(a0, col[i], v[i]);
            M::mac(a1, col[i + 1], v[i + 1]);
          }
          if (i < m) M::mac(a0, col[i], v[i]);
          const R r = M::acc_get(a0) + M::acc_get(a1);
          if (q < nc) Yp[j * p + k + 1 + q] = r;
          else cf[q - nc] = r;
        }
#else
        for (int q = wid; q < nc + 2 * j; q += nw) {
          typename M::acc_t a;
          M::acc_init(a);
          if (q < nc) {
            const R* col = A + (int64_t)(k + 1 + q) * m;
            for (int i = k + lane; i < m; i += PEPS_WARP) M::mac(a, col[i], v[i]);
          } else {
            const int l = q - nc;  // l < j: V^T v, else W^T v
            const R* x = l < j ? Vp + l * m : Wp + (l - j) * m;
            for (int i = k + lane; i < m; i += PEPS_WARP) M::mac(a, x[i], v[i]);
          }
          const R r = warp_sum<R>(M::acc_get(a));
          if (lane == 0) {
            if (q < nc) Yp[j * p + k + 1 + q] = r;
            else cf[q - nc] = r;
          }
        }
#endif
      }
      __syncthreads();
      for (int c = t; c < p; c += nt) {
        R y = M::zero();
        if (c > k && M::hi(tq) != 0) {
          typename M::acc_t a;
          M::acc_init(a);
          M::mac(a, M::one(), Yp[j * p + c]);
          for (int l = 0; l < j; ++l) {
            M::mac(a, Yp[l * p + c], -cf[l]);
            M::mac(a, Up[l * p + c], -cf[j + l]);
          }
          y = tq * M::acc_get(a);
        }
        Yp[j * p + c] = y;
      }
      // (d) reads Y[0..j] only in the columns c that this thread has just
      // written (the same c = t + q nt): PEPS_BIDIAG_FUSE leaves out the
      // barrier between the two loops
#if !PEPS_BIDIAG_FUSE
      __syncthreads();
#endif
      // (d) row k of the current matrix after the left reflector, columns
      //     k+1..p-1, into Up[:, j]
      for (int c = t; c < p; c += nt) {
        R x = M::zero();
        if (c > k) {
          typename M::acc_t a;
          M::acc_init(a);
          M::mac(a, M::one(), A[(int64_t)c * m + k]);
          for (int l = 0; l <= j; ++l) M::mac(a, Vp[l * m + k], -Yp[l * p + c]);
          for (int l = 0; l < j; ++l) M::mac(a, Wp[l * m + k], -Up[l * p + c]);
          x = M::acc_get(a);
        }
        u[c] = x;
      }
      __syncthreads();
      // (e) the right reflector on u[k+1..p-1]: e_k, tau_p, u (u_{k+1} = 1)
      if (wid == 0) {
        typename M::acc_t a;
        M::acc_init(a);
        for (int c = k + 2 + lane; c < p; c += PEPS_WARP) M::mac(a, u[c], u[c]);
        const R xn2 = warp_sum<R>(M::acc_get(a));
        if (lane == 0) {
          const R alpha = u[k + 1];
          if (!(M::hi(xn2) > 0)) {
            sc[1] = M::zero();
            e[k] = alpha;
            sc[2] = M::zero();
          } else {
            const R nrm = M::sqrt_(alpha * alpha + xn2);
            const R beta = M::hi(alpha) >= 0 ? -nrm : nrm;
            sc[1] = (beta - alpha) / beta;
            sc[2] = M::one() / (alpha - beta);
            e[k] = beta;
          }
        }
        __syncwarp();
        const R tp = sc[1], scl = sc[2];
        for (int c = k + 2 + lane; c < p; c += PEPS_WARP) u[c] = M::hi(tp) != 0 ? u[c] * scl : M::zero();
        if (lane == 0) u[k + 1] = M::one();
      }
      __syncthreads();
      // (f) W[:, j] = tau_p (A' u) over rows k+1..m-1, with
      //     A' u = A u - V (Y^T u) - W (U^T u)   (Y, V including column j)
      const R tp = sc[1];
      if (M::hi(tp) != 0) {
        // coefficients: Y^T u (j + 1 of them), U^T u (j of them)
        for (int q = wid; q < 2 * j + 1; q += nw) {
          const R* x = q <= j ? Yp + q * p : Up + (q - j - 1) * p;
          typename M::acc_t a;
          M::acc_init(a);
          for (int c = k + 1 + lane; c < p; c += PEPS_WARP) M::mac(a, x[c], u[c]);
          const R r = warp_sum<R>(M::acc_get(a));
          if (lane == 0) cf[q] = r;
        }
        // A u: one warp per 32-row chunk, every column
        for (int ch = wid; ch * PEPS_WARP + k + 1 < m; ch += nw) {
          const int i = k + 1 + ch * PEPS_WARP + lane;
          typename M::acc_t a0, a1;
          M::acc_init(a0);
          M::acc_init(a1);
          if (i < m) {
            int c = k + 1;
            for (; c + 1 < p; c += 2) {
              M::mac(a0, A[(int64_t)c * m + i], u[c]);
              M::mac(a1, A[(int64_t)(c + 1) * m + i], u[c + 1]);
            }
            if (c < p) M::mac(a0, A[(int64_t)c * m + i], u[c]);
            Wp[j * m + i] = M::acc_get(a0) + M::acc_get(a1);
          }
        }
      }
      __syncthreads();
      for (int i = t; i < m; i += nt) {
        R x = M::zero();
        if (i > k && M::hi(tp) != 0) {
          typename M::acc_t a;
          M::acc_init(a);
          M::mac(a, M::one(), Wp[j * m + i]);
          for (int l = 0; l <= j; ++l) M::mac(a, Vp[l * m + i], -cf[l]);
          for (int l = 0; l < j; ++l) M::mac(a, Wp[l * m + i], -cf[j + 1 + l]);
          x = tp * M::acc_get(a);
        }
        Wp[j * m + i] = x;
      }
      // the next step's (a) reads W[.][i] only in the rows i that this
      // thread has just written (the same i = t + q nt), and its other
      // readers of W come after the barriers of (a) and (b):
      // PEPS_BIDIAG_FUSE keeps this barrier only after the panel's last step
#if PEPS_BIDIAG_FUSE
      if (j + 1 == nbp) __syncthreads();
#else
      __syncthreads();
#endif
    }
    // the panel's update of the trailing matrix (rows, columns >= i0 + nbp)
    const int k1 = i0 + nbp;
    for (int c = k1 + wid; c < p; c += nw) {
      R* col = A + (int64_t)c * m;
      for (int i = k1 + lane; i < m; i += PEPS_WARP) {
        typename M::acc_t a;
        M::acc_init(a);
        M::mac(a, M::one(), col[i]);
        for (int l = 0; l < nbp; ++l) {
          M::mac(a, Vp[l * m + i], -Yp[l * p + c]);
          M::mac(a, Wp[l * m + i], -Up[l * p + c]);
        }
        col[i] = M::acc_get(a);
      }
    }
    __syncthreads();
  }
}

// Arithmetic of the inverse-iteration recurrences: FP64 unless the form is
// FP32 (its workspace is sized in FP32 words).
template <class R> struct InvType { typedef double T; };
template <> struct InvType<float> { typedef float T; };

// ---------------------------------------------------------------------------
// Top-kk right singular vectors of X (rr x n row-major, 1 <= rr <= n) by
// Golub-Kahan bidiagonalisation, bisection and inverse iteration:
//   1. A = X^T (n x rr, column c = row c of X) = Q B P^T with B upper
//      bidiagonal (diagonal d, superdiagonal e); Householder reflectors from
//      the left (kept: they form Q) and from the right (applied and dropped).
//   2. The kk largest singular values of B by bisection on the count of
//      singular values below x, from the stationary qd transform of
//      B^T B - x^2 (relative accuracy in FP32; Demmel-Kahan).
//   3. For each, inverse iteration (FP64; FP32 in the FP32 form) on the
//      Golub-Kahan tridiagonal (zero diagonal, off-diagonals d0,e0,d1,...),
//      whose eigenvector for +sigma interleaves (v_0, u_0, v_1, u_1, ...) with
//      B v = sigma u; three solves with a partially pivoted LU.
//   4. Gram-Schmidt on the u's (largest first), then V_i = Q [u_i; 0]: the
//      right singular vectors of X.  Directions whose singular value is at or
//      below eps * sigma_max are written as zero rows, so that the kept basis
//      stays orthonormal (the truncation stays an orthogonal projection).
// VT (kk x n) receives the vectors in decreasing order of sigma.
// aux: >= 3 rr + 8 scalars; inv: >= kk (13 rr) scalars; fsh: 1024
// floats of shared memory; ush: 256 scalars of shared memory.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned peps_hash(unsigned a, unsigned b) {
  unsigned h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 15; h *= 0x2C1B3C6Du; h ^= h >> 12; h *= 0x297A2D39u; h ^= h >> 15;
  return h;
}

// number of singular values of the bidiagonal (d, e) below x (FP32)
__device__ __forceinline__ int bidiag_count(const float* d, const float* e, int p, float x) {
  const float x2 = x * x;
  const float pivmin = 1e-36f;
  float t = -x2;
  int c = 0;
  for (int i = 0; i < p; ++i) {
    float D = d[i] * d[i] + t;
    if (fabsf(D) < pivmin) D = -pivmin;
    c += D < 0.0f;
    if (i + 1 < p) t = t * (e[i] * e[i] / D) - x2;
  }
  return c;
}

template <class R>
__device__ __noinline__ void svd_topk_rows(R* X, int rr, int n, int kk, R* VT, R* aux, R* inv,
                              float* fsh, R* ush, double* red, R* vsh) {
  typedef Arith<R> M;
  const int t = threadIdx.x, nt = blockDim.x;
  const int lane = t % PEPS_WARP, wid = t / PEPS_WARP, nw = (nt + PEPS_WARP - 1) / PEPS_WARP;
  const int m = n, p = rr;
  R* d = aux;
  R* e = aux + p;
  R* tau = aux + 2 * p;
  R* sc = aux + 3 * p;  // scalars
  // ---- 1. bidiagonalisation ---------------------------------------------
  const int nbb = vsh ? (PEPS_QR_NB * PEPS_QR_ROWS) / (2 * m + 2 * p) : 0;
  if (nbb >= 2) {
    bidiag_blocked<R>(X, m, p, nbb < 8 ? nbb : 8, d, e, tau, vsh, ush);
  } else
  for (int k = 0; k < p; ++k) {
    R* ck = X + (int64_t)k * n;
    if (wid == 0) {
      typename M::acc_t a;
      M::acc_init(a);
      for (int i = k + 1 + lane; i < m; i += PEPS_WARP) M::mac(a, ck[i], ck[i]);
      R xn2 = warp_sum<R>(M::acc_get(a));
      if (lane == 0) {
        R alpha = ck[k];
        if (!(M::hi(xn2) > 0)) {
          tau[k] = M::zero();
          d[k] = alpha;
        } else {
          R nrm = M::sqrt_(alpha * alpha + xn2);
          R beta = M::hi(alpha) >= 0 ? -nrm : nrm;
          tau[k] = (beta - alpha) / beta;
          sc[0] = M::one() / (alpha - beta);
          d[k] = beta;
          ck[k] = beta;
        }
      }
      __syncwarp();
      if (M::hi(tau[k]) != 0) {
        const R scl = sc[0];
        for (int i = k + 1 + lane; i < m; i += PEPS_WARP) ck[i] = ck[i] * scl;
      }
    }
    __syncthreads();
    const R tk = tau[k];
    if (M::hi(tk) != 0) reflect_columns<R>(X, n, k, k + 1, p, ck, tk);
    __syncthreads();
    if (k + 1 < p) {
      // row k of A over columns k+1..p-1: the entries X[c*n + k]
      if (k + 2 < p) {
        if (wid == 0) {
          typename M::acc_t a;
          M::acc_init(a);
          for (int c = k + 2 + lane; c < p; c += PEPS_WARP) {
            R x = X[(int64_t)c * n + k];
            M::mac(a, x, x);
          }
          R xn2 = warp_sum<R>(M::acc_get(a));
          if (lane == 0) {
            R alpha = X[(int64_t)(k + 1) * n + k];
            if (!(M::hi(xn2) > 0)) {
              sc[1] = M::zero();
              e[k] = alpha;
            } else {
              R nrm = M::sqrt_(alpha * alpha + xn2);
              R beta = M::hi(alpha) >= 0 ? -nrm : nrm;
              sc[1] = (beta - alpha) / beta;
              sc[2] = M::one() / (alpha - beta);
              e[k] = beta;
              X[(int64_t)(k + 1) * n + k] = beta;
            }
          }
          __syncwarp();
          const bool on = M::hi(sc[1]) != 0;
          const R scl = sc[2];
          for (int c = k + 1 + lane; c < p; c += PEPS_WARP) {
            R u = M::one();
            if (c > k + 1) {
              u = on ? X[(int64_t)c * n + k] * scl : M::zero();
              X[(int64_t)c * n + k] = u;
            }
            ush[c] = u;
          }
        }
        __syncthreads();
        const R tr = sc[1];
        if (M::hi(tr) != 0) {
          for (int i = k + 1 + t; i < m; i += nt) {
            typename M::acc_t a, b;
            M::acc_init(a);
            M::acc_init(b);
            int c = k + 1;
            for (; c + 1 < p; c += 2) {
              M::mac(a, ush[c], X[(int64_t)c * n + i]);
              M::mac(b, ush[c + 1], X[(int64_t)(c + 1) * n + i]);
            }
            if (c < p) M::mac(a, ush[c], X[(int64_t)c * n + i]);
            const R s = tr * (M::acc_get(a) + M::acc_get(b));
            for (c = k + 1; c < p; ++c) X[(int64_t)c * n + i] = X[(int64_t)c * n + i] - ush[c] * s;
          }
        }
        __syncthreads();
      } else {
        if (t == 0) e[k] = X[(int64_t)(k + 1) * n + k];
        __syncthreads();
      }
    }
  }
  // ---- 2. singular values: FP32 bisection ---------------------------------
  float* df = fsh;
  float* ef = fsh + 256;
  float* sg = fsh + 512;
  double amax = 0.0;
  for (int i = t; i < p; i += nt) {
    amax = fmax(amax, fabs((double)M::hi(d[i])));
    if (i + 1 < p) amax = fmax(amax, fabs((double)M::hi(e[i])));
  }
  const double smax = block_max(amax, red);
  const float rs = smax > 0.0 ? (float)(1.0 / smax) : 0.0f;
  for (int i = t; i < p; i += nt) {
    df[i] = (float)M::hi(d[i]) * rs;
    ef[i] = (i + 1 < p) ? (float)M::hi(e[i]) * rs : 0.0f;
  }
  __syncthreads();
  // multisection: G threads per singular value probe G points of its
  // bracket each round (geometric spacing once the bracket excludes 0)
  float* lo_s = fsh + 768;  // kk <= 256
  float* hi_s = sg;
  int* flag = reinterpret_cast<int*>(ush);
  if (t == 0) {
    float bound = 0.0f;
    for (int i = 0; i < p; ++i)
      bound = fmaxf(bound, fabsf(df[i]) + fabsf(ef[i]) + (i > 0 ? fabsf(ef[i - 1]) : 0.0f));
    for (int q = 0; q < kk; ++q) {
      lo_s[q] = 0.0f;
      hi_s[q] = bound * 1.0001f + 1e-30f;
    }
  }
  __syncthreads();
  {
    const int G = nt / kk >= 1 ? nt / kk : 1;
    const int ngroups = nt / G;
    for (int round = 0; round < 64; ++round) {
      int busy = 0;
      for (int q0 = 0; q0 < kk; q0 += ngroups) {
        const int gq = t / G, r = t % G, q = q0 + gq;
        const bool mine = gq < ngroups && q < kk;
        float lo = 0.0f, hi = 0.0f;
        bool conv = true;
        if (mine) {
          lo = lo_s[q];
          hi = hi_s[q];
          conv = hi - lo <= 2e-7f * hi || hi < 1e-30f;
        }
        const bool geo = lo > 0.0f && hi > 4.0f * lo;
        int f = 0;
        if (mine && !conv) {
          const float fr = (float)(r + 1) / (float)(G + 1);
          float x = geo ? lo * powf(hi / lo, fr) : lo + (hi - lo) * fr;
          f = bidiag_count(df, ef, p, x) > p - 1 - q;
          busy = 1;
        }
        flag[t] = f;
        __syncthreads();
        if (mine && !conv && r == 0) {
          int r1 = 0;  // first probe above sigma_q
          while (r1 < G && !flag[t + r1]) ++r1;
          const float f0 = (float)r1 / (float)(G + 1), f1 = (float)(r1 + 1) / (float)(G + 1);
          if (r1 > 0) lo_s[q] = geo ? lo * powf(hi / lo, f0) : lo + (hi - lo) * f0;
          if (r1 < G) hi_s[q] = geo ? lo * powf(hi / lo, f1) : lo + (hi - lo) * f1;
        }
        __syncthreads();
      }
      if (!__syncthreads_or(busy)) break;
    }
    for (int q = t; q < kk; q += nt) sg[q] = 0.5f * (lo_s[q] + hi_s[q]);  // in units of smax
  }
  __syncthreads();
  // ---- 3. inverse iteration on the Golub-Kahan tridiagonal ----------------
  const int N2 = 2 * p;
  const int stride = 6 * N2 + p;
  const float zero_tol = (float)(M::eps() * 4.0);
  // The recurrences below are serial in j, 24-odd lanes wide and bound by
  // latency, not throughput: they run in FP64 for the FP64 and float-float
  // forms (shorter dependency chains than float-float, and more accurate),
  // in FP32 for the FP32 form.
  typedef typename InvType<R>::T T;
  for (int q = t; q < kk; q += nt) {
    // private rows of the factorisation (no aliasing: the recurrences keep
    // their carried values in registers and the loads can run ahead)
    T* __restrict__ U0 = reinterpret_cast<T*>(inv + (int64_t)q * stride);  // reciprocal pivots
    T* __restrict__ U1 = U0 + N2;
    T* __restrict__ U2 = U1 + N2;
    T* __restrict__ Lm = U2 + N2;
    T* __restrict__ z = Lm + N2;
    T* __restrict__ y = z + N2;
    R* __restrict__ u = inv + (int64_t)q * stride + 6 * N2;
    if (!(sg[q] > zero_tol)) {
      for (int i = 0; i < p; ++i) u[i] = M::zero();
      continue;
    }
    const T mu = (T)((double)sg[q] * smax);
    const T tiny = (T)(smax * 1e-30 + 1e-300);
    // g_j: off-diagonal j of the Golub-Kahan matrix
#define PEPS_GK(j) ((T)M::to(((j) & 1) ? e[(j) >> 1] : d[(j) >> 1]))
    T ca = -mu, cb = PEPS_GK(0), cc = 0;
    for (int j = 0; j + 1 < N2; ++j) {
      const T gs = PEPS_GK(j);
      const T gn = (j + 2 < N2) ? PEPS_GK(j + 1) : (T)0;
      if (fabs(ca) >= fabs(gs)) {
        const T a0 = (ca == 0) ? tiny : ca;
        const T ra = (T)1 / a0;
        const T l = gs * ra;
        U0[j] = ra; U1[j] = cb; U2[j] = cc; Lm[j] = l;
        z[j] = 0;  // pivot flag 0
        ca = -mu - l * cb;
        cb = gn - l * cc;
      } else {
        const T rg = (T)1 / gs;
        const T l = ca * rg;
        U0[j] = rg; U1[j] = -mu; U2[j] = gn; Lm[j] = l;
        z[j] = 1;  // pivot flag 1
        const T na = cb + l * mu;
        cb = cc - l * gn;
        ca = na;
      }
      cc = 0;
    }
    U0[N2 - 1] = (T)1 / ((ca == 0) ? tiny : ca);
    U1[N2 - 1] = 0;
    U2[N2 - 1] = 0;
    // start vector
    for (int j = 0; j < N2; ++j)
      y[j] = (T)(1.0 + (double)(peps_hash((unsigned)q, (unsigned)j) & 0xffff) * (1.0 / 65536.0));
    for (int iter = 0; iter < 3; ++iter) {
      // forward: row interchanges and eliminations (the running entry is
      // carried in a register)
      T cur = y[0];
#pragma unroll 4
      for (int j = 0; j + 1 < N2; ++j) {
        T nxt = y[j + 1];
        if (z[j] != 0) { const T tmp = cur; cur = nxt; nxt = tmp; }
        y[j] = cur;
        cur = nxt - Lm[j] * cur;
      }
      y[N2 - 1] = cur;
      // back substitution
      T x1 = 0, x2 = 0, ymax = 0;
#pragma unroll 4
      for (int j = N2 - 1; j >= 0; --j) {
        const T xj = (y[j] - U1[j] * x1 - U2[j] * x2) * U0[j];
        y[j] = xj;
        x2 = x1;
        x1 = xj;
        ymax = fmax(ymax, fabs(xj));
      }
      // to unit max-abs, then to unit norm
      const T r0 = ymax > 0 ? (T)1 / ymax : (T)1;
      T nrm = 0;
      for (int j = 0; j < N2; ++j) {
        const T v = y[j] * r0;
        y[j] = v;
        nrm += v * v;
      }
      const T sn = (T)1 / sqrt(nrm);
      for (int j = 0; j < N2; ++j) y[j] = y[j] * sn;
    }
    for (int i = 0; i < p; ++i) u[i] = M::from((double)y[2 * i + 1]);
#undef PEPS_GK
  }
  __syncthreads();
  // ---- 4a. Gram-Schmidt on the u's (in order of decreasing sigma) --------
  for (int q = 0; q < kk; ++q) {
    R* uq = inv + (int64_t)q * stride + 6 * N2;
    if (!(sg[q] > zero_tol)) continue;  // zero row
    for (int pass = 0; pass < 2; ++pass) {
      // coefficients against the earlier vectors (warp per vector)
      for (int r = wid; r < q; r += nw) {
        const R* ur = inv + (int64_t)r * stride + 6 * N2;
        typename M::acc_t a;
        M::acc_init(a);
        for (int i = lane; i < p; i += PEPS_WARP) M::mac(a, ur[i], uq[i]);
        R cf = warp_sum<R>(M::acc_get(a));
        if (lane == 0) ush[r] = (sg[r] > zero_tol) ? cf : M::zero();
      }
      __syncthreads();
      for (int i = t; i < p; i += nt) {
        R v = uq[i];
        for (int r = 0; r < q; ++r) v = v - ush[r] * (inv + (int64_t)r * stride + 6 * N2)[i];
        uq[i] = v;
      }
      __syncthreads();
    }
    typename M::acc_t a;
    M::acc_init(a);
    for (int i = t; i < p; i += nt) M::mac(a, uq[i], uq[i]);
    R n2 = block_sum<R>(M::acc_get(a), reinterpret_cast<R*>(red));
    const R s = (M::hi(n2) > 0) ? M::one() / M::sqrt_(n2) : M::zero();
    for (int i = t; i < p; i += nt) uq[i] = uq[i] * s;
    __syncthreads();
  }
  // ---- 4b. V_i = Q [u_i; 0] (reflectors in reverse order): each warp
  //      transforms up to three vectors together (one load of the reflector
  //      per element for all three, interleaved reductions)
  for (int q0 = wid; q0 < kk; q0 += 3 * nw) {
    R* vv[3];
    bool on[3];
#pragma unroll
    for (int g = 0; g < 3; ++g) {
      const int q = q0 + g * nw;
      on[g] = q < kk;
      vv[g] = VT + (int64_t)(on[g] ? q : q0) * n;
      if (on[g]) {
        const R* uq = inv + (int64_t)q * stride + 6 * N2;
        for (int i = lane; i < n; i += PEPS_WARP) vv[g][i] = (i < p) ? uq[i] : M::zero();
      }
    }
    __syncwarp();
    for (int k = p - 1; k >= 0; --k) {
      const R tk = tau[k];
      if (M::hi(tk) == 0) continue;
      const R* ck = X + (int64_t)k * n;
      typename M::acc_t a[3];
#pragma unroll
      for (int g = 0; g < 3; ++g) {
        M::acc_init(a[g]);
        if (on[g] && lane == 0) M::mac(a[g], M::one(), vv[g][k]);
      }
      for (int i = k + 1 + lane; i < n; i += PEPS_WARP) {
        const R c = ck[i];
#pragma unroll
        for (int g = 0; g < 3; ++g)
          if (on[g]) M::mac(a[g], c, vv[g][i]);
      }
      R sg3[3];
#pragma unroll
      for (int g = 0; g < 3; ++g) sg3[g] = M::acc_get(a[g]);
#pragma unroll
      for (int o = PEPS_WARP / 2; o > 0; o >>= 1) {
#pragma unroll
        for (int g = 0; g < 3; ++g) sg3[g] = sg3[g] + shfl_xor_r(sg3[g], o);
      }
#pragma unroll
      for (int g = 0; g < 3; ++g) sg3[g] = tk * sg3[g];
      __syncwarp();
      if (lane == 0) {
#pragma unroll
        for (int g = 0; g < 3; ++g)
          if (on[g]) vv[g][k] = vv[g][k] - sg3[g];
      }
      for (int i = k + 1 + lane; i < n; i += PEPS_WARP) {
        const R c = ck[i];
#pragma unroll
        for (int g = 0; g < 3; ++g)
          if (on[g]) vv[g][i] = M::sub_mul(vv[g][i], c, sg3[g]);
      }
      __syncwarp();
    }
  }
  __syncthreads();
}
