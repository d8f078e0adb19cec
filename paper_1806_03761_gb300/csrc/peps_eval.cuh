// peps_eval.cuh -- the fused per-sample evaluation (PEPS++, arXiv:1806.03761,
// Fig. "contraction" Steps 2, 4, 5 and Eqs. ess, delta):
// lower environments -> for each row: one-row strip (amplitude, horizontal
// ratios, B tensors), two-row strip (vertical and J2 ratios), upper
// environment of the row -> E(S) -> Delta sums.
#pragma once
#include "peps_mps.cuh"
#include "peps_args.h"


template <class R>
__device__ Work<R> make_work(const PepsPlan& P, R* ws, double* wsd, int slot) {
  Work<R> w;
  w.qrv = nullptr;  // the shared-memory pointers are bound by the kernel
  R* base = ws + (int64_t)slot * P.slot_elems;
  double* bd = wsd + (int64_t)slot * P.slot_doubles;
  w.dn = base + P.off_dn;
  w.up = base + P.off_up;
  w.rst = base + P.off_rst;
  w.b0 = base + P.off_b0;
  w.b1 = base + P.off_b1;
  w.b2 = base + P.off_b2;
  w.y = base + P.off_y;
  w.xj = base + P.off_xj;
  w.vt = base + P.off_vt;
  w.c0 = base + P.off_c0;
  w.c1 = base + P.off_c1;
  w.l1 = base + P.off_l1;
  w.r1 = base + P.off_r1;
  w.l2 = base + P.off_l2;
  w.r2 = base + P.off_r2;
  w.scl = bd + P.doff_scale;
  w.delta = bd + P.doff_delta;
  w.alpha = base + P.off_alpha;
  w.inv = base + P.off_inv;
  w.dnf = base + P.off_dnf;
  w.upf = base + P.off_upf;
  return w;
}

// Column dims of a strip between an upper env (step su) and a lower env
// (step sd); step -1 = the trivial environment.
__device__ __forceinline__ Col1 col_dims(const PepsPlan& P, const EnvDims& U,
                                         const EnvDims& Dn, int j) {
  Col1 k;
  k.au = ed_a(U, j); k.pu = U.p; k.bu = ed_b(U, j);
  k.ad = ed_a(Dn, j); k.pd = Dn.p; k.bd = ed_b(Dn, j);
  k.Dl = (j == 0) ? 1 : P.D;
  k.Dr = (j == P.L - 1) ? 1 : P.D;
  return k;
}
__device__ __forceinline__ int env1_size(const PepsPlan& P, const EnvDims& U, const EnvDims& Dn, int j) {
  if (j == P.L) return 1;
  return ed_a(U, j) * ((j == 0) ? 1 : P.D) * ed_a(Dn, j);
}
__device__ __forceinline__ int env2_size(const PepsPlan& P, const EnvDims& U, const EnvDims& Dn, int j) {
  if (j == P.L) return 1;
  int Dl = (j == 0) ? 1 : P.D;
  return ed_a(U, j) * Dl * Dl * ed_a(Dn, j);
}

// Build the trivial environment (every site the 1x1x1 tensor [1]).
template <class R>
__device__ void set_trivial(const PepsPlan& P, R* env) {
  for (int j = threadIdx.x; j < P.L; j += blockDim.x) env[(int64_t)j * P.site_cap] = Arith<R>::one();
  __syncthreads();
}

template <class R>
__device__ __forceinline__ const R* tens(const PepsPlan& P, const R* As, int m, int s) {
  return As + ((int64_t)m * 2 + s) * P.D4;
}

// Build the lower environments of the current spins: Dn_{L-1} .. Dn_1 at
// w.dn + row*env_cap, their log-scales in dnlog[row]; Dn_L (trivial) at L.
template <class R>
__device__ void build_lower(const PepsPlan& P, const PepsStep* steps, const R* As,
                            const uint8_t* sp, const Work<R>& w, double* dnlog) {
  const int L = P.L;
  set_trivial<R>(P, w.dn + (int64_t)L * P.env_cap);
  if (threadIdx.x == 0) dnlog[L] = 0.0;
  const R* Min = w.dn + (int64_t)L * P.env_cap;
  double lg = 0.0;
  for (int t = 0; t < L - 1; ++t) {
    int row = L - 1 - t;
    R* Mout = w.dn + (int64_t)row * P.env_cap;
    lg = compress_row<R>(P, steps[t], false, row, As, sp, Min, lg, Mout, w);
    if (threadIdx.x == 0) dnlog[row] = lg;
    Min = Mout;
  }
  __syncthreads();
}

// One-row strip of row i between U (dims Ud) and Dn (dims Dd): left and
// right environments normalised by powers of two; scale logs in
// cl[0..L], cr[0..L].
template <class R>
__device__ void strip1_build(const PepsPlan& P, int i, const uint8_t* sp, const R* As,
                             const R* U, const EnvDims& Ud, const R* Dn,
                             const EnvDims& Dd, const Work<R>& w, double* cl,
                             double* cr) {
  const int L = P.L;
  const int64_t SC = P.site_cap;
  if (threadIdx.x == 0) {
    w.l1[0] = Arith<R>::one();
    w.r1[(int64_t)L * SC] = Arith<R>::one();
    cl[0] = 0.0;
    cr[L] = 0.0;
  }
  __syncthreads();
  for (int j = 0; j < L; ++j) {
    Col1 k = col_dims(P, Ud, Dd, j);
    int m = i * L + j;
    R* out = w.l1 + (int64_t)(j + 1) * SC;
    strip1_left_step<R>(P, k, w.l1 + (int64_t)j * SC, U + j * SC, tens(P, As, m, sp[m]),
                        Dn + j * SC, out, w);
    double c = normalize_pow2<R>(out, env1_size(P, Ud, Dd, j + 1), w.red);
    if (threadIdx.x == 0) cl[j + 1] = cl[j] + c;
  }
  for (int j = L - 1; j >= 0; --j) {
    Col1 k = col_dims(P, Ud, Dd, j);
    int m = i * L + j;
    R* out = w.r1 + (int64_t)j * SC;
    strip1_right_step<R>(P, k, w.r1 + (int64_t)(j + 1) * SC, U + j * SC, tens(P, As, m, sp[m]),
                         Dn + j * SC, out, w);
    double c = normalize_pow2<R>(out, env1_size(P, Ud, Dd, j), w.red);
    if (threadIdx.x == 0) cr[j] = cr[j + 1] + c;
  }
  __syncthreads();
}

template <class R>
__device__ void strip2_build(const PepsPlan& P, int i, const uint8_t* sp, const R* As,
                             const R* U, const EnvDims& Ud, const R* Dn,
                             const EnvDims& Dd, const Work<R>& w, double* cl) {
  const int L = P.L;
  const int64_t SC = P.site_cap, EC = P.env2_cap;
  if (threadIdx.x == 0) {
    w.l2[0] = Arith<R>::one();
    w.r2[(int64_t)L * EC] = Arith<R>::one();
    cl[0] = 0.0;
  }
  __syncthreads();
  for (int j = 0; j < L; ++j) {
    Col1 k = col_dims(P, Ud, Dd, j);
    int m1 = i * L + j, m2 = (i + 1) * L + j;
    R* out = w.l2 + (int64_t)(j + 1) * EC;
    strip2_left_step<R>(P, k, w.l2 + (int64_t)j * EC, U + j * SC, tens(P, As, m1, sp[m1]),
                        tens(P, As, m2, sp[m2]), Dn + j * SC, out, w);
    double c = normalize_pow2<R>(out, env2_size(P, Ud, Dd, j + 1), w.red);
    if (threadIdx.x == 0) cl[j + 1] = cl[j] + c;
  }
  for (int j = L - 1; j >= 0; --j) {
    Col1 k = col_dims(P, Ud, Dd, j);
    int m1 = i * L + j, m2 = (i + 1) * L + j;
    R* out = w.r2 + (int64_t)j * EC;
    strip2_right_step<R>(P, k, w.r2 + (int64_t)(j + 1) * EC, U + j * SC, tens(P, As, m1, sp[m1]),
                         tens(P, As, m2, sp[m2]), Dn + j * SC, out, w);
    normalize_pow2<R>(out, env2_size(P, Ud, Dd, j), w.red);
  }
  __syncthreads();
}

// Ratio of the horizontal exchange (i,j)-(i,j+1) on the one-row strip.
template <class R>
__device__ double ratio_h(const PepsPlan& P, int i, int j, const uint8_t* sp, const R* As,
                          const R* U, const EnvDims& Ud, const R* Dn, const EnvDims& Dd,
                          const Work<R>& w, const double* cl) {
  const int L = P.L;
  const int64_t SC = P.site_cap;
  int m1 = i * L + j, m2 = m1 + 1;
  Col1 k0 = col_dims(P, Ud, Dd, j), k1 = col_dims(P, Ud, Dd, j + 1);
  strip1_left_step<R>(P, k0, w.l1 + (int64_t)j * SC, U + j * SC, tens(P, As, m1, sp[m2]),
                      Dn + j * SC, w.y, w);
  strip1_left_step<R>(P, k1, w.y, U + (j + 1) * SC, tens(P, As, m2, sp[m1]),
                      Dn + (j + 1) * SC, w.xj, w);
  int n = env1_size(P, Ud, Dd, j + 2);
  const R* Rr = w.r1 + (int64_t)(j + 2) * SC;
  double num = dot_blk<R>(w.xj, Rr, n, w);
  double den = dot_blk<R>(w.l1 + (int64_t)(j + 2) * SC, Rr, n, w);
  return num / den * exp(cl[j] - cl[j + 2]);
}

// Ratio of a two-row-strip exchange.  kind 0: vertical (i,j)-(i+1,j);
// 1: diagonal (i,j)-(i+1,j+1); 2: anti-diagonal (i,j+1)-(i+1,j).
template <class R>
__device__ double ratio_2(const PepsPlan& P, int kind, int i, int j, const uint8_t* sp,
                          const R* As, const R* U, const EnvDims& Ud, const R* Dn,
                          const EnvDims& Dd, const Work<R>& w, const double* cl) {
  const int L = P.L;
  const int64_t SC = P.site_cap, EC = P.env2_cap;
  int t00 = i * L + j, t10 = (i + 1) * L + j;
  Col1 k0 = col_dims(P, Ud, Dd, j);
  int ncol = (kind == 0) ? 1 : 2;
  int s00 = sp[t00], s10 = sp[t10];
  if (kind == 0) {
    strip2_left_step<R>(P, k0, w.l2 + (int64_t)j * EC, U + j * SC, tens(P, As, t00, s10),
                        tens(P, As, t10, s00), Dn + j * SC, w.y, w);
  } else {
    int t01 = t00 + 1, t11 = t10 + 1;
    int s01 = sp[t01], s11 = sp[t11];
    Col1 k1 = col_dims(P, Ud, Dd, j + 1);
    if (kind == 1) {  // swap (i,j) <-> (i+1,j+1)
      strip2_left_step<R>(P, k0, w.l2 + (int64_t)j * EC, U + j * SC, tens(P, As, t00, s11),
                          tens(P, As, t10, s10), Dn + j * SC, w.xj, w);
      strip2_left_step<R>(P, k1, w.xj, U + (j + 1) * SC, tens(P, As, t01, s01),
                          tens(P, As, t11, s00), Dn + (j + 1) * SC, w.y, w);
    } else {          // swap (i,j+1) <-> (i+1,j)
      strip2_left_step<R>(P, k0, w.l2 + (int64_t)j * EC, U + j * SC, tens(P, As, t00, s00),
                          tens(P, As, t10, s01), Dn + j * SC, w.xj, w);
      strip2_left_step<R>(P, k1, w.xj, U + (j + 1) * SC, tens(P, As, t01, s10),
                          tens(P, As, t11, s11), Dn + (j + 1) * SC, w.y, w);
    }
  }
  int n = env2_size(P, Ud, Dd, j + ncol);
  const R* Rr = w.r2 + (int64_t)(j + ncol) * EC;
  double num = dot_blk<R>(w.y, Rr, n, w);
  double den = dot_blk<R>(w.l2 + (int64_t)(j + ncol) * EC, Rr, n, w);
  return num / den * exp(cl[j] - cl[j + ncol]);
}

// Shared memory of the per-sample kernels.
template <class R>
struct BlockShared {
  double red[PEPS_NT];
  __align__(16) unsigned char redR_raw[PEPS_NT * sizeof(R)];
  __align__(16) unsigned char wsh_raw[256 * sizeof(R)];
  __align__(16) unsigned char qrv_raw[PEPS_QR_NB * PEPS_QR_ROWS * sizeof(R)];
  double rot[512];
  uint8_t sp[PEPS_MAXL * PEPS_MAXL];
  uint8_t sp2[PEPS_MAXL * PEPS_MAXL];  // a second configuration (correlations)
  double dnlog[PEPS_MAXL + 1];
  double dnlogf[PEPS_MAXL + 1];
  double uplog[3];
  double uplogf[3];
  int count;
};

template <class R>
__device__ Work<R> bind_work(const PepsPlan& P, R* ws, double* wsd, BlockShared<R>& sh, int* flags) {
  Work<R> w = make_work<R>(P, ws, wsd, blockIdx.x);
  w.red = sh.red;
  w.redR = reinterpret_cast<R*>(sh.redR_raw);
  w.wsh = reinterpret_cast<R*>(sh.wsh_raw);
  w.qrv = reinterpret_cast<R*>(sh.qrv_raw);
  w.rot = sh.rot;
  w.flags = flags;
  return w;
}

// Evaluate sample b (spins in sh.sp): amplitude, E(S), ratios, Delta staged
// and added to the slot partial sums ps.  dn_ready: the lower environments
// of these spins are already in w.dn (dnlog filled).
template <class R>
__device__ __forceinline__ void evaluate_one(const EvalArgs<R>& a, int64_t b, BlockShared<R>& sh,
                             const Work<R>& w, double* ps, bool dn_ready) {
  const PepsPlan& P = a.P;
  const int L = P.L, N = P.N, D4 = P.D4;
  const uint8_t* sp = sh.sp;
  double* dnlog = sh.dnlog;
  double* uplog = sh.uplog;
  double* cl1 = w.scl;
  double* cr1 = w.scl + (L + 1);
  double* cl2 = w.scl + 2 * (L + 1);
  const int64_t PSN = (int64_t)N * 2 * D4;
  if (!dn_ready) build_lower<R>(P, a.steps, a.As, sp, w, dnlog);
  // the trivial upper environment
  set_trivial<R>(P, w.up);
  if (threadIdx.x == 0) uplog[0] = 0.0;
  __syncthreads();
  // diagonal part of E(S) and the flip count
  double e = 0.0;
  int nflip = 0;
  if (a.want_energy) {
    for (int i = 0; i < L; ++i)
      for (int j = 0; j < L; ++j) {
        int m = i * L + j;
        double sm = sp[m] ? -1.0 : 1.0;
        if (j + 1 < L) { double s2 = sp[m + 1] ? -1.0 : 1.0; e += P.J1 * sm * s2 * 0.25; nflip += sp[m] != sp[m + 1]; }
        if (i + 1 < L) { double s2 = sp[m + L] ? -1.0 : 1.0; e += P.J1 * sm * s2 * 0.25; nflip += sp[m] != sp[m + L]; }
        if (i + 1 < L && j + 1 < L) { double s2 = sp[m + L + 1] ? -1.0 : 1.0; e += P.J2 * sm * s2 * 0.25; nflip += sp[m] != sp[m + L + 1]; }
        if (i + 1 < L && j + 1 < L) { double s2 = sp[m + L] ? -1.0 : 1.0; double s1 = sp[m + 1] ? -1.0 : 1.0; e += P.J2 * s1 * s2 * 0.25; nflip += sp[m + 1] != sp[m + L]; }
      }
  }
  double* rout = a.ratios ? a.ratios + b * P.nbonds : nullptr;
  if (rout) {
    for (int o = threadIdx.x; o < P.nbonds; o += blockDim.x) rout[o] = 0.0;
    __syncthreads();
  }
  int ucur = 0;  // index of U_{i-1} among the three upper buffers
  const bool full = a.want_energy || a.want_delta;
  for (int i = 0; i < L; ++i) {
    const R* U = w.up + (int64_t)ucur * P.env_cap;
    EnvDims Ud = env_dims(P, a.steps, i - 1);
    const R* Dn = w.dn + (int64_t)(i + 1) * P.env_cap;
    EnvDims Dd = env_dims(P, a.steps, (i + 1 <= L - 1) ? (L - 2 - i) : -1);
    PEPS_TIC(t_s1);
    strip1_build<R>(P, i, sp, a.As, U, Ud, Dn, Dd, w, cl1, cr1);
    PEPS_TOC(t_s1, PH_STRIP1);
    double wv = Arith<R>::to(w.l1[(int64_t)L * P.site_cap]);
    double logw = log(fabs(wv)) + cl1[L] + uplog[ucur] + dnlog[i + 1];
    if (i == 0) {
      if (threadIdx.x == 0) {
        if (a.log_abs) a.log_abs[b] = logw;
        if (a.sign) a.sign[b] = (int8_t)((wv > 0.0) - (wv < 0.0));
        if (wv == 0.0) atomicOr(a.flags, 2);
        if (!isfinite(wv)) atomicOr(a.flags, 1);
      }
      if (!full) break;
    }
    if (a.want_energy) {
      for (int j = 0; j + 1 < L; ++j) {
        int m = i * L + j;
        if (sp[m] == sp[m + 1]) continue;
        PEPS_TIC(t_rh);
        double r = ratio_h<R>(P, i, j, sp, a.As, U, Ud, Dn, Dd, w, cl1);
        PEPS_TOC(t_rh, PH_RATIO_H);
        e += P.J1 * 0.5 * r;
        if (threadIdx.x == 0) {
          if (rout) rout[i * (L - 1) + j] = r;
          if (!isfinite(r)) atomicOr(a.flags, 1);
        }
      }
    }
    if (a.want_delta) {
      PEPS_TIC(t_bt);
      for (int j = 0; j < L; ++j) {
        int m = i * L + j;
        Col1 k = col_dims(P, Ud, Dd, j);
        R* Bt = w.vt;  // D^4 scalars
        for (int o = threadIdx.x; o < D4; o += blockDim.x) Bt[o] = Arith<R>::zero();
        __syncthreads();
        strip1_btensor<R>(P, k, w.l1 + (int64_t)j * P.site_cap, U + j * P.site_cap,
                          w.r1 + (int64_t)(j + 1) * P.site_cap, Dn + j * P.site_cap, Bt, w);
        double f = exp(cl1[j] + cr1[j + 1] - cl1[L]) / wv;
        for (int o = threadIdx.x; o < D4; o += blockDim.x)
          w.delta[(int64_t)m * D4 + o] = Arith<R>::to(Bt[o]) * f;
        __syncthreads();
      }
      PEPS_TOC(t_bt, PH_BTENS);
    }
    if (a.want_energy && i + 1 < L) {
      const R* Dn2 = w.dn + (int64_t)(i + 2) * P.env_cap;
      EnvDims Dd2 = env_dims(P, a.steps, (i + 2 <= L - 1) ? (L - 3 - i) : -1);
      PEPS_TIC(t_s2);
      strip2_build<R>(P, i, sp, a.As, U, Ud, Dn2, Dd2, w, cl2);
      PEPS_TOC(t_s2, PH_STRIP2);
      PEPS_TIC(t_r2);
      for (int j = 0; j < L; ++j) {
        int m1 = i * L + j, m2 = m1 + L;
        if (sp[m1] != sp[m2]) {
          double r = ratio_2<R>(P, 0, i, j, sp, a.As, U, Ud, Dn2, Dd2, w, cl2);
          e += P.J1 * 0.5 * r;
          if (threadIdx.x == 0 && rout) rout[L * (L - 1) + i * L + j] = r;
        }
        if (j + 1 < L) {
          if (sp[m1] != sp[m2 + 1]) {
            double r = ratio_2<R>(P, 1, i, j, sp, a.As, U, Ud, Dn2, Dd2, w, cl2);
            e += P.J2 * 0.5 * r;
            if (threadIdx.x == 0 && rout) rout[2 * L * (L - 1) + i * (L - 1) + j] = r;
          }
          if (sp[m1 + 1] != sp[m2]) {
            double r = ratio_2<R>(P, 2, i, j, sp, a.As, U, Ud, Dn2, Dd2, w, cl2);
            e += P.J2 * 0.5 * r;
            if (threadIdx.x == 0 && rout)
              rout[2 * L * (L - 1) + (L - 1) * (L - 1) + i * (L - 1) + j] = r;
          }
        }
      }
      PEPS_TOC(t_r2, PH_RATIO_2);
    }
    // U_i for the next row
    if (i + 1 < L) {
      int unext = (ucur == 1) ? 2 : 1;
      double lg = compress_row<R>(P, a.steps[i], true, i, a.As, sp, U,
                                  uplog[ucur], w.up + (int64_t)unext * P.env_cap, w);
      __syncthreads();
      if (threadIdx.x == 0) uplog[unext] = lg;
      __syncthreads();
      ucur = unext;
    }
  }
  if (threadIdx.x == 0) {
    if (a.want_energy) {
      if (a.e_loc) a.e_loc[b] = e;
      if (a.n_flips) a.n_flips[b] = nflip;
      if (!isfinite(e)) atomicOr(a.flags, 1);
    }
  }
  if (a.want_delta) {
    double eb = a.want_energy ? e : a.e_in[b];
    for (int64_t o = threadIdx.x; o < (int64_t)N * D4; o += blockDim.x) {
      int m = (int)(o / D4), kx = (int)(o % D4);
      double d = w.delta[o];
      int64_t idx = ((int64_t)m * 2 + sp[m]) * D4 + kx;
      ps[idx] += d;
      ps[PSN + idx] += d * eb;
      if (a.delta) a.delta[b * (int64_t)N * D4 + o] = d;
    }
    if (threadIdx.x == 0) ps[2 * PSN] += eb;
  }
  __syncthreads();
}

template <class R>
__global__ void __launch_bounds__(PEPS_NT, PEPS_MINB) peps_eval_kernel(EvalArgs<R> a) {
  __shared__ BlockShared<R> sh;
  const PepsPlan& P = a.P;
  const int N = P.N, D4 = P.D4;
  Work<R> w = bind_work<R>(P, a.ws, a.wsd, sh, a.flags);
  double* ps = a.psum + (int64_t)blockIdx.x * (2 * (int64_t)N * 2 * D4 + 1);
  const int64_t PSN = (int64_t)N * 2 * D4;
  if (a.want_delta) {
    for (int64_t o = threadIdx.x; o < 2 * PSN + 1; o += blockDim.x) ps[o] = 0.0;
  }
  __syncthreads();
  for (int64_t b = blockIdx.x; b < a.B; b += gridDim.x) {
    for (int m = threadIdx.x; m < N; m += blockDim.x) sh.sp[m] = a.spins[b * N + m];
    __syncthreads();
    evaluate_one<R>(a, b, sh, w, ps, false);
  }
}

template <class R>
__global__ void peps_convert_kernel(const double* A, R* As, int64_t n, int* flags) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double x = A[k];
    if (!isfinite(x)) atomicOr(flags, 1);
    As[k] = Arith<R>::from(x);
  }
}

// GO update: A[e] -= p_e dt sign(g_e), g = 2 sde/M - 2 (sd/M)(se/M); the step
// number from step_dev when given (read at run time: graph replay)
template <class R>
__global__ void peps_grad_kernel(const double* sd, const double* sde, const double* se,
                                 double M, double dt, uint32_t k0, uint32_t k1,
                                 uint32_t step_in, const uint32_t* step_dev, double* A, R* As,
                                 int64_t n) {
  const uint32_t step = step_dev ? *step_dev : step_in;
  const double mE = se[0] / M;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double g = 2.0 * (sde[e] / M) - 2.0 * (sd[e] / M) * mE;
    double sg = (double)((g > 0.0) - (g < 0.0));
    u32x4 c;
    c.x = (uint32_t)e;
    c.y = (uint32_t)((uint64_t)e >> 32);
    c.z = step;
    c.w = 2u;
    double p = uniform_open52(philox_word64(philox4x32_10(c, k0, k1)));
    double an = A[e] - p * dt * sg;
    A[e] = an;
    As[e] = Arith<R>::from(an);
  }
}
