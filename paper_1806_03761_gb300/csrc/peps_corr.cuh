// peps_corr.cuh -- spin-spin correlations of sampled configurations (PEPS++,
// arXiv:1806.03761, Sec. "Experiment Setup" and its results: the map
// <S_0 . S_m> and the structure factor m_s^2(k) over the bulk).
//
// Local value of S_a . S_m on a configuration S drawn from W(S)^2:
//   sigma_a sigma_m / 4 + [s_a != s_m] (1/2) W(S')/W(S),  3/4 for m = a,
// S' = S with s_a and s_m exchanged.  The ratio is taken on the one-row strip
// of the target's row i = i(m), each configuration with its own
// environments: W_i(S') / W_i(S).  S' agrees with S^a (S with s_a flipped)
// outside row i, so the numerator is the strip of row i of S^a between
// U_{i-1}(S^a) and Dn_{i+1}(S^a), with column j(m) given the spin s_a:
// one left column step from the strip's left environment, closed against
// its right one.  U_{i-1}(S^a) = U_{i-1}(S) above the source row and
// Dn_{i+1}(S^a) = Dn_{i+1}(S) below it, so one item (sample, source) costs
// the lower environments of S and S^a down to the source row, the upper
// environments of S and S^a from it, and two one-row strips per row.
#pragma once
#include "peps_eval.cuh"

// Left environments of the one-row strip of row i (no right ones): returns
// log|W_i| and writes the sign.
template <class R>
__device__ double strip1_value(const PepsPlan& P, int i, const uint8_t* sp, const R* As,
                               const R* U, const EnvDims& Ud, const R* Dn, const EnvDims& Dd,
                               const Work<R>& w, double* sign) {
  const int L = P.L;
  const int64_t SC = P.site_cap;
  if (threadIdx.x == 0) w.l1[0] = Arith<R>::one();
  __syncthreads();
  double lg = 0.0;
  for (int j = 0; j < L; ++j) {
    Col1 k = col_dims(P, Ud, Dd, j);
    const int m = i * L + j;
    R* out = w.l1 + (int64_t)(j + 1) * SC;
    strip1_left_step<R>(P, k, w.l1 + (int64_t)j * SC, U + j * SC, tens(P, As, m, sp[m]),
                        Dn + j * SC, out, w);
    lg += normalize_pow2<R>(out, env1_size(P, Ud, Dd, j + 1), w.red);
  }
  const double v = Arith<R>::to(w.l1[(int64_t)L * SC]);
  *sign = (double)((v > 0.0) - (v < 0.0));
  return log(fabs(v)) + lg;
}

// Lower environments Dn_k(S^a), k = i0 .. 1, into w.dnf (k > i0: those of S).
template <class R>
__device__ void build_lower_flipped(const PepsPlan& P, const PepsStep* steps, const R* As,
                                    const uint8_t* spf, int i0, const Work<R>& w,
                                    const double* dnlog, double* dnlogf) {
  const int L = P.L;
  for (int k = i0; k >= 1; --k) {
    const R* Min = (k == i0) ? w.dn + (int64_t)(k + 1) * P.env_cap : w.dnf + (int64_t)(k + 1) * P.env_cap;
    const double lin = (k == i0) ? dnlog[k + 1] : dnlogf[k + 1];
    R* Mout = w.dnf + (int64_t)k * P.env_cap;
    const double lg = compress_row<R>(P, steps[L - 1 - k], false, k, As, spf, Min, lin, Mout, w);
    __syncthreads();
    if (threadIdx.x == 0) dnlogf[k] = lg;
    __syncthreads();
  }
}

template <class R>
__device__ void correlate_one(const CorrArgs<R>& a, int64_t b, int q, BlockShared<R>& sh,
                              const Work<R>& w) {
  const PepsPlan& P = a.P;
  const int L = P.L, N = P.N;
  const int64_t SC = P.site_cap;
  const int src = a.src[q];
  const int i0 = src / L;
  uint8_t* sp = sh.sp;
  uint8_t* spf = sh.sp2;
  for (int m = threadIdx.x; m < N; m += blockDim.x) {
    const uint8_t s = a.spins[b * N + m];
    sp[m] = s;
    spf[m] = (m == src) ? (uint8_t)(1 - s) : s;
  }
  __syncthreads();
  const uint8_t s_a = sp[src];
  double* out = a.ss + ((int64_t)b * a.n_src + q) * N;
  // diagonal part (and 3/4 at the source); the exchange parts are added below
  for (int m = threadIdx.x; m < N; m += blockDim.x) {
    const double sz = (sp[m] == s_a) ? 0.25 : -0.25;
    out[m] = (m == src) ? 0.75 : sz;
  }
  __syncthreads();
  // lower environments of S, then of S^a down to the source row
  build_lower<R>(P, a.steps, a.As, sp, w, sh.dnlog);
  build_lower_flipped<R>(P, a.steps, a.As, spf, i0, w, sh.dnlog, sh.dnlogf);
  // upper environments of S (ring w.up) and of S^a (ring w.upf from row i0)
  set_trivial<R>(P, w.up);
  if (threadIdx.x == 0) { sh.uplog[0] = 0.0; sh.uplogf[0] = 0.0; }
  __syncthreads();
  int ucur = 0, fcur = -1;  // fcur < 0: U(S^a) = U(S) (rows above the source)
  double* cl = w.scl;
  double* cr = w.scl + (L + 1);
  for (int i = 0; i < L; ++i) {
    const R* U = w.up + (int64_t)ucur * P.env_cap;
    const R* Uf = fcur < 0 ? U : w.upf + (int64_t)fcur * P.env_cap;
    const double ul = sh.uplog[ucur], ulf = fcur < 0 ? ul : sh.uplogf[fcur];
    const EnvDims Ud = env_dims(P, a.steps, i - 1);
    const EnvDims Dd = env_dims(P, a.steps, (i + 1 <= L - 1) ? (L - 2 - i) : -1);
    const R* Dn = w.dn + (int64_t)(i + 1) * P.env_cap;
    const R* Dnf = (i + 1 <= i0) ? w.dnf + (int64_t)(i + 1) * P.env_cap : Dn;
    const double dl = sh.dnlog[i + 1], dlf = (i + 1 <= i0) ? sh.dnlogf[i + 1] : dl;
    bool any = false;
    for (int j = 0; j < L; ++j) any |= (i * L + j != src) && (sp[i * L + j] != s_a);
    if (any) {
      // W_i(S)
      double sg0;
      const double lw0 = strip1_value<R>(P, i, sp, a.As, U, Ud, Dn, Dd, w, &sg0) + ul + dl;
      // the strip of row i of S^a, then one window per target
      strip1_build<R>(P, i, spf, a.As, Uf, Ud, Dnf, Dd, w, cl, cr);
      for (int j = 0; j < L; ++j) {
        const int m = i * L + j;
        if (m == src || sp[m] == s_a) continue;
        const Col1 k = col_dims(P, Ud, Dd, j);
        strip1_left_step<R>(P, k, w.l1 + (int64_t)j * SC, Uf + j * SC, tens(P, a.As, m, s_a),
                            Dnf + j * SC, w.y, w);
        const double v = dot_blk<R>(w.y, w.r1 + (int64_t)(j + 1) * SC, env1_size(P, Ud, Dd, j + 1), w);
        if (threadIdx.x == 0) {
          double r = 0.0;
          if (v != 0.0 && sg0 != 0.0) {
            const double lw = log(fabs(v)) + cl[j] + cr[j + 1] + ulf + dlf;
            r = (double)((v > 0.0) - (v < 0.0)) * sg0 * exp(lw - lw0);
          }
          if (!isfinite(r) || sg0 == 0.0) atomicOr(a.flags, 1);
          out[m] += 0.5 * r;
        }
        __syncthreads();
      }
    }
    if (i + 1 < L) {
      // U_i(S), and U_i(S^a) from the source row on
      const int unext = (ucur == 1) ? 2 : 1;
      const double lg = compress_row<R>(P, a.steps[i], true, i, a.As, sp, U, ul,
                                        w.up + (int64_t)unext * P.env_cap, w);
      __syncthreads();
      if (i >= i0) {
        const int fnext = (fcur == 1) ? 2 : 1;
        const double lgf = compress_row<R>(P, a.steps[i], true, i, a.As, spf, Uf, ulf,
                                           w.upf + (int64_t)fnext * P.env_cap, w);
        __syncthreads();
        if (threadIdx.x == 0) sh.uplogf[fnext] = lgf;
        fcur = fnext;
      }
      if (threadIdx.x == 0) sh.uplog[unext] = lg;
      __syncthreads();
      ucur = unext;
    }
  }
}

template <class R>
__global__ void __launch_bounds__(PEPS_NT, PEPS_MINB) peps_corr_kernel(CorrArgs<R> a) {
  __shared__ BlockShared<R> sh;
  Work<R> w = bind_work<R>(a.P, a.ws, a.wsd, sh, a.flags);
  const int64_t items = a.B * a.n_src;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    correlate_one<R>(a, it / a.n_src, (int)(it % a.n_src), sh, w);
    __syncthreads();
  }
}
