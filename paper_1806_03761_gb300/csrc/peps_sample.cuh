// peps_sample.cuh -- Metropolis sampling of configurations with weight
// W(S)^2 (PEPS++, arXiv:1806.03761: Fig. "contraction", Steps 1-3;
// Eq. energy-MC).  One thread block runs one chain at a time.  A sweep
// rebuilds the lower environments, then for each row i: proposes the
// horizontal exchanges left to right on the one-row strip (right
// environments built once, the left one advanced after every decision),
// then the vertical exchanges (i,j)-(i+1,j) on the two-row strip, then
// absorbs the updated row i into the upper environment.
#pragma once
#include "peps_eval.cuh"


template <class R>
__device__ void strip1_right_all(const PepsPlan& P, int i, const uint8_t* sp, const R* As,
                                 const R* U, const EnvDims& Ud, const R* Dn,
                                 const EnvDims& Dd, const Work<R>& w) {
  const int L = P.L;
  const int64_t SC = P.site_cap;
  if (threadIdx.x == 0) w.r1[(int64_t)L * SC] = Arith<R>::one();
  __syncthreads();
  for (int j = L - 1; j >= 0; --j) {
    Col1 k = col_dims(P, Ud, Dd, j);
    int m = i * L + j;
    R* out = w.r1 + (int64_t)j * SC;
    strip1_right_step<R>(P, k, w.r1 + (int64_t)(j + 1) * SC, U + j * SC, tens(P, As, m, sp[m]),
                         Dn + j * SC, out, w);
    normalize_pow2<R>(out, env1_size(P, Ud, Dd, j), w.red);
  }
}

template <class R>
__device__ void strip2_right_all(const PepsPlan& P, int i, const uint8_t* sp, const R* As,
                                 const R* U, const EnvDims& Ud, const R* Dn,
                                 const EnvDims& Dd, const Work<R>& w) {
  const int L = P.L;
  const int64_t SC = P.site_cap, EC = P.env2_cap;
  if (threadIdx.x == 0) w.r2[(int64_t)L * EC] = Arith<R>::one();
  __syncthreads();
  for (int j = L - 1; j >= 0; --j) {
    Col1 k = col_dims(P, Ud, Dd, j);
    int m1 = i * L + j, m2 = (i + 1) * L + j;
    R* out = w.r2 + (int64_t)j * EC;
    strip2_right_step<R>(P, k, w.r2 + (int64_t)(j + 1) * EC, U + j * SC, tens(P, As, m1, sp[m1]),
                         tens(P, As, m2, sp[m2]), Dn + j * SC, out, w);
    normalize_pow2<R>(out, env2_size(P, Ud, Dd, j), w.red);
  }
}

// One Metropolis sweep of the spins in sh.sp (updated in place); returns the
// number of accepted exchanges (uniform over the block).  dn_ready: the lower
// environments of these spins are already in w.dn.
template <class R>
__device__ __forceinline__ int sweep_one(const PepsPlan& P, const PepsStep* steps, const R* As,
                         uint32_t k0, uint32_t k1, uint32_t chain, uint32_t sweep,
                         BlockShared<R>& sh, const Work<R>& w, bool dn_ready) {
  const int L = P.L;
  const int64_t SC = P.site_cap, EC = P.env2_cap;
  uint8_t* sp = sh.sp;
  if (threadIdx.x == 0) sh.count = 0;
  __syncthreads();
  if (!dn_ready) build_lower<R>(P, steps, As, sp, w, sh.dnlog);
  set_trivial<R>(P, w.up);
  int ucur = 0;
  for (int i = 0; i < L; ++i) {
    const R* U = w.up + (int64_t)ucur * P.env_cap;
    EnvDims Ud = env_dims(P, steps, i - 1);
    const R* Dn = w.dn + (int64_t)(i + 1) * P.env_cap;
    EnvDims Dd = env_dims(P, steps, (i + 1 <= L - 1) ? (L - 2 - i) : -1);
    // ---- horizontal moves on the one-row strip --------------------------
    PEPS_TIC(t_h);
    strip1_right_all<R>(P, i, sp, As, U, Ud, Dn, Dd, w);
    if (threadIdx.x == 0) w.l1[0] = Arith<R>::one();
    __syncthreads();
    for (int j = 0; j + 1 < L; ++j) {
      int m = i * L + j;
      // the left environment over column j with the current spins: the
      // denominator's first column step when a move is proposed here (the
      // numerator's when it is accepted), else computed on its own
      R* out = w.l1 + (int64_t)(j + 1) * SC;
      if (sp[m] != sp[m + 1]) {
        Col1 kc0 = col_dims(P, Ud, Dd, j), kc1 = col_dims(P, Ud, Dd, j + 1);
        int n = env1_size(P, Ud, Dd, j + 2);
        const R* Rr = w.r1 + (int64_t)(j + 2) * SC;
        const R* Lj = w.l1 + (int64_t)j * SC;
        strip1_left_step<R>(P, kc0, Lj, U + j * SC, tens(P, As, m, sp[m + 1]), Dn + j * SC, w.y, w);
        strip1_left_step<R>(P, kc1, w.y, U + (j + 1) * SC, tens(P, As, m + 1, sp[m]), Dn + (j + 1) * SC, w.xj, w);
        double num = dot_blk<R>(w.xj, Rr, n, w);
        strip1_left_step<R>(P, kc0, Lj, U + j * SC, tens(P, As, m, sp[m]), Dn + j * SC, out, w);
        strip1_left_step<R>(P, kc1, out, U + (j + 1) * SC, tens(P, As, m + 1, sp[m + 1]), Dn + (j + 1) * SC, w.xj, w);
        double den = dot_blk<R>(w.xj, Rr, n, w);
        double r = num / den;
        u32x4 ctr = {(uint32_t)(i * (L - 1) + j), sweep, chain, 1u};
        double u = uniform53(philox_word64(philox4x32_10(ctr, k0, k1)));
        if (!isfinite(r) && threadIdx.x == 0) atomicOr(w.flags, 1);
        if (u < r * r) {
          // accepted: column j now carries the other spin, whose column
          // step is the numerator's first one
          const int n1 = env1_size(P, Ud, Dd, j + 1);
          for (int o = threadIdx.x; o < n1; o += blockDim.x) out[o] = w.y[o];
          __syncthreads();
          if (threadIdx.x == 0) {
            uint8_t tmp = sp[m]; sp[m] = sp[m + 1]; sp[m + 1] = tmp;
            sh.count++;
          }
          __syncthreads();
        }
      } else {
        Col1 k = col_dims(P, Ud, Dd, j);
        strip1_left_step<R>(P, k, w.l1 + (int64_t)j * SC, U + j * SC, tens(P, As, m, sp[m]), Dn + j * SC, out, w);
      }
      normalize_pow2<R>(out, env1_size(P, Ud, Dd, j + 1), w.red);
    }
    PEPS_TOC(t_h, PH_SWEEP_1);
    if (i + 1 < L) {
      // ---- vertical moves on the two-row strip ---------------------------
      const R* Dn2 = w.dn + (int64_t)(i + 2) * P.env_cap;
      EnvDims Dd2 = env_dims(P, steps, (i + 2 <= L - 1) ? (L - 3 - i) : -1);
      PEPS_TIC(t_r2);
      strip2_right_all<R>(P, i, sp, As, U, Ud, Dn2, Dd2, w);
      PEPS_TOC(t_r2, PH_SWEEP_R2);
      PEPS_TIC(t_v);
      if (threadIdx.x == 0) w.l2[0] = Arith<R>::one();
      __syncthreads();
      for (int j = 0; j < L; ++j) {
        int m1 = i * L + j, m2 = m1 + L;
        Col1 k = col_dims(P, Ud, Dd2, j);
        const R* L2j = w.l2 + (int64_t)j * EC;
        // the left environment over column j with the current spins: the
        // denominator when a move is proposed here (the numerator when it is
        // accepted), else computed on its own
        R* out = w.l2 + (int64_t)(j + 1) * EC;
        if (sp[m1] != sp[m2]) {
          int n = env2_size(P, Ud, Dd2, j + 1);
          const R* Rr = w.r2 + (int64_t)(j + 1) * EC;
          strip2_left_step<R>(P, k, L2j, U + j * SC, tens(P, As, m1, sp[m2]),
                              tens(P, As, m2, sp[m1]), Dn2 + j * SC, w.y, w);
          double num = dot_blk<R>(w.y, Rr, n, w);
          strip2_left_step<R>(P, k, L2j, U + j * SC, tens(P, As, m1, sp[m1]),
                              tens(P, As, m2, sp[m2]), Dn2 + j * SC, out, w);
          double den = dot_blk<R>(out, Rr, n, w);
          double r = num / den;
          u32x4 ctr = {(uint32_t)(L * (L - 1) + i * L + j), sweep, chain, 1u};
          double u = uniform53(philox_word64(philox4x32_10(ctr, k0, k1)));
          if (!isfinite(r) && threadIdx.x == 0) atomicOr(w.flags, 1);
          if (u < r * r) {
            for (int o = threadIdx.x; o < n; o += blockDim.x) out[o] = w.y[o];
            __syncthreads();
            if (threadIdx.x == 0) {
              uint8_t tmp = sp[m1]; sp[m1] = sp[m2]; sp[m2] = tmp;
              sh.count++;
            }
            __syncthreads();
          }
        } else {
          strip2_left_step<R>(P, k, L2j, U + j * SC, tens(P, As, m1, sp[m1]),
                              tens(P, As, m2, sp[m2]), Dn2 + j * SC, out, w);
        }
        normalize_pow2<R>(out, env2_size(P, Ud, Dd2, j + 1), w.red);
      }
      PEPS_TOC(t_v, PH_SWEEP_2);
      // ---- absorb the updated row i into the upper environment -----------
      int unext = (ucur == 1) ? 2 : 1;
      compress_row<R>(P, steps[i], true, i, As, sp, U, 0.0,
                      w.up + (int64_t)unext * P.env_cap, w);
      ucur = unext;
    }
  }
  __syncthreads();
  return sh.count;
}

// Fisher-Yates start of a chain (thread 0) or its given state.
template <class R>
__device__ void load_chain(BlockShared<R>& sh, const uint8_t* state, int64_t c, int N,
                           uint32_t chain, uint32_t k0, uint32_t k1) {
  if (state) {
    for (int m = threadIdx.x; m < N; m += blockDim.x) sh.sp[m] = state[c * N + m];
  } else if (threadIdx.x == 0) {
    for (int m = 0; m < N; ++m) sh.sp[m] = (m < N / 2) ? 0 : 1;
    for (int k = N - 1; k >= 1; --k) {
      u32x4 ctr = {(uint32_t)k, 0u, chain, 0u};
      uint64_t x = philox_word64(philox4x32_10(ctr, k0, k1));
      int j = (int)(x % (uint64_t)(k + 1));
      uint8_t tmp = sh.sp[k]; sh.sp[k] = sh.sp[j]; sh.sp[j] = tmp;
    }
  }
  __syncthreads();
}

template <class R>
__global__ void __launch_bounds__(PEPS_NT, PEPS_MINB) peps_sample_kernel(SampleArgs<R> a) {
  __shared__ BlockShared<R> sh;
  const PepsPlan& P = a.P;
  const int N = P.N;
  Work<R> w = bind_work<R>(P, a.ws, a.wsd, sh, a.flags);
  for (int64_t c = blockIdx.x; c < a.n_chains; c += gridDim.x) {
    const uint32_t chain = (uint32_t)(a.chain_offset + c);
    load_chain<R>(sh, a.state, c, N, chain, a.k0, a.k1);
    const int total = a.n_burn + a.spc * a.n_thin;
    int rec = 0;
    int64_t acc = 0;
    for (int t = 1; t <= total; ++t) {
      const uint32_t sweep = (uint32_t)(a.first_sweep + (uint64_t)(t - 1));
      acc += sweep_one<R>(P, a.steps, a.As, a.k0, a.k1, chain, sweep, sh, w, false);
      if (t > a.n_burn && (t - a.n_burn) % a.n_thin == 0) {
        uint8_t* o = a.out + (c * a.spc + rec) * (int64_t)N;
        for (int m = threadIdx.x; m < N; m += blockDim.x) o[m] = sh.sp[m];
        ++rec;
      }
      __syncthreads();
    }
    if (a.state)
      for (int m = threadIdx.x; m < N; m += blockDim.x) a.state[c * N + m] = sh.sp[m];
    if (threadIdx.x == 0 && a.accepted) a.accepted[c] = acc;
    __syncthreads();
  }
}

// One VMC step per chain: evaluate the chain's configuration (as
// peps_eval_kernel), then one Metropolis sweep (as peps_sample_kernel)
// that reuses the lower environments the evaluation built.
template <class R>
__global__ void __launch_bounds__(PEPS_NT, PEPS_MINB) peps_vmc_kernel(EvalArgs<R> a, SampleArgs<R> s) {
  __shared__ BlockShared<R> sh;
  const PepsPlan& P = a.P;
  const int N = P.N, D4 = P.D4;
  Work<R> w = bind_work<R>(P, a.ws, a.wsd, sh, a.flags);
  double* ps = a.psum + (int64_t)blockIdx.x * (2 * (int64_t)N * 2 * D4 + 1);
  const int64_t PSN = (int64_t)N * 2 * D4;
  for (int64_t o = threadIdx.x; o < 2 * PSN + 1; o += blockDim.x) ps[o] = 0.0;
  __syncthreads();
  for (int64_t c = blockIdx.x; c < a.B; c += gridDim.x) {
    const uint32_t chain = (uint32_t)(s.chain_offset + c);
    load_chain<R>(sh, s.state, c, N, chain, s.k0, s.k1);
    PEPS_TIC(t_ev);
    evaluate_one<R>(a, c, sh, w, ps, false);
    PEPS_TOC(t_ev, PH_EVAL);
    const uint32_t sw = s.sweep_dev ? *s.sweep_dev : (uint32_t)s.first_sweep;
    PEPS_TIC(t_sw);
    const int acc = sweep_one<R>(P, a.steps, a.As, s.k0, s.k1, chain, sw,
                                 sh, w, true);
    PEPS_TOC(t_sw, PH_SWEEP);
    for (int m = threadIdx.x; m < N; m += blockDim.x) s.state[c * N + m] = sh.sp[m];
    if (threadIdx.x == 0 && s.accepted) s.accepted[c] = acc;
    __syncthreads();
  }
}
