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

template <class R>
__global__ void __launch_bounds__(PEPS_NT) peps_sample_kernel(SampleArgs<R> a) {
  __shared__ double red[PEPS_NT];
  __shared__ __align__(16) unsigned char redR_raw[PEPS_NT * sizeof(R)];
  __shared__ __align__(16) unsigned char wsh_raw[256 * sizeof(R)];
  __shared__ double rot[512];
  __shared__ int ish[264];
  __shared__ uint8_t sp[PEPS_MAXL * PEPS_MAXL];
  __shared__ double dnlog[PEPS_MAXL + 1];
  __shared__ int acc_sh;
  const PepsPlan& P = a.P;
  const int L = P.L, N = P.N;
  const int64_t SC = P.site_cap, EC = P.env2_cap;
  Work<R> w = make_work<R>(P, a.ws, a.wsd, blockIdx.x);
  w.red = red;
  w.redR = reinterpret_cast<R*>(redR_raw);
  w.wsh = reinterpret_cast<R*>(wsh_raw);
  w.rot = rot;
  w.ish = ish;
  w.flags = a.flags;
  for (int64_t c = blockIdx.x; c < a.n_chains; c += gridDim.x) {
    const uint32_t chain = (uint32_t)(a.chain_offset + c);
    if (a.state) {
      for (int m = threadIdx.x; m < N; m += blockDim.x) sp[m] = a.state[c * N + m];
    } else if (threadIdx.x == 0) {
      // Fisher-Yates shuffle of floor(N/2) up spins
      for (int m = 0; m < N; ++m) sp[m] = (m < N / 2) ? 0 : 1;
      for (int k = N - 1; k >= 1; --k) {
        u32x4 ctr = {(uint32_t)k, 0u, chain, 0u};
        uint64_t x = philox_word64(philox4x32_10(ctr, a.k0, a.k1));
        int j = (int)(x % (uint64_t)(k + 1));
        uint8_t tmp = sp[k]; sp[k] = sp[j]; sp[j] = tmp;
      }
    }
    if (threadIdx.x == 0) acc_sh = 0;
    __syncthreads();
    const int total = a.n_burn + a.spc * a.n_thin;
    int rec = 0;
    for (int t = 1; t <= total; ++t) {
      const uint32_t sweep = (uint32_t)(a.first_sweep + (uint64_t)(t - 1));
      build_lower<R>(P, a.steps, a.As, sp, w, dnlog);
      set_trivial<R>(P, w.up);
      int ucur = 0;
      for (int i = 0; i < L; ++i) {
        const R* U = w.up + (int64_t)ucur * P.env_cap;
        EnvDims Ud = env_dims(P, a.steps, i - 1);
        const R* Dn = w.dn + (int64_t)(i + 1) * P.env_cap;
        EnvDims Dd = env_dims(P, a.steps, (i + 1 <= L - 1) ? (L - 2 - i) : -1);
        // ---- horizontal moves on the one-row strip --------------------
        strip1_right_all<R>(P, i, sp, a.As, U, Ud, Dn, Dd, w);
        if (threadIdx.x == 0) w.l1[0] = Arith<R>::one();
        __syncthreads();
        for (int j = 0; j + 1 < L; ++j) {
          int m = i * L + j;
          if (sp[m] != sp[m + 1]) {
            Col1 k0 = col_dims(P, Ud, Dd, j), k1 = col_dims(P, Ud, Dd, j + 1);
            int n = env1_size(P, Ud, Dd, j + 2);
            const R* Rr = w.r1 + (int64_t)(j + 2) * SC;
            const R* Lj = w.l1 + (int64_t)j * SC;
            strip1_left_step<R>(P, k0, Lj, U + j * SC, tens(P, a.As, m, sp[m + 1]), Dn + j * SC, w.y, w);
            strip1_left_step<R>(P, k1, w.y, U + (j + 1) * SC, tens(P, a.As, m + 1, sp[m]), Dn + (j + 1) * SC, w.xj, w);
            double num = dot_blk<R>(w.xj, Rr, n, w);
            strip1_left_step<R>(P, k0, Lj, U + j * SC, tens(P, a.As, m, sp[m]), Dn + j * SC, w.y, w);
            strip1_left_step<R>(P, k1, w.y, U + (j + 1) * SC, tens(P, a.As, m + 1, sp[m + 1]), Dn + (j + 1) * SC, w.xj, w);
            double den = dot_blk<R>(w.xj, Rr, n, w);
            double r = num / den;
            u32x4 ctr = {(uint32_t)(i * (L - 1) + j), sweep, chain, 1u};
            double u = uniform53(philox_word64(philox4x32_10(ctr, a.k0, a.k1)));
            if (!isfinite(r) && threadIdx.x == 0) atomicOr(a.flags, 1);
            if (u < r * r) {
              __syncthreads();
              if (threadIdx.x == 0) {
                uint8_t tmp = sp[m]; sp[m] = sp[m + 1]; sp[m + 1] = tmp;
                acc_sh++;
              }
              __syncthreads();
            }
          }
          // advance the left environment over column j with the current spins
          Col1 k = col_dims(P, Ud, Dd, j);
          R* out = w.l1 + (int64_t)(j + 1) * SC;
          strip1_left_step<R>(P, k, w.l1 + (int64_t)j * SC, U + j * SC, tens(P, a.As, m, sp[m]), Dn + j * SC, out, w);
          normalize_pow2<R>(out, env1_size(P, Ud, Dd, j + 1), w.red);
        }
        if (i + 1 < L) {
          // ---- vertical moves on the two-row strip ---------------------
          const R* Dn2 = w.dn + (int64_t)(i + 2) * P.env_cap;
          EnvDims Dd2 = env_dims(P, a.steps, (i + 2 <= L - 1) ? (L - 3 - i) : -1);
          strip2_right_all<R>(P, i, sp, a.As, U, Ud, Dn2, Dd2, w);
          if (threadIdx.x == 0) w.l2[0] = Arith<R>::one();
          __syncthreads();
          for (int j = 0; j < L; ++j) {
            int m1 = i * L + j, m2 = m1 + L;
            Col1 k = col_dims(P, Ud, Dd2, j);
            const R* L2j = w.l2 + (int64_t)j * EC;
            if (sp[m1] != sp[m2]) {
              int n = env2_size(P, Ud, Dd2, j + 1);
              const R* Rr = w.r2 + (int64_t)(j + 1) * EC;
              strip2_left_step<R>(P, k, L2j, U + j * SC, tens(P, a.As, m1, sp[m2]),
                                  tens(P, a.As, m2, sp[m1]), Dn2 + j * SC, w.y, w);
              double num = dot_blk<R>(w.y, Rr, n, w);
              strip2_left_step<R>(P, k, L2j, U + j * SC, tens(P, a.As, m1, sp[m1]),
                                  tens(P, a.As, m2, sp[m2]), Dn2 + j * SC, w.y, w);
              double den = dot_blk<R>(w.y, Rr, n, w);
              double r = num / den;
              u32x4 ctr = {(uint32_t)(L * (L - 1) + i * L + j), sweep, chain, 1u};
              double u = uniform53(philox_word64(philox4x32_10(ctr, a.k0, a.k1)));
              if (!isfinite(r) && threadIdx.x == 0) atomicOr(a.flags, 1);
              if (u < r * r) {
                __syncthreads();
                if (threadIdx.x == 0) {
                  uint8_t tmp = sp[m1]; sp[m1] = sp[m2]; sp[m2] = tmp;
                  acc_sh++;
                }
                __syncthreads();
              }
            }
            R* out = w.l2 + (int64_t)(j + 1) * EC;
            strip2_left_step<R>(P, k, L2j, U + j * SC, tens(P, a.As, m1, sp[m1]),
                                tens(P, a.As, m2, sp[m2]), Dn2 + j * SC, out, w);
            normalize_pow2<R>(out, env2_size(P, Ud, Dd2, j + 1), w.red);
          }
          // ---- absorb the updated row i into the upper environment -----
          int unext = (ucur == 1) ? 2 : 1;
          compress_row<R>(P, a.steps[i], true, i, a.As, sp, U, 0.0,
                          w.up + (int64_t)unext * P.env_cap, w);
          ucur = unext;
        }
      }
      if (t > a.n_burn && (t - a.n_burn) % a.n_thin == 0) {
        uint8_t* o = a.out + (c * a.spc + rec) * (int64_t)N;
        for (int m = threadIdx.x; m < N; m += blockDim.x) o[m] = sp[m];
        ++rec;
      }
      __syncthreads();
    }
    if (a.state)
      for (int m = threadIdx.x; m < N; m += blockDim.x) a.state[c * N + m] = sp[m];
    if (threadIdx.x == 0 && a.accepted) a.accepted[c] = acc_sh;
    __syncthreads();
  }
}
