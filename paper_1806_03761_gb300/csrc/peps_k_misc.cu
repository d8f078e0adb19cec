// Small kernels: slot-sum reduction, tensor conversion, GO update.
#include "peps_eval.cuh"
#include "peps_launch.h"
#include "../../include/peps.h"

// sums[k] (+)= sum over slots of the slot partial sums (fixed order)
__global__ void peps_reduce_slots(const double* psum, int nslots, int64_t len,
                                  double* sd, double* sde, double* se, int accumulate) {
  const int64_t stride = len;
  const int64_t half = (len - 1) / 2;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < nslots; ++q) s += psum[(int64_t)q * stride + k];
    double* dst = (k < half) ? sd + k : (k < 2 * half ? sde + (k - half) : se);
    *dst = accumulate ? *dst + s : s;
  }
}

cudaError_t peps_launch_reduce(const double* psum, int nslots, int64_t len, double* sd,
                               double* sde, double* se, int accumulate, cudaStream_t st) {
  int rg = (int)((len + 255) / 256 < 4096 ? (len + 255) / 256 : 4096);
  peps_reduce_slots<<<rg, 256, 0, st>>>(psum, nslots, len, sd, sde, se, accumulate);
  return cudaGetLastError();
}

cudaError_t peps_launch_convert(int precision, const double* A, void* As, int64_t n, int* flags,
                                cudaStream_t st) {
  int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  if (precision == PEPS_FP64)
    peps_convert_kernel<double><<<grid, 256, 0, st>>>(A, static_cast<double*>(As), n, flags);
  else if (precision == PEPS_FP32)
    peps_convert_kernel<float><<<grid, 256, 0, st>>>(A, static_cast<float*>(As), n, flags);
  else
    peps_convert_kernel<ff><<<grid, 256, 0, st>>>(A, static_cast<ff*>(As), n, flags);
  return cudaGetLastError();
}

cudaError_t peps_launch_grad(int precision, const double* sd, const double* sde, const double* se,
                             double M, double dt, uint32_t k0, uint32_t k1, uint32_t step,
                             const uint32_t* step_dev, double* A, void* As, int64_t n,
                             cudaStream_t st) {
  int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  if (precision == PEPS_FP64)
    peps_grad_kernel<double><<<grid, 256, 0, st>>>(sd, sde, se, M, dt, k0, k1, step, step_dev, A,
                                                   static_cast<double*>(As), n);
  else if (precision == PEPS_FP32)
    peps_grad_kernel<float><<<grid, 256, 0, st>>>(sd, sde, se, M, dt, k0, k1, step, step_dev, A,
                                                  static_cast<float*>(As), n);
  else
    peps_grad_kernel<ff><<<grid, 256, 0, st>>>(sd, sde, se, M, dt, k0, k1, step, step_dev, A,
                                               static_cast<ff*>(As), n);
  return cudaGetLastError();
}

// mean[k] = (1/B) sum_b ss[b][k], b in order (bit-reproducible)
__global__ void peps_corr_mean(const double* ss, int64_t B, int64_t len, double* mean) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t b = 0; b < B; ++b) s += ss[b * len + k];
    mean[k] = s / (double)B;
  }
}

cudaError_t peps_launch_corr_mean(const double* ss, int64_t B, int64_t len, double* mean,
                                  cudaStream_t st) {
  int grid = (int)((len + 255) / 256 < 4096 ? (len + 255) / 256 : 4096);
  peps_corr_mean<<<grid, 256, 0, st>>>(ss, B, len, mean);
  return cudaGetLastError();
}

// m_s^2(k) = (1/n^2) sum_{a, m in bulk} C[pos[a]][m] cos(k . (r_a - r_m)): one
// block, each thread a fixed set of (a, m) pairs, then a fixed-order tree.
__global__ void peps_structure_factor_kernel(const double* mean, int L, int N, const int32_t* pos,
                                             int nbulk, const int32_t* bulk, double kx, double ky,
                                             double* out) {
  __shared__ double red[256];
  double s = 0.0;
  const int64_t pairs = (int64_t)nbulk * nbulk;
  for (int64_t t = threadIdx.x; t < pairs; t += blockDim.x) {
    const int a = bulk[t / nbulk], m = bulk[t % nbulk];
    const int ia = a / L, ja = a % L, im = m / L, jm = m % L;
    s += mean[(int64_t)pos[t / nbulk] * N + m] * cos(kx * (ia - im) + ky * (ja - jm));
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] / ((double)nbulk * (double)nbulk);
}

cudaError_t peps_launch_structure_factor(const double* mean, int L, int N, const int32_t* pos,
                                         int nbulk, const int32_t* bulk, double kx, double ky,
                                         double* out, cudaStream_t st) {
  peps_structure_factor_kernel<<<1, 256, 0, st>>>(mean, L, N, pos, nbulk, bulk, kx, ky, out);
  return cudaGetLastError();
}

// counters[i] += inc (one thread): advances the device-resident sweep and
// step numbers between replays of a captured VMC step
__global__ void peps_counters_add(uint32_t* c, int n, uint32_t inc) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    for (int i = 0; i < n; ++i) c[i] += inc;
}

cudaError_t peps_launch_counters(uint32_t* c, int n, uint32_t inc, cudaStream_t st) {
  peps_counters_add<<<1, 32, 0, st>>>(c, n, inc);
  return cudaGetLastError();
}
