// Spin-correlation kernel, f64 form.
#include "peps_corr.cuh"
#include "peps_launch.h"

cudaError_t peps_launch_corr_f64(const CorrArgs<double>& a, int grid, cudaStream_t st) {
  peps_corr_kernel<double><<<grid, PEPS_NT, 0, st>>>(a);
  return cudaGetLastError();
}
