// Spin-correlation kernel, ff form.
#include "peps_corr.cuh"
#include "peps_launch.h"

cudaError_t peps_launch_corr_ff(const CorrArgs<ff>& a, int grid, cudaStream_t st) {
  peps_corr_kernel<ff><<<grid, PEPS_NT, 0, st>>>(a);
  return cudaGetLastError();
}
