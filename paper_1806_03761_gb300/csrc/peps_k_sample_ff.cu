// Metropolis sampling kernel, ff form.
#include "peps_sample.cuh"
#include "peps_launch.h"

cudaError_t peps_launch_sample_ff(const SampleArgs<ff>& a, int grid, cudaStream_t st) {
  peps_sample_kernel<ff><<<grid, PEPS_NT, 0, st>>>(a);
  return cudaGetLastError();
}
