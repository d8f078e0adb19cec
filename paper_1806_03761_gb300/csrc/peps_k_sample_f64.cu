// Metropolis sampling kernel, f64 form.
#include "peps_sample.cuh"
#include "peps_launch.h"

cudaError_t peps_launch_sample_f64(const SampleArgs<double>& a, int grid, cudaStream_t st) {
  peps_sample_kernel<double><<<grid, PEPS_NT, 0, st>>>(a);
  return cudaGetLastError();
}
