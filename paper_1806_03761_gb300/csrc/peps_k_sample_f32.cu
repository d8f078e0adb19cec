// Metropolis sampling kernel, f32 form.
#include "peps_sample.cuh"
#include "peps_launch.h"

cudaError_t peps_launch_sample_f32(const SampleArgs<float>& a, int grid, cudaStream_t st) {
  peps_sample_kernel<float><<<grid, PEPS_NT, 0, st>>>(a);
  return cudaGetLastError();
}
