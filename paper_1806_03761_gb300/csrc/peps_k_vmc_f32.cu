// Fused VMC-step kernel (evaluation + one Metropolis sweep), f32 form.
#include "peps_sample.cuh"
#include "peps_launch.h"

cudaError_t peps_launch_vmc_f32(const EvalArgs<float>& a, const SampleArgs<float>& s, int grid,
                              cudaStream_t st) {
  peps_vmc_kernel<float><<<grid, PEPS_NT, 0, st>>>(a, s);
  return cudaGetLastError();
}

PEPS_PHASE_READER(peps_phase_read_f32)
