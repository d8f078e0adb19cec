// Fused VMC-step kernel (evaluation + one Metropolis sweep), f64 form.
#include "peps_sample.cuh"
#include "peps_launch.h"

cudaError_t peps_launch_vmc_f64(const EvalArgs<double>& a, const SampleArgs<double>& s, int grid,
                              cudaStream_t st) {
  peps_vmc_kernel<double><<<grid, PEPS_NT, 0, st>>>(a, s);
  return cudaGetLastError();
}

PEPS_PHASE_READER(peps_phase_read_f64)
