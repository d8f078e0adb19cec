// Fused VMC-step kernel (evaluation + one Metropolis sweep), ff form.
#include "peps_sample.cuh"
#include "peps_launch.h"

cudaError_t peps_launch_vmc_ff(const EvalArgs<ff>& a, const SampleArgs<ff>& s, int grid,
                              cudaStream_t st) {
  peps_vmc_kernel<ff><<<grid, PEPS_NT, 0, st>>>(a, s);
  return cudaGetLastError();
}

PEPS_PHASE_READER(peps_phase_read_ff)
