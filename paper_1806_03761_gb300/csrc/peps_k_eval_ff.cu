// Evaluation kernel, ff form.
#include "peps_eval.cuh"
#include "peps_launch.h"

cudaError_t peps_launch_eval_ff(const EvalArgs<ff>& a, int grid, cudaStream_t st) {
  peps_eval_kernel<ff><<<grid, PEPS_NT, 0, st>>>(a);
  return cudaGetLastError();
}
