// Evaluation kernel, double form.
#include "peps_eval.cuh"
#include "peps_launch.h"

cudaError_t peps_launch_eval_f64(const EvalArgs<double>& a, int grid, cudaStream_t st) {
  peps_eval_kernel<double><<<grid, PEPS_NT, 0, st>>>(a);
  return cudaGetLastError();
}
