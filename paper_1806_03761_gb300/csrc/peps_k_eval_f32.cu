// Evaluation kernel, FP32 form.
#include "peps_eval.cuh"
#include "peps_launch.h"

cudaError_t peps_launch_eval_f32(const EvalArgs<float>& a, int grid, cudaStream_t st) {
  peps_eval_kernel<float><<<grid, PEPS_NT, 0, st>>>(a);
  return cudaGetLastError();
}
