// Multi-job evaluation kernel, ff form.
#include "peps_multi.cuh"
#include "peps_launch.h"

cudaError_t peps_launch_multi_ff(const MultiJobDev<ff>* jobs, int n_jobs, int64_t n_items,
                                  unsigned long long* next, ff* ws, double* wsd,
                                  int64_t slot_elems, int64_t slot_doubles, int* flags, int grid,
                                  cudaStream_t st) {
  peps_multi_kernel<ff><<<grid, PEPS_NT, 0, st>>>(jobs, n_jobs, n_items, next, ws, wsd, slot_elems,
                                                  slot_doubles, flags);
  return cudaGetLastError();
}
