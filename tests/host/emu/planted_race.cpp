// A kernel with a planted race, for the test that the emulation's schedule
// orders expose one: each thread writes its slot of a block-shared array and
// reads its neighbour's, with or without a barrier in between.
#include "cuda_runtime.h"

static void neighbour_kernel(int* out, int with_barrier) {
  __shared__ int buf[64];
  buf[threadIdx.x] = (int)threadIdx.x + 1;
  if (with_barrier) __syncthreads();
  out[threadIdx.x] = buf[(threadIdx.x + 1) % blockDim.x];
  __syncthreads();
  buf[threadIdx.x] = 0;
}

extern "C" void planted_race(int* out, int with_barrier) {
  emu_launch(dim3(1), dim3(64), [=]() { neighbour_kernel(out, with_barrier); });
}
