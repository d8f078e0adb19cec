// Host emulation of the CUDA runtime and device built-ins the library's
// kernels use, for CPU tests of the kernel code (tests/_emu.py builds the
// library's translation units against this header with g++).
//
// A kernel launch runs one block at a time; its blockDim.x threads are
// fibers of one host thread, resumed in turn; __syncthreads parks a fiber
// until the whole block has arrived, __syncwarp and the warp shuffles until
// its group of 32 has; __shared__ variables are function-local statics (one
// block runs at a time on a host thread, so one copy per host thread serves
// every block); atomics are std::atomic_ref.
// "Device" memory is host memory: cudaMalloc is malloc, every copy is
// memcpy, streams are synchronous.  FP32 intrinsics are IEEE binary32
// operations (the build uses -ffp-contract=off).
#pragma once
// system headers first: the qualifier macros below would clash with their
// own attribute spellings
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

// ---- qualifiers -------------------------------------------------------------
#define __global__
#define __device__
#define __host__
#define __forceinline__ inline
#define __noinline__ __attribute__((noinline))
#define __shared__ static thread_local
#define __restrict__ __restrict
#define __align__(n) alignas(n)
#define __launch_bounds__(...)

// ---- built-in indices -------------------------------------------------------
struct uint3 { unsigned x, y, z; };
struct dim3 {
  unsigned x, y, z;
  dim3(unsigned a = 1, unsigned b = 1, unsigned c = 1) : x(a), y(b), z(c) {}
};
// set by the scheduler before it resumes a thread; per host thread, so that
// launches from different host threads (the serving loop's worker) do not
// share them
extern thread_local uint3 threadIdx;
extern thread_local uint3 blockIdx;
extern thread_local dim3 blockDim;
extern thread_local dim3 gridDim;

// ---- synchronisation --------------------------------------------------------
// The threads of a block are fibers of one host thread; a barrier parks the
// fiber until every thread it counts has arrived.
struct EmuBarrier {
  long gen;
  int count, n;
};
void emu_wait(EmuBarrier& b);
extern thread_local EmuBarrier emu_block_bar;
extern thread_local EmuBarrier emu_warp_bar[32];
extern thread_local uint64_t emu_slot[32][32];  // per-warp shuffle exchange
extern thread_local int emu_acc;
extern thread_local EmuBarrier emu_named_bar[16];  // bar.sync 1..15, 64 threads

// the kernels' inline-PTX statements (peps_core.cuh): the L1 prefetch is a
// hint (nothing to do), the warp pair's named barrier a 64-thread barrier
#define PEPS_PREFETCH_L1(ptr) ((void)(ptr))
#define PEPS_PAIR_SYNC(p) emu_wait(emu_named_bar[1 + (p)])

inline void __syncthreads() { emu_wait(emu_block_bar); }
inline void __syncwarp(unsigned = 0xffffffffu) { emu_wait(emu_warp_bar[threadIdx.x / 32]); }
inline int __syncthreads_or(int p) {
  __syncthreads();
  if (threadIdx.x == 0) emu_acc = 0;
  __syncthreads();
  if (p) emu_acc = 1;
  __syncthreads();
  return emu_acc;
}
template <class T>
inline T __shfl_xor_sync(unsigned, T v, int o) {
  static_assert(sizeof(T) <= 8, "shuffle of a scalar");
  const unsigned w = threadIdx.x / 32, l = threadIdx.x % 32;
  uint64_t bits = 0;
  std::memcpy(&bits, &v, sizeof(T));
  emu_slot[w][l] = bits;
  emu_wait(emu_warp_bar[w]);
  bits = emu_slot[w][l ^ (unsigned)o];
  emu_wait(emu_warp_bar[w]);
  T r;
  std::memcpy(&r, &bits, sizeof(T));
  return r;
}

// ---- atomics and clocks -----------------------------------------------------
// (atomic also across host threads: two launches may share a flag word)
inline int atomicOr(int* p, int v) { return std::atomic_ref<int>(*p).fetch_or(v); }
inline int atomicAdd(int* p, int v) { return std::atomic_ref<int>(*p).fetch_add(v); }
inline unsigned long long atomicAdd(unsigned long long* p, unsigned long long v) {
  return std::atomic_ref<unsigned long long>(*p).fetch_add(v);
}
// EMU_COUNT_OPS: every FP32 rounding intrinsic and fmaf counts one operation
// in emu_ops, and clock64() returns that count, so that a build with the
// kernels' phase counters (PEPS_PHASES) reports FP32 operations per phase.
// EMU_COUNT_BARRIERS instead: clock64() returns the number of completed
// block-wide barriers (__syncthreads) of the host thread's launches.
extern thread_local unsigned long long emu_ops;
extern thread_local unsigned long long emu_block_barriers;
#ifdef EMU_COUNT_OPS
#define EMU_OP() (++emu_ops)
inline long long clock64() { return (long long)emu_ops; }
#else
#define EMU_OP() ((void)0)
#ifdef EMU_COUNT_BARRIERS
inline long long clock64() { return (long long)emu_block_barriers; }
#else
inline long long clock64() { return 0; }
#endif
#endif

// ---- FP32 intrinsics ----------------------------------------------------------
inline float __fadd_rn(float a, float b) { EMU_OP(); return a + b; }
inline float __fsub_rn(float a, float b) { EMU_OP(); return a - b; }
inline float __fmul_rn(float a, float b) { EMU_OP(); return a * b; }
inline float __fdiv_rn(float a, float b) { EMU_OP(); return a / b; }
inline float __fsqrt_rn(float a) { EMU_OP(); return std::sqrt(a); }
using std::fabs; using std::fma; using std::fmaf; using std::isfinite; using std::sqrt;
using std::exp; using std::log; using std::frexp; using std::ldexp; using std::fmax; using std::fmin;
#ifdef EMU_COUNT_OPS
inline float emu_fmaf(float a, float b, float c) { EMU_OP(); return std::fmaf(a, b, c); }
#define fmaf emu_fmaf
#endif


// ---- runtime ------------------------------------------------------------------
typedef int cudaError_t;
enum : int {
  cudaSuccess = 0, cudaErrorInvalidValue = 1, cudaErrorMemoryAllocation = 2,
  cudaErrorInvalidDevice = 101, cudaErrorNotReady = 600
};
typedef void* cudaStream_t;
typedef void* cudaEvent_t;
enum { cudaStreamNonBlocking = 1, cudaEventDisableTiming = 2 };
enum cudaMemcpyKind {
  cudaMemcpyHostToHost = 0, cudaMemcpyHostToDevice = 1, cudaMemcpyDeviceToHost = 2,
  cudaMemcpyDeviceToDevice = 3, cudaMemcpyDefault = 4
};
enum cudaDeviceAttr { cudaDevAttrMultiProcessorCount = 16 };

// SMs the emulated device reports (the default slot count scales with it)
#ifndef EMU_SMS
#define EMU_SMS 2
#endif

inline cudaError_t cudaMalloc(void** p, size_t n) {
  *p = std::calloc(n ? n : 1, 1);
  return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}
template <class T> inline cudaError_t cudaMalloc(T** p, size_t n) {
  return cudaMalloc(reinterpret_cast<void**>(p), n);
}
inline cudaError_t cudaFree(void* p) { std::free(p); return cudaSuccess; }
inline cudaError_t cudaMemcpy(void* d, const void* s, size_t n, cudaMemcpyKind) {
  if (n) std::memmove(d, s, n);
  return cudaSuccess;
}
inline cudaError_t cudaMemcpyAsync(void* d, const void* s, size_t n, cudaMemcpyKind k, cudaStream_t = nullptr) {
  return cudaMemcpy(d, s, n, k);
}
inline cudaError_t cudaMemset(void* d, int v, size_t n) { std::memset(d, v, n); return cudaSuccess; }
inline cudaError_t cudaMemsetAsync(void* d, int v, size_t n, cudaStream_t = nullptr) {
  return cudaMemset(d, v, n);
}
inline cudaError_t cudaStreamSynchronize(cudaStream_t) { return cudaSuccess; }
// streams and events: every operation is complete when its call returns
inline cudaError_t cudaStreamCreateWithFlags(cudaStream_t* s, unsigned) {
  *s = reinterpret_cast<cudaStream_t>(new char(0));
  return cudaSuccess;
}
inline cudaError_t cudaStreamDestroy(cudaStream_t s) { delete static_cast<char*>(s); return cudaSuccess; }
inline cudaError_t cudaEventCreateWithFlags(cudaEvent_t* e, unsigned) {
  *e = reinterpret_cast<cudaEvent_t>(new char(0));
  return cudaSuccess;
}
inline cudaError_t cudaEventDestroy(cudaEvent_t e) { delete static_cast<char*>(e); return cudaSuccess; }
inline cudaError_t cudaEventRecord(cudaEvent_t, cudaStream_t = nullptr) { return cudaSuccess; }
inline cudaError_t cudaEventQuery(cudaEvent_t) { return cudaSuccess; }
inline cudaError_t cudaMallocAsync(void** p, size_t n, cudaStream_t) { return cudaMalloc(p, n); }
inline cudaError_t cudaFreeAsync(void* p, cudaStream_t) { return cudaFree(p); }
// the emulated device's memory (the serving loop's default budget is 90 % of
// the free part)
#ifndef EMU_MEM_BYTES
#define EMU_MEM_BYTES (8ull << 30)
#endif
template <class T> inline cudaError_t cudaMemcpyFromSymbol(void* dst, const T& sym, size_t n) {
  std::memcpy(dst, &sym, n);
  return cudaSuccess;
}
template <class T> inline cudaError_t cudaMemcpyToSymbol(T& sym, const void* src, size_t n) {
  std::memcpy(&sym, src, n);
  return cudaSuccess;
}
inline cudaError_t cudaMemGetInfo(size_t* free_b, size_t* total_b) {
  *free_b = EMU_MEM_BYTES;
  *total_b = EMU_MEM_BYTES;
  return cudaSuccess;
}
inline cudaError_t cudaGetLastError() { return cudaSuccess; }
inline const char* cudaGetErrorString(cudaError_t) { return "emulated CUDA error"; }
inline cudaError_t cudaGetDevice(int* d) { *d = 0; return cudaSuccess; }
inline cudaError_t cudaSetDevice(int) { return cudaSuccess; }
inline cudaError_t cudaDeviceGetAttribute(int* v, cudaDeviceAttr, int) { *v = EMU_SMS; return cudaSuccess; }

// ---- launches -------------------------------------------------------------------
// Runs body() on every thread of every block of the grid; aborts with a
// message when a barrier can never complete (a thread missed it).
void emu_launch(dim3 grid, dim3 block, const std::function<void()>& body);
