// peps_launch.h -- host-side launchers of the kernels, one translation unit
// per kernel family and form so that the library compiles in parallel.
#pragma once
#include <cuda_runtime.h>
#include "peps_arith.cuh"
#include "peps_plan.h"

template <class R> struct EvalArgs;
template <class R> struct SampleArgs;
template <class R> struct CorrArgs;
template <class R> struct MultiJobDev;

cudaError_t peps_launch_eval_f64(const EvalArgs<double>& a, int grid, cudaStream_t st);
cudaError_t peps_launch_eval_ff(const EvalArgs<ff>& a, int grid, cudaStream_t st);
cudaError_t peps_launch_eval_f32(const EvalArgs<float>& a, int grid, cudaStream_t st);
cudaError_t peps_launch_sample_f64(const SampleArgs<double>& a, int grid, cudaStream_t st);
cudaError_t peps_launch_sample_ff(const SampleArgs<ff>& a, int grid, cudaStream_t st);
cudaError_t peps_launch_sample_f32(const SampleArgs<float>& a, int grid, cudaStream_t st);
cudaError_t peps_launch_vmc_f64(const EvalArgs<double>& a, const SampleArgs<double>& s, int grid, cudaStream_t st);
cudaError_t peps_launch_vmc_ff(const EvalArgs<ff>& a, const SampleArgs<ff>& s, int grid, cudaStream_t st);
cudaError_t peps_launch_vmc_f32(const EvalArgs<float>& a, const SampleArgs<float>& s, int grid, cudaStream_t st);
// per-phase cycle counters of the fused kernel (PEPS_PHASES builds; else 0)
int peps_phase_read_f64(unsigned long long* out, int n);
int peps_phase_read_ff(unsigned long long* out, int n);
int peps_phase_read_f32(unsigned long long* out, int n);
cudaError_t peps_launch_reduce(const double* psum, int nslots, int64_t len, double* sd,
                               double* sde, double* se, int accumulate, cudaStream_t st);
cudaError_t peps_launch_convert(int precision, const double* A, void* As, int64_t n, int* flags,
                                cudaStream_t st);
cudaError_t peps_launch_grad(int precision, const double* sd, const double* sde, const double* se,
                             double M, double dt, uint32_t k0, uint32_t k1, uint32_t step,
                             const uint32_t* step_dev, double* A, void* As, int64_t n,
                             cudaStream_t st);
cudaError_t peps_launch_counters(uint32_t* c, int n, uint32_t inc, cudaStream_t st);
cudaError_t peps_launch_corr_f64(const CorrArgs<double>& a, int grid, cudaStream_t st);
cudaError_t peps_launch_corr_ff(const CorrArgs<ff>& a, int grid, cudaStream_t st);
cudaError_t peps_launch_corr_mean(const double* ss, int64_t B, int64_t len, double* mean,
                                  cudaStream_t st);
cudaError_t peps_launch_structure_factor(const double* mean, int L, int N, const int32_t* pos,
                                         int nbulk, const int32_t* bulk, double kx, double ky,
                                         double* out, cudaStream_t st);
cudaError_t peps_launch_multi_f64(const MultiJobDev<double>* jobs, int n_jobs, int64_t n_items,
                                  unsigned long long* next, double* ws, double* wsd,
                                  int64_t slot_elems, int64_t slot_doubles, int* flags, int grid,
                                  cudaStream_t st);
cudaError_t peps_launch_multi_ff(const MultiJobDev<ff>* jobs, int n_jobs, int64_t n_items,
                                 unsigned long long* next, ff* ws, double* wsd,
                                 int64_t slot_elems, int64_t slot_doubles, int* flags, int grid,
                                 cudaStream_t st);
