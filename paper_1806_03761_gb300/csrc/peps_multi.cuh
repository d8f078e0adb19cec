// peps_multi.cuh -- one persistent launch over the samples of several jobs of
// different lattice sizes and bond dimensions (one precision form): local
// energies, amplitudes and flip ratios of every sample (PEPS++,
// arXiv:1806.03761, Eq. ess; Fig. "contraction", Steps 4-5), the per-sample
// path of peps_eval_kernel unchanged.
//
// Work queue: the items are (job, sample) pairs numbered job by job; a block
// claims the next item with one atomic add, loads that job's arguments into
// shared memory, binds its slot of the pool with the job's layout, and
// evaluates the sample.  Blocks that finish cheap items take the next ones,
// so items of very different cost share the SMs without waves.
#pragma once
#include "peps_eval.cuh"

// The scratch of one sample at explicit bases (the pool's slot stride is the
// largest layout among the jobs, the offsets are the job's own).
template <class R>
__device__ Work<R> make_work_at(const PepsPlan& P, R* base, double* bd) {
  Work<R> w;
  w.qrv = nullptr;
  w.dn = base + P.off_dn;  w.up = base + P.off_up;  w.rst = base + P.off_rst;
  w.b0 = base + P.off_b0;  w.b1 = base + P.off_b1;  w.b2 = base + P.off_b2;
  w.y = base + P.off_y;    w.xj = base + P.off_xj;  w.vt = base + P.off_vt;
  w.c0 = base + P.off_c0;  w.c1 = base + P.off_c1;  w.l1 = base + P.off_l1;
  w.r1 = base + P.off_r1;  w.l2 = base + P.off_l2;  w.r2 = base + P.off_r2;
  w.scl = bd + P.doff_scale;  w.delta = bd + P.doff_delta;
  w.alpha = base + P.off_alpha;  w.inv = base + P.off_inv;
  w.dnf = base + P.off_dnf;  w.upf = base + P.off_upf;
  return w;
}

template <class R>
__global__ void __launch_bounds__(PEPS_NT, PEPS_MINB)
peps_multi_kernel(const MultiJobDev<R>* jobs, int n_jobs, int64_t n_items,
                  unsigned long long* next, R* ws, double* wsd, int64_t slot_elems,
                  int64_t slot_doubles, int* flags) {
  __shared__ BlockShared<R> sh;
  __shared__ EvalArgs<R> ja;
  __shared__ long long item;
  __shared__ int job;
  R* base = ws + (int64_t)blockIdx.x * slot_elems;
  double* bd = wsd + (int64_t)blockIdx.x * slot_doubles;
  for (;;) {
    if (threadIdx.x == 0) {
      item = (long long)atomicAdd(next, 1ull);
      int j = 0;
      if (item < n_items)
        while (j + 1 < n_jobs && jobs[j + 1].first_item <= item) ++j;
      job = j;
    }
    __syncthreads();
    const long long it = item;
    if (it >= n_items) break;
    // the job's arguments into shared memory (as 32-bit words)
    const int nw = (int)(sizeof(EvalArgs<R>) / 4);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&jobs[job].a);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&ja);
    for (int q = threadIdx.x; q < nw; q += blockDim.x) dst[q] = src[q];
    __syncthreads();
    const int64_t b = it - jobs[job].first_item;
    Work<R> w = make_work_at<R>(ja.P, base, bd);
    w.red = sh.red;
    w.redR = reinterpret_cast<R*>(sh.redR_raw);
    w.wsh = reinterpret_cast<R*>(sh.wsh_raw);
    w.qrv = reinterpret_cast<R*>(sh.qrv_raw);
    w.rot = sh.rot;
    w.flags = flags;
    const int N = ja.P.N;
    for (int m = threadIdx.x; m < N; m += blockDim.x) sh.sp[m] = ja.spins[b * N + m];
    __syncthreads();
    evaluate_one<R>(ja, b, sh, w, nullptr, false);
    __syncthreads();
  }
}
