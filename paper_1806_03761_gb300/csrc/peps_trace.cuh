// peps_trace.cuh -- optional per-phase cycle counters of the fused VMC-step
// kernel (compile-time knob PEPS_PHASES=1, off by default), the counterpart
// of the paper's hardware-counter measurement of its kernels (Sec.
// "Performance Measurement").  Thread 0 of every block adds the clock64()
// cycles of each phase to a device array; peps_phase_cycles() reads and
// clears it.  Phases nest: PH_COMPRESS contains PH_QR, PH_SVD_QR and PH_SVD;
// PH_EVAL and PH_SWEEP contain the phases below them.  Off, the macros
// expand to nothing and the kernels are unchanged.
#pragma once

#ifndef PEPS_PHASES
#define PEPS_PHASES 0
#endif

enum PepsPhase {
  PH_EVAL = 0,     // evaluation of one chain's configuration
  PH_SWEEP,        // one Metropolis sweep
  PH_COMPRESS,     // boundary-MPS compressions (absorption + truncation)
  PH_QR,           // Householder R factors of the QR sweep
  PH_SVD_QR,       // QR of tall bond matrices before their SVD
  PH_SVD,          // truncated SVDs
  PH_STRIP1,       // one-row strip environments (evaluation)
  PH_RATIO_H,      // horizontal flip ratios
  PH_BTENS,        // B tensors (log-derivatives)
  PH_STRIP2,       // two-row strip environments (evaluation)
  PH_RATIO_2,      // vertical and diagonal flip ratios
  PH_SWEEP_1,      // sweep: horizontal moves on the one-row strips
  PH_SWEEP_R2,     // sweep: right environments of the two-row strips
  PH_SWEEP_2,      // sweep: vertical moves on the two-row strips
  PH_N
};

#if PEPS_PHASES
static __device__ unsigned long long g_peps_phase[PH_N];
#define PEPS_TIC(v) const long long v = clock64()
#define PEPS_TOC(v, ph)                                                              \
  do {                                                                               \
    if (threadIdx.x == 0)                                                            \
      atomicAdd(&g_peps_phase[ph], (unsigned long long)(clock64() - (v)));           \
  } while (0)
// host: copy the counters out and clear them; returns PH_N (0 on error)
#define PEPS_PHASE_READER(name)                                                      \
  int name(unsigned long long* out, int n) {                                         \
    unsigned long long h[PH_N];                                                      \
    if (cudaMemcpyFromSymbol(h, g_peps_phase, sizeof(h)) != cudaSuccess) return 0;   \
    for (int i = 0; i < PH_N && i < n; ++i) out[i] = h[i];                           \
    unsigned long long z[PH_N] = {};                                                 \
    if (cudaMemcpyToSymbol(g_peps_phase, z, sizeof(z)) != cudaSuccess) return 0;     \
    return PH_N;                                                                     \
  }
#else
#define PEPS_TIC(v) do {} while (0)
#define PEPS_TOC(v, ph) do {} while (0)
#define PEPS_PHASE_READER(name) \
  int name(unsigned long long*, int) { return 0; }
#endif
