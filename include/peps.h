/*
 * peps.h -- C ABI of the GB300 (sm_103a) per-sample PEPS contraction library
 * (libpeps.so): the data-parallel hot path of PEPS++ (He et al.,
 * arXiv:1806.03761) for the open-boundary J1-J2 spin-1/2 model.
 *
 * For every sampled spin configuration S the library contracts the
 * single-layer network a PEPS forms once each site's physical index is fixed
 * (Eq. PEPS; Fig. 1(b)), row by row as a boundary MPS truncated to bond D_c
 * (Fig. 1(c); Sec. "PEPS++ Algorithm"), and reuses the cached upper, lower,
 * left and right environments (Fig. "contraction", Step 4) for the amplitude
 * W(S), every J1 and J2 flip ratio of the local energy E(S) (Eq. ess), the
 * log-derivatives Delta = dlnW/dA (Eq. delta) and their sums for the energy
 * gradient (Eq. gradients), and for the sign-gradient update of the GO step.
 *
 * Conventions (every entry point):
 *   - L x L open square lattice, N = L*L sites, site m = i*L + j, row 0 on top.
 *   - Site tensors A: float64[N][2][D][D][D][D], axes (s, l, r, u, d), C order.
 *     Outward legs of boundary sites use index 0 only (open boundary).
 *   - Spins: uint8[B][N], s = 0 spin up (sigma = +1), s = 1 spin down.
 *   - Canonical bond order (n_bonds = 2L(L-1) + 2(L-1)^2): horizontal J1
 *     (i,j)-(i,j+1) row-major; vertical J1 (i,j)-(i+1,j); diagonal J2
 *     (i,j)-(i+1,j+1); anti-diagonal J2 (i,j+1)-(i+1,j).
 *   - All array arguments are DEVICE pointers owned by the caller, unless a
 *     comment says "host".  The library owns its workspace (environments,
 *     scratch) inside the opaque context.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls only
 *     enqueue work on it and return; results are ready when the stream is.
 *   - Return value: PEPS_OK or a negative PEPS_E* code; peps_last_error()
 *     gives a message.  No C++ exception crosses this ABI.  Errors found on the
 *     device (non-finite input, zero amplitude) are
 *     recorded in the context and returned by peps_sync_status().
 *   - One context per host thread at a time; calls on one context must not
 *     overlap on the device (they share the context's workspace).
 */
#ifndef PEPS_GB300_H
#define PEPS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  PEPS_OK = 0,
  PEPS_EINVAL = -1,   /* bad argument (NULL, size, alignment, shape) */
  PEPS_ENOMEM = -2,   /* device allocation failed */
  PEPS_ECUDA = -3,    /* CUDA runtime error (launch, copy, no device) */
  PEPS_ENUMERIC = -4, /* non-finite input or zero amplitude */
  PEPS_ETIMEOUT = -5, /* a bounded device wait ran out */
  PEPS_ESCRATCH = -6  /* peps_amplitudes_noalloc: the shape does not fit the
                         fixed device scratch */
};

enum {
  PEPS_FP64 = 0,  /* every contraction and factorisation in FP64 */
  PEPS_MIXED = 1, /* tensors, contractions and the QR/SVD truncation in
                     float-float (a pair of FP32 numbers, about 48
                     significand bits) on the FP32 pipes; log-scales, flip
                     ratios, energies and the Delta and gradient sums in FP64 */
  PEPS_FP32 = 2   /* tensors, contractions and truncation in plain FP32,
                     scalars as PEPS_MIXED.  Diagnostic form: its error grows
                     with the cancellation in W(S) and is not held to the
                     1e-4 tolerance */
};

/* Device-side error bits reported by peps_sync_status() through *flags. */
enum {
  PEPS_FLAG_NONFINITE = 1,   /* NaN/Inf met in a tensor or ratio */
  PEPS_FLAG_ZERO_AMP = 2,    /* W(S) = 0 for some sample (its sign is 0) */
  PEPS_FLAG_NO_CONVERGE = 4  /* reserved */
};

typedef struct peps_ctx peps_ctx;

typedef struct {
  int32_t L;          /* lattice side, 2 <= L <= 32 */
  int32_t D;          /* PEPS bond dimension, 1 <= D <= 8 */
  int32_t Dc;         /* boundary-MPS truncation D_c, 1 <= Dc, Dc*D <= 256 */
  double J1, J2;      /* couplings of the J1-J2 Hamiltonian (Sec. Experiment
                         Setup; the paper sets J1 = 1) */
  int32_t precision;  /* PEPS_FP64, PEPS_MIXED or PEPS_FP32 */
} peps_shape;

/* Create a context on the current CUDA device.  workspace_slots = number of
 * samples processed concurrently (0 = 2 per SM); the workspace
 * (about slots x 8 (L*L*Dc*D*Dc + ...) bytes, see peps_workspace_bytes) is
 * allocated here with cudaMalloc.  EINVAL on a bad shape, ENOMEM if the
 * workspace does not fit. */
int peps_create(const peps_shape* shape, int32_t workspace_slots,
                peps_ctx** out);
int peps_destroy(peps_ctx* ctx);
const char* peps_last_error(const peps_ctx* ctx);
/* Bytes of device workspace a context with this shape and slot count holds
 * (host call, no allocation). */
size_t peps_workspace_bytes(const peps_shape* shape, int32_t workspace_slots);
/* Number of workspace slots of a context (the persistent kernels' grid):
 * samples are processed in waves of this many.  Host call; EINVAL on a null
 * argument. */
int peps_slots(const peps_ctx* ctx, int32_t* slots);

/* Copy the site tensors A (float64[N][2][D^4], device) into the context
 * (converting to the context's precision).  Must precede every evaluation.
 * The caller may free or change A after the stream reaches this call. */
int peps_set_tensors(peps_ctx* ctx, const double* A, void* stream);

/* W(S) for B configurations (Eq. PEPS; Fig. 1(b,c)): the lower environments
 * Dn_{L-1} .. Dn_1 are built by boundary-MPS absorption and truncation, and
 * the row-0 strip is closed against Dn_1.  Outputs log|W| (float64[B]) and
 * sign (int8[B], 0 for a zero amplitude). */
int peps_amplitudes(peps_ctx* ctx, const uint8_t* spins, int64_t B,
                    double* log_abs, int8_t* sign, void* stream);

/* Local energy E(S) of Eq. ess for B configurations: the total (not per
 * site) sum over all J1 and J2 bonds of J [sigma_i sigma_j / 4 + (for an
 * antiparallel pair) W(S')/W(S) / 2], each ratio taken on the one-row strip
 * (horizontal bonds) or two-row strip (vertical and J2 bonds) between the
 * cached upper and lower environments.  Outputs: e_loc float64[B]; log_abs
 * float64[B] and sign int8[B] as peps_amplitudes; ratios (nullable)
 * float64[B][n_bonds] in canonical bond order, 0 for parallel pairs;
 * n_flips (nullable) int32[B], the number of antiparallel pairs. */
int peps_local_energy(peps_ctx* ctx, const uint8_t* spins, int64_t B,
                      double* e_loc, double* log_abs, int8_t* sign,
                      double* ratios, int32_t* n_flips, void* stream);

/* Log-derivatives Delta^{s_m}_{lrud}(S) = B^{s_m}_{lrud}(S) / W(S) of
 * Eq. delta, B taken from the one-row strip of site m's row, and their sums
 * over the batch for Eq. gradients:
 *   sum_delta[m][s][k]   (+)= sum_b [s_b,m == s] Delta_b[m][k]
 *   sum_delta_e[m][s][k] (+)= sum_b [s_b,m == s] Delta_b[m][k] * e_loc[b]
 *   sum_e[0]             (+)= sum_b e_loc[b]
 * with k = ((l*D + r)*D + u)*D + d.  e_loc: float64[B] (input, e.g. from
 * peps_local_energy).  delta (nullable): float64[B][N][D^4], the s_m slice
 * only.  sum_delta, sum_delta_e: float64[N][2][D^4]; sum_e: float64[1].
 * accumulate = 0 overwrites the sums, 1 adds to them.  Sums are formed in a
 * fixed order (bit-reproducible for a fixed slot count). */
int peps_logderiv(peps_ctx* ctx, const uint8_t* spins, int64_t B,
                  const double* e_loc, double* delta, double* sum_delta,
                  double* sum_delta_e, double* sum_e, int32_t accumulate,
                  void* stream);

/* peps_local_energy and peps_logderiv in one pass over the batch (the
 * environments are built once); the sums use the e_loc computed here.
 * Any of ratios, n_flips, delta may be NULL. */
int peps_evaluate(peps_ctx* ctx, const uint8_t* spins, int64_t B,
                  double* e_loc, double* log_abs, int8_t* sign,
                  double* ratios, int32_t* n_flips, double* delta,
                  double* sum_delta, double* sum_delta_e, double* sum_e,
                  int32_t accumulate, void* stream);

/* One GO step (the sign update after Eq. delta, with the gradient of
 * Eq. gradients):
 *   g = 2 sum_delta_e / M - 2 (sum_delta / M) (sum_e[0] / M)
 *   A[e] -= p_e * dt * sign(g[e]),   sign(0) = 0,
 * p_e in (0,1) from Philox4x32-10 with key = seed and counter
 * (e mod 2^32, e >> 32, step, 2): p = ((x >> 12) + 1/2) 2^-52, x the 64-bit
 * word out[1]:out[0].  A_inout: float64[N][2][D^4] (device, updated in
 * place); also refreshes the context's copy of the tensors.  step < 2^32. */
int peps_grad_step(peps_ctx* ctx, const double* sum_delta,
                   const double* sum_delta_e, const double* sum_e, int64_t M,
                   double dt, uint64_t seed, uint64_t step, double* A_inout,
                   void* stream);

/* Metropolis sampling with weight W(S)^2 (Fig. "contraction", Steps 1-3;
 * Eq. energy-MC) of chains chain_offset .. chain_offset+n_chains-1.
 * Moves: exchanges of antiparallel nearest-neighbour spins (S^z kept).  A
 * chain starts from chain_state (uint8[n_chains][N]) if non-NULL, else from
 * a Fisher-Yates shuffle of floor(N/2) up spins (Philox key seed, counter
 * (k, 0, chain, 0), j = x mod (k+1)).  A sweep rebuilds the lower
 * environments and visits row i = 0..L-1: horizontal bonds left to right on
 * the one-row strip, then vertical bonds (i,j)-(i+1,j) on the two-row strip,
 * then absorbs row i into the upper environment.  Bond b in sweep t draws
 * u = (x >> 11) 2^-53 from counter (b, t, chain, 1) and accepts iff
 * u < (W(S')/W(S))^2.  Sweeps of this call are numbered first_sweep,
 * first_sweep+1, ...; the configuration after the call's sweep number
 * n (n = 1, 2, ...) is recorded when n > n_burn and (n - n_burn) % n_thin
 * == 0.  spins_out: uint8[n_chains * samples_per_chain][N], chain-major.
 * chain_state (nullable) receives the final configurations.  accepted
 * (nullable): int64[n_chains] accepted moves. */
int peps_sample_batch(peps_ctx* ctx, uint64_t seed, int64_t n_chains,
                      int64_t chain_offset, int32_t n_burn, int32_t n_thin,
                      int32_t samples_per_chain, uint64_t first_sweep,
                      uint8_t* spins_out, uint8_t* chain_state,
                      int64_t* accepted, void* stream);

/* peps_amplitudes without any device allocation, for callers that may not
 * call cudaMalloc (inside a stream capture whose owner forbids allocation, a
 * real-time loop with a fixed memory budget, a plug-in whose host owns all
 * device memory).  The paper has no counterpart: it is an interface for
 * such callers, computing exactly what peps_amplitudes computes (FP64 form
 * only; shape->precision must be PEPS_FP64).
 *   A: float64[N][2][D^4] site tensors (device, read only); spins, log_abs,
 *   sign as in peps_amplitudes; no context.
 * The workspace (a converted copy of A, the bond-dimension table and the
 * per-sample environments) lives in one fixed 64 MiB device array that every
 * GPU loading the library holds until process exit.  Shapes whose per-sample
 * workspace does not fit return PEPS_ESCRATCH (e.g. 16x16, D=6, Dc=24 fits
 * three samples at a time, 8x8, D=4, Dc=16 fits 39, 24x24, D=8, Dc=32 does not fit);
 * when fewer samples fit than the GPU could run, they run fewer at a
 * time.  Calls no allocating routine.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current:
 * make that first call before any stream capture.  The address is kept with
 * the id of the device's context and looked up again when the context has
 * changed (after cudaDeviceReset the next call is again a first call).  Every
 * call reuses the
 * same array, so calls that overlap on the GPU (other streams, other host
 * threads) race: order them.  Device-side conditions (zero amplitude,
 * non-finite input) are only reflected in sign = 0 / log_abs. */
int peps_amplitudes_noalloc(const peps_shape* shape, const double* A,
                            const uint8_t* spins, int64_t B, double* log_abs,
                            int8_t* sign, void* stream);

/* One variational Monte Carlo step for chains chain_offset ..
 * chain_offset+n_chains-1 in a single fused launch: each chain's current
 * configuration chain_state[c] (uint8[n_chains][N], device, in/out) is
 * evaluated exactly as by peps_evaluate (e_loc, log_abs, sign per chain;
 * sum_delta, sum_delta_e, sum_e over the chains, accumulate as there), then
 * advanced by one Metropolis sweep numbered `sweep` exactly as by
 * peps_sample_batch (n_burn 0, n_thin 1, one sample), reusing the lower
 * environments the evaluation built (Fig. "contraction", Steps 1-6).
 * log_abs, sign, accepted (int64[n_chains]) may be NULL. */
int peps_vmc_step(peps_ctx* ctx, uint64_t seed, int64_t n_chains,
                  int64_t chain_offset, uint64_t sweep, uint8_t* chain_state,
                  double* e_loc, double* log_abs, int8_t* sign,
                  double* sum_delta, double* sum_delta_e, double* sum_e,
                  int32_t accumulate, int64_t* accepted, void* stream);

/* Spin-spin correlations (Sec. "Experiment Setup" and the results after it:
 * the map <S_0 . S_m> and the structure factor m_s^2(k)).  For every sample b
 * and source site src[q], the local values of S_src . S_m at every site m,
 *     ss[b][q][m] = sigma_src sigma_m / 4 + [s_src != s_m] W(S')/W(S) / 2,
 * ss[b][q][src] = 3/4, S' = S with s_src and s_m exchanged; their mean over
 * configurations drawn from W^2 is <S_src . S_m>.  The ratio is taken on the
 * one-row strip of row i(m), each configuration with its own environments
 * (W_i(S') / W_i(S); for a pair in one row the horizontal-bond window).
 *   spins: uint8[B][N] (device); src: int32[n_src] (HOST), 1 <= n_src <= N,
 *   0 <= src[q] < N; ss: float64[B][n_src][N] (device, written);
 *   ss_mean: float64[n_src][N] (device, nullable): the mean over the batch,
 *   summed in sample order (bit-reproducible).
 * FP64 and mixed forms (PEPS_EINVAL for PEPS_FP32).  Items (sample, source)
 * run one per thread block; each costs about one evaluation.  Zero or
 * non-finite amplitudes set PEPS_FLAG_NONFINITE (ratio 0).  The source list is
 * copied into the context: calls on one context are ordered on one stream. */
int peps_correlations(peps_ctx* ctx, const uint8_t* spins, int64_t B, int32_t n_src,
                      const int32_t* src, double* ss, double* ss_mean, void* stream);

/* m_s^2(k) = (1/n^2) sum_{a, m in the bulk} C[a][m] cos(k . (r_a - r_m)) over
 * the n = (L-4)^2 central sites (all sites for L <= 4), C[a][m] =
 * ss_mean[q(a)][m] from peps_correlations with sources src (HOST int32[n_src];
 * every bulk site must be among them, else PEPS_EINVAL); k = (kx, ky) along
 * (rows, columns); M^2 = m_s^2(pi, pi).  m2: float64[1] (device, written). */
int peps_structure_factor(peps_ctx* ctx, const double* ss_mean, int32_t n_src,
                          const int32_t* src, double kx, double ky, double* m2,
                          void* stream);

/* Batched contraction C_b = A_b B_b (A_b: float64[M][K] row-major, B_b:
 * float64[K][N] row-major, C_b: float64[M][N]; batch elements contiguous, B
 * shared by the batch when b_shared = 1) on the tcgen05 tensor cores at
 * FP64-class accuracy: every row of A and column of B is split error-free
 * into `slices` BF16 integer slices of 7 bits at a common exponent (Ozaki et
 * al., 2012); the slice products of equal order add up exactly in FP32 TMEM
 * accumulators (K * slices <= 1024) and are combined exactly into FP64
 * (c_format = PEPS_FP64: C is float64[M][N]) or into float-float
 * (c_format = PEPS_MIXED: C holds (hi, lo) FP32 pairs, the persistent
 * kernels' form); slices = 7 keeps about 49 significant bits of the row and
 * column scales.  One CTA per SM walks the tiles, holding its TMEM columns.  The paper's column
 * steps (Fig. 1(c); Fig. "contraction", Step 4) are such contractions; this
 * entry point measures the tensor-core form of them against peps_cc_gemm.
 *   workspace: device, 256-byte aligned, peps_tc_workspace_bytes() bytes
 *   (the slice images and exponents); status: device int32, bit 1 / 2 set
 *   when a bounded wait on the copies / MMAs ran out (C not written).
 * 1 <= slices <= 8.  Asynchronous on `stream`. */
size_t peps_tc_workspace_bytes(int32_t M, int32_t N, int32_t K, int64_t batch,
                               int32_t slices, int32_t b_shared);
int peps_tc_gemm(const double* A, const double* B, void* C, int32_t M,
                 int32_t N, int32_t K, int64_t batch, int32_t b_shared,
                 int32_t slices, int32_t c_format, void* workspace,
                 size_t workspace_bytes, int32_t* status, void* stream);

/* The same batched contraction on the CUDA cores with the persistent kernels'
 * contract() routine in the arithmetic of `precision` (PEPS_FP64, PEPS_MIXED
 * float-float, PEPS_FP32), one thread block per batch element.  convert = 1:
 * A and B are converted into the workspace and C converted back; convert = 0
 * runs the contraction alone on operands an earlier call converted (for
 * timing).  workspace: peps_cc_workspace_bytes() bytes, device. */
size_t peps_cc_workspace_bytes(int32_t precision, int32_t M, int32_t N, int32_t K,
                               int64_t batch, int32_t b_shared);
int peps_cc_gemm(int32_t precision, const double* A, const double* B, double* C,
                 int32_t M, int32_t N, int32_t K, int64_t batch, int32_t b_shared,
                 void* workspace, size_t workspace_bytes, int32_t convert, void* stream);

/* Several jobs of different lattice sizes and bond dimensions (one precision
 * form) in ONE persistent launch: the local energies of every job's samples
 * (Eq. ess), computed exactly as peps_local_energy computes them.  A pool
 * holds the slot workspaces (sized for the largest of `shapes`) and the
 * work queue: the blocks claim (job, sample) items one at a time with an
 * atomic counter, the costliest jobs' items first, so that items of very
 * different cost share the SMs without waves.
 *   peps_pool_create: precision PEPS_FP64 or PEPS_MIXED; slots (0: two per
 *   SM); shapes: HOST array of the shapes the pool will run (their
 *   precision must be the pool's); max_jobs: jobs per launch.
 *   peps_multi_job: ctx (a context of the job's shape, tensors set; its own
 *   workspace is not used), spins uint8[B][N] (device), outputs as in
 *   peps_local_energy (e_loc required; log_abs, sign, ratios, n_flips
 *   nullable).  Errors: PEPS_EINVAL for a shape larger than the pool's, a
 *   context of another form or device, n_jobs > max_jobs.  Device-side
 *   conditions collect in the pool's flags (peps_pool_sync_status).
 * Calls on one pool are ordered on one stream (the queue counter and the
 * job table are the pool's). */
typedef struct peps_pool peps_pool;
typedef struct {
  peps_ctx* ctx;
  const uint8_t* spins;
  int64_t B;
  double* e_loc;
  double* log_abs;
  int8_t* sign;
  double* ratios;
  int32_t* n_flips;
} peps_multi_job;
int peps_pool_create(int32_t precision, int32_t slots, const peps_shape* shapes,
                     int32_t n_shapes, int32_t max_jobs, peps_pool** out);
int peps_pool_destroy(peps_pool* pool);
int peps_pool_slots(const peps_pool* pool, int32_t* slots);
int peps_local_energy_multi(peps_pool* pool, const peps_multi_job* jobs, int32_t n_jobs,
                            void* stream);
int peps_pool_sync_status(peps_pool* pool, void* stream, int32_t* flags);

/* peps_vmc_step from and to HOST memory, for callers that hold the chains on
 * the host: chain_state (uint8[n_chains][N], host, in/out) is copied in, the
 * fused step runs (Fig. "contraction", Steps 1-6), and the advanced states,
 * e_loc (float64[n_chains], host), log_abs and sign (host, nullable) and
 * sum_e (float64[1], host, nullable: the batch's sum of E(S)) are copied
 * back; the call returns when they are there (stream synchronised).  The
 * gradient sums stay on the device: sum_delta, sum_delta_e, sum_e_dev as in
 * peps_vmc_step (all three NULL: the context's own, not returned).  Pinned
 * host memory makes the copies asynchronous with respect to other streams.
 * The context's device staging grows on the first call with a larger
 * n_chains (an allocation). */
int peps_vmc_step_host(peps_ctx* ctx, uint64_t seed, int64_t n_chains,
                       int64_t chain_offset, uint64_t sweep, uint8_t* chain_state,
                       double* e_loc, double* log_abs, int8_t* sign, double* sum_e,
                       double* sum_delta, double* sum_delta_e, double* sum_e_dev,
                       void* stream);

/* The fused VMC step and the GO update with their Philox counters in device
 * memory, for capture in a CUDA graph: counters is uint32[2] (device) with
 * counters[0] the sweep number (as `sweep` of peps_vmc_step) and counters[1]
 * the GO step number (as `step` of peps_grad_step), read by the kernels when
 * they run; peps_counters_advance adds `inc` to counters[0 .. n-1] in a
 * one-thread kernel.  A graph holding peps_vmc_step_dc, peps_grad_step_dc and
 * peps_counters_advance(counters, 2, 1) therefore replays as successive VMC
 * steps (Fig. "contraction", Steps 1-6 and the GO update), with results
 * identical to the same steps called directly.  Arguments and errors
 * otherwise as peps_vmc_step / peps_grad_step. */
int peps_vmc_step_dc(peps_ctx* ctx, uint64_t seed, int64_t n_chains,
                     int64_t chain_offset, const uint32_t* counters,
                     uint8_t* chain_state, double* e_loc, double* log_abs,
                     int8_t* sign, double* sum_delta, double* sum_delta_e,
                     double* sum_e, int32_t accumulate, int64_t* accepted,
                     void* stream);
int peps_grad_step_dc(peps_ctx* ctx, const double* sum_delta,
                      const double* sum_delta_e, const double* sum_e, int64_t M,
                      double dt, uint64_t seed, const uint32_t* counters,
                      double* A_inout, void* stream);
int peps_counters_advance(uint32_t* counters, int32_t n, uint32_t inc, void* stream);

/* Wait for `stream` and return the device-side error state: PEPS_OK, or
 * PEPS_ENUMERIC with *flags (host, nullable) set to the PEPS_FLAG_* bits
 * seen since the last call (the bits are cleared). */
int peps_sync_status(peps_ctx* ctx, void* stream, int32_t* flags);

/* Algorithmic floating-point operation count per chain, as the kernels
 * perform it (contractions, Householder QR, bidiagonalisation, inverse
 * iteration, back-transformation; a multiply-add counts 2; ratios at half
 * filling): what = 0 one peps_evaluate sample, 1 one Metropolis sweep,
 * 2 one peps_vmc_step (evaluation + sweep sharing the lower environments).
 * Host call for roofline reporting; 0 for an invalid shape or `what`. */
double peps_flops_per_sample(const peps_shape* shape, int32_t what);

/* Per-phase cycle counters of the fused VMC-step kernel (peps_vmc_step) of
 * ctx's precision form, the counterpart of the paper's hardware-counter
 * measurement (Sec. "Performance Measurement").  Only a library built with
 * the compile-time knob PEPS_PHASES=1 counts: thread 0 of every block adds
 * the clock64() cycles of each phase (summed over blocks and launches since
 * the last call).  Copies min(n, *n_phases) counters to out (host array),
 * clears them and sets *n_phases to the number of phases (0 for a build
 * without the counters).  Phase order: evaluation, sweep, compressions, QR
 * R factors, QR before an SVD, truncated SVDs, one-row strip environments,
 * horizontal ratios, B tensors, two-row strip environments, vertical and
 * diagonal ratios, sweep horizontal moves, sweep two-row right
 * environments, sweep vertical moves (the first two contain the others,
 * compressions contain the three after them).  Synchronises the device.
 * PEPS_EINVAL for a null ctx or n_phases, n < 0, or n > 0 with a null out. */
int peps_phase_cycles(const peps_ctx* ctx, uint64_t* out, int32_t n, int32_t* n_phases);

/* ------------------------------------------------------------------------
 * Serving: a request loop with continuous batching.  The paper runs one
 * large job; serving many independent VMC users at once has no counterpart
 * there.  A server owns a worker thread on the current device.  Jobs (the
 * amplitudes and local energies of a batch of configurations of one PEPS,
 * of any lattice size, D, Dc and precision form) are submitted from any host
 * thread and admitted in arrival order while the sum of the admitted jobs'
 * device footprints (workspace, tensors, spins and outputs) stays within the
 * HBM budget.  An admitted job gets its own context and stream and keeps its
 * tensors and environments resident until it completes; its configurations
 * run one wave (its slot count) at a time, so that jobs that arrive while
 * others are on the GPU start as soon as memory allows and their waves
 * overlap on the device.  A job's results do not depend on what runs beside
 * it: every configuration is evaluated by the same per-sample code as
 * peps_local_energy.
 * ------------------------------------------------------------------------ */
typedef struct peps_server peps_server;

typedef struct {
  peps_shape shape;       /* lattice, D, Dc, couplings, precision form */
  const double* A;        /* host float64[N][2][D^4]; read at admission */
  const uint8_t* spins;   /* host uint8[B][N]; read at admission */
  int64_t B;              /* configurations, >= 1 */
  double* e_loc;          /* host float64[B] out: E(S) */
  double* log_abs;        /* host float64[B] out (nullable) */
  int8_t* sign;           /* host int8[B] out (nullable) */
} peps_job;

typedef struct {
  double submit_s, admit_s, done_s; /* host monotonic clock, seconds */
  int64_t footprint_bytes;          /* device bytes the job held */
  int32_t status;                   /* PEPS_OK or the job's error code */
  int32_t flags;                    /* PEPS_FLAG_* bits seen by the job */
} peps_job_stats;

/* Create a server on the current device.  hbm_budget_bytes: device memory
 * the admitted jobs may hold together (0 = 90 % of the free memory);
 * slots_per_job: wave size of a job (0 = 2 per SM; a job uses
 * min(B, slots_per_job)).  ECUDA without a device. */
int peps_server_create(size_t hbm_budget_bytes, int32_t slots_per_job,
                       peps_server** out);
/* Queue a job (thread-safe).  The host buffers the job names must stay valid
 * and untouched until peps_server_wait returns for it.  EINVAL for a bad
 * shape or buffer, ENOMEM if the job alone exceeds the budget. */
int peps_server_submit(peps_server* srv, const peps_job* job, int64_t* job_id);
/* Block until job_id completes (timeout_s <= 0: no limit; ETIMEOUT when it
 * runs out, the job keeps running).  Returns the job's status; *stats
 * (nullable) receives its timings.  A job can be waited for once. */
int peps_server_wait(peps_server* srv, int64_t job_id, double timeout_s,
                     peps_job_stats* stats);
/* Finish every queued job, stop the worker and free the server. */
int peps_server_destroy(peps_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* PEPS_GB300_H */
