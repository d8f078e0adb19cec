// peps_tc.cu -- batched contractions C_b = A_b B_b on the tcgen05 tensor cores
// at FP64-class accuracy, and the same contractions on the CUDA cores through
// the persistent kernels' contract() routine, for measuring one against the
// other on the shapes of the strip and absorption steps (PEPS++,
// arXiv:1806.03761, Fig. 1(c) and Fig. "contraction", Step 4: every column
// step is a small dense contraction).
//
// Error-free splitting (Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59,
// 2012).  Row i of A is scaled by 2^-e_i (e_i: the exponent of its largest
// entry) and cut into s slices of 7 bits: slice t holds the digit q_t of
// x 2^-e_i = sum_t q_t 2^-7(t+1) + (a remainder of at most 2^-7s-1), digits
// balanced and rounded to nearest (|q_0| <= 128, |q_t| <= 64 after), read
// off the bits of x with integer operations only (exact in BF16); column j
// of B likewise with f_j.  A product of slices t_a and t_b
// is an integer multiple of 2^-7(t_a+t_b+2) of magnitude < 2^14, so the K
// products of every pair with the same g = t_a + t_b (at most s pairs) add up
// exactly in an FP32 accumulator while K s <= 1024.  One TMEM accumulator per
// g < s collects those pairs; the epilogue forms
//     C_ij = 2^(e_i + f_j) sum_g acc_g[i][j] 2^-7(g+2)
// in FP64.  With s = 7 the result carries about 49 significant bits of the
// row/column scales (the float-float form keeps about 48).
//
// Tensor-core tile: one CTA of 128 threads per (128-row tile, column tile,
// batch element).  The slice images are laid out in global memory in the
// no-swizzle K-major core-matrix order the MMA reads (8 rows x 16 bytes per
// core matrix, core matrices along K 128 bytes apart, 8-row groups 768 bytes
// apart) in chunks of 48 along K, so that a slice's chunk lands in shared
// memory with one bulk copy (cp.async.bulk) completing on an mbarrier; the
// chunks are copied and multiplied in turn.  One thread issues the
// tcgen05.mma chain (kind::f16, BF16 x BF16 -> F32, M = 128) and commits it to
// the mbarrier; the four warps read their 32 TMEM lanes with tcgen05.ld.
// Every wait is bounded: on expiry the kernel records an error, waits (again
// bounded) for its copies and MMAs, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "../../include/peps.h"
#include "peps_core.cuh"

namespace {

constexpr int TC_ROWS = 128;        // M of one MMA tile (TMEM lanes)
constexpr int TC_COLS_MAX = 512;    // TMEM columns of one CTA
constexpr int TC_SLICE_BITS = 7;
constexpr unsigned long long TC_WAIT_NS = 1000000000ull;  // bound of one mbarrier wait: 1 s

constexpr int TC_KC = 48;          // K chunk: one bulk copy per slice and chunk
__host__ __device__ inline int tc_kpad(int K) { return (K + TC_KC - 1) / TC_KC * TC_KC; }
__host__ __device__ inline int tc_ntile(int N, int s) {
  // columns of one CTA: a multiple of 16, s * ntile TMEM columns <= 512
  int cap = (TC_COLS_MAX / s) / 16 * 16;
  if (cap > 256) cap = 256;
  int n16 = (N + 15) / 16 * 16;
  return n16 < cap ? n16 : cap;
}
// byte offset of element (row r, k) inside the block of one K chunk (TC_KC
// columns) of an image of `rows` rows (a multiple of 8): no-swizzle K-major
// core-matrix order, core matrices along K 128 bytes apart, 8-row groups
// TC_KC / 8 * 128 bytes apart
__host__ __device__ inline int64_t tc_core_off(int r, int kc) {
  return (int64_t)(r >> 3) * (TC_KC >> 3) * 128 + (int64_t)(kc >> 3) * 128 + (r & 7) * 16 + (kc & 7) * 2;
}

// ---------------------------------------------------------------------------
// Split: rows x K matrix X (element (r, k) at X[b*sb + r*rs + k*cs]) into s
// BF16 slice images.  Block of batch b, tile T (tile_rows rows), slice t,
// K chunk c: img + (((b * n_tiles + T) * s + t) * n_chunks + c) * tile_rows *
// TC_KC (BF16 elements).
// One warp per row; the row's exponent goes to expo[b * rows_pad + r].
// ---------------------------------------------------------------------------
__global__ void tc_split_kernel(const double* X, int64_t sb, int64_t rs, int64_t cs, int rows,
                                int K, int rows_pad, int tile_rows, int Kp, int s, int64_t batch,
                                __nv_bfloat16* img, int* expo) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int n_tiles = rows_pad / tile_rows;
  for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < batch * rows_pad;
       w += warps) {
    const int64_t b = w / rows_pad;
    const int r = (int)(w % rows_pad);
    const double* x = X + b * sb + (int64_t)r * rs;
    double mx = 0.0;
    if (r < rows)
      for (int k = lane; k < K; k += 32) mx = fmax(mx, fabs(x[(int64_t)k * cs]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);  // mx = f 2^e, f in [1/2, 1): |x| 2^-e < 1
    if (lane == 0) expo[b * rows_pad + r] = e;
    const int T = r / tile_rows, rr = r % tile_rows;
    const int nch = Kp / TC_KC;
    const int64_t blk = (int64_t)tile_rows * TC_KC;
    __nv_bfloat16* base = img + ((b * n_tiles + T) * (int64_t)s) * nch * blk;
    for (int k = lane; k < Kp; k += 32) {
      const double xv = (r < rows && k < K) ? x[(int64_t)k * cs] : 0.0;
      // |x| 2^(62-e) truncated to an integer, from the bits of x: no FP64
      // arithmetic (the mantissa shifted by the exponent difference)
      const unsigned long long bits = (unsigned long long)__double_as_longlong(xv);
      const int ex = (int)((bits >> 52) & 0x7FF);
      const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
      const int sh = ex - 1075 + 62 - e;  // |x| = mant 2^(ex-1075) < 2^e
      unsigned long long mag = 0;
      if (ex != 0) mag = sh >= 0 ? (mant << sh) : (-sh < 64 ? (mant >> -sh) : 0ull);
      const bool neg = (bits >> 63) != 0;
      const int64_t off = (k / TC_KC) * blk + tc_core_off(rr, k % TC_KC) / 2;
      // balanced base-128 digits, each rounded to nearest (half up): digit
      // t = round(rem / 2^(55-7t)), rem -= digit 2^(55-7t); the first lies in
      // [0, 128], the others in [-64, 64], so the digits of different rows
      // and columns carry both signs and the omitted high-order slice
      // products cancel on average; |remainder| <= 2^-7s-1 of the scale
      long long rem = (long long)mag;
      for (int t = 0; t < s; ++t) {
        const int sh = 55 - TC_SLICE_BITS * t;
        const long long d = (rem + (1ll << (sh - 1))) >> sh;  // arithmetic shift
        rem -= d * (1ll << sh);
        const int di = (int)d;  // |d| <= 128: a 32-bit conversion
        base[(int64_t)t * nch * blk + off] = __int2bfloat16_rn(neg ? -di : di);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Inline PTX: mbarrier, bulk copy, tcgen05.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// wait on phase `parity` for at most TC_WAIT_NS; false when the time ran out
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > TC_WAIT_NS) return false;
  }
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// UMMA shared-memory descriptor: start, leading (K) and stride (8-row group)
// byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor of kind::f16: D F32, A and B BF16, both K-major
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}
// 32 lanes x 16 columns of 32 bits from TMEM; the values may be read only
// after tmem_wait()
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}
__device__ __forceinline__ void tmem_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---------------------------------------------------------------------------
// The tensor-core kernel.  grid (M tiles, N tiles, batch), 128 threads.
// ---------------------------------------------------------------------------
struct TcArgs {
  const __nv_bfloat16* aimg;  // [batch][m_tiles][s][Kp / TC_KC][128][TC_KC]
  const __nv_bfloat16* bimg;  // [batch or 1][s][Kp / TC_KC][Np][TC_KC]
  const int* ea;              // [batch][Mp]
  const int* eb;              // [batch or 1][Np]
  void* C;                    // element (i, j) of batch b at C[b*sc + i*ldc + j] (double or ff)
  int64_t sc, ldc;
  int M, N, Kp, Mp, Np, ntile, s;
  int64_t batch;
  int b_shared;               // B (and its image) shared by the batch
  int* status;                // error bits: 1 copy wait, 2 MMA wait ran out
};

// 2^k as FP32 / FP64 from the exponent bits (exact; k in the normal range)
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }
__device__ __forceinline__ double pow2d(int k) {
  return __longlong_as_double((long long)(1023 + k) << 52);
}

// Persistent: each CTA walks the (batch, row tile, column tile) tiles with a
// stride of the grid, holding its TMEM columns throughout; the next tile's
// first chunk is copied while the current tile's accumulators are read out.
// FF: write C as float-float (hi, lo), the form the persistent kernels use;
// else FP64.
template <bool FF>
__global__ void __launch_bounds__(128, 1) tc_gemm_kernel(TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int s = a.s, ntile = a.ntile, nch = a.Kp / TC_KC;
  const int m_tiles = a.Mp / TC_ROWS, n_tiles = a.Np / ntile;
  const int64_t tiles = a.batch * m_tiles * n_tiles;
  const uint32_t a_blk = (uint32_t)TC_ROWS * TC_KC * 2;   // one slice, one chunk
  const uint32_t b_blk = (uint32_t)ntile * TC_KC * 2;
  unsigned char* sa = smem;
  unsigned char* sb = smem + (size_t)s * a_blk;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sb + (size_t)s * b_blk);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tcols = s * ntile <= 32 ? 32 : s * ntile <= 64 ? 64 : s * ntile <= 128 ? 128
                  : s * ntile <= 256 ? 256 : 512;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_async_smem();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tslot)),
                 "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = umma_idesc(TC_ROWS, ntile);
  const uint32_t sbo = (uint32_t)(TC_KC / 8) * 128;
  // thread 0: the bulk copies of chunk c of tile `tl`
  auto issue_copy = [&](int64_t tl, int c) {
    const int nt = (int)(tl % n_tiles);
    const int mt = (int)((tl / n_tiles) % m_tiles);
    const int64_t b = tl / ((int64_t)n_tiles * m_tiles);
    const int64_t bb = a.b_shared ? 0 : b;
    const __nv_bfloat16* ga = a.aimg + ((b * m_tiles + mt) * (int64_t)s) * nch * (TC_ROWS * TC_KC);
    const __nv_bfloat16* gb = a.bimg + (bb * (int64_t)s) * nch * ((int64_t)a.Np * TC_KC) +
                              (int64_t)nt * ntile * TC_KC;
    mbar_expect_tx(bar, (uint32_t)s * (a_blk + b_blk));
    for (int t = 0; t < s; ++t) {
      bulk_g2s(sa + (size_t)t * a_blk, ga + ((int64_t)t * nch + c) * (TC_ROWS * TC_KC), a_blk, bar);
      bulk_g2s(sb + (size_t)t * b_blk, gb + ((int64_t)t * nch + c) * ((int64_t)a.Np * TC_KC), b_blk, bar);
    }
  };
  uint32_t phase = 0;
  int err = 0;  // 1: a copy wait ran out, 2: an MMA wait ran out
  if (threadIdx.x == 0 && (int64_t)blockIdx.x < tiles) issue_copy(blockIdx.x, 0);
  for (int64_t tl = blockIdx.x; tl < tiles && !err; tl += gridDim.x) {
    for (int c = 0; c < nch; ++c) {
      if (c > 0 && threadIdx.x == 0) issue_copy(tl, c);  // chunk 0 was prefetched
      if (!__syncthreads_and(mbar_wait(bar, phase & 1))) { err = 1; break; }
      ++phase;
      // the MMAs of chunk c: accumulator g collects the slice pairs with
      // t_a + t_b = g; the first MMA into each accumulator overwrites it
      if (threadIdx.x == 0) {
        tc_fence_after();
        for (int g = 0; g < s; ++g)
          for (int ta = 0; ta <= g; ++ta) {
            const int tb = g - ta;
            for (int kk = 0; kk < TC_KC / 16; ++kk) {
              const uint64_t da = umma_desc(smem_addr(sa + (size_t)ta * a_blk + kk * 256), 128, sbo);
              const uint64_t db = umma_desc(smem_addr(sb + (size_t)tb * b_blk + kk * 256), 128, sbo);
              umma_bf16(tmem + (uint32_t)(g * ntile), da, db, idesc, (c | ta | kk) ? 1u : 0u);
            }
          }
        umma_commit(bar);
      }
      if (!__syncthreads_and(mbar_wait(bar, phase & 1))) { err = 2; break; }
      ++phase;
    }
    if (err) break;
    // the shared buffers are free: prefetch the next tile's first chunk
    if (threadIdx.x == 0 && tl + gridDim.x < tiles) issue_copy(tl + gridDim.x, 0);
    tc_fence_after();
    // epilogue: row i = 32 warp + lane of the tile
    const int nt = (int)(tl % n_tiles);
    const int mt = (int)((tl / n_tiles) % m_tiles);
    const int64_t b = tl / ((int64_t)n_tiles * m_tiles);
    const int64_t bb = a.b_shared ? 0 : b;
    const int i = mt * TC_ROWS + warp * 32 + lane;
    const int ei = a.ea[b * a.Mp + i];
    for (int j0 = 0; j0 < ntile; j0 += 16) {
      float v[8][16];
#pragma unroll
      for (int g = 0; g < 8; ++g)
        if (g < s) tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(g * ntile + j0), v[g]);
      tmem_wait();
      if (i < a.M) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int j = nt * ntile + j0 + q;
          if (j >= a.N) continue;
          const int sc = ei + a.eb[bb * a.Np + j];
          const int64_t at = b * a.sc + (int64_t)i * a.ldc + j;
          if (FF) {
            // sum_g acc_g 2^-7(g+2), smallest first, in float-float (every
            // term exact in FP32), then the row/column scale
            ff acc = {0.0f, 0.0f};
#pragma unroll
            for (int g = 7; g >= 0; --g)
              if (g < s) {
                const ff t = ff_two_sum(acc.hi, v[g][q] * pow2f(-TC_SLICE_BITS * (g + 2)));
                acc = ff_fast_two_sum(t.hi, __fadd_rn(acc.lo, t.lo));
              }
            const float p2 = pow2f(sc);
            static_cast<ff*>(a.C)[at] = ff{acc.hi * p2, acc.lo * p2};
          } else {
            // exact integer combination in two parts (|acc_g| < 2^24), one
            // rounding: sum_g acc_g 2^-7(g+2) = H 2^-28 + Lo 2^-56
            long long H = 0, Lo = 0;
#pragma unroll
            for (int g = 0; g < 8; ++g)
              if (g < s) {
                const long long x = (long long)__float2int_rn(v[g][q]);
                if (g < 3) H += x << (TC_SLICE_BITS * (2 - g));
                else Lo += x << (TC_SLICE_BITS * (6 - g));
              }
            const double val = fma((double)H, pow2d(-28), (double)Lo * pow2d(-56));
            static_cast<double*>(a.C)[at] = val * pow2d(sc);
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();  // every TMEM read done before the next tile's MMAs
    tc_fence_after();
  }
  if (err && threadIdx.x == 0) {
    atomicOr(a.status, err);
    // let the copies or the MMAs in flight finish, within the same bound,
    // before the shared memory and the TMEM columns are released
    mbar_wait(bar, phase & 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
}

// ---------------------------------------------------------------------------
// CUDA-core reference: one block per batch element runs contract() (the
// persistent kernels' routine) on C = A B in the form's arithmetic.
// ---------------------------------------------------------------------------
template <class R>
__global__ void __launch_bounds__(PEPS_NT, PEPS_MINB) cc_gemm_kernel(const R* A, const R* B, R* C,
                                                                      int M, int N, int K,
                                                                      int64_t sa, int64_t sb,
                                                                      int64_t sc, int64_t batch) {
  for (int64_t b = blockIdx.x; b < batch; b += gridDim.x) {
    Ctr c = ctr_init();
    c.e[0] = M; c.e[1] = N;
    c.sa[0] = K; c.sb[1] = 1;
    c.sc[0] = N; c.sc[1] = 1;
    c.k1 = K; c.ka1 = 1; c.kb1 = N;
    contract<R>(c, A + b * sa, B + b * sb, C + b * sc);
  }
}

template <class R>
__global__ void to_form(const double* x, R* y, int64_t n) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    y[k] = Arith<R>::from(x[k]);
}
template <class R>
__global__ void from_form(const R* y, double* x, int64_t n) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    x[k] = Arith<R>::to(y[k]);
}

struct TcLayout {
  int Kp, Mp, Np, ntile, m_tiles, n_tiles;
  size_t aimg, bimg, ea, eb, total, smem;
};

bool tc_layout(int M, int N, int K, int64_t batch, int s, int b_shared, TcLayout* L) {
  if (M < 1 || N < 1 || K < 1 || batch < 1 || s < 1 || s > 8) return false;
  if ((int64_t)K * s > 1024) return false;  // exact FP32 accumulation of a group
  L->Kp = tc_kpad(K);
  L->ntile = tc_ntile(N, s);
  L->n_tiles = (N + L->ntile - 1) / L->ntile;
  L->Np = L->n_tiles * L->ntile;
  L->m_tiles = (M + TC_ROWS - 1) / TC_ROWS;
  L->Mp = L->m_tiles * TC_ROWS;
  const int64_t bb = b_shared ? 1 : batch;
  auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
  L->aimg = up((size_t)batch * L->Mp * L->Kp * s * 2);
  L->bimg = up((size_t)bb * L->Np * L->Kp * s * 2);
  L->ea = up((size_t)batch * L->Mp * 4);
  L->eb = up((size_t)bb * L->Np * 4);
  L->total = L->aimg + L->bimg + L->ea + L->eb;
  L->smem = (size_t)s * (TC_ROWS + L->ntile) * TC_KC * 2 + 16;
  return L->smem <= 227 * 1024;
}

}  // namespace

extern "C" {

size_t peps_tc_workspace_bytes(int32_t M, int32_t N, int32_t K, int64_t batch, int32_t slices,
                               int32_t b_shared) {
  TcLayout L;
  if (!tc_layout(M, N, K, batch, slices, b_shared, &L)) return 0;
  return L.total;
}

int peps_tc_gemm(const double* A, const double* B, void* C, int32_t M, int32_t N, int32_t K,
                 int64_t batch, int32_t b_shared, int32_t slices, int32_t c_format, void* workspace,
                 size_t workspace_bytes, int32_t* status, void* stream) {
  TcLayout L;
  if (!A || !B || !C || !workspace || !status) return PEPS_EINVAL;
  if (c_format != PEPS_FP64 && c_format != PEPS_MIXED) return PEPS_EINVAL;
  if (!tc_layout(M, N, K, batch, slices, b_shared, &L)) return PEPS_EINVAL;
  if (workspace_bytes < L.total) return PEPS_EINVAL;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return PEPS_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* w = static_cast<unsigned char*>(workspace);
  __nv_bfloat16* aimg = reinterpret_cast<__nv_bfloat16*>(w);
  __nv_bfloat16* bimg = reinterpret_cast<__nv_bfloat16*>(w + L.aimg);
  int* ea = reinterpret_cast<int*>(w + L.aimg + L.bimg);
  int* eb = reinterpret_cast<int*>(w + L.aimg + L.bimg + L.ea);
  const int64_t bb = b_shared ? 1 : batch;
  // A: rows i (stride K), k (stride 1); B as N rows j (stride 1), k (stride N)
  auto grid_for = [](int64_t rows) { return (int)std::min<int64_t>((rows + 7) / 8, 4096); };
  tc_split_kernel<<<grid_for(batch * L.Mp), 256, 0, st>>>(A, (int64_t)M * K, K, 1, M, K, L.Mp, TC_ROWS,
                                                          L.Kp, slices, batch, aimg, ea);
  tc_split_kernel<<<grid_for(bb * L.Np), 256, 0, st>>>(B, (int64_t)K * N, 1, N, N, K, L.Np, L.Np,
                                                       L.Kp, slices, bb, bimg, eb);
  if (cudaGetLastError() != cudaSuccess) return PEPS_ECUDA;
  const bool ffout = c_format == PEPS_MIXED;
  if (cudaFuncSetAttribute(ffout ? tc_gemm_kernel<true> : tc_gemm_kernel<false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem) != cudaSuccess)
    return PEPS_ECUDA;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PEPS_ECUDA;
  TcArgs a;
  a.aimg = aimg;
  a.bimg = bimg;
  a.ea = ea;
  a.eb = eb;
  a.C = C;
  a.sc = (int64_t)M * N;
  a.ldc = N;
  a.M = M; a.N = N; a.Kp = L.Kp; a.Mp = L.Mp; a.Np = L.Np; a.ntile = L.ntile; a.s = slices;
  a.batch = batch;
  a.b_shared = b_shared;
  a.status = status;
  const int64_t tiles = batch * L.m_tiles * L.n_tiles;
  const int grid = (int)std::min<int64_t>(tiles, sms);  // one CTA per SM (TMEM, shared memory)
  if (ffout) tc_gemm_kernel<true><<<grid, 128, L.smem, st>>>(a);
  else tc_gemm_kernel<false><<<grid, 128, L.smem, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? PEPS_OK : PEPS_ECUDA;
}

size_t peps_cc_workspace_bytes(int32_t precision, int32_t M, int32_t N, int32_t K, int64_t batch,
                               int32_t b_shared) {
  if (M < 1 || N < 1 || K < 1 || batch < 1) return 0;
  const size_t es = precision == PEPS_FP64 ? 8 : precision == PEPS_MIXED ? 8 : 4;
  const int64_t bb = b_shared ? 1 : batch;
  return es * ((size_t)batch * M * K + (size_t)bb * K * N + (size_t)batch * M * N) + 1024;
}

int peps_cc_gemm(int32_t precision, const double* A, const double* B, double* C, int32_t M, int32_t N,
                 int32_t K, int64_t batch, int32_t b_shared, void* workspace, size_t workspace_bytes,
                 int32_t convert, void* stream) {
  if (!A || !B || !C || !workspace || M < 1 || N < 1 || K < 1 || batch < 1) return PEPS_EINVAL;
  if (workspace_bytes < peps_cc_workspace_bytes(precision, M, N, K, batch, b_shared)) return PEPS_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t bb = b_shared ? 1 : batch;
  const int64_t na = batch * (int64_t)M * K, nb = bb * (int64_t)K * N, nc = batch * (int64_t)M * N;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PEPS_ECUDA;
  const int grid = (int)std::min<int64_t>(batch, (int64_t)PEPS_MINB * sms);
  auto run = [&](auto tag) -> int {
    typedef decltype(tag) R;
    R* wa = static_cast<R*>(workspace);
    R* wb = wa + na;
    R* wc = wb + nb;
    // convert: 1 = convert the operands, run, convert C back; 0 = run only
    // (operands already converted by an earlier call on this workspace)
    if (convert) {
      to_form<R><<<1024, 256, 0, st>>>(A, wa, na);
      to_form<R><<<1024, 256, 0, st>>>(B, wb, nb);
    }
    cc_gemm_kernel<R><<<grid, PEPS_NT, 0, st>>>(wa, wb, wc, M, N, K, (int64_t)M * K,
                                                b_shared ? 0 : (int64_t)K * N, (int64_t)M * N, batch);
    if (convert) from_form<R><<<1024, 256, 0, st>>>(wc, C, nc);
    return cudaGetLastError() == cudaSuccess ? PEPS_OK : PEPS_ECUDA;
  };
  if (precision == PEPS_FP64) return run(double());
  if (precision == PEPS_MIXED) return run(ff());
  return run(float());
}

}  // extern "C"
