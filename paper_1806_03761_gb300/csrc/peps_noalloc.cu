// peps_noalloc.cu -- peps_amplitudes_noalloc: amplitudes without any device
// allocation.
//
// Some callers cannot call cudaMalloc: code running inside a region where the
// allocator must not be touched (a stream being captured by a framework that
// forbids allocation, a real-time loop with a fixed memory budget, a plug-in
// whose host application owns all device memory).  This entry point serves
// them: its workspace is a file-scope device array of fixed size that exists
// on every GPU that loads the library, from load until process exit.  The
// caller passes only the site tensors, the spins and the two output arrays.
//
// The array is shared by every call on a device, keeps the previous call's
// contents, and is not protected against concurrent use: two calls that
// overlap on the GPU (different streams, or different host threads without
// ordering) race and produce wrong results.  Order them on one stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../include/peps.h"
#include "peps_eval.cuh"
#include "peps_launch.h"

// Workspace of peps_amplitudes_noalloc: 64 MiB per device.
#define PEPS_NOALLOC_BYTES (64ull << 20)
static __device__ __align__(256) unsigned char peps_noalloc_scratch[PEPS_NOALLOC_BYTES];

namespace {

struct NoallocSteps {
  PepsStep s[PEPS_MAXL - 1];
};

// Copy the bond-dimension table into the scratch (parameters by value: no
// host buffer, no allocation).
__global__ void noalloc_put_steps(NoallocSteps st, int n, PepsStep* dst, int* flags) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = st.s[k];
  if (threadIdx.x == 0) *flags = 0;  // the flags must start at zero every call
}

// The amplitude-only variant of the evaluation kernel: lower environments,
// then the row-0 strip closed against Dn_1 (Eq. PEPS; Fig. 1(b,c)).
__global__ void __launch_bounds__(PEPS_NT, PEPS_MINB) peps_amp_noalloc_kernel(EvalArgs<double> a) {
  __shared__ double red[PEPS_NT];
  __shared__ __align__(16) unsigned char redR_raw[PEPS_NT * sizeof(double)];
  __shared__ __align__(16) unsigned char wsh_raw[256 * sizeof(double)];
  __shared__ __align__(16) unsigned char qrv_raw[PEPS_QR_NB * PEPS_QR_ROWS * sizeof(double)];
  __shared__ double rot[512];
  __shared__ uint8_t sp[PEPS_MAXL * PEPS_MAXL];
  __shared__ double dnlog[PEPS_MAXL + 1];
  const PepsPlan& P = a.P;
  const int L = P.L, N = P.N;
  Work<double> w = make_work<double>(P, a.ws, a.wsd, blockIdx.x);
  w.red = red;
  w.redR = reinterpret_cast<double*>(redR_raw);
  w.wsh = reinterpret_cast<double*>(wsh_raw);
  w.qrv = reinterpret_cast<double*>(qrv_raw);
  w.rot = rot;
  w.flags = a.flags;
  for (int64_t b = blockIdx.x; b < a.B; b += gridDim.x) {
    for (int m = threadIdx.x; m < N; m += blockDim.x) sp[m] = a.spins[b * N + m];
    __syncthreads();
    build_lower<double>(P, a.steps, a.As, sp, w, dnlog);
    set_trivial<double>(P, w.up);
    EnvDims Ud = env_dims(P, a.steps, -1);
    EnvDims Dd = env_dims(P, a.steps, L - 2);
    strip1_build<double>(P, 0, sp, a.As, w.up, Ud, w.dn + P.env_cap, Dd, w, w.scl, w.scl + (L + 1));
    const double wv = w.l1[(int64_t)L * P.site_cap];
    if (threadIdx.x == 0) {
      a.log_abs[b] = log(fabs(wv)) + w.scl[L] + dnlog[1];
      a.sign[b] = (int8_t)((wv > 0.0) - (wv < 0.0));
      if (wv == 0.0) atomicOr(a.flags, PEPS_FLAG_ZERO_AMP);
      if (!isfinite(wv)) atomicOr(a.flags, PEPS_FLAG_NONFINITE);
    }
    __syncthreads();
  }
}

int64_t up32(int64_t x) { return (x + 31) & ~int64_t(31); }

// The bond dimensions and the per-slot workspace layout of the FP64 form
// (the same recurrences as the context's plan).
void plan_fp64(const peps_shape& s, PepsPlan* P, NoallocSteps* steps) {
  const int L = s.L, D = s.D, Dc = s.Dc;
  std::memset(P, 0, sizeof(*P));
  std::memset(steps, 0, sizeof(*steps));
  P->L = L; P->D = D; P->Dc = Dc; P->N = L * L;
  P->D2 = D * D; P->D3 = D * D * D; P->D4 = D * D * D * D;
  P->nbonds = 2 * L * (L - 1) + 2 * (L - 1) * (L - 1);
  P->J1 = s.J1; P->J2 = s.J2;
  P->nsteps = L - 1;
  for (int t = 0; t < L - 1; ++t) {
    PepsStep& st = steps->s[t];
    for (int j = 0; j < L; ++j) {
      if (t == 0) { st.ia[j] = 1; st.ip[j] = 1; st.ib[j] = 1; }
      else { st.ia[j] = steps->s[t - 1].oa[j]; st.ip[j] = D; st.ib[j] = steps->s[t - 1].ob[j]; }
    }
    int rprev = 1;
    for (int j = 0; j < L - 1; ++j) {
      int r = std::min(rprev * D, st.ib[j] * D);
      st.r[j] = (int16_t)r;
      rprev = r;
    }
    int cn = 1;
    for (int j = L - 1; j >= 1; --j) {
      int k = std::min(Dc, std::min((int)st.r[j - 1], D * cn));
      st.oa[j] = (int16_t)k;
      st.ob[j] = (int16_t)cn;
      cn = k;
    }
    st.oa[0] = 1;
    st.ob[0] = (int16_t)cn;
  }
  P->site_cap = (int64_t)Dc * D * Dc;
  P->env_cap = (int64_t)L * P->site_cap;
  P->big_cap = (int64_t)Dc * Dc * D * D * D;
  P->mat_cap = (int64_t)(Dc * D) * (Dc * D);
  P->env2_cap = (int64_t)Dc * D * D * Dc;
  int64_t o = 0;
  auto take = [&](int64_t n) { int64_t r = o; o += up32(n); return r; };
  P->off_dn = take((int64_t)(L + 1) * P->env_cap);
  P->off_up = take(3 * P->env_cap);
  P->off_rst = take((int64_t)L * P->mat_cap);
  P->off_b0 = take(P->big_cap);
  P->off_b1 = take(P->big_cap);
  P->off_b2 = take(P->big_cap);
  P->off_y = take(P->mat_cap);
  P->off_xj = take(P->mat_cap);
  P->off_vt = take(std::max<int64_t>(P->site_cap, P->D4));
  P->off_c0 = take(P->site_cap);
  P->off_c1 = take(P->site_cap);
  P->off_l1 = take((int64_t)(L + 1) * P->site_cap);
  P->off_r1 = take((int64_t)(L + 1) * P->site_cap);
  P->off_l2 = 0;  // the two-row strip is not used by this entry point
  P->off_r2 = 0;
  P->off_alpha = take(3 * (int64_t)Dc * D + 16);
  P->off_inv = take(13 * (int64_t)Dc * Dc * D);
  P->off_tmp = take(32);
  P->slot_elems = o;
  int64_t d = 0;
  auto taked = [&](int64_t n) { int64_t r = d; d += up32(n); return r; };
  P->doff_scale = taked(4 * (L + 1));
  P->doff_delta = 0;
  P->doff_alpha = 0;
  P->slot_doubles = d;
}

// Device address of the scratch array, looked up once per device with that
// device current (the array's name is only a host-side stand-in).
std::mutex g_mu;
void* g_addr[64] = {nullptr};

cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, peps_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int peps_amplitudes_noalloc(const peps_shape* shape, const double* A,
                                       const uint8_t* spins, int64_t B, double* log_abs,
                                       int8_t* sign, void* stream) {
  if (!shape || shape->L < 2 || shape->L > PEPS_MAXL || shape->D < 1 || shape->D > 8 ||
      shape->Dc < 1 || shape->Dc * shape->D > 256 || shape->precision != PEPS_FP64)
    return PEPS_EINVAL;
  if (B < 0) return PEPS_EINVAL;
  if (B == 0) return PEPS_OK;
  if (!A || !spins || !log_abs || !sign) return PEPS_EINVAL;
  PepsPlan P;
  NoallocSteps steps;
  plan_fp64(*shape, &P, &steps);
  // layout inside the scratch: flags | steps | tensors | slot workspaces
  const int64_t n_tensor = (int64_t)P.N * 2 * P.D4;
  const size_t off_steps = 256;
  const size_t off_as = off_steps + ((sizeof(PepsStep) * (P.L - 1) + 255) & ~size_t(255));
  const size_t off_ws = off_as + ((n_tensor * sizeof(double) + 255) & ~size_t(255));
  const size_t slot_bytes = (size_t)(P.slot_elems + P.slot_doubles) * sizeof(double);
  if (off_ws + slot_bytes > PEPS_NOALLOC_BYTES) return PEPS_ESCRATCH;
  const int64_t fit = (int64_t)((PEPS_NOALLOC_BYTES - off_ws) / slot_bytes);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PEPS_ECUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PEPS_ECUDA;
  const int nslots = (int)std::min<int64_t>(std::min<int64_t>(fit, PEPS_MINB * (int64_t)sms), B);
  unsigned char* base = nullptr;
  if (scratch_address(dev, (void**)&base) != cudaSuccess) return PEPS_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* flags = reinterpret_cast<int*>(base);
  PepsStep* dsteps = reinterpret_cast<PepsStep*>(base + off_steps);
  double* As = reinterpret_cast<double*>(base + off_as);
  double* ws = reinterpret_cast<double*>(base + off_ws);
  double* wsd = ws + (int64_t)nslots * P.slot_elems;
  noalloc_put_steps<<<1, 64, 0, st>>>(steps, P.L - 1, dsteps, flags);
  if (cudaGetLastError() != cudaSuccess) return PEPS_ECUDA;
  if (peps_launch_convert(PEPS_FP64, A, As, n_tensor, flags, st) != cudaSuccess) return PEPS_ECUDA;
  EvalArgs<double> a;
  std::memset(&a, 0, sizeof(a));
  a.P = P;
  a.steps = dsteps;
  a.As = As;
  a.spins = spins;
  a.B = B;
  a.log_abs = log_abs;
  a.sign = sign;
  a.ws = ws;
  a.wsd = wsd;
  a.psum = wsd;  // unused: no sums are formed
  a.flags = flags;
  peps_amp_noalloc_kernel<<<nslots, PEPS_NT, 0, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? PEPS_OK : PEPS_ECUDA;
}
