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

// The bond dimensions and the amplitude-only slot layout of the FP64 form:
// the context's plan (peps_plan.h) without the two-row strip environments
// and the Delta staging, which this entry point never touches.
void plan_fp64(const peps_shape& s, PepsPlan* P, NoallocSteps* steps) {
  std::memset(steps, 0, sizeof(*steps));
  peps_plan_steps(s.L, s.D, s.Dc, s.J1, s.J2, P, steps->s);
  peps_plan_layout(P, true);
}

// Device address of the scratch array, looked up with the device current
// (the array's name is only a host-side stand-in).  The address belongs to the
// device's current context: it is cached together with that context's id and
// looked up again when the id changes (cudaDeviceReset ends the primary
// context, and the next call on the device runs in a new one).  The driver's
// context calls are reached through the runtime's entry-point query, so the
// library does not link against the driver library.
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);

std::mutex g_mu;
void* g_addr[64] = {nullptr};
unsigned long long g_ctx_id[64] = {0};

bool current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    cudaDriverEntryPointQueryResult q1, q2;
    void* f1 = nullptr;
    void* f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) ==
            cudaSuccess && q1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) ==
            cudaSuccess && q2 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
      get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
  }
  void* ctx = nullptr;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx) return false;
  return get_id(ctx, id) == 0;
}

cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  unsigned long long id = 0;
  const bool have_id = current_context_id(&id);
  if (!g_addr[dev] || !have_id || id != g_ctx_id[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, peps_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
    // the id is read again: the lookup above may have created the context
    if (have_id || current_context_id(&id)) g_ctx_id[dev] = id;
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
