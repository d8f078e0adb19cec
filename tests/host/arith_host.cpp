// Host build of the device arithmetic header (peps_arith.cuh) for CPU tests:
// the CUDA rounding intrinsics map to IEEE binary32 operations with
// round-to-nearest (compiled with -ffp-contract=off so that no product is
// fused that the device code keeps separate), fmaf to the correctly rounded
// libm fmaf, and a warp shuffle returns the value the test queued for the
// partner lane.  Exposes the float-float operations, the compensated
// accumulator and Philox4x32-10 through extern "C" wrappers.
#include <cmath>
#include <cstdint>

#define __device__
#define __forceinline__ inline
#define __align__(n) alignas(n)
#define PEPS_HD inline

static float g_partner[8];
static int g_partner_next = 0;
template <class T> static inline T peps_host_partner(T) {
  return (T)g_partner[g_partner_next++ & 7];
}
#define __shfl_xor_sync(mask, v, o) peps_host_partner(v)
static inline float __fadd_rn(float a, float b) { return a + b; }
static inline float __fsub_rn(float a, float b) { return a - b; }
static inline float __fmul_rn(float a, float b) { return a * b; }
static inline float __fdiv_rn(float a, float b) { return a / b; }
static inline float __fsqrt_rn(float a) { return std::sqrt(a); }
using std::fabs;
using std::fma;
using std::fmaf;
using std::isfinite;
using std::sqrt;

#include "peps_arith.cuh"

extern "C" {

void h_two_sum(float a, float b, float* out) {
  ff r = ff_two_sum(a, b);
  out[0] = r.hi; out[1] = r.lo;
}
void h_add(const float* a, const float* b, float* out) {
  ff r = ff{a[0], a[1]} + ff{b[0], b[1]};
  out[0] = r.hi; out[1] = r.lo;
}
void h_mul(const float* a, const float* b, float* out) {
  ff r = ff{a[0], a[1]} * ff{b[0], b[1]};
  out[0] = r.hi; out[1] = r.lo;
}
void h_div(const float* a, const float* b, float* out) {
  ff r = ff{a[0], a[1]} / ff{b[0], b[1]};
  out[0] = r.hi; out[1] = r.lo;
}
void h_sqrt(const float* a, float* out) {
  ff r = ff_sqrt(ff{a[0], a[1]});
  out[0] = r.hi; out[1] = r.lo;
}
void h_from_double(double x, float* out) {
  ff r = Arith<ff>::from(x);
  out[0] = r.hi; out[1] = r.lo;
}
// sum_i x_i y_i with the compensated accumulator (x, y: n float-float pairs)
void h_dot(const float* x, const float* y, int n, float* out) {
  Arith<ff>::acc_t a;
  Arith<ff>::acc_init(a);
  for (int i = 0; i < n; ++i) Arith<ff>::mac(a, ff{x[2 * i], x[2 * i + 1]}, ff{y[2 * i], y[2 * i + 1]});
  ff r = Arith<ff>::acc_get(a);
  out[0] = r.hi; out[1] = r.lo;
}
// two accumulators (s, c) merged as the warp reduction merges lanes
void h_acc_merge(float s1, float c1, float s2, float c2, float* out) {
  Arith<ff>::acc_t a{s1, c1};
  g_partner[0] = s2; g_partner[1] = c2; g_partner_next = 0;
  Arith<ff>::acc_shfl_add(a, 1);
  out[0] = a.s; out[1] = a.c;
}
// x - sum_s v_s w_s: the compensated update (acc_set, mac with -w) and the
// chain of fused multiply-subtracts, both as the QR's trailing update forms them
void h_update(const float* x, const float* v, const float* w, int n, float* acc_out,
              float* chain_out) {
  Arith<ff>::acc_t u;
  Arith<ff>::acc_set(u, ff{x[0], x[1]});
  ff c = ff{x[0], x[1]};
  for (int s = 0; s < n; ++s) {
    ff vs{v[2 * s], v[2 * s + 1]}, ws{w[2 * s], w[2 * s + 1]};
    Arith<ff>::mac(u, vs, -ws);
    c = Arith<ff>::sub_mul(c, vs, ws);
  }
  ff r = Arith<ff>::acc_get(u);
  acc_out[0] = r.hi; acc_out[1] = r.lo;
  chain_out[0] = c.hi; chain_out[1] = c.lo;
}
void h_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out) {
  u32x4 r = philox4x32_10(u32x4{ctr[0], ctr[1], ctr[2], ctr[3]}, k0, k1);
  out[0] = r.x; out[1] = r.y; out[2] = r.z; out[3] = r.w;
}
double h_uniform53(uint64_t x) { return uniform53(x); }
double h_uniform_open52(uint64_t x) { return uniform_open52(x); }
uint64_t h_word64(const uint32_t* o) { return philox_word64(u32x4{o[0], o[1], o[2], o[3]}); }

}  // extern "C"
