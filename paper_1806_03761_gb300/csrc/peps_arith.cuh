// peps_arith.cuh -- scalar types of the two precision forms and the
// Philox4x32-10 generator.
//
//   double : the FP64 form.
//   float  : the FP32 form (FP32 tensors, factorisations and contractions).
//   ff     : a float-float value hi + lo (two FP32, |lo| <= ulp(hi)/2), about
//            48 significand bits, computed on the FP32 pipes.  The
//            error-free transformations are the classical ones: TwoSum
//            (Knuth, TAOCP vol. 2, 4.2.2), FastTwoSum (Dekker 1971) and the
//            FMA form of TwoProduct; addition, product, quotient and square
//            root follow the double-word algorithms of Hida, Li and Bailey
//            (ARITH 2001) with one correction step each.
#pragma once
#include <stdint.h>
#include <math.h>

#ifndef PEPS_HD
#define PEPS_HD __device__ __forceinline__
#endif

// 8-byte aligned so that a value moves in one 64-bit load or store (every ff
// array in the workspaces and in shared memory starts on an 8-byte boundary)
struct __align__(8) ff {
  float hi, lo;
};

PEPS_HD ff ff_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ff{s, e};
}
PEPS_HD ff ff_fast_two_sum(float a, float b) {  // requires |a| >= |b|
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return ff{s, e};
}
PEPS_HD ff ff_from_double(double x) {
  float h = (float)x;
  float l = (float)(x - (double)h);
  return ff{h, l};
}
PEPS_HD double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

PEPS_HD ff operator+(ff a, ff b) {
  ff s = ff_two_sum(a.hi, b.hi);
  ff t = ff_two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = ff_fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return ff_fast_two_sum(s.hi, s.lo);
}
PEPS_HD ff operator-(ff a) { return ff{-a.hi, -a.lo}; }
PEPS_HD ff operator-(ff a, ff b) { return a + (-b); }
PEPS_HD ff operator*(ff a, ff b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return ff_fast_two_sum(p, e);
}
PEPS_HD ff operator/(ff a, ff b) {
  float q1 = __fdiv_rn(a.hi, b.hi);
  ff r = a - b * ff{q1, 0.0f};
  float q2 = __fdiv_rn(r.hi, b.hi);
  return ff_fast_two_sum(q1, q2);
}
PEPS_HD ff ff_sqrt(ff a) {
  if (a.hi <= 0.0f) return ff{0.0f, 0.0f};
  float s = __fsqrt_rn(a.hi);
  ff r = a - ff{s, 0.0f} * ff{s, 0.0f};
  float c = __fdiv_rn(r.hi, __fmul_rn(2.0f, s));
  return ff_fast_two_sum(s, c);
}

// ---------------------------------------------------------------------------
// Uniform interface used by the templated kernels.
// ---------------------------------------------------------------------------
template <class R> struct Arith;

template <> struct Arith<double> {
  typedef double acc_t;
  PEPS_HD static double zero() { return 0.0; }
  PEPS_HD static double one() { return 1.0; }
  PEPS_HD static double from(double x) { return x; }
  PEPS_HD static double to(double x) { return x; }
  PEPS_HD static double hi(double x) { return x; }
  PEPS_HD static void acc_init(acc_t& a) { a = 0.0; }
  PEPS_HD static void mac(acc_t& a, double x, double y) { a = fma(x, y, a); }
  PEPS_HD static double acc_get(const acc_t& a) { return a; }
  PEPS_HD static void acc_set(acc_t& a, double x) { a = x; }
  // a += the accumulator of lane (this lane ^ o)
  PEPS_HD static void acc_shfl_add(acc_t& a, int o) { a = a + __shfl_xor_sync(0xffffffffu, a, o); }
  // x - v w in one rounding
  PEPS_HD static double sub_mul(double x, double v, double w) { return fma(-v, w, x); }
  PEPS_HD static double sqrt_(double x) { return sqrt(x); }
  PEPS_HD static double scale(double x, double s) { return x * s; }
  // relative rounding unit of the form
  PEPS_HD static double eps() { return 1.1102230246251565e-16; }
};

template <> struct Arith<float> {
  typedef float acc_t;
  PEPS_HD static float zero() { return 0.0f; }
  PEPS_HD static float one() { return 1.0f; }
  PEPS_HD static float from(double x) { return (float)x; }
  PEPS_HD static double to(float x) { return (double)x; }
  PEPS_HD static float hi(float x) { return x; }
  PEPS_HD static void acc_init(acc_t& a) { a = 0.0f; }
  PEPS_HD static void mac(acc_t& a, float x, float y) { a = fmaf(x, y, a); }
  PEPS_HD static float acc_get(const acc_t& a) { return a; }
  PEPS_HD static void acc_set(acc_t& a, float x) { a = x; }
  PEPS_HD static void acc_shfl_add(acc_t& a, int o) { a = a + __shfl_xor_sync(0xffffffffu, a, o); }
  PEPS_HD static float sub_mul(float x, float v, float w) { return fmaf(-v, w, x); }
  PEPS_HD static float sqrt_(float x) { return sqrtf(x); }
  PEPS_HD static float scale(float x, double s) { return x * (float)s; }
  PEPS_HD static double eps() { return 5.9604644775390625e-08; }  // 2^-24
};

// Compensated dot-product accumulator: the products' high parts are summed
// with TwoSum, every rounding error and low-order product term goes to c.
struct ffacc {
  float s, c;
};

template <> struct Arith<ff> {
  typedef ffacc acc_t;
  PEPS_HD static ff zero() { return ff{0.0f, 0.0f}; }
  PEPS_HD static ff one() { return ff{1.0f, 0.0f}; }
  PEPS_HD static ff from(double x) { return ff_from_double(x); }
  PEPS_HD static double to(ff x) { return ff_to_double(x); }
  PEPS_HD static float hi(ff x) { return x.hi; }
  PEPS_HD static void acc_init(acc_t& a) { a.s = 0.0f; a.c = 0.0f; }
  PEPS_HD static void mac(acc_t& a, ff x, ff y) {
    float p = __fmul_rn(x.hi, y.hi);
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    ff t = ff_two_sum(a.s, p);
    a.s = t.hi;
    a.c = __fadd_rn(a.c, __fadd_rn(t.lo, e));
  }
  PEPS_HD static ff acc_get(const acc_t& a) { return ff_fast_two_sum(a.s, a.c); }
  PEPS_HD static void acc_set(acc_t& a, ff x) { a.s = x.hi; a.c = x.lo; }
  // merge with the accumulator of lane (this lane ^ o): TwoSum of the two
  // leading sums, their error and both correction terms into c (commutative,
  // so both lanes of a pair end with the same value)
  PEPS_HD static void acc_shfl_add(acc_t& a, int o) {
    const float s2 = __shfl_xor_sync(0xffffffffu, a.s, o);
    const float c2 = __shfl_xor_sync(0xffffffffu, a.c, o);
    const ff t = ff_two_sum(a.s, s2);
    a.s = t.hi;
    a.c = __fadd_rn(__fadd_rn(a.c, c2), t.lo);
  }
  // x - v w: the high parts of x and of the exact product v.hi w.hi meet in
  // one TwoSum; the product's rounding error (FMA), its cross terms and the
  // low parts are summed in FP32 and renormalised (error a few 2^-48 of
  // |x| + |v w|, the bound the Householder updates need).
  PEPS_HD static ff sub_mul(ff x, ff v, ff w) {
    float p = __fmul_rn(v.hi, w.hi);
    float e = fmaf(v.hi, w.hi, -p);
    e = fmaf(v.hi, w.lo, e);
    e = fmaf(v.lo, w.hi, e);
    ff t = ff_two_sum(x.hi, -p);
    float l = __fadd_rn(__fsub_rn(x.lo, e), t.lo);
    return ff_two_sum(t.hi, l);  // t.hi may have cancelled below |l|
  }
  PEPS_HD static ff sqrt_(ff x) { return ff_sqrt(x); }
  PEPS_HD static ff scale(ff x, double s) { return x * ff_from_double(s); }
  PEPS_HD static double eps() { return 3.552713678800501e-15; }  // 2^-48
};

// Butterfly shuffle of a scalar of the form (components moved separately).
PEPS_HD double shfl_xor_r(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
PEPS_HD float shfl_xor_r(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
PEPS_HD ff shfl_xor_r(ff v, int o) {
  return ff{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its definition:
// ten rounds of two 32x32->64 multiplications mixing the counter with a
// Weyl-sequence key schedule.
// ---------------------------------------------------------------------------
struct u32x4 {
  uint32_t x, y, z, w;
};

PEPS_HD u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)M0 * c.x;
    uint64_t p1 = (uint64_t)M1 * c.z;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    u32x4 n;
    n.x = hi1 ^ c.y ^ k0;
    n.y = lo1;
    n.z = hi0 ^ c.w ^ k1;
    n.w = lo0;
    c = n;
    k0 += W0;
    k1 += W1;
  }
  return c;
}

PEPS_HD uint64_t philox_word64(u32x4 o) { return ((uint64_t)o.y << 32) | o.x; }
// u in [0, 1) from 53 bits
PEPS_HD double uniform53(uint64_t x) { return (double)(x >> 11) * 0x1.0p-53; }
// p in (0, 1) from 52 bits plus one half
PEPS_HD double uniform_open52(uint64_t x) { return ((double)(x >> 12) + 0.5) * 0x1.0p-52; }
