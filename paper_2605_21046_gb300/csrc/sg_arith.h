// Arithmetic policies of the apply kernels.
//
// F64  native IEEE double arithmetic (the FP64 pipe: 2 FMA lanes per clock per
//      SM on GB300).
// DW   double-word arithmetic: a value is an unevaluated sum hi + lo of two
//      floats, computed on the FP32 pipe (128 lanes per clock per SM) with
//      error-free transformations: the exact product error by FMA
//      (p = a*b, e = fma(a, b, -p)) and Knuth's TwoSum for additions.  The
//      significand is about 48 bits; one multiply-add costs 12 FP32
//      instructions.  Conversions to and from double are done with integer
//      bit operations, so the FP64 pipe is not used at all.
//
// Both policies expose the same operations:
//   T     value type (8 bytes; shared-memory storage type)
//   in(double)            convert an input
//   cmul(c, x) / cfma(c, x, acc)   multiply by / accumulate a compile-time
//                         constant c = {double, float hi, float lo}
//   mul(a, b) / fma(a, b, acc)     runtime operands
//   fin(acc)              normalise an accumulated value
//   add_out(y, v)         atomically add v into the double at y
#pragma once
#include <cuda_runtime.h>

namespace sg {

// A compile-time constant with its double-word split (hi + lo floats).
struct Cf {
  double c;
  float h, l;
};

struct F64 {
  using T = double;
  using IO = double;
  static constexpr bool kDW = false;
  __device__ __forceinline__ static T in(double x) { return x; }
  __device__ __forceinline__ static T zero() { return 0.0; }
  __device__ __forceinline__ static T cmul(Cf c, T x) { return c.c * x; }
  __device__ __forceinline__ static void cfma(Cf c, T x, T& acc) { acc = ::fma(c.c, x, acc); }
  __device__ __forceinline__ static T mul(T a, T b) { return a * b; }
  __device__ __forceinline__ static void fma(T a, T b, T& acc) { acc = ::fma(a, b, acc); }
  __device__ __forceinline__ static T add(T a, T b) { return a + b; }
  __device__ __forceinline__ static T neg(T a) { return -a; }
  __device__ __forceinline__ static T fin(T a) { return a; }
  __device__ __forceinline__ static void add_out(double* y, T v) { atomicAdd(y, v); }
};

struct __align__(8) dw {
  float h, l;
};

struct DW {
  using T = dw;
  using IO = double;
  static constexpr bool kDW = true;

  __device__ __forceinline__ static void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  }

  // double -> (hi, lo) with integer operations: hi keeps the leading 24
  // significant bits (truncated), lo is the rounded remainder.  Relative
  // error <= 2^-48 for 2^-74 <= |x| < 2^127; smaller magnitudes keep only hi
  // (subnormal and zero inputs give 0).
  __device__ __forceinline__ static T in(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int top = (unsigned int)(b >> 32);
    const int e = (int)((top >> 20) & 0x7ff);
    const unsigned int sign = top & 0x80000000u;
    const int ef = e - 1023 + 127;
    if (ef <= 0) return {0.0f, 0.0f};
    if (e == 0x7ff) return {__uint_as_float(sign | 0x7f800000u | ((b & 0x000fffffffffffffull) ? 0x400000u : 0u)), 0.0f};
    if (ef >= 255) return {__uint_as_float(sign | 0x7f800000u), 0.0f};
    const unsigned long long frac = b & 0x000fffffffffffffull;
    const float h = __uint_as_float(sign | ((unsigned int)ef << 23) | (unsigned int)(frac >> 29));
    const unsigned int r = (unsigned int)(frac & 0x1fffffffu);   // 29 low bits
    float l = 0.0f;
    const int es = ef - 52;                                      // exponent field of 2^(E-52)
    if (es >= 1 && r) {
      l = __fmul_rn(__uint2float_rn(r), __uint_as_float((unsigned int)es << 23));
      if (sign) l = -l;
    }
    return {h, l};
  }

  // float -> the bits of the same value as a double (exact; subnormal -> 0)
  __device__ __forceinline__ static double widen(float f) {
    const unsigned int u = __float_as_uint(f);
    const unsigned int ef = (u >> 23) & 0xffu;
    if (ef == 0) return 0.0;
    if (ef == 0xffu)
      return __longlong_as_double((long long)(((unsigned long long)(u & 0x80000000u) << 32) | 0x7ff0000000000000ull |
                                              ((unsigned long long)(u & 0x7fffffu) << 29)));
    const unsigned long long bits = ((unsigned long long)(u & 0x80000000u) << 32) |
                                    ((unsigned long long)(ef - 127 + 1023) << 52) |
                                    ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)bits);
  }

  __device__ __forceinline__ static T zero() { return {0.0f, 0.0f}; }

  // c * x for a compile-time constant c
  __device__ __forceinline__ static T cmul(Cf c, T x) {
    if (c.c == 1.0) return x;
    if (c.c == -1.0) return {-x.h, -x.l};
    const float p = __fmul_rn(c.h, x.h);
    float e = __fmaf_rn(c.h, x.h, -p);
    e = __fmaf_rn(c.h, x.l, e);
    if (c.l != 0.0f) e = __fmaf_rn(c.l, x.h, e);
    return {p, e};
  }
  __device__ __forceinline__ static void acc_add(T& acc, float ph, float pl) {
    float s, err;
    two_sum(acc.h, ph, s, err);
    acc.h = s;
    acc.l = __fadd_rn(acc.l, __fadd_rn(pl, err));
  }
  __device__ __forceinline__ static void cfma(Cf c, T x, T& acc) {
    const T p = cmul(c, x);
    acc_add(acc, p.h, p.l);
  }
  __device__ __forceinline__ static T mul(T a, T b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return {p, e};
  }
  __device__ __forceinline__ static void fma(T a, T b, T& acc) {
    const T p = mul(a, b);
    acc_add(acc, p.h, p.l);
  }
  __device__ __forceinline__ static T add(T a, T b) {
    T s = a;
    acc_add(s, b.h, b.l);
    return s;
  }
  __device__ __forceinline__ static T neg(T a) { return {-a.h, -a.l}; }
  __device__ __forceinline__ static T fin(T a) {
    float s, e;
    two_sum(a.h, a.l, s, e);
    return {s, e};
  }
  __device__ __forceinline__ static void add_out(double* y, T v) {
    atomicAdd(y, widen(v.h));
    if (v.l != 0.0f) atomicAdd(y, widen(v.l));
  }
};

// Native single precision (the FP32 pipe); used by the multigrid
// preconditioner, whose vectors are float.
struct F32 {
  using T = float;
  using IO = float;
  static constexpr bool kDW = false;
  __device__ __forceinline__ static T in(double x) { return (float)x; }
  __device__ __forceinline__ static T in(float x) { return x; }
  __device__ __forceinline__ static T zero() { return 0.0f; }
  __device__ __forceinline__ static T cmul(Cf c, T x) { return c.h * x; }
  __device__ __forceinline__ static void cfma(Cf c, T x, T& acc) { acc = fmaf(c.h, x, acc); }
  __device__ __forceinline__ static T mul(T a, T b) { return a * b; }
  __device__ __forceinline__ static void fma(T a, T b, T& acc) { acc = fmaf(a, b, acc); }
  __device__ __forceinline__ static T add(T a, T b) { return a + b; }
  __device__ __forceinline__ static T neg(T a) { return -a; }
  __device__ __forceinline__ static T fin(T a) { return a; }
  __device__ __forceinline__ static void add_out(float* y, T v) { atomicAdd(y, v); }
};

}  // namespace sg
