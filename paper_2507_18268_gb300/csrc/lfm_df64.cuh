// Double-float ("df64") arithmetic on the FP32 pipe.
//
// GB300 issues FP64 instructions at about 1/64 of its FP32 rate, so a step that does every
// per-cell operation in FP64 is bound by the FP64 pipe long before HBM. A df64 value is the
// unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2: a 48-bit significand
// (unit roundoff 2^-48, about 3.6e-15) with FP32's exponent range. Every operation below is
// built from error-free transformations of FP32 operations:
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s = fl(a + b) and e with s + e = a + b exactly;
//   Fast2Sum (Dekker 1971): the same in three operations when |a| >= |b|;
//   the exact product: p = fl(a b), e = fma(a, b, -p), p + e = a b exactly.
// The compositions (sum, product, fused multiply-add, Newton reciprocal) follow the
// double-word algorithms of Dekker (1971) and Hida, Li & Bailey ("Library for double-double
// and quad-double arithmetic", 2001). All FP32 operations are written with the _rn
// intrinsics so that the compiler neither contracts nor reorders them.
#pragma once

#include <cuda_runtime.h>

namespace lfm {
namespace {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df mkdf(float h, float l) { return df{h, l}; }
__device__ __forceinline__ df ld_df(const float2* p) {
  const float2 v = *p;
  return df{v.x, v.y};
}
__device__ __forceinline__ df ldg_df(const float2* p) {
  const float2 v = __ldg(p);
  return df{v.x, v.y};
}
__device__ __forceinline__ void st_df(float2* p, df v) { *p = make_float2(v.hi, v.lo); }

// s + e == a + b exactly (any a, b).
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df{s, e};
}

// s + e == a + b exactly when |a| >= |b| or a == 0.
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}

// p + e == a * b exactly (barring underflow).
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return df{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }
__device__ __forceinline__ df df_abs(df a) { return a.hi < 0.0f ? df_neg(a) : a; }

// a + b: exact sum of the leading parts, the trailing parts added to its error.
__device__ __forceinline__ df df_add(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, e);
}
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// a * b: exact product of the leading parts plus the two cross terms (lo * lo is below
// the format's precision).
__device__ __forceinline__ df df_mul(df a, df b) {
  const df p = two_prod(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.lo, p.lo);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p.hi, e);
}

// a * b + c with one renormalisation.
__device__ __forceinline__ df df_fma(df a, df b, df c) {
  const df p = two_prod(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.lo, p.lo);
  e = __fmaf_rn(a.lo, b.hi, e);
  const df s = two_sum(p.hi, c.hi);
  const float t = __fadd_rn(s.lo, __fadd_rn(e, c.lo));
  return fast_two_sum(s.hi, t);
}

// 1 / a: the FP32 reciprocal of the leading part, refined by one Newton step
// y' = y + y (1 - a y) evaluated in df64 (quadratic convergence: 2^-24 -> ~2^-47).
__device__ __forceinline__ df df_rcp(df a) {
  const float y = __frcp_rn(a.hi);
  const df ay = df_mul(a, df{y, 0.0f});
  const df e = df_sub(df{1.0f, 0.0f}, ay);
  return fast_two_sum(y, __fmul_rn(y, e.hi));
}

// Conversions (the FP64 side runs once per cell per launch, or in set-up kernels).
__device__ __forceinline__ df df_from_double(double d) {
  const float h = __double2float_rn(d);
  return df{h, __double2float_rn(d - (double)h)};
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// ---- triple-float: the field ------------------------------------------------------------
// T itself is kept as hi + mid + lo (three FP32 numbers, ~72 significand bits): every flux
// and every ddt term is a difference of two field values, formed exactly from the three
// parts, so the field's rounding never enters the method at the 2^-48 level of df64 (it
// would otherwise be injected every step at 2^-48 |T|, far above FP64's 2^-53 |T|).
struct tf {
  float hi, mid, lo;
};

__device__ __forceinline__ tf ld_tf(const float2* hm, const float* l, int c) {
  const float2 v = hm[c];
  return tf{v.x, v.y, l[c]};
}
__device__ __forceinline__ void st_tf(float2* hm, float* l, int c, tf v) {
  hm[c] = make_float2(v.hi, v.mid);
  l[c] = v.lo;
}

// x + d (d df64, |d| typically far below |x|): exact sums of the matching parts, then
// renormalised so that each part is below half an ulp of the one before.
__device__ __forceinline__ tf tf_add_df(tf a, df b) {
  const df s0 = two_sum(a.hi, b.hi);
  const df s1 = two_sum(a.mid, b.lo);
  const df t = two_sum(s1.hi, s0.lo);
  const float r2 = __fadd_rn(__fadd_rn(s1.lo, t.lo), a.lo);
  const df u = two_sum(s0.hi, t.hi);
  const df v = two_sum(u.lo, r2);
  const df w = fast_two_sum(u.hi, v.hi);
  return tf{w.hi, w.lo, v.lo};
}

// a - b as df64, for field values: the leading difference is exact (Sterbenz) when the two
// are within a factor of two, and every rounding error is collected, so the difference
// keeps df64's relative accuracy.
__device__ __forceinline__ df tf_diff(tf a, tf b) {
  const df s0 = two_sum(a.hi, -b.hi);
  const df s1 = two_sum(a.mid, -b.mid);
  const float s2 = __fsub_rn(a.lo, b.lo);
  const df t = two_sum(s1.hi, s0.lo);
  const df h = two_sum(s0.hi, t.hi);
  const float l = __fadd_rn(h.lo, __fadd_rn(t.lo, __fadd_rn(s1.lo, s2)));
  return fast_two_sum(h.hi, l);
}

__device__ __forceinline__ df tf_to_df(tf a) { return fast_two_sum(a.hi, a.mid); }

__device__ __forceinline__ tf tf_from_double(double d) {
  const float h = __double2float_rn(d);
  const double r = d - (double)h;  // exact
  const float m = __double2float_rn(r);
  return tf{h, m, __double2float_rn(r - (double)m)};
}
__device__ __forceinline__ double tf_to_double(tf a) { return ((double)a.hi + (double)a.mid) + (double)a.lo; }

// Per-thread running sum of df64 terms: the leading parts through TwoSum, their rounding
// errors and the trailing parts collected in lo. Converted to FP64 once per thread; the
// block and team reductions then run in FP64.
struct DfAcc {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add(df v) {
    const df s = two_sum(hi, v.hi);
    hi = s.hi;
    lo = __fadd_rn(lo, __fadd_rn(s.lo, v.lo));
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

}  // namespace
}  // namespace lfm
