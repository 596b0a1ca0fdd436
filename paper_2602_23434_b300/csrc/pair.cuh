// pair.cuh -- paired-f32 arithmetic: a value is the unevaluated sum h + l of
// two floats, |l| <= ulp(h)/2 once normalised, about 48 significant bits.
//
// B300 runs FP64 (and every f64 <-> f32 conversion) at about 1/64 of the f32
// rate, so work that needs more than f32 but not all of FP64's 53 bits is
// cheaper as float pairs on the f32 pipes.  Built from error-free
// transformations: Knuth's TwoSum, Dekker's FastTwoSum, and the FMA product
// error (a*b - fl(a*b) = fma(a, b, -fl(a*b)) exactly).  Sums of products are
// accumulated as in Ogita, Rump & Oishi (2005), Algorithm Dot2: the running
// sum's high part is updated with TwoSum, and every rounding error (of the
// sums and of the products) is added into the low part.
//
// The adds here are the "sloppy" (Dekker) form: their error is about 2^-47
// of |a| + |b|, i.e. absolute, not relative to a + b.  Callers use them
// where absolute accuracy is what is needed (positions, weights, offsets).
#pragma once
#include <cuda_runtime.h>

struct f2 {
  float h, l;
};

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ f2 f2_two_sum(float a, float b) {
  const float s = a + b;
  const float bp = s - a;
  return {s, (a - (s - bp)) + (b - bp)};
}
// s + e = a + b exactly, given |a| >= |b| or a == 0 (Dekker)
__device__ __forceinline__ f2 f2_fast(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
// the pair nearest a double (its top 48 bits, rounded twice to nearest)
__device__ __forceinline__ f2 f2_of(double v) {
  const float h = __double2float_rn(v);
  return {h, __double2float_rn(v - (double)h)};
}
__host__ inline f2 f2_host(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}
__device__ __forceinline__ double f2_to(f2 a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ f2 f2_neg(f2 a) { return {-a.h, -a.l}; }

__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  const f2 s = f2_two_sum(a.h, b.h);
  return f2_fast(s.h, s.l + (a.l + b.l));
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) { return f2_add(a, f2_neg(b)); }
// a + f for a float f
__device__ __forceinline__ f2 f2_addf(f2 a, float f) {
  const f2 s = f2_two_sum(a.h, f);
  return f2_fast(s.h, s.l + a.l);
}
// product, left unnormalised: h = fl(a.h b.h), l = its rounding error plus
// the cross terms (|l| within a few ulp(h)); the a.l b.l term (2^-48 of the
// product) is dropped
__device__ __forceinline__ f2 f2_mul_u(f2 a, f2 b) {
  const float p = a.h * b.h;
  return {p, fmaf(a.l, b.h, fmaf(a.h, b.l, fmaf(a.h, b.h, -p)))};
}
__device__ __forceinline__ f2 f2_norm(f2 a) { return f2_fast(a.h, a.l); }
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) { return f2_norm(f2_mul_u(a, b)); }
__device__ __forceinline__ f2 f2_sqr_u(f2 a) {
  const float p = a.h * a.h;
  return {p, fmaf(2.0f * a.h, a.l, fmaf(a.h, a.h, -p))};
}
// scaling by a power of two is exact
__device__ __forceinline__ f2 f2_scale(f2 a, float s) { return {a.h * s, a.l * s}; }
// a < b on the represented values (both normalised)
__device__ __forceinline__ bool f2_lt(f2 a, f2 b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }
// 1/sqrt(a) for a > 0: the f32 estimate refined by one Newton step whose
// residual 1 - a y^2 is formed in pair arithmetic (quadratic convergence
// from ~2^-23 gives ~2^-46)
__device__ __forceinline__ f2 f2_rsqrt(f2 a) {
  const float y = rsqrtf(a.h);
  const f2 y2 = f2_sqr_u({y, 0.0f});                 // y^2 exactly (h + l)
  const f2 ay2 = f2_mul_u(a, f2_norm(y2));
  const f2 r = f2_add({1.0f, 0.0f}, f2_neg(f2_norm(ay2)));  // 1 - a y^2
  return f2_fast(y, 0.5f * y * r.h);
}
// sqrt(a) = a / sqrt(a), for a > 0
__device__ __forceinline__ f2 f2_sqrt(f2 a) { return f2_mul(a, f2_rsqrt(a)); }

// ---- two components at once on packed f32x2 instructions
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);  // a - b, one rounding
}
// Dot2 step for two components sharing the weight w:
// (ah, al) += w * (fh + fl), componentwise
__device__ __forceinline__ void dot2_acc2(float2& ah, float2& al, f2 w, float2 fh, float2 fl) {
  const float2 wh = make_float2(w.h, w.h), wl = make_float2(w.l, w.l);
  const float2 p = __fmul2_rn(wh, fh);
  const float2 pe = __ffma2_rn(wh, fh, make_float2(-p.x, -p.y));  // exact product error
  const float2 s = __fadd2_rn(ah, p);
  const float2 bp = sub2(s, ah);
  const float2 se = __fadd2_rn(sub2(ah, sub2(s, bp)), sub2(p, bp));  // exact sum error
  ah = s;
  al = __ffma2_rn(wl, fh, __ffma2_rn(wh, fl, __fadd2_rn(al, __fadd2_rn(se, pe))));
}
