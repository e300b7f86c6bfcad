// Float-float (hi + lo, unevaluated sum of two float32) arithmetic from
// error-free transformations: Knuth's two-sum, Dekker's product with FMA,
// and Dekker/Karp-Markstein one-step corrections for quotient and square
// root.  About 46-48 significant bits on the FP32 pipe, which on this GPU
// issues 64x the FP64 pipe's lane rate.
#pragma once

namespace bf {
namespace dev {

struct FF {
  float h, l;
};

// s + e == a + b exactly (Knuth)
__device__ __forceinline__ FF two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
// s + e == a + b exactly when |a| >= |b| or a == 0 (Dekker)
__device__ __forceinline__ FF fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
// p + e == a * b exactly (FMA)
__device__ __forceinline__ FF two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ FF ff_sq(FF a) {
  FF p = two_prod(a.h, a.h);
  p.l = fmaf(2.0f * a.h, a.l, p.l);
  return p;
}
// renormalise an unnormalised pair (no ordering assumed)
__device__ __forceinline__ FF ff_norm(FF a) {
  return two_sum(a.h, a.l);
}
__device__ __forceinline__ FF ff_neg(FF a) { return {-a.h, -a.l}; }
// a + b (the low words added in float32: error ~2^-46 (|a| + |b|))
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  FF s = two_sum(a.h, b.h);
  s.l += a.l + b.l;
  return fast_two_sum(s.h, s.l);
}
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  FF p = two_prod(a.h, b.h);
  p.l = fmaf(a.h, b.l, fmaf(a.l, b.h, p.l));
  return fast_two_sum(p.h, p.l);
}
// acc += a * b with acc left unnormalised: the high words are summed
// error-free, every rounding error and the cross terms collect in acc.l
// (the a.l * b.l term, 2^-48 relative, is dropped)
__device__ __forceinline__ void ff_mac(FF& acc, FF a, FF b) {
  const float p = a.h * b.h;
  const float e = fmaf(a.h, b.h, -p);
  const FF s = two_sum(acc.h, p);
  acc.h = s.h;
  acc.l += s.l + fmaf(a.h, b.l, fmaf(a.l, b.h, e));
}
// a / b: float32 quotient q, then q + (a - q b) / b with the residual
// formed from the exact product q * b.h (Dekker)
__device__ __forceinline__ FF ff_div(FF a, FF b) {
  const float q = a.h / b.h;
  const FF p = two_prod(q, b.h);
  const float r = ((a.h - p.h) - p.l) + a.l - q * b.l;
  return fast_two_sum(q, r / b.h);
}
// sqrt(a), a >= 0: float32 root y, then y + (a - y^2) / (2 y) (Karp-Markstein)
__device__ __forceinline__ FF ff_sqrt(FF a) {
  if (!(a.h > 0.0f)) return {0.0f, 0.0f};
  const float y = sqrtf(a.h);
  const FF p = two_prod(y, y);
  const float r = ((a.h - p.h) - p.l) + a.l;
  return fast_two_sum(y, r / (2.0f * y));
}

}  // namespace dev
}  // namespace bf
