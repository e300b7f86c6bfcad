// Kernel-entry formulas of the built-in operators, shared by the sketch kernels.
//
// FP64 path: distance, phase k*r and its reduction modulo 2*pi in FP64, then
// sincos.  Mixed path, no FP64 instruction: points and k are float-float
// pairs (hi + lo); the distance is formed in float-float with Dekker/Knuth
// error-free transformations (its square root from an rsqrt estimate, one
// Newton step and a float-float correction), the phase k*r in float-float is
// reduced by pi/2 (Cody & Waite: the first product subtracted exactly by
// FMA, the second in float32), and sin/cos of the reduced argument
// |t| <= pi/4 come from near-minimax polynomials (degree 7 and 8, errors
// below 2e-9) with the quadrant applied afterwards.  Entries keep ~1.5e-7
// relative accuracy at k*r ~ 2e4.
#pragma once
#include "bf_internal.h"
#include "cx.cuh"
#include "ff.cuh"

namespace bf {
namespace dev {

__device__ __forceinline__ double2 kernel_value(int type, double wn, double tx, double ty,
                                                double tz, double sx, double sy, double sz) {
  if (type == BF_KERNEL_DFT) {
    double sn, cs;
    sincospi(-2.0 * tx * sx, &sn, &cs);
    return make_double2(cs, sn);
  }
  const double dx = tx - sx, dy = ty - sy, dz = tz - sz;
  const double r = sqrt(dx * dx + dy * dy + dz * dz);
  const double ph = wn * r;
  // reduce the phase to [-pi, pi] before the trigonometric evaluation
  const double q = rint(ph * 0.15915494309189535);
  const double red = fma(-q, 6.283185307179586, ph) - q * 2.4492935982947064e-16;
  double sn, cs;
  sincos(red, &sn, &cs);
  if (type == BF_KERNEL_HELMHOLTZ_2D) {   // exp(-i k r) / r
    const double ir = 1.0 / r;
    return make_double2(cs * ir, -sn * ir);
  }
  const double ir = 0.07957747154594767 / r;   // exp(i k r) / (4 pi r)
  return make_double2(cs * ir, sn * ir);
}

// pi/2 ~ C1 + C2 (each the float nearest to the remainder; the next term,
// -1.7e-15, is below what the reduction needs) and 2/pi
#define BF_PIO2_1 1.57079637050628662e+00f
#define BF_PIO2_2 -4.37113882867379289e-08f
#define BF_2OPI 6.36619746685028076e-01f

// sin t and cos t for |t| <= pi/4: near-minimax polynomials (absolute error
// 1.8e-9 and 5.4e-11 before float32 rounding; coefficients from a Remez
// exchange, fit_sincos.py)
#define BF_S3 -1.666665077e-01f
#define BF_S5 8.331978694e-03f
#define BF_S7 -1.949563593e-04f
#define BF_C2 -5.000000000e-01f
#define BF_C4 4.166662320e-02f
#define BF_C6 -1.388676348e-03f
#define BF_C8 2.439045056e-05f
__device__ __forceinline__ void sincos_poly(float t, float& s, float& c) {
  const float t2 = t * t;
  float ps = fmaf(t2, BF_S7, BF_S5);
  ps = fmaf(t2, ps, BF_S3);
  s = fmaf(t * t2, ps, t);
  float pc = fmaf(t2, BF_C8, BF_C6);
  pc = fmaf(t2, pc, BF_C4);
  pc = fmaf(t2, pc, BF_C2);
  c = fmaf(t2, pc, 1.0f);
}

// 1/sqrt(x), the hardware approximation (PTX rsqrt.approx.ftz.f32)
__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Magic constant 1.5 * 2^23: for |v| < 2^22, fmaf(x, y, MAGIC) - MAGIC is
// x*y rounded to the nearest integer, and the low bits of the sum's encoding
// hold that integer modulo 2^22 (two's complement).
#define BF_RND_MAGIC 12582912.0f

// e^{i phi} for a float-float phase ph (|ph.l| <= ulp(ph.h)): phi = q pi/2
// + t.  ph.h - q C1 is exact in one FMA (C1, the float nearest pi/2, is a
// multiple of 2^-23 and |result| < 1); the C2 term and ph.l are ~1e-3 and
// added in float32 (error ~1e-10), the C3 term (< 1e-10) is dropped; t then
// carries one rounding (<= 4.7e-8).  The quadrant q mod 4 swaps sin/cos and
// sets signs; `neg` (0 or the sign bit) also flips sin.  Returns
// (cos phi, +-sin phi).
__device__ __forceinline__ float2 expi_ff(FF ph, unsigned neg) {
  const float qm = fmaf(ph.h, BF_2OPI, BF_RND_MAGIC);
  const float q = qm - BF_RND_MAGIC;
  const unsigned qi = (unsigned)__float_as_int(qm);
  const float t = fmaf(-q, BF_PIO2_1, ph.h) + fmaf(-q, BF_PIO2_2, ph.l);
  float sv, cv;
  sincos_poly(t, sv, cv);
  float sn = (qi & 1) ? cv : sv, cs = (qi & 1) ? sv : cv;
  sn = __uint_as_float(__float_as_uint(sn) ^ (((qi & 2u) << 30) ^ neg));
  cs = __uint_as_float(__float_as_uint(cs) ^ (((qi + 1u) & 2u) << 30));
  return make_float2(cs, sn);
}

// Float-float difference and sum left unnormalised (hi + lo with |lo| a
// few ulps of hi): their consumers below (squares, the square root's
// correction, the phase) use both parts.
__device__ __forceinline__ FF ff_sub_u(float ah, float al, float bh, float bl) {
  FF d = two_sum(ah, -bh);
  d.l += al - bl;
  return d;
}
__device__ __forceinline__ FF ff_add_u(FF a, FF b) {
  FF s = two_sum(a.h, b.h);
  s.l += a.l + b.l;
  return s;
}

// Helmholtz kernel entry at the float-float row point rp = (x, y, z as
// hi/lo pairs) and column point (cxh + cxl, cyh + cyl, czh + czl):
// returns (cos(k r) a, +-sin(k r) a) with a = 1/r (2D) or 1/(4 pi r) (3D),
// the sine negated when neg is the sign bit (exp(-i k r) in 2D, conjugates).
template <bool D3>
__device__ __forceinline__ float2 helmholtz_ff(const float (&rp)[6], float cxh, float cxl, float cyh, float cyl,
                                               float czh, float czl, float kh, float kl, unsigned neg) {
  FF r2 = ff_sq(ff_sub_u(rp[0], rp[1], cxh, cxl));
  r2 = ff_add_u(r2, ff_sq(ff_sub_u(rp[2], rp[3], cyh, cyl)));
  if (D3) r2 = ff_add_u(r2, ff_sq(ff_sub_u(rp[4], rp[5], czh, czl)));
  // 1/sqrt(r2): estimate and one Newton step; r = sqrt(r2) = rh0 + rl
  // corrected in float-float
  float rs = rsqrt_approx(r2.h);
  rs = rs * fmaf(-0.5f * r2.h * rs, rs, 1.5f);
  const float rh0 = r2.h * rs;
  const FF e = two_prod(rh0, rh0);
  const float num = ((r2.h - e.h) - e.l) + r2.l;
  const float rl = num * (0.5f * rs);
  // phase k * r
  FF ph = two_prod(kh, rh0);
  ph.l = fmaf(kh, rl, fmaf(kl, rh0, ph.l));
  const float2 c = expi_ff(ph, neg);
  const float a = D3 ? 0.0795774715f * rs : rs;
  return make_float2(c.x * a, c.y * a);
}

// DFT entry exp(-2 pi i t s) at float-float t = th + tl, s = sh + sl.
__device__ __forceinline__ float2 dft_ff(float th, float tl, float sh, float sl) {
  FF u = two_prod(th, sh);
  u.l = fmaf(th, sl, fmaf(tl, sh, u.l));
  const float q = rintf(u.h);
  const FF f = two_sum(u.h - q, u.l);     // u.h - q exact (Sterbenz)
  float sn, cs;
  sincospif(-2.0f * f.h, &sn, &cs);
  const float d = -6.28318531f * f.l;     // first-order correction
  return make_float2(cs - d * sn, sn + d * cs);
}

// Per-thread evaluation context of one job's entries, held in registers so
// that the entry loop neither reloads the job descriptor nor the thread's row
// point.  The kernels depend on the points only through |t - s| (the DFT
// through the symmetric product t*s), so the adjoint (op C) evaluates the same
// formula with sources as rows and targets as columns, then conjugates.
template <typename R>
struct Entry;

template <>
struct Entry<float> {
  int kind, type, conj;
  float kh, kl;
  const float* colp;   // float-float SoA of the column point set
  int64_t coln;
  const float2* A;
  int64_t lda;
  int opN;
  float rp[6];         // this thread's row point (x, y, z as hi/lo)

  __device__ __forceinline__ void init(const SketchJob& J, int64_t row, bool valid) {
    kind = J.kind;
    type = J.ktype;
    opN = J.op == BF_OP_N;
    conj = !opN;
    kh = J.kh;
    kl = J.kl;
    A = (const float2*)J.A;
    lda = J.lda;
    const float* rowp = opN ? J.tgtF : J.srcF;
    const int64_t rown = opN ? J.m : J.n;
    colp = opN ? J.srcF : J.tgtF;
    coln = opN ? J.n : J.m;
#pragma unroll
    for (int d = 0; d < 6; ++d) rp[d] = (kind == 1 && valid) ? rowp[d * rown + row] : 0.f;
  }

  __device__ __forceinline__ float2 get(int64_t row, int64_t kk) const {
    float2 v;
    if (kind == 0) {
      if (opN) return A[row + kk * lda];
      v = A[kk + row * lda];
    } else {
      v = value(kk);
    }
    if (conj) v.y = -v.y;
    return v;
  }

  // K(row point, column point kk)
  __device__ __forceinline__ float2 value(int64_t kk) const {
    const float* c = colp + kk;
    if (type == BF_KERNEL_DFT) return dft_ff(rp[0], rp[1], c[0], c[coln]);
    if (type == BF_KERNEL_HELMHOLTZ_3D)
      return helmholtz_ff<true>(rp, c[0], c[coln], c[2 * coln], c[3 * coln], c[4 * coln], c[5 * coln], kh, kl, 0u);
    // exp(-i k r) / r
    return helmholtz_ff<false>(rp, c[0], c[coln], c[2 * coln], c[3 * coln], 0.f, 0.f, kh, kl, 0x80000000u);
  }
};

template <>
struct Entry<double> {
  int kind, type, opN;
  double wn;
  const double* colp;
  int64_t coln;
  const double2* A;
  int64_t lda;
  double rp[3];

  __device__ __forceinline__ void init(const SketchJob& J, int64_t row, bool valid) {
    kind = J.kind;
    type = J.ktype;
    opN = J.op == BF_OP_N;
    wn = J.wn;
    A = (const double2*)J.A;
    lda = J.lda;
    const double* rowp = opN ? J.tgt : J.src;
    const int64_t rown = opN ? J.m : J.n;
    colp = opN ? J.src : J.tgt;
    coln = opN ? J.n : J.m;
#pragma unroll
    for (int d = 0; d < 3; ++d) rp[d] = (kind == 1 && valid) ? rowp[d * rown + row] : 0.0;
  }

  __device__ __forceinline__ double2 get(int64_t row, int64_t kk) const {
    double2 v;
    if (kind == 0) {
      if (opN) return A[row + kk * lda];
      v = A[kk + row * lda];
    } else {
      const double* c = colp + kk;
      v = kernel_value(type, wn, rp[0], rp[1], rp[2], c[0], c[coln], c[2 * coln]);
      if (opN) return v;
    }
    v.y = -v.y;
    return v;
  }
};

}  // namespace dev
}  // namespace bf
