// Sketch products of the built-in black boxes (Alg. 2 input; Sec. 4.1):
// Y = A X or Y = A^H X in tree order for a dense stored A or for entries
// K(t_i, s_j) formed on the fly from the point sets, with the structured
// random matrices of Sec. 4.1 handled by skipping their zero blocks: output
// column group g only sums over the input rows of node g,
//   op N: Y[:, g*k + c] = sum_{j in S_g} A[:, j] X[j, c]
//   op C: Y[:, g*k + c] = sum_{i in T_g} conj(A[i, :]) X[i, c].
//
// Complex GEMM on the SIMT pipes: a GM x GN output tile per 256-thread CTA,
// K streamed in chunks of 16 through shared memory.  GN covers the whole
// sketch width (up to 64 columns) so each kernel entry is formed once per
// row tile.  FP64 path: complex128 throughout.  Mixed path: complex64
// operands, each 16-term chunk accumulated in FP32 and merged into a
// (hi, lo) FP32 pair with Knuth's TwoSum, so the long dot products (K up to
// n) keep ~FP32 accuracy instead of losing sqrt(K).
//
// Kernel entries.  FP64 path: distance, phase k*r and its reduction modulo
// 2*pi in FP64, then sincos.  Mixed path: no FP64 instruction at all -- the
// points and k are held as float-float pairs (hi + lo), the distance, k*r
// and the reduction by a three-part split of 2*pi (Cody & Waite) are
// carried in float-float (Dekker/Knuth error-free transformations), and the
// reduced phase theta_hi + theta_lo is evaluated as sincosf(theta_hi)
// corrected to first order in theta_lo.  The phase of an oscillatory kernel
// with k*r ~ 1e4 keeps ~1e-9 rad absolute accuracy.
#include <algorithm>

#include "bf_internal.h"
#include "cx.cuh"

namespace bf {

namespace {
constexpr int GM = 64, GK = 16, GT = 256;

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

// ---- float-float (hi + lo) arithmetic: error-free transformations ----
struct FF {
  float h, l;
};
__device__ __forceinline__ FF two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ FF fast_two_sum(float a, float b) {   // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ FF two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ FF ff_sub(float ah, float al, float bh, float bl) {
  FF d = two_sum(ah, -bh);
  d.l += al - bl;
  return fast_two_sum(d.h, d.l);
}
__device__ __forceinline__ FF ff_sq(FF a) {
  FF p = two_prod(a.h, a.h);
  p.l = fmaf(2.0f * a.h, a.l, p.l);
  return p;
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  FF s = two_sum(a.h, b.h);
  s.l += a.l + b.l;
  return fast_two_sum(s.h, s.l);
}

// 2*pi = C1 + C2 + C3 (each the float nearest to the remainder)
#define BF_2PI_1 6.28318548202514648f
#define BF_2PI_2 -1.74845553146951716e-07f
#define BF_2PI_3 -6.86049804002352749e-15f
#define BF_INV_2PI 0.159154943091895336f

struct PointsFF {
  const float* p;   // [x_hi, x_lo, y_hi, y_lo, z_hi, z_lo] x count
  int64_t count;
  __device__ __forceinline__ float c(int d, int64_t i) const { return p[d * count + i]; }
};

// exp(-i k r)/r or exp(i k r)/(4 pi r) (or the DFT phase) in float-float.
__device__ __forceinline__ float2 kernel_value_ff(int type, float kh, float kl, const PointsFF& T,
                                                  int64_t it, const PointsFF& S, int64_t is) {
  if (type == BF_KERNEL_DFT) {
    // phase in turns u = t * s with t = t_hi + t_lo, s exact integer
    FF u = two_prod(T.c(0, it), S.c(0, is));
    u.l = fmaf(T.c(1, it), S.c(0, is), u.l);
    const float q = rintf(u.h);
    FF f = two_sum(u.h - q, u.l);     // u.h - q exact (Sterbenz)
    float sn, cs;
    sincospif(-2.0f * f.h, &sn, &cs);
    const float d = -6.28318531f * f.l;   // first-order correction
    return make_float2(cs - d * sn, sn + d * cs);
  }
  FF r2 = ff_sq(ff_sub(T.c(0, it), T.c(1, it), S.c(0, is), S.c(1, is)));
  r2 = ff_add(r2, ff_sq(ff_sub(T.c(2, it), T.c(3, it), S.c(2, is), S.c(3, is))));
  r2 = ff_add(r2, ff_sq(ff_sub(T.c(4, it), T.c(5, it), S.c(4, is), S.c(5, is))));
  // r = sqrt(r2) with one Newton correction in float-float
  const float rh0 = sqrtf(r2.h);
  const FF e = two_prod(rh0, rh0);
  const float num = ((r2.h - e.h) - e.l) + r2.l;
  const FF r = fast_two_sum(rh0, num * (0.5f / rh0));
  // phase k * r
  FF ph = two_prod(kh, r.h);
  ph.l = fmaf(kh, r.l, fmaf(kl, r.h, ph.l));
  ph = fast_two_sum(ph.h, ph.l);
  // reduction: theta = ph - q * 2 pi, q * C1 subtracted exactly by FMA
  const float q = rintf(ph.h * BF_INV_2PI);
  const float t1 = fmaf(-q, BF_2PI_1, ph.h);
  const FF m2 = two_prod(q, BF_2PI_2);
  FF th = two_sum(t1, -m2.h);
  th.l += (ph.l - m2.l) - q * BF_2PI_3;
  th = fast_two_sum(th.h, th.l);
  float sn, cs;
  sincosf(th.h, &sn, &cs);
  const float s1 = fmaf(th.l, cs, sn), c1 = fmaf(-th.l, sn, cs);
  if (type == BF_KERNEL_HELMHOLTZ_2D) {
    const float ir = 1.0f / r.h;
    return make_float2(c1 * ir, -s1 * ir);
  }
  const float ir = 0.0795774715f / r.h;
  return make_float2(c1 * ir, s1 * ir);
}

template <typename R, int Q>
struct Acc;
template <int Q>
struct Acc<double, Q> {
  double2 v[Q];
  __device__ void zero() {
#pragma unroll
    for (int q = 0; q < Q; ++q) v[q] = make_double2(0.0, 0.0);
  }
  __device__ __forceinline__ double2& chunk(int q) { return v[q]; }
  __device__ __forceinline__ void begin_chunk() {}
  __device__ __forceinline__ void end_chunk() {}
  __device__ __forceinline__ double2 result(int q) const { return v[q]; }
};
template <int Q>
struct Acc<float, Q> {
  float2 part[Q], hi[Q], lo[Q];
  __device__ void zero() {
#pragma unroll
    for (int q = 0; q < Q; ++q)
      part[q] = make_float2(0.f, 0.f), hi[q] = make_float2(0.f, 0.f), lo[q] = make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ float2& chunk(int q) { return part[q]; }
  __device__ __forceinline__ void begin_chunk() {
#pragma unroll
    for (int q = 0; q < Q; ++q) part[q] = make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ void end_chunk() {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      FF a = two_sum(hi[q].x, part[q].x);
      FF b = two_sum(hi[q].y, part[q].y);
      hi[q].x = a.h, lo[q].x += a.l;
      hi[q].y = b.h, lo[q].y += b.l;
    }
  }
  __device__ __forceinline__ float2 result(int q) const {
    return make_float2(hi[q].x + lo[q].x, hi[q].y + lo[q].y);
  }
};
}  // namespace

// Element (r, kk) of the job's operator in the orientation of its product.
template <typename R>
struct JobElem;
template <>
struct JobElem<double> {
  static __device__ __forceinline__ double2 get(const SketchJob& J, int64_t r, int64_t kk) {
    double2 v;
    if (J.kind == 0) {
      const double2* A = (const double2*)J.A;
      if (J.op == BF_OP_N) return A[r + kk * J.lda];
      v = A[kk + r * J.lda];
    } else {
      const int64_t it = J.op == BF_OP_N ? r : kk, is = J.op == BF_OP_N ? kk : r;
      v = kernel_value(J.ktype, J.wn, J.tgt[it], J.tgt[J.m + it], J.tgt[2 * J.m + it], J.src[is],
                       J.src[J.n + is], J.src[2 * J.n + is]);
      if (J.op == BF_OP_N) return v;
    }
    v.y = -v.y;
    return v;
  }
};
template <>
struct JobElem<float> {
  static __device__ __forceinline__ float2 get(const SketchJob& J, int64_t r, int64_t kk) {
    float2 v;
    if (J.kind == 0) {
      const float2* A = (const float2*)J.A;
      if (J.op == BF_OP_N) return A[r + kk * J.lda];
      v = A[kk + r * J.lda];
    } else {
      const PointsFF T{J.tgtF, J.m}, S{J.srcF, J.n};
      if (J.op == BF_OP_N) return kernel_value_ff(J.ktype, J.kh, J.kl, T, r, S, kk);
      v = kernel_value_ff(J.ktype, J.kh, J.kl, T, kk, S, r);
    }
    v.y = -v.y;
    return v;
  }
};

struct SketchTile {
  int32_t job, group, col0, pad;
  int64_t row0;
};

// One CTA computes a GM x GN tile of one job's group; each thread owns one
// row and GN/4 columns.
template <typename R, int GN>
__global__ void __launch_bounds__(GT)
sketch_job_kernel(const SketchJob* __restrict__ jobs, const SketchTile* __restrict__ tiles) {
  using V = typename Cx<R>::V;
  constexpr int Q = GN / 4;
  __shared__ V sA[GK][GM + 1];
  __shared__ V sB[GK][GN + 1];
  __shared__ SketchJob J;
  __shared__ SketchTile T;
  if (threadIdx.x == 0) {
    T = tiles[blockIdx.x];
    J = jobs[T.job];
  }
  __syncthreads();
  const int64_t row0 = T.row0;
  const int col0 = T.col0, g = T.group;
  const int64_t M = J.M, kcols = J.kcols;
  const int64_t klo = J.d_off ? J.d_off[g] : 0;
  const int64_t khi = J.d_off ? J.d_off[g + 1] : J.Ktot;
  const V* __restrict__ X = (const V*)J.X;
  V* __restrict__ Y = (V*)J.Y;
  const int64_t ldx = J.ldx, ldy = J.ldy;
  const int tr = threadIdx.x % GM, tc = threadIdx.x / GM;   // tc 0..3
  Acc<R, Q> acc;
  acc.zero();
  const bool kf = J.kind == 0 && J.op != BF_OP_N;   // dense adjoint: K is contiguous
  for (int64_t k0 = klo; k0 < khi; k0 += GK) {
    acc.begin_chunk();
#pragma unroll
    for (int e = 0; e < (GM * GK) / GT; ++e) {
      const int idx = threadIdx.x + e * GT;
      int i, kk;
      if (kf) {
        kk = idx % GK;
        i = idx / GK;
      } else {
        i = idx % GM;
        kk = idx / GM;
      }
      const int64_t gi = row0 + i, gk = k0 + kk;
      V v = Cx<R>::make(0, 0);
      if (gi < M && gk < khi) v = JobElem<R>::get(J, gi, gk);
      sA[kk][i] = v;
    }
#pragma unroll
    for (int e = 0; e < (GK * GN) / GT; ++e) {
      const int idx = threadIdx.x + e * GT;
      const int kk = idx % GK, c = idx / GK;
      const int64_t gk = k0 + kk;
      V v = Cx<R>::make(0, 0);
      if (gk < khi && col0 + c < kcols) v = X[gk + (int64_t)(col0 + c) * ldx];
      sB[kk][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      const V a = sA[kk][tr];
#pragma unroll
      for (int q = 0; q < Q; ++q) cmac(acc.chunk(q), a, sB[kk][tc + 4 * q]);
    }
    acc.end_chunk();
    __syncthreads();
  }
  const int64_t gi = row0 + tr;
  if (gi < M) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int c = col0 + tc + 4 * q;
      if (c < kcols) Y[gi + ((int64_t)g * kcols + c) * ldy] = acc.result(q);
    }
  }
}

int launch_sketch_jobs(const std::vector<SketchJob>& jobs, int dtype, MemTracker* mt, cudaStream_t s) {
  if (jobs.empty()) return BF_OK;
  int64_t maxk = 0;
  for (const auto& j : jobs) maxk = std::max(maxk, j.kcols);
  const int GN = maxk > 32 ? 64 : 32;
  std::vector<SketchTile> tiles;
  for (size_t ji = 0; ji < jobs.size(); ++ji) {
    const SketchJob& j = jobs[ji];
    if (j.M <= 0 || j.kcols <= 0) continue;
    for (int g = 0; g < j.groups; ++g)
      for (int64_t r0 = 0; r0 < j.M; r0 += GM)
        for (int c0 = 0; c0 < j.kcols; c0 += GN) tiles.push_back({(int32_t)ji, g, c0, 0, r0});
  }
  if (tiles.empty()) return BF_OK;
  const size_t jb = jobs.size() * sizeof(SketchJob), tb = tiles.size() * sizeof(SketchTile);
  DevBuf d;
  BF_TRY(d.alloc(mt, jb + tb, s));
  int rc = BF_OK;
  if (cudaMemcpyAsync(d.p, jobs.data(), jb, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync((char*)d.p + jb, tiles.data(), tb, cudaMemcpyHostToDevice, s) != cudaSuccess)
    rc = fail(BF_ECUDA, "upload of sketch jobs failed");
  const SketchJob* dj = (const SketchJob*)d.p;
  const SketchTile* dt = (const SketchTile*)((char*)d.p + jb);
  const unsigned nt = (unsigned)tiles.size();
  if (!rc) {
    if (dtype == BF_C128) {
      if (GN == 64)
        sketch_job_kernel<double, 64><<<nt, GT, 0, s>>>(dj, dt);
      else
        sketch_job_kernel<double, 32><<<nt, GT, 0, s>>>(dj, dt);
    } else {
      if (GN == 64)
        sketch_job_kernel<float, 64><<<nt, GT, 0, s>>>(dj, dt);
      else
        sketch_job_kernel<float, 32><<<nt, GT, 0, s>>>(dj, dt);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) rc = fail(BF_ECUDA, std::string("sketch launch: ") + cudaGetErrorString(e));
  }
  d.release(s);
  return rc;
}

SketchJob dense_job(int op, const void* A, int64_t lda, int64_t m, int64_t n, const GemmGroups& g,
                    const void* X, int64_t ldx, void* Y, int64_t ldy) {
  SketchJob j{};
  j.kind = 0;
  j.op = op;
  j.groups = g.groups;
  j.M = op == BF_OP_N ? m : n;
  j.Ktot = op == BF_OP_N ? n : m;
  j.kcols = g.kcols;
  j.d_off = g.d_off;
  j.A = A;
  j.lda = lda;
  j.m = m;
  j.n = n;
  j.X = X;
  j.ldx = ldx;
  j.Y = Y;
  j.ldy = ldy;
  return j;
}

SketchJob kernel_job(const Plan* P, int op, const GemmGroups& g, const void* X, int64_t ldx, void* Y,
                     int64_t ldy) {
  SketchJob j{};
  j.kind = 1;
  j.op = op;
  j.ktype = P->kern.type;
  j.groups = g.groups;
  j.M = op == BF_OP_N ? P->m : P->n;
  j.Ktot = op == BF_OP_N ? P->n : P->m;
  j.kcols = g.kcols;
  j.d_off = g.d_off;
  j.tgt = (const double*)P->d_tgt.p;
  j.src = (const double*)P->d_src.p;
  j.tgtF = (const float*)P->d_tgtF.p;
  j.srcF = (const float*)P->d_srcF.p;
  j.m = P->m;
  j.n = P->n;
  j.wn = P->kern.wavenumber;
  j.kh = P->kh;
  j.kl = P->kl;
  j.X = X;
  j.ldx = ldx;
  j.Y = Y;
  j.ldy = ldy;
  return j;
}

int launch_dense_gemm(int op, const void* A, int64_t lda, int64_t m, int64_t n, const GemmGroups& g,
                      const void* X, int64_t ldx, void* Y, int64_t ldy, int dtype, cudaStream_t s) {
  return launch_sketch_jobs({dense_job(op, A, lda, m, n, g, X, ldx, Y, ldy)}, dtype, nullptr, s);
}

int launch_kernel_gemm(const Plan* P, int op, const GemmGroups& g, const void* X, int64_t ldx,
                       void* Y, int64_t ldy, int dtype, cudaStream_t s) {
  return launch_sketch_jobs({kernel_job(P, op, g, X, ldx, Y, ldy)}, dtype, nullptr, s);
}

}  // namespace bf
