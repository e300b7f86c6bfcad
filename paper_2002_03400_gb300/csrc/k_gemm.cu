// Sketch products of the built-in black boxes (Alg. 2 input; Sec. 4.1):
// Y = A X or Y = A^H X in tree order for a dense stored A or for entries
// K(t_i, s_j) formed on the fly from the point sets, with the structured
// random matrices of Sec. 4.1 handled by skipping their zero blocks: output
// column group g only sums over the input rows of node g,
//   op N: Y[:, g*k + c] = sum_{j in S_g} A[:, j] X[j, c]
//   op C: Y[:, g*k + c] = sum_{i in T_g} conj(A[i, :]) X[i, c].
//
// Complex GEMM on the SIMT pipes: a 64 x 32 output tile per 256-thread CTA,
// K streamed in chunks of 16 through shared memory, each thread holding 8
// complex accumulators.  FP64 path: complex128 throughout.  Mixed path:
// complex64 operands, each 16-term chunk accumulated in FP32 and merged
// into a (hi, lo) FP32 pair with Knuth's TwoSum, so the long dot products
// (K up to n) keep ~FP32 accuracy per chunk instead of growing with sqrt(K).
// Kernel entries: the distance and the phase k*r are formed in FP64 and
// reduced modulo 2*pi before the trigonometric evaluation, so the phase of
// an oscillatory kernel with k*r ~ 1e4 stays accurate in both paths.
#include "bf_internal.h"
#include "cx.cuh"

namespace bf {

namespace {
constexpr int GM = 64, GN = 32, GK = 16, GT = 256;

struct PointsSoA {
  const double* x;
  const double* y;
  const double* z;
};

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

template <typename V>
struct DenseLoader {
  const V* A;
  int64_t lda;
  int op;
  __device__ __forceinline__ V get(int64_t r, int64_t kk) const {
    if (op == BF_OP_N) return A[r + kk * lda];
    V v = A[kk + r * lda];
    v.y = -v.y;
    return v;
  }
  __device__ __forceinline__ bool k_fastest() const { return op != BF_OP_N; }
};

template <typename V>
struct KernelLoader {
  PointsSoA tgt, src;
  int type;
  double wn;
  int op;
  __device__ __forceinline__ V get(int64_t r, int64_t kk) const {
    double2 v;
    if (op == BF_OP_N) {
      v = kernel_value(type, wn, tgt.x[r], tgt.y[r], tgt.z[r], src.x[kk], src.y[kk], src.z[kk]);
    } else {
      v = kernel_value(type, wn, tgt.x[kk], tgt.y[kk], tgt.z[kk], src.x[r], src.y[r], src.z[r]);
      v.y = -v.y;
    }
    return from_d2<V>(v);
  }
  __device__ __forceinline__ bool k_fastest() const { return false; }
};

__device__ __forceinline__ void two_sum(float& hi, float& lo, float b) {
  const float s = hi + b;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (b - bb);
  hi = s;
  lo += err;
}

template <typename R>
struct Acc;
template <>
struct Acc<double> {
  double2 v[8];
  __device__ void zero() {
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = make_double2(0.0, 0.0);
  }
  __device__ __forceinline__ double2& chunk(int q) { return v[q]; }
  __device__ __forceinline__ void begin_chunk() {}
  __device__ __forceinline__ void end_chunk() {}
  __device__ __forceinline__ double2 result(int q) const { return v[q]; }
};
template <>
struct Acc<float> {
  float2 part[8], hi[8], lo[8];
  __device__ void zero() {
#pragma unroll
    for (int q = 0; q < 8; ++q)
      part[q] = make_float2(0.f, 0.f), hi[q] = make_float2(0.f, 0.f), lo[q] = make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ float2& chunk(int q) { return part[q]; }
  __device__ __forceinline__ void begin_chunk() {
#pragma unroll
    for (int q = 0; q < 8; ++q) part[q] = make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ void end_chunk() {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      two_sum(hi[q].x, lo[q].x, part[q].x);
      two_sum(hi[q].y, lo[q].y, part[q].y);
    }
  }
  __device__ __forceinline__ float2 result(int q) const {
    return make_float2(hi[q].x + lo[q].x, hi[q].y + lo[q].y);
  }
};
}  // namespace

template <typename R, class Loader>
__global__ void __launch_bounds__(GT)
sketch_gemm_kernel(Loader ld, int64_t M, const int64_t* __restrict__ goff, int64_t Ktot,
                   int64_t kcols, const typename Cx<R>::V* __restrict__ X, int64_t ldx,
                   typename Cx<R>::V* __restrict__ Y, int64_t ldy) {
  using V = typename Cx<R>::V;
  __shared__ V sA[GK][GM + 1];
  __shared__ V sB[GK][GN + 1];
  const int64_t row0 = (int64_t)blockIdx.x * GM;
  const int col0 = blockIdx.y * GN;
  const int g = blockIdx.z;
  const int64_t klo = goff ? goff[g] : 0;
  const int64_t khi = goff ? goff[g + 1] : Ktot;
  const int tr = threadIdx.x % GM, tc = threadIdx.x / GM;   // tc 0..3
  Acc<R> acc;
  acc.zero();
  const bool kf = ld.k_fastest();
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
      if (gi < M && gk < khi) v = ld.get(gi, gk);
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
      for (int q = 0; q < 8; ++q) cmac(acc.chunk(q), a, sB[kk][tc + 4 * q]);
    }
    acc.end_chunk();
    __syncthreads();
  }
  const int64_t gi = row0 + tr;
  if (gi < M) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int c = col0 + tc + 4 * q;
      if (c < kcols) Y[gi + ((int64_t)g * kcols + c) * ldy] = acc.result(q);
    }
  }
}

template <typename R, class Loader>
static int run_gemm(const Loader& ld, int64_t M, const GemmGroups& g, int64_t Ktot, const void* X,
                    int64_t ldx, void* Y, int64_t ldy, cudaStream_t s) {
  using V = typename Cx<R>::V;
  if (M <= 0 || g.kcols <= 0 || g.groups <= 0) return BF_OK;
  dim3 grid((unsigned)((M + GM - 1) / GM), (unsigned)((g.kcols + GN - 1) / GN), (unsigned)g.groups);
  if (grid.y > 65535 || grid.z > 65535) return fail(BF_EINVAL, "sketch grid too large");
  sketch_gemm_kernel<R, Loader><<<grid, GT, 0, s>>>(ld, M, g.d_off, Ktot, g.kcols, (const V*)X, ldx,
                                                    (V*)Y, ldy);
  BF_CUDA_TRY(cudaGetLastError());
  return BF_OK;
}

int launch_dense_gemm(int op, const void* A, int64_t lda, int64_t m, int64_t n, const GemmGroups& g,
                      const void* X, int64_t ldx, void* Y, int64_t ldy, int dtype, cudaStream_t s) {
  const int64_t M = op == BF_OP_N ? m : n;
  const int64_t K = op == BF_OP_N ? n : m;
  if (dtype == BF_C128) {
    DenseLoader<double2> ld{(const double2*)A, lda, op};
    return run_gemm<double>(ld, M, g, K, X, ldx, Y, ldy, s);
  }
  DenseLoader<float2> ld{(const float2*)A, lda, op};
  return run_gemm<float>(ld, M, g, K, X, ldx, Y, ldy, s);
}

int launch_kernel_gemm(const Plan* P, int op, const GemmGroups& g, const void* X, int64_t ldx,
                       void* Y, int64_t ldy, int dtype, cudaStream_t s) {
  const double* src = (const double*)P->d_src.p;
  const double* tgt = (const double*)P->d_tgt.p;
  PointsSoA ps{src, src + P->n, src + 2 * P->n};
  PointsSoA pt{tgt, tgt + P->m, tgt + 2 * P->m};
  const int64_t M = op == BF_OP_N ? P->m : P->n;
  const int64_t K = op == BF_OP_N ? P->n : P->m;
  if (dtype == BF_C128) {
    KernelLoader<double2> ld{pt, ps, P->kern.type, P->kern.wavenumber, op};
    return run_gemm<double>(ld, M, g, K, X, ldx, Y, ldy, s);
  }
  KernelLoader<float2> ld{pt, ps, P->kern.type, P->kern.wavenumber, op};
  return run_gemm<float>(ld, M, g, K, X, ldx, Y, ldy, s);
}

}  // namespace bf
