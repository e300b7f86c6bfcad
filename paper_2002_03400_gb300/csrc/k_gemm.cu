// Sketch products of the built-in black boxes (Alg. 2 input; Sec. 4.1):
// Y = A X or Y = A^H X in tree order for a dense stored A or for entries
// K(t_i, s_j) formed on the fly from the point sets, with the structured
// random matrices of Sec. 4.1 handled by skipping their zero blocks: output
// column group g only sums over the input rows of node g,
//   op N: Y[:, g*k + c] = sum_{j in S_g} A[:, j] X[j, c]
//   op C: Y[:, g*k + c] = sum_{i in T_g} conj(A[i, :]) X[i, c].
//
// SIMT complex GEMM (the FP64 path, and the mixed path when the tensor-core
// kernel of k_sketch_tc.cu does not apply): a GM x GN output tile per
// 256-thread CTA, K streamed in chunks of 16 through shared memory, GN
// covering the whole sketch width (up to 64 columns) so each entry is formed
// once per row tile.  Mixed path: each 16-term chunk is accumulated in FP32
// and merged into a (hi, lo) FP32 pair with Knuth's TwoSum, so long dot
// products (K up to n) keep ~FP32 accuracy instead of losing sqrt(K).
#include <algorithm>

#include "bf_internal.h"
#include "cx.cuh"
#include "kentry.cuh"

namespace bf {

using namespace dev;

namespace {
constexpr int GM = 64, GK = 16, GT = 256;

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
  // entries of kernel jobs: each thread always forms row tr of the tile
  Entry<R> en;
  en.init(J, row0 + tr, row0 + tr < M);
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
      if (gi < M && gk < khi) v = en.get(gi, gk);
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

// 0: tensor cores where they apply (split depth from each job), 1: SIMT only,
// 2 / 3: tensor cores with the split depth forced to 2 / 3
static int g_sketch_engine = 0;
static int g_entry_images = 1;

int set_entry_images(int on) {
  if (on != 0 && on != 1) return fail(BF_EINVAL, "entry images: 0 (off) or 1 (on)");
  g_entry_images = on;
  return BF_OK;
}
int entry_images_enabled() { return g_entry_images; }

int set_sketch_engine(int e) {
  if (e < 0 || e > 3) return fail(BF_EINVAL, "sketch engine must be 0 (auto), 1 (SIMT), 2 or 3 (tensor split)");
  g_sketch_engine = e;
  return BF_OK;
}

int launch_sketch_jobs(const std::vector<SketchJob>& jobs, int dtype, MemTracker* mt, cudaStream_t s) {
  if (jobs.empty()) return BF_OK;
  if (dtype == BF_C64 && g_sketch_engine != 1 && sketch_tc_applies(jobs)) {
    if (g_sketch_engine == 0) return launch_sketch_jobs_tc(jobs, mt, s);
    std::vector<SketchJob> forced(jobs);
    for (auto& j : forced) {
      if (j.split != g_sketch_engine) j.img = nullptr;   // images hold the bf16 split only
      j.split = g_sketch_engine;
    }
    return launch_sketch_jobs_tc(forced, mt, s);
  }
  return launch_sketch_jobs_simt(jobs, dtype, mt, s);
}

int launch_sketch_jobs_simt(const std::vector<SketchJob>& jobs, int dtype, MemTracker* mt, cudaStream_t s) {
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
  if (upload_async(d.p, jobs.data(), jb, s) != BF_OK || upload_async((char*)d.p + jb, tiles.data(), tb, s) != BF_OK)
    rc = fail(BF_ECUDA, "upload of sketch jobs failed");
  const SketchJob* dj = (const SketchJob*)d.p;
  const SketchTile* dt = (const SketchTile*)((char*)d.p + jb);
  const unsigned nt = (unsigned)tiles.size();
  if (!rc) {
    note_launch();
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
  j.split = 3;
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
  j.split = 3;
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
                       void* Y, int64_t ldy, int dtype, cudaStream_t s, const void* img) {
  SketchJob j = kernel_job(P, op, g, X, ldx, Y, ldy);
  if (img && dtype == BF_C64 && (op == BF_OP_N || op == BF_OP_C) && entry_image_fits(j)) {
    j.img = img;
    j.img_nch = entry_image_chunks(j.Ktot);
  }
  return launch_sketch_jobs({j}, dtype, nullptr, s);
}

}  // namespace bf
