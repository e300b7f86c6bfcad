// Block-sparse stage products of the butterfly: one launch applies every
// block of one factor (V^0, W^j, B, R^j or U^L, or their adjoints) to a block
// of vectors.  The same kernel serves the apply (eq. hybrid_butterfly_mat),
// the peeling of already-recovered factors from the sketches (Alg. 2, the
// lines that project K(T_tau,S_nu)^T Gamma_tau and K(T_tau,S_nu) Omega_nu
// and form V^T Omega_nu) and the projection of the centre level.
//
// Each task is one output block (or a column slice of it):
//   out[M x N] = sum_t op_t(mat_t)[M x K_t] * in_t[K_t x N],  t < nterms <= 2
// One warp owns one task at a time (blocks have ranks ~10-60, far too small
// for a CTA each).  Lanes own output columns; the factor block is staged in
// 16 x 16 tiles through the warp's slice of shared memory, where every lane
// reads the same element (broadcast), with the conjugate transpose folded
// into that load; each lane keeps 16 input values and 16 accumulators in
// registers.  Operand layouts (per StageTerm/StageTask):
//   ld > 0: column-major, element (k, c) at off + k + c*ld
//   ld < 0: row-major,    element (k, c) at off + k*(-ld) + c
//   ld = 0: row-major with the launch's column count N: off is a row index,
//           element (k, c) at (off + k)*N + c  (apply intermediates)
// Row-major intermediates make the loads of a K-chunk and the stores of an
// output row contiguous across the warp's lanes.
#include "bf_internal.h"
#include "cx.cuh"

namespace bf {

namespace {
constexpr int MT = 16, KC = 16, WARPS = 4, THREADS = 32 * WARPS;

struct Strides {
  int64_t off, rs, cs;
};
__device__ __forceinline__ Strides strides(int64_t off, int64_t ld, int N) {
  if (ld > 0) return {off, 1, ld};
  if (ld < 0) return {off, -ld, 1};
  return {off * N, N, 1};
}
}  // namespace

template <typename R>
__global__ void __launch_bounds__(THREADS)
stage_kernel(const StageTask* __restrict__ tasks, int ntasks, StageBases bases, int Noverride) {
  using V = typename Cx<R>::V;
  __shared__ V smat[WARPS][MT][KC + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  V (*sm)[KC + 1] = smat[warp];
  for (int ti = blockIdx.x * WARPS + warp; ti < ntasks; ti += gridDim.x * WARPS) {
    const StageTask& tk = tasks[ti];
    const int M = tk.M, nterms = tk.nterms;
    const int N = Noverride > 0 ? Noverride : tk.N;
    const Strides so = strides(tk.out_off, tk.ldo, N);
    V* __restrict__ out = (V*)bases.p[tk.out_base] + so.off;
    for (int c0 = 0; c0 < N; c0 += 32) {
      const int c = c0 + lane;
      const bool cv = c < N;
      for (int i0 = 0; i0 < M; i0 += MT) {
        V acc[MT];
#pragma unroll
        for (int i = 0; i < MT; ++i) acc[i] = Cx<R>::make(0, 0);
        for (int term = 0; term < nterms; ++term) {
          const StageTerm& T = tk.t[term];
          const V* __restrict__ mat = (const V*)T.mat;
          const int K = T.K, ldm = T.ldm, conjT = T.conjT;
          const Strides si = strides(T.in_off, T.ldi, N);
          const V* __restrict__ in = (const V*)bases.p[T.in_base] + si.off + (int64_t)c * si.cs;
          for (int k0 = 0; k0 < K; k0 += KC) {
            // factor tile (MT x KC) of op(mat) into shared memory
#pragma unroll
            for (int e = 0; e < (MT * KC) / 32; ++e) {
              const int idx = lane + 32 * e;
              int i, kk;
              if (!conjT) {
                i = idx % MT;
                kk = idx / MT;
              } else {
                kk = idx % KC;
                i = idx / KC;
              }
              const int gi = i0 + i, gk = k0 + kk;
              V v = Cx<R>::make(0, 0);
              if (gi < M && gk < K) {
                if (!conjT) {
                  v = mat[gi + (int64_t)gk * ldm];
                } else {
                  v = mat[gk + (int64_t)gi * ldm];
                  v.y = -v.y;
                }
              }
              sm[i][kk] = v;
            }
            V x[KC];
#pragma unroll
            for (int kk = 0; kk < KC; ++kk)
              x[kk] = (cv && k0 + kk < K) ? in[(int64_t)(k0 + kk) * si.rs] : Cx<R>::make(0, 0);
            __syncwarp();
#pragma unroll
            for (int i = 0; i < MT; ++i)
#pragma unroll
              for (int kk = 0; kk < KC; ++kk) cmac(acc[i], sm[i][kk], x[kk]);
            __syncwarp();
          }
        }
        if (cv) {
#pragma unroll
          for (int i = 0; i < MT; ++i)
            if (i0 + i < M) out[(int64_t)(i0 + i) * so.rs + (int64_t)c * so.cs] = acc[i];
        }
      }
    }
  }
}

int launch_stage(const StageTask* d_tasks, int ntasks, int maxM, int maxN, int Noverride,
                 const StageBases& bases, int dtype, cudaStream_t s) {
  if (Noverride > 0) maxN = Noverride;
  if (ntasks <= 0 || maxM <= 0 || maxN <= 0) return BF_OK;
  int blocks = (ntasks + WARPS - 1) / WARPS;
  if (blocks > 152 * 16) blocks = 152 * 16;
  note_launch();
  if (dtype == BF_C128)
    stage_kernel<double><<<blocks, THREADS, 0, s>>>(d_tasks, ntasks, bases, Noverride);
  else
    stage_kernel<float><<<blocks, THREADS, 0, s>>>(d_tasks, ntasks, bases, Noverride);
  BF_CUDA_TRY(cudaGetLastError());
  return BF_OK;
}

}  // namespace bf
