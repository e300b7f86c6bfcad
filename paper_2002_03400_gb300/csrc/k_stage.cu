// Block-sparse stage products of the butterfly: one launch applies every
// block of one factor (V^0, W^j, B, R^j or U^L, or their adjoints) to a block
// of vectors.  The same kernel serves the apply (eq. hybrid_butterfly_mat),
// the peeling of already-recovered factors from the sketches (Alg. 2, the
// lines that project K(T_tau,S_nu)^T Gamma_tau and K(T_tau,S_nu) Omega_nu
// and form V^T Omega_nu) and the projection C = R^H P of eq. Bij.
//
// Each task is one output block (or a column slice of it):
//   out[M x N] = sum_t op_t(mat_t)[M x K_t] * in_t[K_t x N],  t < nterms <= 2
// A CTA computes a TM x TN tile of one task, streaming K in chunks of KC
// through shared memory; operands arrive coalesced along their contiguous
// dimension and the conjugate transpose is folded into the tile load.
#include "bf_internal.h"
#include "cx.cuh"

namespace bf {

namespace {
constexpr int TM = 32, TN = 32, KC = 16, THREADS = 128;
}

template <typename R>
__global__ void __launch_bounds__(THREADS) stage_kernel(const StageTask* __restrict__ tasks, StageBases bases, int Noverride) {
  using V = typename Cx<R>::V;
  __shared__ StageTask t;
  __shared__ V sA[KC][TM + 1];
  __shared__ V sB[KC][TN + 1];
  if (threadIdx.x == 0) {
    t = tasks[blockIdx.x];
    if (Noverride > 0) t.N = Noverride;
  }
  __syncthreads();
  const int row0 = blockIdx.z * TM, col0 = blockIdx.y * TN;
  if (row0 >= t.M || col0 >= t.N) return;
  const int tr = threadIdx.x & 31;        // output row within tile
  const int tc = threadIdx.x >> 5;        // 0..3: output columns tc + 4q
  V acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q] = Cx<R>::make(0, 0);

  for (int term = 0; term < t.nterms; ++term) {
    const StageTerm& T = t.t[term];
    const V* __restrict__ mat = (const V*)T.mat;
    const V* __restrict__ in = (const V*)bases.p[T.in_base] + T.in_off;
    for (int k0 = 0; k0 < T.K; k0 += KC) {
      // A tile: element (i, kk) of op(mat); 512 elements, 4 per thread
#pragma unroll
      for (int e = 0; e < (TM * KC) / THREADS; ++e) {
        const int idx = threadIdx.x + e * THREADS;
        int i, kk;
        if (!T.conjT) {
          i = idx % TM;
          kk = idx / TM;            // contiguous along i
        } else {
          kk = idx % KC;
          i = idx / KC;             // contiguous along kk
        }
        V v = Cx<R>::make(0, 0);
        const int gi = row0 + i, gk = k0 + kk;
        if (gi < t.M && gk < T.K) {
          if (!T.conjT) {
            v = mat[gi + (int64_t)gk * T.ldm];
          } else {
            v = mat[gk + (int64_t)gi * T.ldm];
            v.y = -v.y;
          }
        }
        sA[kk][i] = v;
      }
      // B tile: element (kk, c) of in
#pragma unroll
      for (int e = 0; e < (KC * TN) / THREADS; ++e) {
        const int idx = threadIdx.x + e * THREADS;
        const int kk = idx % KC, c = idx / KC;
        V v = Cx<R>::make(0, 0);
        const int gk = k0 + kk, gc = col0 + c;
        if (gk < T.K && gc < t.N) v = in[gk + (int64_t)gc * T.ldi];
        sB[kk][c] = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < KC; ++kk) {
        const V a = sA[kk][tr];
#pragma unroll
        for (int q = 0; q < 8; ++q) cmac(acc[q], a, sB[kk][tc + 4 * q]);
      }
      __syncthreads();
    }
  }
  V* out = (V*)bases.p[t.out_base] + t.out_off;
  const int gi = row0 + tr;
  if (gi < t.M) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int gc = col0 + tc + 4 * q;
      if (gc < t.N) out[gi + (int64_t)gc * t.ldo] = acc[q];
    }
  }
}

int launch_stage(const StageTask* d_tasks, int ntasks, int maxM, int maxN, int Noverride,
                 const StageBases& bases, int dtype, cudaStream_t s) {
  if (Noverride > 0) maxN = Noverride;
  if (ntasks <= 0 || maxM <= 0 || maxN <= 0) return BF_OK;
  dim3 grid(ntasks, (maxN + TN - 1) / TN, (maxM + TM - 1) / TM);
  if (grid.y > 65535 || grid.z > 65535) return fail(BF_EINVAL, "stage tile grid too large");
  if (dtype == BF_C128)
    stage_kernel<double><<<grid, THREADS, 0, s>>>(d_tasks, bases, Noverride);
  else
    stage_kernel<float><<<grid, THREADS, 0, s>>>(d_tasks, bases, Noverride);
  BF_CUDA_TRY(cudaGetLastError());
  return BF_OK;
}

}  // namespace bf
