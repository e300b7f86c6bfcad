// Batched truncated column-pivoted Householder QR in FP64 (Alg. 1 step 3).
//
// One CTA of 8 warps factors one block W (s x k): at step j the trailing
// column of largest norm is swapped to position j (ties: lowest index), the
// factorization stops when that norm is <= eps times the first pivot's norm
// (or zero), otherwise a Householder reflector
//   H = I - tau v v^H,  v = x - alpha e1,  alpha = -exp(i arg x0) ||x||
// is built from the column and applied to the trailing columns, one warp per
// column with warp-shuffle dot products; the same warp recomputes that
// column's norm for the next pivot search.  The rank is max(steps, 1) and
// Q = H_0 ... H_{rank-1} [I; 0] is written explicitly (one warp per column).
// The block lives in shared memory when it fits, else in a per-task global
// workspace (same code path, pointer switch).
#include "bf_internal.h"
#include "cx.cuh"

namespace bf {

namespace {
constexpr int QR_THREADS = 256;
constexpr int QR_WARPS = QR_THREADS / 32;
constexpr size_t QR_SMEM_LIMIT = 200 * 1024;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double2 warp_sum2(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

size_t meta_bytes(int maxK) { return (size_t)(2 * maxK + 8) * sizeof(double); }
}  // namespace

template <typename VIn>
__global__ void __launch_bounds__(QR_THREADS)
qr_kernel(const QRTask* __restrict__ tasks, double eps, int32_t* __restrict__ ranks,
          double2* __restrict__ gwork, int64_t work_stride, int maxK, int use_smem) {
  extern __shared__ double smem_d[];
  const QRTask t = tasks[blockIdx.x];
  const int s = t.s, k = t.k;
  double* nrm2 = smem_d;                    // k
  double* tau = smem_d + maxK;              // k
  double* misc = smem_d + 2 * maxK;         // [0]=nrm0 [1]=pivot [2]=stop [3]=steps
  double2* A = use_smem ? (double2*)(smem_d + 2 * maxK + 8) : gwork + blockIdx.x * work_stride;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const VIn* in = (const VIn*)t.in;

  for (int idx = threadIdx.x; idx < s * k; idx += QR_THREADS) {
    const int i = idx % s, c = idx / s;
    A[idx] = to_d2(in[i + (int64_t)c * t.ldi]);
  }
  __syncthreads();
  for (int c = warp; c < k; c += QR_WARPS) {
    double a = 0.0;
    for (int i = lane; i < s; i += 32) {
      const double2 v = A[i + c * s];
      a += v.x * v.x + v.y * v.y;
    }
    a = warp_sum(a);
    if (lane == 0) nrm2[c] = a;
  }
  __syncthreads();

  const int jmax = min(s, k);
  int steps = 0;
  for (int j = 0; j < jmax; ++j) {
    // pivot: largest trailing norm, ties -> lowest index (warp 0)
    if (warp == 0) {
      double best = -1.0;
      int bi = k;
      for (int c = j + lane; c < k; c += 32) {
        const double v = nrm2[c];
        if (v > best) best = v, bi = c;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) best = ob, bi = oi;
      }
      if (lane == 0) {
        const double nrm = sqrt(fmax(best, 0.0));
        if (j == 0) misc[0] = nrm;
        misc[1] = (double)bi;
        misc[2] = (nrm == 0.0 || nrm <= eps * misc[0]) ? 1.0 : 0.0;
      }
    }
    __syncthreads();
    if (misc[2] != 0.0) break;
    const int p = (int)misc[1];
    if (p != j) {
      for (int i = threadIdx.x; i < s; i += QR_THREADS) {
        const double2 a = A[i + j * s];
        A[i + j * s] = A[i + p * s];
        A[i + p * s] = a;
      }
      if (threadIdx.x == 0) {
        const double a = nrm2[j];
        nrm2[j] = nrm2[p];
        nrm2[p] = a;
      }
      __syncthreads();
    }
    // reflector from column j, rows j..s-1 (warp 0)
    if (warp == 0) {
      double sq = 0.0;
      for (int i = j + lane; i < s; i += 32) {
        const double2 v = A[i + j * s];
        sq += v.x * v.x + v.y * v.y;
      }
      sq = warp_sum(sq);
      const double nrm = sqrt(sq);
      const double2 x0 = A[j + j * s];
      const double ax0 = hypot(x0.x, x0.y);
      double px = 1.0, py = 0.0;
      if (ax0 != 0.0) px = x0.x / ax0, py = x0.y / ax0;
      // v0 = x0 - alpha, alpha = -phase*nrm  ->  v0 = x0 + phase*nrm
      const double2 v0 = make_double2(x0.x + px * nrm, x0.y + py * nrm);
      // v^H v = |v0|^2 + (sq - |x0|^2)
      const double beta = (v0.x * v0.x + v0.y * v0.y) + (sq - ax0 * ax0);
      if (lane == 0) {
        A[j + j * s] = v0;
        tau[j] = beta > 0.0 ? 2.0 / beta : 0.0;
      }
    }
    __syncthreads();
    const double tj = tau[j];
    // apply H to trailing columns and refresh their norms (rows j+1..s-1)
    for (int c = j + 1 + warp; c < k; c += QR_WARPS) {
      double2 w = make_double2(0.0, 0.0);
      for (int i = j + lane; i < s; i += 32) {
        const double2 v = A[i + j * s], a = A[i + c * s];
        w.x += v.x * a.x + v.y * a.y;      // conj(v) * a
        w.y += v.x * a.y - v.y * a.x;
      }
      w = warp_sum2(w);
      w.x *= tj;
      w.y *= tj;
      double a2 = 0.0;
      for (int i = j + lane; i < s; i += 32) {
        const double2 v = A[i + j * s];
        double2 a = A[i + c * s];
        a.x -= v.x * w.x - v.y * w.y;
        a.y -= v.x * w.y + v.y * w.x;
        A[i + c * s] = a;
        if (i > j) a2 += a.x * a.x + a.y * a.y;
      }
      a2 = warp_sum(a2);
      if (lane == 0) nrm2[c] = a2;
    }
    ++steps;
    __syncthreads();
  }
  const int rank = steps > 0 ? steps : 1;
  if (threadIdx.x == 0) ranks[blockIdx.x] = rank;

  // Q = H_0 ... H_{steps-1} [I; 0]; column c only meets reflectors j <= c
  double2* q = (double2*)t.q;
  for (int c = warp; c < rank; c += QR_WARPS) {
    for (int i = lane; i < s; i += 32)
      q[i + (int64_t)c * s] = make_double2(i == c ? 1.0 : 0.0, 0.0);
    __syncwarp();
    for (int j = min(c, steps - 1); j >= 0; --j) {
      double2 w = make_double2(0.0, 0.0);
      for (int i = j + lane; i < s; i += 32) {
        const double2 v = A[i + j * s], a = q[i + (int64_t)c * s];
        w.x += v.x * a.x + v.y * a.y;
        w.y += v.x * a.y - v.y * a.x;
      }
      w = warp_sum2(w);
      const double tj = tau[j];
      w.x *= tj;
      w.y *= tj;
      for (int i = j + lane; i < s; i += 32) {
        const double2 v = A[i + j * s];
        double2 a = q[i + (int64_t)c * s];
        a.x -= v.x * w.x - v.y * w.y;
        a.y -= v.x * w.y + v.y * w.x;
        q[i + (int64_t)c * s] = a;
      }
      __syncwarp();
    }
  }
}

size_t qr_workspace_bytes(int ntasks, int maxS, int maxK) {
  const size_t blk = (size_t)maxS * maxK * sizeof(double2);
  if (blk + meta_bytes(maxK) <= QR_SMEM_LIMIT) return 0;
  return blk * (size_t)ntasks;
}

int launch_qr(const QRTask* d_tasks, int ntasks, int maxS, int maxK, double eps, int in_dtype,
              int32_t* d_ranks, void* d_work, size_t work_bytes, cudaStream_t s) {
  if (ntasks <= 0) return BF_OK;
  const size_t blk = (size_t)maxS * maxK * sizeof(double2);
  const int use_smem = (blk + meta_bytes(maxK) <= QR_SMEM_LIMIT) ? 1 : 0;
  const size_t smem = meta_bytes(maxK) + (use_smem ? blk : 0);
  if (!use_smem && (d_work == nullptr || work_bytes < blk * (size_t)ntasks))
    return fail(BF_EINVAL, "QR workspace too small");
  const int64_t stride = (int64_t)maxS * maxK;
  if (in_dtype == BF_C128) {
    BF_CUDA_TRY(cudaFuncSetAttribute(qr_kernel<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)QR_SMEM_LIMIT + 4096));
    qr_kernel<double2><<<ntasks, QR_THREADS, smem, s>>>(d_tasks, eps, d_ranks, (double2*)d_work,
                                                        stride, maxK, use_smem);
  } else {
    BF_CUDA_TRY(cudaFuncSetAttribute(qr_kernel<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)QR_SMEM_LIMIT + 4096));
    qr_kernel<float2><<<ntasks, QR_THREADS, smem, s>>>(d_tasks, eps, d_ranks, (double2*)d_work,
                                                       stride, maxK, use_smem);
  }
  BF_CUDA_TRY(cudaGetLastError());
  return BF_OK;
}

}  // namespace bf
