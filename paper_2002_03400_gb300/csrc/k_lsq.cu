// Batched least-squares solve for the centre coupling B at level l_m (eq. Bij,
// Sec. 4.4), FP64:
//   C = R_{tau,nu}^H P_{tau,nu}            (= U_{tau,nu}^H K(T_tau,S_nu) Omega_nu)
//   X = V_{tau,nu}^H Omega_nu              (r^V x k, k >= r^V + p)
//   B = argmin ||C - B X||_F = C X^+
// solved through the Householder QR X^H = Qx Rx:  B^H = Rx^{-1} Qx^H C^H.
// One CTA per block; X^H and C^H in shared memory when they fit, else in a
// per-task global workspace (same code, pointer switch: weakly admissible
// geometries reach centre ranks of hundreds).
#include "bf_internal.h"
#include "cx.cuh"

namespace bf {

namespace {
constexpr int LSQ_THREADS = 256;
constexpr int LSQ_WARPS = LSQ_THREADS / 32;
__device__ __forceinline__ double2 wsum2(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}
__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
}  // namespace

template <typename VIn>
__global__ void __launch_bounds__(LSQ_THREADS)
lsq_kernel(const LSQTask* __restrict__ tasks, int maxK, int maxR, double2* __restrict__ gwork, int use_smem) {
  extern __shared__ double2 sm[];
  const LSQTask t = tasks[blockIdx.x];
  const int s = t.s, k = t.k, rU = t.rU, rV = t.rV;
  double2* XH = use_smem ? sm : gwork + (int64_t)blockIdx.x * 2 * maxK * maxR;   // k x rV (ld k)
  double2* CH = XH + (int64_t)maxK * maxR;                                       // k x rU (ld k)
  double* tau = (double*)(use_smem ? CH + (int64_t)maxK * maxR : sm);             // rV
  double* rdiag = tau + maxR;                  // rV (real part of alpha unused)
  double2* alpha = (double2*)(rdiag + maxR);   // rV
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const VIn* P = (const VIn*)t.P;
  const double2* Q = (const double2*)t.Q;
  const VIn* X = (const VIn*)t.X;

  // C^H[c, i] = conj( sum_r conj(Q[r,i]) P[r,c] ) = sum_r Q[r,i] conj(P[r,c])
  for (int idx = threadIdx.x; idx < k * rU; idx += LSQ_THREADS) {
    const int c = idx % k, i = idx / k;
    double2 acc = make_double2(0.0, 0.0);
    for (int r = 0; r < s; ++r) {
      const double2 q = Q[r + (int64_t)i * s];
      const double2 p = to_d2(P[r + (int64_t)c * s]);
      acc.x += q.x * p.x + q.y * p.y;
      acc.y += q.y * p.x - q.x * p.y;
    }
    CH[c + i * k] = acc;
  }
  for (int idx = threadIdx.x; idx < k * rV; idx += LSQ_THREADS) {
    const int c = idx % k, i = idx / k;
    const double2 x = to_d2(X[i + (int64_t)c * rV]);
    XH[c + i * k] = make_double2(x.x, -x.y);
  }
  __syncthreads();

  for (int j = 0; j < rV; ++j) {
    if (warp == 0) {
      double sq = 0.0;
      for (int i = j + lane; i < k; i += 32) {
        const double2 v = XH[i + j * k];
        sq += v.x * v.x + v.y * v.y;
      }
      sq = wsum(sq);
      const double nrm = sqrt(sq);
      const double2 x0 = XH[j + j * k];
      const double ax0 = hypot(x0.x, x0.y);
      double px = 1.0, py = 0.0;
      if (ax0 != 0.0) px = x0.x / ax0, py = x0.y / ax0;
      const double2 v0 = make_double2(x0.x + px * nrm, x0.y + py * nrm);
      const double beta = (v0.x * v0.x + v0.y * v0.y) + (sq - ax0 * ax0);
      if (lane == 0) {
        alpha[j] = make_double2(-px * nrm, -py * nrm);   // R_jj
        XH[j + j * k] = v0;
        tau[j] = beta > 0.0 ? 2.0 / beta : 0.0;
      }
    }
    __syncthreads();
    const double tj = tau[j];
    // trailing columns of XH (j+1..rV-1) and all columns of CH
    for (int c = warp; c < (rV - j - 1) + rU; c += LSQ_WARPS) {
      double2* col = c < rV - j - 1 ? XH + (j + 1 + c) * k : CH + (c - (rV - j - 1)) * k;
      double2 w = make_double2(0.0, 0.0);
      for (int i = j + lane; i < k; i += 32) {
        const double2 v = XH[i + j * k], a = col[i];
        w.x += v.x * a.x + v.y * a.y;
        w.y += v.x * a.y - v.y * a.x;
      }
      w = wsum2(w);
      w.x *= tj;
      w.y *= tj;
      for (int i = j + lane; i < k; i += 32) {
        const double2 v = XH[i + j * k];
        double2 a = col[i];
        a.x -= v.x * w.x - v.y * w.y;
        a.y -= v.x * w.y + v.y * w.x;
        col[i] = a;
      }
    }
    __syncthreads();
  }
  // back substitution Rx Y = (Qx^H C^H)[0:rV, :] per column i of C^H; B = Y^H
  double2* B = (double2*)t.B;
  for (int i = threadIdx.x; i < rU; i += LSQ_THREADS) {
    double2* y = CH + i * k;
    for (int j = rV - 1; j >= 0; --j) {
      double2 acc = y[j];
      for (int c = j + 1; c < rV; ++c) {
        const double2 r = XH[j + c * k];      // R[j, c]
        const double2 x = y[c];
        acc.x -= r.x * x.x - r.y * x.y;
        acc.y -= r.x * x.y + r.y * x.x;
      }
      const double2 d = alpha[j];
      const double dd = d.x * d.x + d.y * d.y;
      double2 xj = make_double2(0.0, 0.0);
      if (dd > 1e-300) xj = make_double2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd);
      y[j] = xj;
    }
    for (int j = 0; j < rV; ++j) B[i + (int64_t)j * rU] = make_double2(y[j].x, -y[j].y);
  }
}

namespace {
size_t lsq_block_bytes(int maxK, int maxR) { return (size_t)2 * maxK * maxR * sizeof(double2); }
size_t lsq_meta_bytes(int maxR) { return (size_t)maxR * (2 * sizeof(double) + sizeof(double2)); }
constexpr size_t LSQ_SMEM_LIMIT = 220 * 1024;
}  // namespace

size_t lsq_workspace_bytes(int ntasks, int maxK, int maxR) {
  if (lsq_block_bytes(maxK, maxR) + lsq_meta_bytes(maxR) <= LSQ_SMEM_LIMIT) return 0;
  return lsq_block_bytes(maxK, maxR) * (size_t)ntasks;
}

int launch_lsq(const LSQTask* d_tasks, int ntasks, int maxS, int maxK, int maxR, int in_dtype, void* d_work,
               size_t work_bytes, cudaStream_t s) {
  if (ntasks <= 0) return BF_OK;
  const int use_smem = lsq_block_bytes(maxK, maxR) + lsq_meta_bytes(maxR) <= LSQ_SMEM_LIMIT ? 1 : 0;
  const size_t smem = (use_smem ? lsq_block_bytes(maxK, maxR) : 0) + lsq_meta_bytes(maxR);
  if (smem > LSQ_SMEM_LIMIT) return fail(BF_EUNSUPPORTED, "B least-squares ranks too large");
  if (!use_smem && (d_work == nullptr || work_bytes < lsq_block_bytes(maxK, maxR) * (size_t)ntasks))
    return fail(BF_EINVAL, "B least-squares workspace too small");
  note_launch();
  if (in_dtype == BF_C128) {
    BF_CUDA_TRY(cudaFuncSetAttribute(lsq_kernel<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)LSQ_SMEM_LIMIT));   // the largest size, whatever this launch needs
    lsq_kernel<double2><<<ntasks, LSQ_THREADS, smem, s>>>(d_tasks, maxK, maxR, (double2*)d_work, use_smem);
  } else {
    BF_CUDA_TRY(cudaFuncSetAttribute(lsq_kernel<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)LSQ_SMEM_LIMIT));
    lsq_kernel<float2><<<ntasks, LSQ_THREADS, smem, s>>>(d_tasks, maxK, maxR, (double2*)d_work, use_smem);
  }
  BF_CUDA_TRY(cudaGetLastError());
  return BF_OK;
}

}  // namespace bf
