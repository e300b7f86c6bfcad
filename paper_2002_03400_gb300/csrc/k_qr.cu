// Batched truncated column-pivoted Householder QR in FP64 (Alg. 1 step 3).
//
// One CTA factors one block W (s x k).  At step j the trailing column of
// largest norm is swapped to position j (ties: lowest index); the
// factorization stops when that norm is <= eps times the first pivot's norm
// (or zero); otherwise the reflector
//   H = I - tau v v^H,  v = x - alpha e1,  alpha = -exp(i arg x0) ||x||
// is built from the column and applied to the trailing columns.  The rank is
// max(steps, 1) and Q = H_0 ... H_{rank-1} [I; 0] is formed explicitly.
//
// GB300 retires ~2 FP64 FMAs per clock per SM, so the layout is chosen to
// spend FP64 instructions only on useful lanes: each thread owns one column
// and runs its dot products, updates and norm refreshes sequentially over
// the rows (the reflector is broadcast from shared memory), with no
// shuffle-reduction trees.  The block sits in shared memory with an odd
// leading dimension (conflict-free column-per-thread access) when it fits,
// else in a per-task global workspace (same code, pointer switch).
#include "bf_internal.h"
#include "cx.cuh"

namespace bf {

namespace {
constexpr size_t QR_SMEM_LIMIT = 200 * 1024;
constexpr int QR_MAX_THREADS = 256;

__host__ __device__ inline int ld_of(int s) { return s | 1; }
size_t meta_bytes(int maxK) { return (size_t)(2 * maxK + 8) * sizeof(double); }
size_t block_bytes(int maxS, int maxK) {
  // A (ld x k) and Q (ld x min(s,k)) in complex128
  return (size_t)ld_of(maxS) * (maxK + (maxS < maxK ? maxS : maxK)) * sizeof(double2);
}
int threads_for(int maxK) {
  int t = ((maxK + 31) / 32) * 32;
  return t > QR_MAX_THREADS ? QR_MAX_THREADS : t;
}
}  // namespace

template <typename VIn>
__global__ void qr_kernel(const QRTask* __restrict__ tasks, int32_t* __restrict__ ranks,
                          double2* __restrict__ gwork, int64_t work_stride, int maxK, int use_smem) {
  extern __shared__ double smem_d[];
  const QRTask t = tasks[blockIdx.x];
  const int s = t.s, k = t.k, ld = ld_of(s);
  const int nthr = blockDim.x;
  double* nrm2 = smem_d;                    // k
  double* tau = smem_d + maxK;              // k
  double* misc = smem_d + 2 * maxK;         // [0]=nrm0 [1]=pivot [2]=stop
  double2* A = use_smem ? (double2*)(smem_d + 2 * maxK + 8) : gwork + blockIdx.x * work_stride;
  double2* Qs = A + (size_t)ld * k;         // ld x min(s,k)
  const VIn* in = (const VIn*)t.in;

  for (int idx = threadIdx.x; idx < s * k; idx += nthr) {
    const int i = idx % s, c = idx / s;
    A[i + c * ld] = to_d2(in[i + (int64_t)c * t.ldi]);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < k; c += nthr) {
    double a = 0.0;
    for (int i = 0; i < s; ++i) {
      const double2 v = A[i + c * ld];
      a = fma(v.x, v.x, fma(v.y, v.y, a));
    }
    nrm2[c] = a;
  }
  __syncthreads();

  const int jmax = min(s, k);
  int steps = 0;
  for (int j = 0; j < jmax; ++j) {
    if (threadIdx.x < 32) {              // pivot: largest trailing norm, ties -> lowest index
      const int lane = threadIdx.x;
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
        misc[2] = (nrm == 0.0 || nrm <= t.eps * misc[0]) ? 1.0 : 0.0;
      }
    }
    __syncthreads();
    if (misc[2] != 0.0) break;
    const int p = (int)misc[1];
    if (p != j) {
      for (int i = threadIdx.x; i < s; i += nthr) {
        const double2 a = A[i + j * ld];
        A[i + j * ld] = A[i + p * ld];
        A[i + p * ld] = a;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        const double a = nrm2[j];
        nrm2[j] = nrm2[p];
        nrm2[p] = a;
      }
    }
    if (threadIdx.x == 0) {              // reflector from column j, rows j..s-1
      double sq = 0.0;
      for (int i = j; i < s; ++i) {
        const double2 v = A[i + j * ld];
        sq = fma(v.x, v.x, fma(v.y, v.y, sq));
      }
      const double nrm = sqrt(sq);
      const double2 x0 = A[j + j * ld];
      const double ax0 = hypot(x0.x, x0.y);
      double px = 1.0, py = 0.0;
      if (ax0 != 0.0) px = x0.x / ax0, py = x0.y / ax0;
      const double2 v0 = make_double2(x0.x + px * nrm, x0.y + py * nrm);   // x0 - alpha
      const double beta = (v0.x * v0.x + v0.y * v0.y) + (sq - ax0 * ax0);  // v^H v
      A[j + j * ld] = v0;
      tau[j] = beta > 0.0 ? 2.0 / beta : 0.0;
    }
    __syncthreads();
    const double tj = tau[j];
    const double2* v = A + j * ld;
    for (int c = j + 1 + threadIdx.x; c < k; c += nthr) {
      double2* a = A + c * ld;
      double wx = 0.0, wy = 0.0;             // w = v^H a
      for (int i = j; i < s; ++i) {
        const double2 vi = v[i], ai = a[i];
        wx = fma(vi.x, ai.x, fma(vi.y, ai.y, wx));
        wy = fma(vi.x, ai.y, fma(-vi.y, ai.x, wy));
      }
      wx *= tj;
      wy *= tj;
      double n2 = 0.0;
      for (int i = j; i < s; ++i) {
        const double2 vi = v[i];
        double2 ai = a[i];
        ai.x = fma(-vi.x, wx, fma(vi.y, wy, ai.x));
        ai.y = fma(-vi.x, wy, fma(-vi.y, wx, ai.y));
        a[i] = ai;
        if (i > j) n2 = fma(ai.x, ai.x, fma(ai.y, ai.y, n2));
      }
      nrm2[c] = n2;
    }
    ++steps;
    __syncthreads();
  }
  const int rank = steps > 0 ? steps : 1;
  if (threadIdx.x == 0) ranks[blockIdx.x] = rank;

  // Q e_c = H_0 ... H_c e_c (H_j leaves e_c unchanged for j > c); one column per thread
  for (int c = threadIdx.x; c < rank; c += nthr) {
    double2* q = Qs + c * ld;
    for (int i = 0; i < s; ++i) q[i] = make_double2(i == c ? 1.0 : 0.0, 0.0);
    for (int j = min(c, steps - 1); j >= 0; --j) {
      const double2* vj = A + j * ld;
      double wx = 0.0, wy = 0.0;
      for (int i = j; i < s; ++i) {
        const double2 vi = vj[i], qi = q[i];
        wx = fma(vi.x, qi.x, fma(vi.y, qi.y, wx));
        wy = fma(vi.x, qi.y, fma(-vi.y, qi.x, wy));
      }
      const double tj = tau[j];
      wx *= tj;
      wy *= tj;
      for (int i = j; i < s; ++i) {
        const double2 vi = vj[i];
        double2 qi = q[i];
        qi.x = fma(-vi.x, wx, fma(vi.y, wy, qi.x));
        qi.y = fma(-vi.x, wy, fma(-vi.y, wx, qi.y));
        q[i] = qi;
      }
    }
  }
  __syncthreads();
  double2* out = (double2*)t.q;
  for (int idx = threadIdx.x; idx < s * rank; idx += nthr) {
    const int i = idx % s, c = idx / s;
    out[i + (int64_t)c * s] = Qs[i + c * ld];
  }
}

size_t qr_workspace_bytes(int ntasks, int maxS, int maxK) {
  const size_t blk = block_bytes(maxS, maxK);
  if (blk + meta_bytes(maxK) <= QR_SMEM_LIMIT) return 0;
  return blk * (size_t)ntasks;
}

int launch_qr(const QRTask* d_tasks, int ntasks, int maxS, int maxK, int in_dtype, int32_t* d_ranks,
              void* d_work, size_t work_bytes, cudaStream_t s) {
  if (ntasks <= 0) return BF_OK;
  const size_t blk = block_bytes(maxS, maxK);
  const int use_smem = (blk + meta_bytes(maxK) <= QR_SMEM_LIMIT) ? 1 : 0;
  const size_t smem = meta_bytes(maxK) + (use_smem ? blk : 0);
  if (!use_smem && (d_work == nullptr || work_bytes < blk * (size_t)ntasks))
    return fail(BF_EINVAL, "QR workspace too small");
  const int64_t stride = (int64_t)(blk / sizeof(double2));
  const int nthr = threads_for(maxK);
  note_launch();
  if (in_dtype == BF_C128) {
    BF_CUDA_TRY(cudaFuncSetAttribute(qr_kernel<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(QR_SMEM_LIMIT + 4096)));
    qr_kernel<double2><<<ntasks, nthr, smem, s>>>(d_tasks, d_ranks, (double2*)d_work, stride, maxK, use_smem);
  } else {
    BF_CUDA_TRY(cudaFuncSetAttribute(qr_kernel<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(QR_SMEM_LIMIT + 4096)));
    qr_kernel<float2><<<ntasks, nthr, smem, s>>>(d_tasks, d_ranks, (double2*)d_work, stride, maxK, use_smem);
  }
  BF_CUDA_TRY(cudaGetLastError());
  return BF_OK;
}

}  // namespace bf
