// Small memory-bound kernels: the counter-based Gaussian generator,
// row permutations between user and tree order, structured expansion of a
// compact random matrix, dtype conversion, conjugation and norm reductions.
#include "bf_internal.h"
#include "cx.cuh"

namespace bf {

// ----------------------------------------------------------------- RNG ---
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two
// 32x32->64 multiplies with the published multipliers and Weyl key bumps.
__device__ __forceinline__ void philox4x32_10(uint32_t& c0, uint32_t& c1,
                                              uint32_t& c2, uint32_t& c3,
                                              uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// Entry (g, c): counter (g>>1, c, stream, 0), key = seed; words (0,1) for
// even g, (2,3) for odd g; Box-Muller z = sqrt(-ln u1) exp(2 pi i u2) with
// u = (word + 1/2) 2^-32 (FP64 for complex128 output, FP32 for complex64).
template <typename R>
__global__ void gaussian_kernel(uint64_t seed, uint32_t sid, int64_t row0,
                                int64_t rows, int64_t col0, int64_t ncols,
                                typename Cx<R>::V* out, int64_t ld) {
  const int64_t p0 = row0 >> 1;
  const int64_t npairs = ((row0 + rows + 1) >> 1) - p0;
  const int64_t total = npairs * ncols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pr = p0 + t % npairs;
    const int64_t c = col0 + t / npairs;
    uint32_t w0 = (uint32_t)pr, w1 = (uint32_t)c, w2 = sid, w3 = 0;
    philox4x32_10(w0, w1, w2, w3, (uint32_t)seed, (uint32_t)(seed >> 32));
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t g = 2 * pr + h;
      if (g < row0 || g >= row0 + rows) continue;
      const uint32_t a = h ? w2 : w0, b = h ? w3 : w1;
      if (sizeof(R) == 8) {
        const double u1 = ((double)a + 0.5) * 2.3283064365386963e-10;
        const double u2 = ((double)b + 0.5) * 2.3283064365386963e-10;
        const double rad = sqrt(-log(u1));
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
        out[(g - row0) + (c - col0) * ld] = Cx<R>::make((R)(rad * cs), (R)(rad * sn));
      } else {
        // complex64: the same variates in FP32 (this GPU's FP64 pipe is
        // 1/64 of its FP32 rate); -ln u1 from u1 itself below 1/2 and from
        // 1 - u1 (exact in 32-bit integers) above, so no cancellation
        const float l = a < 0x80000000u ? -logf(((float)a + 0.5f) * 2.3283064e-10f)
                                        : -log1pf(-((float)(0xFFFFFFFFu - a) + 0.5f) * 2.3283064e-10f);
        const float rad = sqrtf(l);
        float sn, cs;
        sincospif(2.0f * (((float)b + 0.5f) * 2.3283064e-10f), &sn, &cs);
        out[(g - row0) + (c - col0) * ld] = Cx<R>::make((R)(rad * cs), (R)(rad * sn));
      }
    }
  }
}

static inline int grid_for(int64_t total, int threads = 256) {
  int64_t b = (total + threads - 1) / threads;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return (int)b;
}

int launch_gaussian(uint64_t seed, uint32_t sid, int64_t row0, int64_t rows,
                    int64_t col0, int64_t col1, void* out, int64_t ld, int dtype,
                    cudaStream_t s) {
  if (rows <= 0 || col1 <= col0) return BF_OK;
  const int64_t npairs = ((row0 + rows + 1) >> 1) - (row0 >> 1);
  const int g = grid_for(npairs * (col1 - col0));
  note_launch();
  if (dtype == BF_C128)
    gaussian_kernel<double><<<g, 256, 0, s>>>(seed, sid, row0, rows, col0, col1 - col0,
                                              (double2*)out, ld);
  else
    gaussian_kernel<float><<<g, 256, 0, s>>>(seed, sid, row0, rows, col0, col1 - col0,
                                             (float2*)out, ld);
  BF_CUDA_TRY(cudaGetLastError());
  return BF_OK;
}

// ------------------------------------------------------------ permutes ---
template <typename V, bool SCATTER>
__global__ void permute_rows_kernel(const int64_t* perm, int64_t rows, int64_t cols,
                                    const V* in, int64_t ldi, V* out, int64_t ldo,
                                    int conj) {
  const int64_t total = rows * cols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % rows, c = t / rows;
    const int64_t p = perm ? perm[i] : i;
    V v = SCATTER ? in[i + c * ldi] : in[p + c * ldi];
    if (conj) v.y = -v.y;
    if (SCATTER)
      out[p + c * ldo] = v;
    else
      out[i + c * ldo] = v;
  }
}

int launch_gather_rows(const int64_t* d_perm, int64_t rows, int64_t cols,
                       const void* in, int64_t ldi, void* out, int64_t ldo,
                       int conj, int dtype, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return BF_OK;
  const int g = grid_for(rows * cols);
  note_launch();
  if (dtype == BF_C128)
    permute_rows_kernel<double2, false><<<g, 256, 0, s>>>(d_perm, rows, cols, (const double2*)in, ldi,
                                                           (double2*)out, ldo, conj);
  else
    permute_rows_kernel<float2, false><<<g, 256, 0, s>>>(d_perm, rows, cols, (const float2*)in, ldi,
                                                          (float2*)out, ldo, conj);
  BF_CUDA_TRY(cudaGetLastError());
  return BF_OK;
}

int launch_scatter_rows(const int64_t* d_perm, int64_t rows, int64_t cols,
                        const void* in, int64_t ldi, void* out, int64_t ldo,
                        int conj, int dtype, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return BF_OK;
  const int g = grid_for(rows * cols);
  note_launch();
  if (dtype == BF_C128)
    permute_rows_kernel<double2, true><<<g, 256, 0, s>>>(d_perm, rows, cols, (const double2*)in, ldi,
                                                          (double2*)out, ldo, conj);
  else
    permute_rows_kernel<float2, true><<<g, 256, 0, s>>>(d_perm, rows, cols, (const float2*)in, ldi,
                                                         (float2*)out, ldo, conj);
  BF_CUDA_TRY(cudaGetLastError());
  return BF_OK;
}

// out (rows x groups*k) = block-diagonal scatter of the compact matrix.
template <typename V>
__global__ void expand_kernel(int groups, const int64_t* off, int64_t rows, int64_t k,
                              const V* in, int64_t ldi, V* out, int64_t ldo) {
  const int64_t total = rows * k * groups;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % rows;
    const int64_t cg = t / rows;          // 0 .. groups*k-1
    const int64_t g = cg / k, c = cg % k;
    V v;
    if (i >= off[g] && i < off[g + 1])
      v = in[i + c * ldi];
    else
      v.x = 0, v.y = 0;
    out[i + cg * ldo] = v;
  }
}

int launch_expand_structured(int groups, const int64_t* d_off, int64_t rows, int64_t k,
                             const void* in, int64_t ldi, void* out, int64_t ldo,
                             int dtype, cudaStream_t s) {
  const int g = grid_for(rows * k * groups);
  note_launch();
  if (dtype == BF_C128)
    expand_kernel<double2><<<g, 256, 0, s>>>(groups, d_off, rows, k, (const double2*)in, ldi,
                                             (double2*)out, ldo);
  else
    expand_kernel<float2><<<g, 256, 0, s>>>(groups, d_off, rows, k, (const float2*)in, ldi,
                                            (float2*)out, ldo);
  BF_CUDA_TRY(cudaGetLastError());
  return BF_OK;
}

template <typename A, typename B>
__global__ void gather2d_kernel(const int64_t* rp, const int64_t* cp, int64_t rows, int64_t cols,
                                const A* in, int64_t ldi, B* out, int64_t ldo) {
  const int64_t total = rows * cols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % rows, j = t / rows;
    const int64_t si = rp ? rp[i] : i, sj = cp ? cp[j] : j;
    const A v = in[si + sj * ldi];
    B w;
    w.x = v.x;
    w.y = v.y;
    out[i + j * ldo] = w;
  }
}

int launch_gather2d(const int64_t* d_rp, const int64_t* d_cp, int64_t rows, int64_t cols,
                    const void* in, int64_t ldi, int in_dtype, void* out, int64_t ldo,
                    int out_dtype, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return BF_OK;
  const int g = grid_for(rows * cols);
  note_launch();
  if (in_dtype == BF_C128 && out_dtype == BF_C128)
    gather2d_kernel<double2, double2><<<g, 256, 0, s>>>(d_rp, d_cp, rows, cols, (const double2*)in, ldi,
                                                         (double2*)out, ldo);
  else if (in_dtype == BF_C128)
    gather2d_kernel<double2, float2><<<g, 256, 0, s>>>(d_rp, d_cp, rows, cols, (const double2*)in, ldi,
                                                        (float2*)out, ldo);
  else if (out_dtype == BF_C128)
    gather2d_kernel<float2, double2><<<g, 256, 0, s>>>(d_rp, d_cp, rows, cols, (const float2*)in, ldi,
                                                        (double2*)out, ldo);
  else
    gather2d_kernel<float2, float2><<<g, 256, 0, s>>>(d_rp, d_cp, rows, cols, (const float2*)in, ldi,
                                                       (float2*)out, ldo);
  BF_CUDA_TRY(cudaGetLastError());
  return BF_OK;
}

template <typename A, typename B>
__global__ void convert_kernel(const A* in, B* out, int64_t count) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x) {
    A v = in[t];
    B w;
    w.x = v.x;
    w.y = v.y;
    out[t] = w;
  }
}

int launch_convert(const void* in, void* out, int64_t count, int in_dtype, int out_dtype,
                   cudaStream_t s) {
  if (count <= 0) return BF_OK;
  const int g = grid_for(count);
  if (in_dtype == out_dtype) {
    BF_CUDA_TRY(cudaMemcpyAsync(out, in, count * elem_bytes(in_dtype), cudaMemcpyDeviceToDevice, s));
    return BF_OK;
  }
  note_launch();
  if (in_dtype == BF_C128)
    convert_kernel<double2, float2><<<g, 256, 0, s>>>((const double2*)in, (float2*)out, count);
  else
    convert_kernel<float2, double2><<<g, 256, 0, s>>>((const float2*)in, (double2*)out, count);
  BF_CUDA_TRY(cudaGetLastError());
  return BF_OK;
}

template <typename V>
__global__ void conj_kernel(V* p, int64_t rows, int64_t cols, int64_t ld) {
  const int64_t total = rows * cols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % rows, c = t / rows;
    p[i + c * ld].y = -p[i + c * ld].y;
  }
}

int launch_conj_inplace(void* p, int64_t rows, int64_t cols, int64_t ld, int dtype,
                        cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return BF_OK;
  const int g = grid_for(rows * cols);
  note_launch();
  if (dtype == BF_C128)
    conj_kernel<double2><<<g, 256, 0, s>>>((double2*)p, rows, cols, ld);
  else
    conj_kernel<float2><<<g, 256, 0, s>>>((float2*)p, rows, cols, ld);
  BF_CUDA_TRY(cudaGetLastError());
  return BF_OK;
}

// ---------------------------------------------------------- reductions ---
template <typename V>
__global__ void diff_norms_kernel(const V* a, const V* b, int64_t rows, int64_t cols,
                                  int64_t lda, int64_t ldb, double* out) {
  double sd = 0.0, sa = 0.0;
  const int64_t total = rows * cols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % rows, c = t / rows;
    const V x = a[i + c * lda], y = b[i + c * ldb];
    const double dx = (double)x.x - (double)y.x, dy = (double)x.y - (double)y.y;
    sd += dx * dx + dy * dy;
    sa += (double)x.x * x.x + (double)x.y * x.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sd += __shfl_down_sync(0xffffffffu, sd, o);
    sa += __shfl_down_sync(0xffffffffu, sa, o);
  }
  __shared__ double red[2][32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[0][w] = sd, red[1][w] = sa;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    sd = l < nw ? red[0][l] : 0.0;
    sa = l < nw ? red[1][l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      sd += __shfl_down_sync(0xffffffffu, sd, o);
      sa += __shfl_down_sync(0xffffffffu, sa, o);
    }
    if (l == 0) {
      atomicAdd(out, sd);
      atomicAdd(out + 1, sa);
    }
  }
}

int launch_diff_norms(const void* a, const void* b, int64_t rows, int64_t cols, int64_t lda,
                      int64_t ldb, int dtype, double* d_out, cudaStream_t s) {
  BF_CUDA_TRY(cudaMemsetAsync(d_out, 0, 2 * sizeof(double), s));
  const int g = grid_for(rows * cols);
  note_launch();
  if (dtype == BF_C128)
    diff_norms_kernel<double2><<<g, 256, 0, s>>>((const double2*)a, (const double2*)b, rows, cols,
                                                 lda, ldb, d_out);
  else
    diff_norms_kernel<float2><<<g, 256, 0, s>>>((const float2*)a, (const float2*)b, rows, cols,
                                                lda, ldb, d_out);
  BF_CUDA_TRY(cudaGetLastError());
  return BF_OK;
}

}  // namespace bf
