// Batched truncated column-pivoted Householder QR (Alg. 1 step 3).
//
// One CTA factors one block W (s x k).  At step j the trailing column of
// largest norm is swapped to position j (ties: lowest index); the
// factorization stops when that norm is <= eps times the first pivot's norm
// (or zero); otherwise the reflector
//   H = I - tau v v^H,  v = x - alpha e1,  alpha = -exp(i arg x0) ||x||,
//   tau = 2 / (v^H v)
// is built from the column and applied to the trailing columns.  The rank is
// max(steps, 1) and Q = H_0 ... H_{rank-1} [I; 0] is formed explicitly.
//
// GB300 retires ~2 FP64 FMAs per clock per SM against 128 FP32 lanes, so
// the complex64 (mixed-precision) blocks are factored in float-float
// arithmetic on the FP32 pipe (qr_ff_kernel, ~2^-46 relative rounding):
// the block is first scaled by a power of two so that its largest entry
// lies in [1/2, 1) (Q, the pivots and the rank are invariant under that),
// column norms for pivoting are float32 sums of the high words, the pivot
// column's norm that builds the reflector is float-float, and the relative
// threshold eps is floored at 2^-40, where the float-float rounding of the
// trailing columns (~2^-46 of the block) would start to decide the rank.  Each column of
// the trailing update is handled by RG consecutive lanes (rows strided by
// RG, float-float partial dot products joined by shuffles), so lanes stay
// busy while the trailing matrix shrinks.  Q is formed in place of the
// reflectors, backwards, one barrier per reflector.
//
// The complex128 blocks (and complex64 ones when FP64 is asked for) use the
// FP64 kernel (qr64_kernel), laid out like the float-float one: RG lanes per
// column of the trailing update (rows strided by RG, partial dot products
// and column norms joined by shuffles), Q formed in place backwards.  The
// FP64 pipe retires ~2 FMAs per clock per SM on this GPU, so the kernel's
// time is its FP64 warp instructions: with one thread per column (the first
// design) each instruction carried ~10 of 32 active lanes.  Either kernel
// keeps its block in shared memory when it fits, else in a per-task global
// workspace (same code, pointer switch).
#include "bf_internal.h"
#include "cx.cuh"
#include "ff.cuh"

namespace bf {

namespace {
constexpr size_t QR_SMEM_LIMIT = 200 * 1024;
constexpr int QR_MAX_THREADS = 256;
}  // namespace

// ---------------------------------------------------------------------------
// complex64 blocks: float-float factorization on the FP32 pipe
// ---------------------------------------------------------------------------
namespace {
// smallest leading dimension >= s with ld = RG (mod 8): the RG lanes of a
// column read consecutive 16-byte rows and the 8 / RG columns of a
// quarter-warp start in distinct bank groups
__host__ __device__ inline int ld_ff(int s, int rg) { return s + (((rg & 7) - (s & 7)) & 7); }
__host__ __device__ inline int meta_ff_bytes(int maxS, int maxK) {
  const int rk = (maxK + 1) & ~1;
  const int head = (4 * rk + 8 * maxK + 48 + 15) & ~15;  // norms, tau, flags, warp maxima
  return head + 32 * maxS;                                // two reflector buffers
}
size_t block_ff_bytes(int maxS, int maxK, int rg) { return (size_t)ld_ff(maxS, rg) * maxK * sizeof(float4); }
int rg_for(int maxS) { return maxS <= 8 ? 2 : (maxS <= 48 ? 4 : 8); }
// the FP64 kernel's lanes per column (measured: 2 lanes for the ~20-row
// blocks of the bench workload took 2.09 ms per factorization against 1.81
// with 4)
int rg64_for(int maxS) { return rg_for(maxS); }
}  // namespace

namespace dev {
__device__ __forceinline__ float4 ff_c(FF re, FF im) { return make_float4(re.h, im.h, re.l, im.l); }

template <int RG>
__device__ __forceinline__ FF group_add(FF a, unsigned gmask) {
#pragma unroll
  for (int o = RG / 2; o > 0; o >>= 1) {
    const FF b{__shfl_xor_sync(gmask, a.h, o), __shfl_xor_sync(gmask, a.l, o)};
    a = ff_add(a, b);   // two-sum is exact in either order: every lane gets the same sum
  }
  return a;
}

// col <- H col = col - v (tau v^H col) over rows j..s-1, by the RG lanes of
// one group (lane g takes rows j+g, j+g+RG, ...).  UNIT: col is e_j
// (its content is not read).  NORM: the float32 squared norm of rows
// j+1..s-1 of the result goes to *nrm_out.
template <int RG, bool NORM, bool UNIT>
__device__ __forceinline__ void reflect_column(float4* __restrict__ col, const float4* __restrict__ v, FF tau,
                                               int j, int s, int g, unsigned gmask, float* nrm_out) {
  FF dr{0.0f, 0.0f}, di{0.0f, 0.0f};   // v^H col
  if (UNIT) {
    const float4 vj = v[j];
    dr = {vj.x, vj.z};
    di = {-vj.y, -vj.w};
  } else {
    for (int i = j + g; i < s; i += RG) {
      const float4 a = v[i], b = col[i];
      const FF vx{a.x, a.z}, vy{a.y, a.w}, ax{b.x, b.z}, ay{b.y, b.w};
      ff_mac(dr, vx, ax);
      ff_mac(dr, vy, ay);
      ff_mac(di, vx, ay);
      ff_mac(di, ff_neg(vy), ax);
    }
    dr = group_add<RG>(ff_norm(dr), gmask);
    di = group_add<RG>(ff_norm(di), gmask);
  }
  const FF wr = ff_mul(tau, dr), wi = ff_mul(tau, di);
  float n = 0.0f;
  for (int i = j + g; i < s; i += RG) {
    const float4 a = v[i];
    const FF vx{a.x, a.z}, vy{a.y, a.w};
    FF ax{0.0f, 0.0f}, ay{0.0f, 0.0f};
    if (UNIT) {
      ax.h = (i == j) ? 1.0f : 0.0f;
    } else {
      const float4 b = col[i];
      ax = {b.x, b.z};
      ay = {b.y, b.w};
    }
    ff_mac(ax, ff_neg(vx), wr);   // re: a - (vx wr - vy wi)
    ff_mac(ax, vy, wi);
    ff_mac(ay, ff_neg(vx), wi);   // im: a - (vx wi + vy wr)
    ff_mac(ay, ff_neg(vy), wr);
    ax = ff_norm(ax);
    ay = ff_norm(ay);
    col[i] = ff_c(ax, ay);
    if (NORM && i > j) n = fmaf(ax.h, ax.h, fmaf(ay.h, ay.h, n));
  }
  if (NORM) {
#pragma unroll
    for (int o = RG / 2; o > 0; o >>= 1) n += __shfl_xor_sync(gmask, n, o);
    if (g == 0) *nrm_out = n;
  }
}
}  // namespace dev

template <int RG>
__global__ void qr_ff_kernel(const QRTask* __restrict__ tasks, int32_t* __restrict__ ranks,
                             float4* __restrict__ gwork, int64_t work_stride, int maxS, int maxK, int use_smem) {
  using namespace dev;
  extern __shared__ float4 smem4[];
  char* base = (char*)smem4;
  const QRTask t = tasks[blockIdx.x];
  const int s = t.s, k = t.k, ld = ld_ff(s, RG);
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31;
  const int rk = (maxK + 1) & ~1;
  float* nrm = (float*)base;                                  // k squared column norms (float32)
  float2* taus = (float2*)(base + 4 * rk);                     // tau_j, float-float
  int* flags = (int*)(base + 4 * rk + 8 * maxK);               // [0] stop, [4..11] warp maxima
  float4* vb = (float4*)(base + ((4 * rk + 8 * maxK + 48 + 15) & ~15));   // 2 x maxS
  float4* A = use_smem ? (float4*)(base + meta_ff_bytes(maxS, maxK)) : gwork + blockIdx.x * work_stride;
  const float2* in = (const float2*)t.in;
  const int grp = tid / RG, g = tid % RG, G = nthr / RG;
  const unsigned gmask = ((1u << RG) - 1u) << (lane & ~(RG - 1));
  const float4 zero = make_float4(0.0f, 0.0f, 0.0f, 0.0f);

  // load; largest |component| of the block (as bits: non-negative floats
  // order like their bit patterns)
  unsigned mx = 0u;
  for (int idx = tid; idx < s * k; idx += nthr) {
    const int i = idx % s, c = idx / s;
    const float2 a = in[i + (int64_t)c * t.ldi];
    A[i + c * ld] = make_float4(a.x, a.y, 0.0f, 0.0f);
    mx = max(mx, max(__float_as_uint(a.x) & 0x7fffffffu, __float_as_uint(a.y) & 0x7fffffffu));
  }
  mx = __reduce_max_sync(0xffffffffu, mx);
  if (lane == 0) flags[4 + (tid >> 5)] = (int)mx;
  __syncthreads();
  for (int w = 0; w < (nthr >> 5); ++w) mx = max(mx, (unsigned)flags[4 + w]);
  const int E = (int)(mx >> 23);
  const float sc = (mx == 0u || E >= 255) ? 1.0f : ldexpf(1.0f, 126 - E);   // largest entry -> [1/2, 1)

  // scale (exact: powers of two) and squared column norms
  for (int c = grp; c < k; c += G) {
    float n = 0.0f;
    for (int i = g; i < s; i += RG) {
      float4 a = A[i + c * ld];
      a.x *= sc;
      a.y *= sc;
      A[i + c * ld] = a;
      n = fmaf(a.x, a.x, fmaf(a.y, a.y, n));
    }
#pragma unroll
    for (int o = RG / 2; o > 0; o >>= 1) n += __shfl_xor_sync(gmask, n, o);
    if (g == 0) nrm[c] = n;
  }
  __syncthreads();

  // float-float rounding leaves trailing columns with noise ~2^-46 of the
  // block, so pivots below 2^-40 of the first are not resolved: the
  // threshold is floored there (this also keeps nu^2 and tau in range)
  const float epsf = fmaxf((float)t.eps, 0x1p-40f);
  float nrm0 = 0.0f;
  int steps = 0;
  const int jmax = min(s, k);
  for (int j = 0; j < jmax; ++j) {
    if (tid < 32) {
      // pivot: largest trailing norm, ties -> lowest index
      float best = -1.0f;
      int bi = k;
      for (int c = j + lane; c < k; c += 32) {
        const float v = nrm[c];
        if (v > best) best = v, bi = c;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) best = ob, bi = oi;
      }
      const int p = bi < k ? bi : j;   // (no finite norm: keep column j)
      if (p != j) {
        for (int i = lane; i < s; i += 32) {
          const float4 a = A[i + j * ld];
          A[i + j * ld] = A[i + p * ld];
          A[i + p * ld] = a;
        }
        if (lane == 0) {
          const float a = nrm[j];
          nrm[j] = nrm[p];
          nrm[p] = a;
        }
      }
      __syncwarp();
      // float-float squared norm of the pivot column below row j
      FF rest{0.0f, 0.0f};
      for (int i = j + 1 + lane; i < s; i += 32) {
        const float4 a = A[i + j * ld];
        rest = ff_add(rest, ff_add(ff_sq({a.x, a.z}), ff_sq({a.y, a.w})));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
        rest = ff_add(rest, FF{__shfl_xor_sync(0xffffffffu, rest.h, o), __shfl_xor_sync(0xffffffffu, rest.l, o)});
      if (lane == 0) {
        const float4 x0 = A[j + j * ld];
        const FF xr{x0.x, x0.z}, xi{x0.y, x0.w};
        const FF ax2 = ff_add(ff_sq(xr), ff_sq(xi));
        const FF nu = ff_sqrt(ff_add(ax2, rest));   // ||x||
        if (j == 0) nrm0 = nu.h;
        const bool stop = !(nu.h > 0.0f) || nu.h <= epsf * nrm0;   // epsf >= 2^-40 (see below)
        flags[0] = stop ? 1 : 0;
        if (!stop) {
          const FF ax0 = ff_sqrt(ax2);
          FF vr = nu, vi{0.0f, 0.0f};
          if (ax0.h > 0.0f) {   // v0 = x0 - alpha = x0 (1 + ||x|| / |x0|)
            const FF f = ff_add(FF{1.0f, 0.0f}, ff_div(nu, ax0));
            vr = ff_mul(xr, f);
            vi = ff_mul(xi, f);
          }
          A[j + j * ld] = ff_c(vr, vi);
          // tau = 2 / (v^H v) from the stored v itself, so H stays unitary to
          // float-float rounding whatever the rounding of ||x||
          const FF vhv = ff_add(ff_add(ff_sq(vr), ff_sq(vi)), rest);
          const FF tau = ff_div(FF{2.0f, 0.0f}, vhv);
          taus[j] = make_float2(tau.h, tau.l);
        }
      }
    }
    __syncthreads();
    if (flags[0]) break;
    const FF tau{taus[j].x, taus[j].y};
    for (int c = j + 1 + grp; c < k; c += G)
      reflect_column<RG, true, false>(A + c * ld, A + j * ld, tau, j, s, g, gmask, nrm + c);
    ++steps;
    __syncthreads();
  }
  const int rank = steps > 0 ? steps : 1;
  if (tid == 0) ranks[blockIdx.x] = rank;

  // Q in place of the reflectors, backwards: at step j the columns > j hold
  // H_{j+1} ... H_{rank-1} [I; 0] (zero above their diagonal), column j
  // starts as e_j; v_j is read from a buffer so that column j can be
  // overwritten in the same step, and v_{j-1} is copied into the other one.
  if (steps == 0) {
    for (int i = tid; i < s; i += nthr) A[i] = i == 0 ? make_float4(1.0f, 0.0f, 0.0f, 0.0f) : zero;
    __syncthreads();
  } else {
    {
      const int j = steps - 1;
      float4* dst = vb + (j & 1) * maxS;
      for (int i = j + tid; i < s; i += nthr) dst[i] = A[i + j * ld];
    }
    __syncthreads();
    for (int j = steps - 1; j >= 0; --j) {
      const float4* v = vb + (j & 1) * maxS;
      if (j > 0) {
        float4* dst = vb + ((j - 1) & 1) * maxS;
        for (int i = j - 1 + tid; i < s; i += nthr) dst[i] = A[i + (j - 1) * ld];
      }
      const FF tau{taus[j].x, taus[j].y};
      for (int c = j + grp; c < rank; c += G) {
        float4* col = A + c * ld;
        if (c == j) {
          for (int i = g; i < j; i += RG) col[i] = zero;
          reflect_column<RG, false, true>(col, v, tau, j, s, g, gmask, nullptr);
        } else {
          reflect_column<RG, false, false>(col, v, tau, j, s, g, gmask, nullptr);
        }
      }
      __syncthreads();
    }
  }
  double2* out = (double2*)t.q;
  for (int idx = tid; idx < s * rank; idx += nthr) {
    const int i = idx % s, c = idx / s;
    const float4 a = A[i + c * ld];
    out[i + (int64_t)c * s] = make_double2((double)a.x + (double)a.z, (double)a.y + (double)a.w);
  }
}


// ---------------------------------------------------------------------------
// FP64 factorization (complex128 blocks, and complex64 ones on request)
// ---------------------------------------------------------------------------
namespace {
// shared-memory head: squared norms and tau (double each), a stop flag,
// then two reflector buffers of maxS entries
__host__ __device__ inline int meta64_head(int maxK) { return (16 * maxK + 64 + 15) & ~15; }
__host__ __device__ inline int meta64_bytes(int maxS, int maxK) { return meta64_head(maxK) + 32 * maxS; }
size_t block64_bytes(int maxS, int maxK, int rg) { return (size_t)ld_ff(maxS, rg) * maxK * sizeof(double2); }
}  // namespace

namespace dev {
template <int RG>
__device__ __forceinline__ double group_sum(double a, unsigned gmask) {
#pragma unroll
  for (int o = RG / 2; o > 0; o >>= 1) a += __shfl_xor_sync(gmask, a, o);   // every lane gets the same sum
  return a;
}

// col <- H col = col - v (tau v^H col) over rows j..s-1 by the RG lanes of one
// group; UNIT: col is e_j (not read); NORM: squared norm of rows j+1..s-1 of
// the result to *nrm_out.
template <int RG, bool NORM, bool UNIT>
__device__ __forceinline__ void reflect64(double2* __restrict__ col, const double2* __restrict__ v, double tau,
                                          int j, int s, int g, unsigned gmask, double* nrm_out) {
  double dr = 0.0, di = 0.0;   // v^H col
  if (UNIT) {
    dr = v[j].x;
    di = -v[j].y;
  } else {
    for (int i = j + g; i < s; i += RG) {
      const double2 a = v[i], b = col[i];
      dr = fma(a.x, b.x, fma(a.y, b.y, dr));
      di = fma(a.x, b.y, fma(-a.y, b.x, di));
    }
    dr = group_sum<RG>(dr, gmask);
    di = group_sum<RG>(di, gmask);
  }
  const double wr = tau * dr, wi = tau * di;
  double n = 0.0;
  for (int i = j + g; i < s; i += RG) {
    const double2 a = v[i];
    double2 b = UNIT ? make_double2(i == j ? 1.0 : 0.0, 0.0) : col[i];
    b.x = fma(-a.x, wr, fma(a.y, wi, b.x));    // re: b - (vx wr - vy wi)
    b.y = fma(-a.x, wi, fma(-a.y, wr, b.y));   // im: b - (vx wi + vy wr)
    col[i] = b;
    if (NORM && i > j) n = fma(b.x, b.x, fma(b.y, b.y, n));
  }
  if (NORM) {
    n = group_sum<RG>(n, gmask);
    if (g == 0) *nrm_out = n;
  }
}
}  // namespace dev

template <typename VIn, int RG>
__global__ void qr64_kernel(const QRTask* __restrict__ tasks, int32_t* __restrict__ ranks,
                            double2* __restrict__ gwork, int64_t work_stride, int maxS, int maxK, int use_smem) {
  using namespace dev;
  extern __shared__ double2 smem64[];
  char* base = (char*)smem64;
  const QRTask t = tasks[blockIdx.x];
  const int s = t.s, k = t.k, ld = ld_ff(s, RG);
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31;
  double* nrm = (double*)base;                                // k squared trailing column norms
  double* taus = nrm + maxK;                                  // tau_j
  int* flags = (int*)(base + 16 * maxK);                      // [0] stop
  double2* vb = (double2*)(base + meta64_head(maxK));         // 2 x maxS reflector buffers
  double2* A = use_smem ? (double2*)(base + meta64_bytes(maxS, maxK)) : gwork + blockIdx.x * work_stride;
  const VIn* in = (const VIn*)t.in;
  const int grp = tid / RG, g = tid % RG, G = nthr / RG;
  const unsigned gmask = ((1u << RG) - 1u) << (lane & ~(RG - 1));
  const double2 zero = make_double2(0.0, 0.0);

  for (int idx = tid; idx < s * k; idx += nthr) {
    const int i = idx % s, c = idx / s;
    A[i + c * ld] = to_d2(in[i + (int64_t)c * t.ldi]);
  }
  __syncthreads();
  for (int c = grp; c < k; c += G) {
    double n = 0.0;
    for (int i = g; i < s; i += RG) {
      const double2 a = A[i + c * ld];
      n = fma(a.x, a.x, fma(a.y, a.y, n));
    }
    n = group_sum<RG>(n, gmask);
    if (g == 0) nrm[c] = n;
  }
  __syncthreads();

  double nrm0 = 0.0;   // first pivot's norm (lane 0 of warp 0)
  int steps = 0;
  const int jmax = min(s, k);
  for (int j = 0; j < jmax; ++j) {
    if (tid < 32) {
      // pivot: largest trailing norm, ties -> lowest index
      double best = -1.0;
      int bi = k;
      for (int c = j + lane; c < k; c += 32) {
        const double v = nrm[c];
        if (v > best) best = v, bi = c;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) best = ob, bi = oi;
      }
      const int p = bi < k ? bi : j;   // (no finite norm: keep column j)
      if (p != j) {
        for (int i = lane; i < s; i += 32) {
          const double2 a = A[i + j * ld];
          A[i + j * ld] = A[i + p * ld];
          A[i + p * ld] = a;
        }
        if (lane == 0) {
          const double a = nrm[j];
          nrm[j] = nrm[p];
          nrm[p] = a;
        }
      }
      __syncwarp();
      double rest = 0.0;   // squared norm of the pivot column below row j
      for (int i = j + 1 + lane; i < s; i += 32) {
        const double2 a = A[i + j * ld];
        rest = fma(a.x, a.x, fma(a.y, a.y, rest));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) rest += __shfl_xor_sync(0xffffffffu, rest, o);
      if (lane == 0) {
        const double2 x0 = A[j + j * ld];
        const double ax2 = fma(x0.x, x0.x, x0.y * x0.y);
        const double nu = sqrt(ax2 + rest);   // ||x||
        if (j == 0) nrm0 = nu;
        const bool stop = !(nu > 0.0) || nu <= t.eps * nrm0;
        flags[0] = stop ? 1 : 0;
        if (!stop) {
          const double ax0 = sqrt(ax2);
          double vr = nu, vi = 0.0;
          if (ax0 > 0.0) {   // v0 = x0 - alpha = x0 (1 + ||x|| / |x0|)
            const double f = 1.0 + nu / ax0;
            vr = x0.x * f;
            vi = x0.y * f;
          }
          A[j + j * ld] = make_double2(vr, vi);
          taus[j] = 2.0 / (fma(vr, vr, vi * vi) + rest);   // 2 / (v^H v) from the stored v
        }
      }
    }
    __syncthreads();
    if (flags[0]) break;
    const double tau = taus[j];
    for (int c = j + 1 + grp; c < k; c += G)
      reflect64<RG, true, false>(A + c * ld, A + j * ld, tau, j, s, g, gmask, nrm + c);
    ++steps;
    __syncthreads();
  }
  const int rank = steps > 0 ? steps : 1;
  if (tid == 0) ranks[blockIdx.x] = rank;

  // Q in place of the reflectors, backwards (as in qr_ff_kernel)
  if (steps == 0) {
    for (int i = tid; i < s; i += nthr) A[i] = i == 0 ? make_double2(1.0, 0.0) : zero;
    __syncthreads();
  } else {
    {
      const int j = steps - 1;
      double2* dst = vb + (j & 1) * maxS;
      for (int i = j + tid; i < s; i += nthr) dst[i] = A[i + j * ld];
    }
    __syncthreads();
    for (int j = steps - 1; j >= 0; --j) {
      const double2* v = vb + (j & 1) * maxS;
      if (j > 0) {
        double2* dst = vb + ((j - 1) & 1) * maxS;
        for (int i = j - 1 + tid; i < s; i += nthr) dst[i] = A[i + (j - 1) * ld];
      }
      const double tau = taus[j];
      for (int c = j + grp; c < rank; c += G) {
        double2* col = A + c * ld;
        if (c == j) {
          for (int i = g; i < j; i += RG) col[i] = zero;
          reflect64<RG, false, true>(col, v, tau, j, s, g, gmask, nullptr);
        } else {
          reflect64<RG, false, false>(col, v, tau, j, s, g, gmask, nullptr);
        }
      }
      __syncthreads();
    }
  }
  double2* out = (double2*)t.q;
  for (int idx = tid; idx < s * rank; idx += nthr) {
    const int i = idx % s, c = idx / s;
    out[i + (int64_t)c * s] = A[i + c * ld];
  }
}

namespace {
template <int RG>
int launch_qr_ff(const QRTask* d_tasks, int ntasks, int maxS, int maxK, int32_t* d_ranks, void* d_work,
                 size_t work_bytes, cudaStream_t s) {
  const size_t blk = block_ff_bytes(maxS, maxK, RG);
  const size_t meta = (size_t)meta_ff_bytes(maxS, maxK);
  const int use_smem = (blk + meta <= QR_SMEM_LIMIT) ? 1 : 0;
  if (meta > QR_SMEM_LIMIT) return fail(BF_EINVAL, "QR block too large");
  if (!use_smem && (d_work == nullptr || work_bytes < blk * (size_t)ntasks))
    return fail(BF_EINVAL, "QR workspace too small");
  const size_t smem = meta + (use_smem ? blk : 0);
  int nthr = ((maxK * RG + 31) / 32) * 32;
  nthr = nthr > QR_MAX_THREADS ? QR_MAX_THREADS : nthr;
  BF_CUDA_TRY(cudaFuncSetAttribute(qr_ff_kernel<RG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(QR_SMEM_LIMIT + 4096)));
  note_launch();
  qr_ff_kernel<RG><<<ntasks, nthr, smem, s>>>(d_tasks, d_ranks, (float4*)d_work, (int64_t)(blk / sizeof(float4)),
                                              maxS, maxK, use_smem);
  BF_CUDA_TRY(cudaGetLastError());
  return BF_OK;
}

template <typename VIn, int RG>
int launch_qr64(const QRTask* d_tasks, int ntasks, int maxS, int maxK, int32_t* d_ranks, void* d_work,
                size_t work_bytes, cudaStream_t s) {
  const size_t blk = block64_bytes(maxS, maxK, RG);
  const size_t meta = (size_t)meta64_bytes(maxS, maxK);
  const int use_smem = (blk + meta <= QR_SMEM_LIMIT) ? 1 : 0;
  if (meta > QR_SMEM_LIMIT) return fail(BF_EINVAL, "QR block too large");
  if (!use_smem && (d_work == nullptr || work_bytes < blk * (size_t)ntasks))
    return fail(BF_EINVAL, "QR workspace too small");
  const size_t smem = meta + (use_smem ? blk : 0);
  int nthr = ((maxK * RG + 31) / 32) * 32;
  nthr = nthr > QR_MAX_THREADS ? QR_MAX_THREADS : nthr;
  BF_CUDA_TRY(cudaFuncSetAttribute(qr64_kernel<VIn, RG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(QR_SMEM_LIMIT + 4096)));
  note_launch();
  qr64_kernel<VIn, RG><<<ntasks, nthr, smem, s>>>(d_tasks, d_ranks, (double2*)d_work,
                                                  (int64_t)(blk / sizeof(double2)), maxS, maxK, use_smem);
  BF_CUDA_TRY(cudaGetLastError());
  return BF_OK;
}
template <typename VIn>
int launch_qr64_rg(const QRTask* d_tasks, int ntasks, int maxS, int maxK, int32_t* d_ranks, void* d_work,
                   size_t work_bytes, cudaStream_t s) {
  switch (rg64_for(maxS)) {
    case 2: return launch_qr64<VIn, 2>(d_tasks, ntasks, maxS, maxK, d_ranks, d_work, work_bytes, s);
    case 4: return launch_qr64<VIn, 4>(d_tasks, ntasks, maxS, maxK, d_ranks, d_work, work_bytes, s);
    default: return launch_qr64<VIn, 8>(d_tasks, ntasks, maxS, maxK, d_ranks, d_work, work_bytes, s);
  }
}
}  // namespace

int qr_lanes(int s, int in_dtype, bool fp64) { return (in_dtype == BF_C64 && !fp64) ? rg_for(s) : rg64_for(s); }

size_t qr_workspace_bytes(int ntasks, int maxS, int maxK, int in_dtype, bool fp64) {
  if (in_dtype == BF_C64 && !fp64) {
    const size_t blk = block_ff_bytes(maxS, maxK, rg_for(maxS));
    if (blk + (size_t)meta_ff_bytes(maxS, maxK) <= QR_SMEM_LIMIT) return 0;
    return blk * (size_t)ntasks;
  }
  const size_t blk = block64_bytes(maxS, maxK, rg64_for(maxS));
  if (blk + (size_t)meta64_bytes(maxS, maxK) <= QR_SMEM_LIMIT) return 0;
  return blk * (size_t)ntasks;
}

int launch_qr(const QRTask* d_tasks, int ntasks, int maxS, int maxK, int in_dtype, bool fp64, int32_t* d_ranks,
              void* d_work, size_t work_bytes, cudaStream_t s) {
  if (ntasks <= 0) return BF_OK;
  if (in_dtype == BF_C64 && !fp64) {
    switch (rg_for(maxS)) {
      case 2: return launch_qr_ff<2>(d_tasks, ntasks, maxS, maxK, d_ranks, d_work, work_bytes, s);
      case 4: return launch_qr_ff<4>(d_tasks, ntasks, maxS, maxK, d_ranks, d_work, work_bytes, s);
      default: return launch_qr_ff<8>(d_tasks, ntasks, maxS, maxK, d_ranks, d_work, work_bytes, s);
    }
  }
  if (in_dtype == BF_C128) return launch_qr64_rg<double2>(d_tasks, ntasks, maxS, maxK, d_ranks, d_work, work_bytes, s);
  return launch_qr64_rg<float2>(d_tasks, ntasks, maxS, maxK, d_ranks, d_work, work_bytes, s);
}

}  // namespace bf
