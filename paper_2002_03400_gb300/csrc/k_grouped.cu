// Grouped apply of a finished factorization (eq. hybrid_butterfly_mat): the
// L + 3 stages in runs of `depth` consecutive stages, one launch per run.
//
// The apply's chain only ever reads the previous stage's output, and in a
// butterfly each block of level j + 1 reads two blocks of level j (W^j: the
// two children of a column-tree node; R^j and the adjoints likewise), so the
// tasks of a few consecutive stages fall into small connected groups (for
// the W levels with depth 3: 4 + 4 + 4 blocks whose inputs are 8 blocks of
// the level below).  Each group has an image, built once per plan: its
// descriptors and its factor blocks packed as tiles, contiguous and
// 16-byte aligned.  One CTA per (group, column slice):
//   - copies the group's image into shared memory in one coalesced pass
//     while it waits for the previous launch (the image does not depend on
//     it; programmatic dependent launch), then the group's input rows of the
//     previous run's output (or of x);
//   - computes the run's stages one after another, the inner stages' blocks
//     in shared memory, and writes only the last stage's blocks to global
//     memory (one of two level buffers, or y).
// Column-major x and y (the first run's input, the last run's output) are
// held column by column in shared memory from 32 columns per slice on, so
// both move along a column's contiguous rows; complex64 products use packed
// FP32 FMAs over pairs of rows; independent single-block groups are merged
// (complex64) so that a CTA has several blocks to work on.
// So an apply takes ceil((L + 3) / depth) launches, each reading its inputs
// once and writing its outputs once.  Every output is the same FMA chain as
// in the stage kernels (terms in order, k ascending): results equal the
// stage apply's bit for bit.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <numeric>

#include "bf_internal.h"
#include "cx.cuh"

namespace bf {

namespace {
constexpr size_t GR_SMEM_LIMIT = 110 * 1024;   // two CTAs per SM
constexpr size_t GR_FAC_LIMIT = 40 * 1024;     // staged factor bytes per group (more: read in place)

struct GroupedArgs {
  const uint8_t* img;   // the run's group images: group (group0 + i) at img + i * stride bytes
  int64_t stride;       // bytes per image (a multiple of 16); the rows follow it in shared memory
  int group0;           // the run's first group
  int N, CW;            // right-hand sides, column-slice width
  const void* x;        // the run's input (row-major N columns when in_ld == 0, else column-major)
  int64_t in_ld;
  void* y;              // the run's output base
};

template <int BYTES>
__device__ __forceinline__ void gr_cp_async(void* dst, const void* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}

__host__ __device__ constexpr size_t gr_align16(size_t b) { return (b + 15) & ~(size_t)15; }
static_assert(sizeof(GroupedTask) % 8 == 0 && sizeof(GroupedSpan) % 8 == 0, "image parts keep 8-byte alignment");

// shared memory of one CTA: the group's image, then the rows of every
// region (CW columns each)
inline size_t gr_smem_bytes(int64_t stride, int rows_max, int CW, size_t es) {
  return (size_t)stride + (size_t)rows_max * CW * es;
}

template <typename V, bool CJ>
__device__ __forceinline__ void gr_fma(V& acc, const V e, const V x) {
  if constexpr (CJ) cmac_conj(acc, e, x);
  else cmac(acc, e, x);
}

// Rows r0 .. r0 + NR - 1 of a staged complex128 term for the lane's column
// c (x: the lane's input column, consecutive k xs elements apart; t: the
// tile, entry (i, k) at t[k tld + i]): acc[r] += op(A)(r0 + r, k) x(k, c),
// k ascending -- the stage kernels' FMA chain (CJ: op(A) = conj(A)^T, the
// staged entries are A's, the conjugate is taken in the multiply).
template <typename V, int NR, bool CJ>
__device__ __forceinline__ void gr_tile_s(const V* __restrict__ x, int xs, const V* __restrict__ t, int tld, int K,
                                          V* acc) {
#pragma unroll 2
  for (int kk = 0; kk < K; ++kk) {
    const V xv = *x;
#pragma unroll
    for (int r = 0; r < NR; ++r) gr_fma<V, CJ>(acc[r], t[r], xv);
    x += xs;
    t += tld;
  }
}

// the same for a term read in place (global memory, the factor's layout)
template <typename V, int NR, bool CJ>
__device__ __forceinline__ void gr_tile_g(const V* __restrict__ x, int xs, const V* __restrict__ mat, int ldm, int K,
                                          int r0, V* acc) {
#pragma unroll 2
  for (int kk = 0; kk < K; ++kk) {
    const V xv = x[kk * xs];
    if constexpr (CJ) {
      const V* __restrict__ m = mat + (int64_t)r0 * ldm + kk;
#pragma unroll
      for (int r = 0; r < NR; ++r) cmac_conj(acc[r], m[r * ldm], xv);
    } else {
      const V* __restrict__ m = mat + (int64_t)kk * ldm + r0;
#pragma unroll
      for (int r = 0; r < NR; ++r) cmac(acc[r], m[r], xv);
    }
  }
}

// Complex64 tiles are planar: column k of a tile holds the real parts of
// its tq rows (tq = M rounded up to 4), then their imaginary parts.  A
// lane's accumulators pair rows (2p, 2p + 1): ax[p] their real parts, ay[p]
// their imaginary parts, so one packed FP32 FMA (__ffma2_rn) serves two rows.
// Each component takes the products in the order of cmac / cmac_conj, so
// every output is still the stage kernels' FMA chain.
template <bool CJ>
__device__ __forceinline__ void gr_pair(float2& ax, float2& ay, const float2 ex, const float2 ey, const float2 XX,
                                        const float2 YY, const float2 NEG) {
  // NEG: (-x.y, -x.y) for A, (-x.x, -x.x) for conj(A)
  ax = __ffma2_rn(ex, XX, ax);
  ax = __ffma2_rn(ey, CJ ? YY : NEG, ax);
  ay = __ffma2_rn(ex, YY, ay);
  ay = __ffma2_rn(ey, CJ ? NEG : XX, ay);
}
template <bool CJ>
__device__ __forceinline__ void gr_one(float& ax, float& ay, const float ex, const float ey, const float2 xv) {
  if constexpr (CJ) {
    ax = fmaf(ex, xv.x, ax);
    ax = fmaf(ey, xv.y, ax);
    ay = fmaf(ex, xv.y, ay);
    ay = fmaf(-ey, xv.x, ay);
  } else {
    ax = fmaf(ex, xv.x, ax);
    ax = fmaf(-ey, xv.y, ax);
    ay = fmaf(ex, xv.y, ay);
    ay = fmaf(ey, xv.x, ay);
  }
}
template <int NR, bool CJ>
__device__ __forceinline__ void gr_tile_p(const float2* __restrict__ x, int xs, const float* __restrict__ t, int tq,
                                          int K, float2* ax, float2* ay) {
#pragma unroll 2
  for (int kk = 0; kk < K; ++kk) {
    const float2 xv = *x;
    const float2 XX = make_float2(xv.x, xv.x), YY = make_float2(xv.y, xv.y);
    const float2 NEG = CJ ? make_float2(-xv.x, -xv.x) : make_float2(-xv.y, -xv.y);
#pragma unroll
    for (int r = 0; r + 3 < NR; r += 4) {   // four rows: two 16-byte loads
      const float4 ex = *(const float4*)(t + r), ey = *(const float4*)(t + tq + r);
      gr_pair<CJ>(ax[r / 2], ay[r / 2], make_float2(ex.x, ex.y), make_float2(ey.x, ey.y), XX, YY, NEG);
      gr_pair<CJ>(ax[r / 2 + 1], ay[r / 2 + 1], make_float2(ex.z, ex.w), make_float2(ey.z, ey.w), XX, YY, NEG);
    }
    if constexpr ((NR & 3) >= 2) {
      constexpr int r = NR & ~3;
      gr_pair<CJ>(ax[r / 2], ay[r / 2], *(const float2*)(t + r), *(const float2*)(t + tq + r), XX, YY, NEG);
    }
    if constexpr (NR & 1) gr_one<CJ>(ax[NR / 2].x, ay[NR / 2].x, t[NR - 1], t[tq + NR - 1], xv);
    x += xs;
    t += 2 * tq;
  }
}
// the same for a term read in place (global memory, the factor's layout)
template <int NR, bool CJ>
__device__ __forceinline__ void gr_tile_gp(const float2* __restrict__ x, int xs, const float2* __restrict__ mat,
                                           int ldm, int K, int r0, float2* ax, float2* ay) {
#pragma unroll 2
  for (int kk = 0; kk < K; ++kk) {
    const float2 xv = x[kk * xs];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const float2 e = CJ ? mat[(int64_t)(r0 + r) * ldm + kk] : mat[(int64_t)kk * ldm + r0 + r];
      if (r & 1) gr_one<CJ>(ax[r / 2].y, ay[r / 2].y, e.x, e.y, xv);
      else gr_one<CJ>(ax[r / 2].x, ay[r / 2].x, e.x, e.y, xv);
    }
  }
}
// one complex64 term for nr (<= GR_RB) rows into the paired accumulators
__device__ __forceinline__ void gr_term_p(const GroupedTerm& Q, const float2* __restrict__ fsm,
                                          const float2* __restrict__ x, int xs, int r0, int nr, float2* ax,
                                          float2* ay) {
  const bool cj = Q.conjT != 0;
  if (Q.fac_off >= 0) {
    const float* t = (const float*)fsm + 2 * (int64_t)Q.fac_off + r0;
    switch (nr) {
#define GR_CASE(n)                                                      \
  case n:                                                               \
    if (cj) gr_tile_p<n, true>(x, xs, t, Q.tld, Q.K, ax, ay);           \
    else gr_tile_p<n, false>(x, xs, t, Q.tld, Q.K, ax, ay);             \
    break;
      GR_CASE(1) GR_CASE(2) GR_CASE(3) GR_CASE(4) GR_CASE(5) GR_CASE(6) GR_CASE(7) GR_CASE(8)
      GR_CASE(9) GR_CASE(10) GR_CASE(11) GR_CASE(12) GR_CASE(13) GR_CASE(14) GR_CASE(15) GR_CASE(16)
#undef GR_CASE
      default: break;
    }
  } else {
    const float2* mat = (const float2*)Q.mat;
    switch (nr) {
#define GR_CASE(n)                                                      \
  case n:                                                               \
    if (cj) gr_tile_gp<n, true>(x, xs, mat, Q.ldm, Q.K, r0, ax, ay);    \
    else gr_tile_gp<n, false>(x, xs, mat, Q.ldm, Q.K, r0, ax, ay);      \
    break;
      GR_CASE(1) GR_CASE(2) GR_CASE(3) GR_CASE(4) GR_CASE(5) GR_CASE(6) GR_CASE(7) GR_CASE(8)
      GR_CASE(9) GR_CASE(10) GR_CASE(11) GR_CASE(12) GR_CASE(13) GR_CASE(14) GR_CASE(15) GR_CASE(16)
#undef GR_CASE
      default: break;
    }
  }
}

// one term for nr (<= MR) rows, nr known at run time and uniform over the
// warp: one fully unrolled body per count, no work on absent rows
template <typename V, int MR>
__device__ __forceinline__ void gr_term(const GroupedTerm& Q, const V* __restrict__ fsm, const V* __restrict__ x,
                                        int xs, int r0, int nr, V* acc) {
  const bool cj = Q.conjT != 0;
  if (Q.fac_off >= 0) {
    const V* t = fsm + Q.fac_off + r0;
    switch (nr) {
#define GR_CASE(n)                                                                           \
  case n:                                                                                    \
    if constexpr (n <= MR) {                                                                 \
      if (cj) gr_tile_s<V, n, true>(x, xs, t, Q.tld, Q.K, acc);                             \
      else gr_tile_s<V, n, false>(x, xs, t, Q.tld, Q.K, acc);                               \
    }                                                                                        \
    break;
      GR_CASE(1) GR_CASE(2) GR_CASE(3) GR_CASE(4) GR_CASE(5) GR_CASE(6) GR_CASE(7) GR_CASE(8)
      GR_CASE(9) GR_CASE(10) GR_CASE(11) GR_CASE(12) GR_CASE(13) GR_CASE(14) GR_CASE(15) GR_CASE(16)
#undef GR_CASE
      default: break;
    }
  } else {
    const V* mat = (const V*)Q.mat;
    switch (nr) {
#define GR_CASE(n)                                                                           \
  case n:                                                                                    \
    if constexpr (n <= MR) {                                                                 \
      if (cj) gr_tile_g<V, n, true>(x, xs, mat, Q.ldm, Q.K, r0, acc);                       \
      else gr_tile_g<V, n, false>(x, xs, mat, Q.ldm, Q.K, r0, acc);                         \
    }                                                                                        \
    break;
      GR_CASE(1) GR_CASE(2) GR_CASE(3) GR_CASE(4) GR_CASE(5) GR_CASE(6) GR_CASE(7) GR_CASE(8)
      GR_CASE(9) GR_CASE(10) GR_CASE(11) GR_CASE(12) GR_CASE(13) GR_CASE(14) GR_CASE(15) GR_CASE(16)
#undef GR_CASE
      default: break;
    }
  }
}
// ---- persistent launch: per-task flags and bounded waits ----
__device__ __forceinline__ unsigned long long gr_now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int gr_ld_acquire(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void gr_st_release(int32_t* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// true once *flag is set; false when the time limit passed or another CTA
// has already given up (the status flag), so one failure ends every wait
__device__ bool gr_wait_flag(const int32_t* flag, const int* status, unsigned long long limit_ns) {
  if (gr_ld_acquire(flag)) return true;
  const unsigned long long t0 = gr_now_ns();
  for (unsigned it = 0;; ++it) {
    if (gr_ld_acquire(flag)) return true;
    if ((it & 15) == 15) {
      if (gr_ld_acquire(status)) return false;
      if (gr_now_ns() - t0 > limit_ns) return false;
    }
    __nanosleep(32);
  }
}

// What a persistent task waits for: the tasks of the same column slice of
// the groups it reads (dep_ptr / dep_idx index groups)
struct GroupedWait {
  const int32_t* dep_ptr;
  const int32_t* dep_idx;
  int32_t* flags;       // one per (group, slice) task, zero at launch
  int* status;          // device status flag: set when a wait gave up
  unsigned long long limit_ns;
  int slices;
};
}  // namespace

// One group of a run for one column slice.  PERSIST: inside the persistent
// launch (task = the group's (group, slice) index): wait for the producer
// tasks' flags where the plain launch waits for the previous grid, read the
// producers' rows around L1 (another SM wrote them in this launch), release
// this task's flag at the end; returns false when a wait gave up.
template <typename R, int NT, bool PERSIST>
__device__ __forceinline__ bool grouped_group(const GroupedArgs& a, int gi, int sl, const GroupedWait* w, int task) {
  using V = typename Cx<R>::V;
  extern __shared__ __align__(16) uint8_t gr_smem[];
  const int tid = threadIdx.x;
  // the group's image (head, task descriptors, spans, row chunks, factor
  // tiles) in one coalesced pass of 16-byte copies; it does not depend on
  // the previous launch, so it is in flight while this CTA waits for it
  {
    const uint8_t* img = a.img + (int64_t)(gi - a.group0) * a.stride;
    const int n16 = (int)(a.stride >> 4);
    for (int v = tid; v < n16; v += NT) gr_cp_async<16>(gr_smem + 16 * v, img + 16 * v);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  const int CW = a.CW, N = a.N;
  const int c0 = sl * CW;
  const int cw = min(CW, N - c0);
  if constexpr (PERSIST) {
    __shared__ int s_abort;
    if (tid == 0) {
      bool ok = true;
      const int g = gi;
      for (int q = w->dep_ptr[g]; q < w->dep_ptr[g + 1] && ok; ++q)
        ok = gr_wait_flag(w->flags + (int64_t)w->dep_idx[q] * w->slices + sl, w->status, w->limit_ns);
      if (!ok) atomicExch(w->status, 1);
      s_abort = ok ? 0 : 1;
    }
    __syncthreads();
    if (s_abort) {
      asm volatile("cp.async.wait_all;" ::: "memory");
      return false;
    }
  } else {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  const GroupedGroup& G = *(const GroupedGroup*)gr_smem;
  const GroupedTask* __restrict__ stask = (const GroupedTask*)(gr_smem + G.off_tasks);
  const GroupedSpan* __restrict__ sspan = (const GroupedSpan*)(gr_smem + G.off_spans);
  const int32_t* __restrict__ schunk = (const int32_t*)(gr_smem + G.off_chunks);   // (first row << 16) | task
  const V* __restrict__ fsm = (const V*)(gr_smem + G.off_fac);                      // staged factor tiles
  V* __restrict__ rsm = (V*)(gr_smem + a.stride);                                   // rows, CW columns each
  // the group's input rows (region 0); inside the persistent launch rows
  // another SM wrote are read around L1
  const V* __restrict__ x = (const V*)a.x;
  auto in_copy = [&](V* dst, const V* src) {
    if constexpr (PERSIST && sizeof(V) == 8) *dst = __ldcg(src);
    else if constexpr (PERSIST) gr_cp_async<16>(dst, src);
    else gr_cp_async<sizeof(V)>(dst, src);
  };
  // row-major inputs: a row's cw columns to a group of lanes (16-byte
  // units where rows and slice allow), the span rows round robin over the
  // CTA's row slots in local-row order; column-major x: column by column
  // column-major x and y staged column by column from 32 columns per slice
  // on (with fewer, a lane's column is read and written in place)
  const bool cmi = G.in_pitch > 0 && cw >= 32, cmo = G.out_pitch > 0 && cw >= 32;
  constexpr int VPU = 16 / (int)sizeof(V);
  const bool vec = a.in_ld == 0 && N % VPU == 0 && CW % VPU == 0 && cw % VPU == 0;   // 16-byte copies (cg)
  const int upr = vec ? cw / VPU : cw;
  int lg = 0;
  while ((1 << lg) < upr && lg < 5) ++lg;
  const int rslots = (NT / 32) << (5 - lg);
  const int rslot = ((tid >> 5) << (5 - lg)) + ((tid & 31) >> lg), u0 = tid & ((1 << lg) - 1);
  for (int sp = 0; sp < G.nspans; ++sp) {
    const GroupedSpan S = sspan[sp];
    if (a.in_ld == 0) {
      for (int i = (rslot - S.l0) & (rslots - 1); i < S.rows; i += rslots) {
        V* d = rsm + (int64_t)(S.l0 + i) * CW;
        const V* s = x + (S.g0 + i) * N + c0;
        for (int u = u0; u < upr; u += 1 << lg) {
          if (vec) gr_cp_async<16>(d + u * VPU, s + u * VPU);
          else in_copy(d + u, s + u);
        }
      }
    } else if (cmi) {   // column-major x, held column by column: lanes along a column's rows
      const int P0 = G.in_pitch;
      for (int c = tid >> 5; c < cw; c += NT / 32) {
        const V* s = x + S.g0 + (int64_t)(c0 + c) * a.in_ld;
        V* d = rsm + (int64_t)c * P0 + S.l0;
        for (int i = tid & 31; i < S.rows; i += 32) in_copy(d + i, s + i);
      }
    } else {   // column-major x into rows (few columns): consecutive threads along a column's rows
      for (int e = tid; e < S.rows * cw; e += NT) {
        const int c = e / S.rows, i = e - c * S.rows;
        in_copy(rsm + (int64_t)(S.l0 + i) * CW + c, x + (S.g0 + i) + (int64_t)(c0 + c) * a.in_ld);
      }
    }
  }
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  V* __restrict__ y = (V*)a.y;
  const int lane = tid & 31, warp = tid >> 5;
  // complex128: chunks in tiles of 8 rows (registers)
  constexpr int MR = sizeof(V) == 16 ? 8 : GR_RB;
  for (int k = 0; k < G.nst; ++k) {
    const int ch0 = G.st_chunk[k], nch = G.st_chunk[k + 1] - ch0;
    // one warp per (row chunk, 32-column slice), lane = column; with few
    // columns one lane per (row, column) instead
    const bool wide = cw >= 16;
    const int ncs = (cw + 31) >> 5;
    const int items = wide ? nch * ncs : nch * GR_RB * cw;
    for (int it = wide ? warp : tid; it < items; it += wide ? NT / 32 : NT) {
      int ch, c, rsub = 0, rcount;
      if (wide) {
        ch = it / ncs;
        c = (it - ch * ncs) * 32 + lane;
      } else {
        c = it % cw;
        const int rr = it / cw;
        ch = rr / GR_RB;
        rsub = rr - ch * GR_RB;
      }
      const int32_t cp = schunk[ch0 + ch];
      const GroupedTask& T = stask[cp & 0xffff];
      const int rbase = (cp >> 16) + rsub;
      rcount = wide ? min(GR_RB, T.M - (cp >> 16)) : (rbase < T.M ? 1 : 0);
      if (c >= cw || rcount <= 0) continue;
      for (int h = 0; h < rcount; h += MR) {
        const int r0 = rbase + h, nr = min(MR, rcount - h);
        if constexpr (sizeof(V) == 8) {   // complex64: planar tiles, paired rows
          float2 ax[GR_RB / 2], ay[GR_RB / 2];
#pragma unroll
          for (int p = 0; p < GR_RB / 2; ++p) ax[p] = ay[p] = make_float2(0.f, 0.f);
          for (int q = 0; q < T.nterms; ++q) {
            const GroupedTerm& Q = T.t[q];
            const bool cm = Q.in_reg == 0 && cmi;
            const V* xin = cm ? rsm + (int64_t)c * G.in_pitch + Q.in_row
                              : rsm + (int64_t)(G.reg_row[Q.in_reg] + Q.in_row) * CW + c;
            gr_term_p(Q, fsm, xin, cm ? 1 : CW, r0, nr, ax, ay);
          }
          V* o;
          int64_t rs;
          if (T.out_reg > 0) {
            o = rsm + (int64_t)(G.reg_row[T.out_reg] + T.out_row + r0) * CW + c;
            rs = CW;
          } else if (cmo) {   // staged column by column
            o = rsm + (int64_t)G.out_row0 * CW + (int64_t)c * G.out_pitch + T.out_loc + r0;
            rs = 1;
          } else {
            rs = T.ldo > 0 ? 1 : N;
            const int64_t cs = T.ldo > 0 ? T.ldo : 1;
            o = y + (T.ldo > 0 ? T.out_row : T.out_row * N) + (int64_t)r0 * rs + (int64_t)(c0 + c) * cs;
          }
#pragma unroll
          for (int r = 0; r < GR_RB; ++r)
            if (r < nr)
              o[r * rs] = (r & 1) ? make_float2(ax[r / 2].y, ay[r / 2].y) : make_float2(ax[r / 2].x, ay[r / 2].x);
        } else {   // complex128: interleaved tiles, a register tile of MR rows
          V acc[MR];
#pragma unroll
          for (int r = 0; r < MR; ++r) acc[r] = Cx<R>::make(0, 0);
          for (int q = 0; q < T.nterms; ++q) {
            const GroupedTerm& Q = T.t[q];
            const bool cm = Q.in_reg == 0 && cmi;
            const V* xin = cm ? rsm + (int64_t)c * G.in_pitch + Q.in_row
                              : rsm + (int64_t)(G.reg_row[Q.in_reg] + Q.in_row) * CW + c;
            gr_term<V, MR>(Q, fsm, xin, cm ? 1 : CW, r0, nr, acc);
          }
          if (T.out_reg > 0) {
            V* o = rsm + (int64_t)(G.reg_row[T.out_reg] + T.out_row + r0) * CW + c;
#pragma unroll
            for (int r = 0; r < MR; ++r)
              if (r < nr) o[r * CW] = acc[r];
          } else if (cmo) {   // staged column by column
            V* o = rsm + (int64_t)G.out_row0 * CW + (int64_t)c * G.out_pitch + T.out_loc + r0;
#pragma unroll
            for (int r = 0; r < MR; ++r)
              if (r < nr) o[r] = acc[r];
          } else {
            const int64_t rs = T.ldo > 0 ? 1 : N, cs = T.ldo > 0 ? T.ldo : 1;
            V* o = y + (T.ldo > 0 ? T.out_row : T.out_row * N) + (int64_t)r0 * rs + (int64_t)(c0 + c) * cs;
#pragma unroll
            for (int r = 0; r < MR; ++r)
              if (r < nr) o[r * rs] = acc[r];
          }
        }
      }
    }
    __syncthreads();   // this stage's blocks are complete
  }
  if (cmo && G.nospans > 0) {   // staged column-major outputs: lanes along a column's rows
    const GroupedSpan* __restrict__ osp = (const GroupedSpan*)(gr_smem + G.off_ospans);
    const int64_t ldo = G.out_ld;
    const V* __restrict__ so = rsm + (int64_t)G.out_row0 * CW;
    for (int sp = 0; sp < G.nospans; ++sp) {
      const GroupedSpan S = osp[sp];
      for (int c = tid >> 5; c < cw; c += NT / 32) {
        V* d = y + S.g0 + (int64_t)(c0 + c) * ldo;
        const V* s = so + (int64_t)c * G.out_pitch + S.l0;
        for (int i = tid & 31; i < S.rows; i += 32) d[i] = s[i];
      }
    }
  }
  if constexpr (PERSIST) {
    if (tid == 0) {
      __threadfence();
      gr_st_release(w->flags + task, 1);
    }
  }
  return true;
}

// complex64 within 128 registers (no spills), 256 threads for slices of 64
// columns and 128 for narrower ones; complex128 (FP64-bound) 256 threads at
// the compiler's register choice.
__global__ void __launch_bounds__(256, 2) grouped_kernel_c64_256(const GroupedArgs a) {
  grouped_group<float, 256, false>(a, a.group0 + blockIdx.x, blockIdx.y, nullptr, 0);
}
__global__ void __launch_bounds__(128, 4) grouped_kernel_c64_128(const GroupedArgs a) {
  grouped_group<float, 128, false>(a, a.group0 + blockIdx.x, blockIdx.y, nullptr, 0);
}
__global__ void __launch_bounds__(256) grouped_kernel_c128_256(const GroupedArgs a) {
  grouped_group<double, 256, false>(a, a.group0 + blockIdx.x, blockIdx.y, nullptr, 0);
}

// Persistent launch: every run's groups, task t = (group t / slices, slice
// t % slices) in run order, CTA c taking tasks c, c + G, ... (all CTAs
// resident: a cooperative launch, so the lowest unfinished task never
// waits).  run_group0[r] is the first group of run r (nruns + 1 entries),
// args[r] that run's arguments (one shared-memory layout for all runs).
struct GroupedPersistArgs {
  const GroupedArgs* args;
  const int32_t* run_group0;
  int nruns, ntasks;
  GroupedWait w;
};
template <typename R, int NT>
__device__ __forceinline__ void grouped_persist_body(const GroupedPersistArgs& p) {
  for (int t = blockIdx.x; t < p.ntasks; t += gridDim.x) {
    const int g = t / p.w.slices, sl = t - g * p.w.slices;
    int r = 0;
    while (r + 1 < p.nruns && g >= p.run_group0[r + 1]) ++r;
    __syncthreads();   // the previous task's shared memory is free
    if (!grouped_group<R, NT, true>(p.args[r], g, sl, &p.w, t)) return;
  }
}
__global__ void __launch_bounds__(256, 2) grouped_persist_c64_256(const GroupedPersistArgs p) {
  grouped_persist_body<float, 256>(p);
}
__global__ void __launch_bounds__(128, 4) grouped_persist_c64_128(const GroupedPersistArgs p) {
  grouped_persist_body<float, 128>(p);
}
__global__ void __launch_bounds__(256) grouped_persist_c128_256(const GroupedPersistArgs p) {
  grouped_persist_body<double, 256>(p);
}

// Packs each term's factor entries into its group's image (once per plan):
// complex128 entry (i, k) of a tile at dst + (k tld + i) elements;
// complex64 planar, its real part at float k 2 tld + i and its imaginary
// part tld floats later.
__global__ void grouped_pack_kernel(const GroupedSeg* __restrict__ segs, int nseg, uint8_t* __restrict__ img,
                                    int es) {
  for (int q = blockIdx.x; q < nseg; q += gridDim.x) {
    const GroupedSeg sg = segs[q];
    const int n = sg.M * sg.K;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      int i, k;
      int64_t so;
      if (sg.conj) {
        i = e / sg.K;
        k = e - i * sg.K;
        so = (int64_t)i * sg.ldm + k;
      } else {
        k = e / sg.M;
        i = e - k * sg.M;
        so = i + (int64_t)k * sg.ldm;
      }
      if (es == 16) {
        *(double2*)(img + sg.dst + ((int64_t)k * sg.tld + i) * 16) = ((const double2*)sg.src)[so];
      } else {   // planar: real parts, then imaginary parts, per column
        const float2 v = ((const float2*)sg.src)[so];
        float* d = (float*)(img + sg.dst) + (int64_t)k * 2 * sg.tld + i;
        d[0] = v.x;
        d[sg.tld] = v.y;
      }
    }
  }
}

// ------------------------------------------------------------------ host --
namespace {

size_t grouped_smem(const GroupedRun& run, int CW, size_t es) {
  return gr_smem_bytes(run.img_stride, run.rows_max, CW, es);
}

struct DSU {
  std::vector<int> p;
  explicit DSU(int n) : p(n) { std::iota(p.begin(), p.end(), 0); }
  int find(int x) {
    while (p[x] != x) x = p[x] = p[p[x]];
    return x;
  }
  void join(int a, int b) {
    a = find(a), b = find(b);
    if (a != b) p[std::max(a, b)] = std::min(a, b);
  }
};

// sorted, disjoint row ranges [a, b) -> consecutive local rows
struct RowMap {
  std::vector<std::pair<int64_t, int64_t>> r;   // (first, end)
  std::vector<int32_t> l0;
  void build(std::vector<std::pair<int64_t, int64_t>> v) {
    std::sort(v.begin(), v.end());
    r.clear();
    for (auto& x : v) {
      if (!r.empty() && x.first <= r.back().second) r.back().second = std::max(r.back().second, x.second);
      else r.push_back(x);
    }
    l0.assign(r.size(), 0);
    for (size_t i = 1; i < r.size(); ++i) l0[i] = l0[i - 1] + (int32_t)(r[i - 1].second - r[i - 1].first);
  }
  int64_t rows() const { return r.empty() ? 0 : l0.back() + (r.back().second - r.back().first); }
  // local row of global row g, -1 when outside
  int64_t at(int64_t g) const {
    auto it = std::upper_bound(r.begin(), r.end(), std::make_pair(g, INT64_MAX));
    if (it == r.begin()) return -1;
    --it;
    if (g >= it->second) return -1;
    return l0[it - r.begin()] + (g - it->first);
  }
};

struct RunTables {
  std::vector<GroupedGroup> groups;
  std::vector<GroupedTask> tasks;
  std::vector<GroupedSpan> spans;
  std::vector<GroupedSeg> segs;
  std::vector<int32_t> chunks;
  std::vector<GroupedSpan> ospans;   // column-major output: staging rows -> global rows
};

// Builds the groups of stages [s0, s0 + d) into T (cleared first; every
// index is absolute: `base` holds the sizes of the tables already built);
// false when a group does not fit (the caller retries with a shorter run).
// cm_in: the run reads x column-major (region 0 is then held column by
// column); a last stage writing y column-major stages its outputs the same
// way.
bool build_run(int dtype, const std::vector<StageTask>& all, const ApplyPlan& tmp, int s0, int d, int merge_min,
               bool cm_in, const RunTables& base, GroupedRun& run, RunTables& T) {
  T.ospans.clear();
  T.groups.clear();
  T.tasks.clear();
  T.spans.clear();
  T.segs.clear();
  T.chunks.clear();
  const size_t es = elem_bytes(dtype);
  // tasks of the run, local numbering (stage by stage)
  int first[GR_MAXD + 1];
  first[0] = 0;
  for (int k = 0; k < d; ++k) first[k + 1] = first[k] + tmp.count[s0 + k];
  const int nt = first[d];
  auto task = [&](int i) -> const StageTask& {
    int k = 0;
    while (i >= first[k + 1]) ++k;
    return all[tmp.first[s0 + k] + (i - first[k])];
  };
  DSU dsu(nt);
  // producers inside the run: stage k's terms read stage k - 1's outputs
  std::vector<std::pair<int64_t, int>> outs;   // (out_off, local index) of stage k - 1
  for (int k = 1; k < d; ++k) {
    outs.clear();
    for (int i = first[k - 1]; i < first[k]; ++i) outs.push_back({task(i).out_off, i});
    std::sort(outs.begin(), outs.end());
    for (int i = first[k]; i < first[k + 1]; ++i) {
      const StageTask& tk = task(i);
      for (int q = 0; q < tk.nterms; ++q) {
        const int64_t lo = tk.t[q].in_off, hi = lo + tk.t[q].K;
        auto it = std::upper_bound(outs.begin(), outs.end(), std::make_pair(lo, INT32_MAX));
        if (it != outs.begin()) --it;
        for (; it != outs.end() && it->first < hi; ++it)
          if (it->first + task(it->second).M > lo) dsu.join(i, it->second);
      }
    }
  }
  // components in order of their smallest task (the root), members
  // ascending (so stage by stage): a counting sort by component
  std::vector<int> gid(nt), cnt, mem(nt);
  int ng = 0;
  for (int i = 0; i < nt; ++i) {
    const int r = dsu.find(i);
    gid[i] = r == i ? ng++ : gid[r];
  }
  // consecutive components merged until each group holds merge_min blocks
  // of the run's last stage (independent components share a CTA: fewer,
  // fuller CTAs where the components are single blocks or pairs)
  if (merge_min > 1 && ng > 1) {
    std::vector<int> last(ng, 0), nid(ng);
    for (int i = first[d - 1]; i < nt; ++i) ++last[gid[i]];
    int m = 0, acc = 0;
    for (int g = 0; g < ng; ++g) {
      nid[g] = m;
      acc += last[g];
      if (acc >= merge_min) {
        ++m;
        acc = 0;
      }
    }
    ng = m + (acc > 0 ? 1 : 0);
    for (int i = 0; i < nt; ++i) gid[i] = nid[gid[i]];
  }
  cnt.assign(ng + 1, 0);
  for (int i = 0; i < nt; ++i) ++cnt[gid[i] + 1];
  for (int g = 0; g < ng; ++g) cnt[g + 1] += cnt[g];
  {
    std::vector<int> pos(cnt.begin(), cnt.end() - 1);
    for (int i = 0; i < nt; ++i) mem[pos[gid[i]]++] = i;
  }
  run.group0 = (int32_t)(base.groups.size());
  run.ngroups = ng;
  run.img_stride = 0;
  run.desc_max = 0;
  run.rows_max = 0;
  RowMap reg[GR_MAXD];
  std::vector<std::pair<int64_t, int64_t>> v;
  for (int g = 0; g < ng; ++g) {
    const int m0 = cnt[g], m1 = cnt[g + 1];
    // members of stage k: [sb[k], sb[k + 1]) within mem
    int sb[GR_MAXD + 1];
    for (int k = 0, m = m0; k < d; ++k) {
      sb[k] = m;
      while (m < m1 && mem[m] < first[k + 1]) ++m;
    }
    sb[d] = m1;
    GroupedGroup G{};
    G.task0 = (int32_t)(base.tasks.size() + T.tasks.size());
    G.span0 = (int32_t)(base.spans.size() + T.spans.size());
    G.seg0 = (int32_t)(base.segs.size() + T.segs.size());
    G.chunk0 = (int32_t)(base.chunks.size() + T.chunks.size());
    G.nst = d;
    // regions: 0 = the stage-0 inputs, k = the outputs of stage k - 1
    v.clear();
    for (int m = sb[0]; m < sb[1]; ++m) {
      const StageTask& tk = task(mem[m]);
      for (int q = 0; q < tk.nterms; ++q) v.push_back({tk.t[q].in_off, tk.t[q].in_off + tk.t[q].K});
    }
    reg[0].build(v);
    for (int k = 1; k < d; ++k) {
      v.clear();
      for (int m = sb[k - 1]; m < sb[k]; ++m) {
        const StageTask& tk = task(mem[m]);
        v.push_back({tk.out_off, tk.out_off + tk.M});
      }
      reg[k].build(v);
    }
    // region 0 of a column-major input: one column after another with an
    // odd pitch (lanes = columns read it without bank conflicts)
    G.reg_row[0] = 0;
    for (int k = 0; k < d; ++k)
      G.reg_row[k + 1] = G.reg_row[k] + (int32_t)reg[k].rows() + (k == 0 && cm_in && !(reg[0].rows() & 1) ? 1 : 0);
    for (int k = d + 1; k <= GR_MAXD; ++k) G.reg_row[k] = G.reg_row[d];
    G.in_pitch = cm_in ? G.reg_row[1] : 0;
    // column-major output: the last stage's blocks staged column by column
    // (odd pitch), written out along columns
    RowMap ro;
    bool cm_out = false;
    v.clear();
    for (int m = sb[d - 1]; m < sb[d]; ++m) {
      const StageTask& tk = task(mem[m]);
      cm_out = cm_out || tk.ldo > 0;
      v.push_back({tk.out_off, tk.out_off + tk.M});
    }
    G.ospan0 = (int32_t)(base.ospans.size() + T.ospans.size());
    if (cm_out) {
      const int64_t ldo = task(mem[sb[d - 1]]).ldo;
      for (int m = sb[d - 1]; m < sb[d]; ++m)
        if (task(mem[m]).ldo != ldo) return false;
      if (ldo > INT32_MAX) return false;
      G.out_ld = (int32_t)ldo;
      ro.build(v);
      G.out_row0 = G.reg_row[d];
      G.out_pitch = (int32_t)(ro.rows() | 1);
      for (size_t sp = 0; sp < ro.r.size(); ++sp)
        T.ospans.push_back({ro.r[sp].first, ro.l0[sp], (int32_t)(ro.r[sp].second - ro.r[sp].first)});
      G.nospans = (int32_t)ro.r.size();
    }
    for (size_t sp = 0; sp < reg[0].r.size(); ++sp)
      T.spans.push_back({reg[0].r[sp].first, reg[0].l0[sp], (int32_t)(reg[0].r[sp].second - reg[0].r[sp].first)});
    G.nspans = (int32_t)reg[0].r.size();
    // each term's entries as a tile of the group's staged factors (entry
    // (i, k) at dst + k tld + i, tld = M rounded up to even; every tile
    // starts at an even element, so complex64 row pairs are 16-byte aligned)
    const size_t t0 = T.tasks.size(), seg0 = T.segs.size(), ch0 = T.chunks.size();
    int64_t fac = 0;
    G.st_chunk[0] = 0;
    for (int k = 0; k < d; ++k) {
      for (int m = sb[k]; m < sb[k + 1]; ++m) {
        const StageTask& tk = task(mem[m]);
        GroupedTask gt{};
        gt.M = tk.M;
        gt.nterms = tk.nterms;
        if (k < d - 1) {
          gt.out_reg = (int16_t)(k + 1);
          gt.out_row = reg[k + 1].at(tk.out_off);
          if (gt.out_row < 0) return false;
          gt.ldo = 0;
        } else {
          gt.out_reg = 0;
          gt.out_row = tk.out_off;
          gt.ldo = tk.ldo;
          gt.out_loc = cm_out && tk.M > 0 ? (int32_t)ro.at(tk.out_off) : 0;
          if (gt.out_loc < 0) return false;
        }
        // tile pitch: complex64 tiles are planar with M rounded up to 4
        // (16-byte row quads), complex128 tiles interleaved with M rounded
        // up to even
        const int tld = es == 8 ? (tk.M + 3) & ~3 : tk.M + (tk.M & 1);
        for (int q = 0; q < tk.nterms; ++q) {
          const StageTerm& S = tk.t[q];
          GroupedTerm& Q = gt.t[q];
          Q.mat = S.mat;
          Q.K = S.K;
          Q.ldm = S.ldm;
          Q.tld = tld;
          Q.conjT = S.conjT;
          Q.in_reg = (int16_t)k;
          const int64_t lr = reg[k].at(S.in_off);
          if (S.K > 0 && (lr < 0 || reg[k].at(S.in_off + S.K - 1) != lr + S.K - 1)) return false;
          Q.in_row = (int32_t)std::max<int64_t>(lr, 0);
          Q.fac_off = (int32_t)fac;
          // (dst: the element offset in the group's tiles until the images are placed)
          if (tk.M > 0 && S.K > 0) T.segs.push_back({S.mat, fac, tk.M, S.K, S.ldm, tld, S.conjT, 0});
          fac += (int64_t)S.K * tld;
        }
        const size_t li = T.tasks.size() - t0;
        if (li >= 0x10000 || tk.M >= 0x8000) return false;
        for (int r0 = 0; r0 < tk.M; r0 += GR_RB) T.chunks.push_back((r0 << 16) | (int32_t)li);
        T.tasks.push_back(gt);
      }
      G.st_chunk[k + 1] = (int32_t)(T.chunks.size() - ch0);
    }
    for (int k = d + 1; k <= GR_MAXD; ++k) G.st_chunk[k] = G.st_chunk[d];
    G.ntasks = (int32_t)(T.tasks.size() - t0);
    if ((size_t)fac * es > GR_FAC_LIMIT) {   // read the factors in place
      for (size_t t = t0; t < T.tasks.size(); ++t)
        for (int q = 0; q < T.tasks[t].nterms; ++q) T.tasks[t].t[q].fac_off = -1;
      T.segs.resize(seg0);
      fac = 0;
    }
    G.fac_elems = (int32_t)fac;
    G.nseg = (int32_t)(T.segs.size() - seg0);
    // the image: head, tasks, spans, chunks, tiles (16-byte aligned parts)
    const size_t o_tasks = gr_align16(sizeof(GroupedGroup));
    const size_t o_spans = o_tasks + gr_align16((size_t)G.ntasks * sizeof(GroupedTask));
    const size_t o_ospans = o_spans + gr_align16((size_t)G.nspans * sizeof(GroupedSpan));
    const size_t o_chunks = o_ospans + gr_align16((size_t)G.nospans * sizeof(GroupedSpan));
    const size_t o_fac = o_chunks + gr_align16((size_t)G.st_chunk[d] * 4);
    const size_t bytes = gr_align16(o_fac + (size_t)fac * es);
    if (bytes > GR_SMEM_LIMIT) return false;
    G.off_tasks = (int32_t)o_tasks;
    G.off_spans = (int32_t)o_spans;
    G.off_ospans = (int32_t)o_ospans;
    G.off_chunks = (int32_t)o_chunks;
    G.off_fac = (int32_t)o_fac;
    T.groups.push_back(G);
    run.img_stride = std::max<int64_t>(run.img_stride, (int64_t)bytes);
    run.desc_max = std::max(run.desc_max, (int32_t)o_fac);
    run.rows_max = std::max(run.rows_max, G.reg_row[d] + G.out_pitch);
  }
  // the smallest slice width (8 columns) must fit
  return grouped_smem(run, 8, es) <= GR_SMEM_LIMIT;
}

}  // namespace

static std::atomic<int> g_grouped_depth{0};
int set_grouped_depth(int depth) {
  if (depth < 0 || depth > GR_MAXD) return fail(BF_EINVAL, "grouped depth must be 0 .. 4");
  g_grouped_depth.store(depth);
  return BF_OK;
}
int grouped_depth() { return g_grouped_depth.load(); }

static std::atomic<int> g_grouped_merge{0};
int set_grouped_merge(int merge) {
  if (merge < 0 || merge > 16) return fail(BF_EINVAL, "grouped merge must be 0 .. 16");
  g_grouped_merge.store(merge);
  return BF_OK;
}
int grouped_merge() { return g_grouped_merge.load(); }

int build_grouped(Fact* F, int opC, int dtype, int depth, cudaStream_t s, int merge) {
  GroupedPlan& gp = F->gp[opC][dtype];
  if (merge <= 0) merge = grouped_merge();
  if (merge <= 0 && gp.tuned_merge > 0) merge = gp.tuned_merge;
  if (merge <= 0) {
    // untuned: complex64 groups of small blocks (ranks <= 16) merged; large
    // blocks fill a CTA alone (merged, their tiles outgrow shared memory
    // and are read in place: 3-D caps with ranks ~53 at 64 columns took
    // 0.83 ms merged against 0.20 ms unmerged)
    int rmax = 0;
    for (const auto& v : F->rV)
      for (int r : v) rmax = std::max(rmax, r);
    for (const auto& v : F->rU)
      for (int r : v) rmax = std::max(rmax, r);
    merge = dtype == BF_C64 && rmax <= 16 ? GR_MERGE_MIN : 1;
  }
  if (gp.built && gp.depth == depth && gp.merge == merge) return BF_OK;
  if (depth < 1 || depth > GR_MAXD) return fail(BF_EINVAL, "grouped apply depth must be 1 .. 4");
  const auto pick = gp.pick, ppick = gp.ppick, tuned = gp.tuned;
  const auto cws = gp.cw;
  const int tuned_depth = gp.tuned_depth, tuned_merge = gp.tuned_merge;
  const int64_t uses = gp.untuned_uses;
  gp.dev.release(s);
  gp = GroupedPlan();
  gp.built = true;
  gp.depth = depth;
  gp.pick = pick;
  gp.ppick = ppick;
  gp.tuned = tuned;
  gp.cw = cws;
  gp.tuned_depth = tuned_depth;
  gp.tuned_merge = tuned_merge;
  gp.merge = merge;
  gp.untuned_uses = uses;
  ApplyPlan tmp;
  std::vector<StageTask> all;
  apply_tasks_host(F, opC, dtype, tmp, all);
  if (debug_checks()) BF_TRY(check_apply_tasks(F, opC, dtype, tmp, all));
  const int nst = (int)tmp.first.size();
  // the chain the runs rely on: stage 0 reads x (base 0), stage i > 0 reads
  // only stage i - 1's output buffer (row-major), the last stage writes y
  int prev_out = 0;
  int64_t in_ld0 = -1;
  for (int i = 0; i < nst; ++i) {
    int out = -1;
    for (int t = tmp.first[i]; t < tmp.first[i] + tmp.count[i]; ++t) {
      const StageTask& tk = all[t];
      if (out >= 0 && tk.out_base != out) return BF_OK;
      out = tk.out_base;
      if (tk.nterms > 2) return BF_OK;
      for (int q = 0; q < tk.nterms; ++q) {
        if (tk.t[q].in_base != prev_out) return BF_OK;
        if (i == 0) {
          if (in_ld0 >= 0 && tk.t[q].ldi != in_ld0) return BF_OK;
          in_ld0 = tk.t[q].ldi;
        } else if (tk.t[q].ldi != 0) {
          return BF_OK;
        }
      }
      if (i < nst - 1 && (tk.ldo != 0 || (tk.out_base != 1 && tk.out_base != 2))) return BF_OK;
      if (i == nst - 1 && tk.out_base != 3) return BF_OK;
    }
    prev_out = out;
  }
  if (in_ld0 < 0) in_ld0 = 0;
  RunTables T, R;
  int64_t lvl_max = 0;
  int buf = 1;
  for (int s0 = 0; s0 < nst;) {
    int d = std::min(depth, nst - s0);
    GroupedRun run{};
    // groups merged up to `merge` last-stage blocks; unmerged when that does
    // not fit, then shorter runs
    for (;; --d) {
      const bool cm_in = s0 == 0 && in_ld0 > 0;
      if (build_run(dtype, all, tmp, s0, d, merge, cm_in, T, run, R) ||
          (merge > 1 && build_run(dtype, all, tmp, s0, d, 1, cm_in, T, run, R))) {
        T.groups.insert(T.groups.end(), R.groups.begin(), R.groups.end());
        T.tasks.insert(T.tasks.end(), R.tasks.begin(), R.tasks.end());
        T.spans.insert(T.spans.end(), R.spans.begin(), R.spans.end());
        T.segs.insert(T.segs.end(), R.segs.begin(), R.segs.end());
        T.chunks.insert(T.chunks.end(), R.chunks.begin(), R.chunks.end());
        T.ospans.insert(T.ospans.end(), R.ospans.begin(), R.ospans.end());
        break;
      }
      if (d == 1) return BF_OK;   // a single stage does not fit: not applicable
    }
    run.in_base = s0 == 0 ? 0 : (buf == 1 ? 2 : 1);
    run.in_ld = s0 == 0 ? in_ld0 : 0;
    const bool last = s0 + d == nst;
    run.out_base = last ? 3 : buf;
    run.out_rows = 0;
    for (int t = tmp.first[s0 + d - 1]; t < tmp.first[s0 + d - 1] + tmp.count[s0 + d - 1]; ++t)
      run.out_rows = std::max(run.out_rows, all[t].out_off + all[t].M);
    if (!last) {
      lvl_max = std::max(lvl_max, run.out_rows);
      buf = 3 - buf;
    }
    gp.runs.push_back(run);
    s0 += d;
  }
  gp.level_rows_max = std::max<int64_t>(lvl_max, 1);
  // persistent launch: a group of run r reads rows written by the last
  // stage of run r - 1; its producers are the groups whose last-stage
  // blocks meet one of its input spans
  std::vector<int32_t> dep_ptr(T.groups.size() + 1, 0), dep_idx;
  {
    std::vector<int32_t> dg;
    for (size_t r = 0; r < gp.runs.size(); ++r) {
      const GroupedRun& run = gp.runs[r];
      std::vector<std::pair<int64_t, std::pair<int64_t, int32_t>>> outs;   // (first row, (end, group))
      if (r > 0) {
        const GroupedRun& pr = gp.runs[r - 1];
        for (int g = pr.group0; g < pr.group0 + pr.ngroups; ++g) {
          const GroupedGroup& G = T.groups[g];
          for (int t = G.task0; t < G.task0 + G.ntasks; ++t)
            if (T.tasks[t].out_reg == 0) outs.push_back({T.tasks[t].out_row, {T.tasks[t].out_row + T.tasks[t].M, g}});
        }
        std::sort(outs.begin(), outs.end());
      }
      for (int g = run.group0; g < run.group0 + run.ngroups; ++g) {
        dg.clear();
        const GroupedGroup& G = T.groups[g];
        for (int sp = G.span0; r > 0 && sp < G.span0 + G.nspans; ++sp) {
          const int64_t lo = T.spans[sp].g0, hi = lo + T.spans[sp].rows;
          // blocks are disjoint and sorted: the first that can meet [lo, hi)
          auto it = std::upper_bound(outs.begin(), outs.end(), std::make_pair(lo, std::make_pair(INT64_MAX, INT32_MAX)));
          if (it != outs.begin()) --it;
          for (; it != outs.end() && it->first < hi; ++it)
            if (it->second.first > lo) dg.push_back(it->second.second);
        }
        std::sort(dg.begin(), dg.end());
        dg.erase(std::unique(dg.begin(), dg.end()), dg.end());
        for (int32_t x : dg)
          if (x >= g) return fail(BF_EINTERNAL, "grouped apply: a group depends on a later group");
        dep_idx.insert(dep_idx.end(), dg.begin(), dg.end());
        dep_ptr[g + 1] = (int32_t)dep_idx.size();
      }
    }
  }
  gp.ngroups = (int32_t)T.groups.size();
  // place the images: run r's groups at img_off + i * img_stride; each
  // tile's destination becomes a byte offset into the images
  int64_t img_bytes = 0;
  for (GroupedRun& run : gp.runs) {
    run.img_off = img_bytes;
    img_bytes += (int64_t)run.ngroups * run.img_stride;
  }
  const size_t es = elem_bytes(dtype);
  for (const GroupedRun& run : gp.runs)
    for (int g = run.group0; g < run.group0 + run.ngroups; ++g) {
      const GroupedGroup& G = T.groups[g];
      const int64_t base = run.img_off + (int64_t)(g - run.group0) * run.img_stride + G.off_fac;
      for (int q = G.seg0; q < G.seg0 + G.nseg; ++q) {
        GroupedSeg& sg = T.segs[q];
        // every tile inside its group's staged elements, every image inside its slot
        if (sg.dst < 0 || sg.dst + (int64_t)sg.K * sg.tld > G.fac_elems ||
            G.off_fac + (int64_t)G.fac_elems * (int64_t)es > run.img_stride)
          return fail(BF_EINTERNAL, "grouped apply: a factor tile outside its image");
        sg.dst = base + sg.dst * (int64_t)es;
      }
    }
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t b0 = al((size_t)std::max<int64_t>(img_bytes, 16)), b1 = dep_ptr.size() * sizeof(int32_t),
               b2 = std::max<size_t>(1, dep_idx.size()) * sizeof(int32_t),
               b3 = std::max<size_t>(1, T.segs.size()) * sizeof(GroupedSeg);
  std::vector<char> tail(al(b1) + al(b2) + b3, 0);
  memcpy(tail.data(), dep_ptr.data(), b1);
  if (!dep_idx.empty()) memcpy(tail.data() + al(b1), dep_idx.data(), dep_idx.size() * sizeof(int32_t));
  if (!T.segs.empty()) memcpy(tail.data() + al(b1) + al(b2), T.segs.data(), T.segs.size() * sizeof(GroupedSeg));
  // over the memory cap the plan stays unusable and the applies use the
  // stage launches
  const int arc = gp.dev.alloc(&F->mem, b0 + tail.size(), nullptr);
  if (arc == BF_ENOMEM) return BF_OK;
  BF_TRY(arc);
  char* p = (char*)gp.dev.p;
  BF_CUDA_TRY(cudaMemsetAsync(p, 0, b0, s));
  BF_CUDA_TRY(cudaMemcpyAsync(p + b0, tail.data(), tail.size(), cudaMemcpyHostToDevice, s));
  // the descriptor parts of each run's images (one strided copy per run),
  // then the factor tiles packed on the device
  std::vector<char> desc;
  for (const GroupedRun& run : gp.runs) {
    const size_t dm = (size_t)run.desc_max;
    if (dm == 0 || run.ngroups == 0) continue;
    desc.assign(dm * run.ngroups, 0);
    for (int g = run.group0; g < run.group0 + run.ngroups; ++g) {
      const GroupedGroup& G = T.groups[g];
      char* d = desc.data() + (size_t)(g - run.group0) * dm;
      memcpy(d, &G, sizeof(GroupedGroup));
      if (G.ntasks) memcpy(d + G.off_tasks, &T.tasks[G.task0], (size_t)G.ntasks * sizeof(GroupedTask));
      if (G.nspans) memcpy(d + G.off_spans, &T.spans[G.span0], (size_t)G.nspans * sizeof(GroupedSpan));
      if (G.nospans) memcpy(d + G.off_ospans, &T.ospans[G.ospan0], (size_t)G.nospans * sizeof(GroupedSpan));
      if (G.st_chunk[G.nst]) memcpy(d + G.off_chunks, &T.chunks[G.chunk0], (size_t)G.st_chunk[G.nst] * 4);
    }
    BF_CUDA_TRY(cudaMemcpy2DAsync(p + run.img_off, (size_t)run.img_stride, desc.data(), dm, dm,
                                  (size_t)run.ngroups, cudaMemcpyHostToDevice, s));
  }
  if (!T.segs.empty()) {
    const int grid = (int)std::min<size_t>(T.segs.size(), 4096);
    note_launch();
    grouped_pack_kernel<<<grid, 128, 0, s>>>((const GroupedSeg*)(p + b0 + al(b1) + al(b2)), (int)T.segs.size(),
                                             (uint8_t*)p, (int)es);
    BF_CUDA_TRY(cudaGetLastError());
  }
  BF_CUDA_TRY(host_sync(s));
  gp.d_img = (const uint8_t*)p;
  gp.d_dep_ptr = (const int32_t*)(p + b0);
  gp.d_dep_idx = (const int32_t*)(p + b0 + al(b1));
  gp.ok = true;
  return BF_OK;
}

int run_grouped(Fact* F, int opC, int dtype, int64_t nrhs, const void* xt, void* yt, void* ping, void* pong,
                cudaStream_t s, int cw_override) {
  const GroupedPlan& gp = F->gp[opC][dtype];
  if (!gp.ok) return fail(BF_EINTERNAL, "grouped apply not built");
  if (nrhs > INT32_MAX) return fail(BF_EINVAL, "too many right-hand sides");
  const size_t es = elem_bytes(dtype);
  void* bases[4] = {const_cast<void*>(xt), ping, pong, yt};
  for (size_t r = 0; r < gp.runs.size(); ++r) {
    const GroupedRun& run = gp.runs[r];
    // the tuned (or asked) slice width, else the widest up to 64 columns;
    // narrower while the rows and factors do not fit
    const int tuned = cw_override > 0 ? cw_override : gp.cw[nrhs_class(nrhs)];
    int CW = (int)std::min<int64_t>(nrhs, tuned > 0 ? tuned : 64);
    auto bytes = [&](int cw) { return grouped_smem(run, cw, es); };
    while (CW > 1 && bytes(CW) > GR_SMEM_LIMIT) CW = (CW + 1) / 2;
    if (bytes(CW) > GR_SMEM_LIMIT) return fail(BF_EINTERNAL, "grouped apply: a group does not fit");
    GroupedArgs a{};
    a.img = gp.d_img + run.img_off;
    a.stride = run.img_stride;
    a.group0 = run.group0;
    a.N = (int)nrhs;
    a.CW = CW;
    a.x = bases[run.in_base];
    a.in_ld = run.in_ld;
    a.y = bases[run.out_base];
    const int slices = (int)((nrhs + CW - 1) / CW);
    // 256 threads (8 warps) for 64-column slices, 128 for narrower ones
    // (complex128: 256)
    const int NT = CW > 32 || dtype == BF_C128 ? 256 : 128;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)run.ngroups, (unsigned)slices);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = bytes(CW);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = r > 0 ? 1 : 0;
    // the attribute is each kernel's largest size, set once per process
    // (never lowered under a launch of another host thread)
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [&] {
      const void* k[3] = {(const void*)grouped_kernel_c64_256, (const void*)grouped_kernel_c64_128,
                          (const void*)grouped_kernel_c128_256};
      for (int i = 0; i < 3 && attr_err == cudaSuccess; ++i)
        attr_err = cudaFuncSetAttribute(k[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GR_SMEM_LIMIT);
    });
    BF_CUDA_TRY(attr_err);
    note_launch();
    cudaError_t e;
    if (dtype == BF_C128)
      e = cudaLaunchKernelEx(&cfg, grouped_kernel_c128_256, a);
    else
      e = NT == 256 ? cudaLaunchKernelEx(&cfg, grouped_kernel_c64_256, a) : cudaLaunchKernelEx(&cfg, grouped_kernel_c64_128, a);
    if (e != cudaSuccess) return fail(BF_ECUDA, std::string("grouped apply launch: ") + cudaGetErrorString(e));
    BF_CUDA_TRY(cudaGetLastError());
  }
  return BF_OK;
}

// ----------------------------------------------------- persistent launch --
namespace {
size_t gr_al256(size_t b) { return (b + 255) & ~(size_t)255; }

// one column-slice width for every run: the widest (<= 64, or the tuned /
// asked width) at which every run's image and rows fit; *smem: the largest
// run's shared memory at that width
int persist_cw(const GroupedPlan& gp, int64_t nrhs, int dtype, int cw_override, size_t* smem) {
  const size_t es = elem_bytes(dtype);
  auto bytes = [&](int cw) {
    size_t b = 0;
    for (const GroupedRun& r : gp.runs) b = std::max(b, grouped_smem(r, cw, es));
    return b;
  };
  const int tuned = cw_override > 0 ? cw_override : gp.cw[nrhs_class(nrhs)];
  int CW = (int)std::min<int64_t>(nrhs, tuned > 0 ? tuned : 64);
  while (CW > 1 && bytes(CW) > GR_SMEM_LIMIT) CW = (CW + 1) / 2;
  if (smem) *smem = bytes(CW);
  return bytes(CW) <= GR_SMEM_LIMIT ? CW : 0;
}

int launch_persist(const GroupedPersistArgs& pa, int dtype, int NT, size_t smem, cudaStream_t s) {
  const void* k = dtype == BF_C128 ? (const void*)grouped_persist_c128_256
                  : NT == 256      ? (const void*)grouped_persist_c64_256
                                   : (const void*)grouped_persist_c64_128;
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [&] {
    const void* ks[3] = {(const void*)grouped_persist_c64_256, (const void*)grouped_persist_c64_128,
                         (const void*)grouped_persist_c128_256};
    for (int i = 0; i < 3 && attr_err == cudaSuccess; ++i)
      attr_err = cudaFuncSetAttribute(ks[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GR_SMEM_LIMIT);
  });
  BF_CUDA_TRY(attr_err);
  int dev = 0, sms = 0, per_sm = 0;
  BF_CUDA_TRY(cudaGetDevice(&dev));
  BF_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  BF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, smem));
  if (per_sm < 1) return fail(BF_ECUDA, "persistent apply: no CTA fits on an SM");
  const int grid = std::max(1, std::min(pa.ntasks, per_sm * sms));   // all resident
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  note_launch();
  cudaError_t e;
  if (dtype == BF_C128) e = cudaLaunchKernelEx(&cfg, grouped_persist_c128_256, pa);
  else if (NT == 256) e = cudaLaunchKernelEx(&cfg, grouped_persist_c64_256, pa);
  else e = cudaLaunchKernelEx(&cfg, grouped_persist_c64_128, pa);
  if (e != cudaSuccess) return fail(BF_ECUDA, std::string("persistent apply launch: ") + cudaGetErrorString(e));
  BF_CUDA_TRY(cudaGetLastError());
  return BF_OK;
}
}  // namespace

// scratch: every run's output rows but the last (stacked), the task flags,
// the per-run arguments and the runs' first groups
size_t grouped_persist_scratch_bytes(const GroupedPlan& gp, int64_t nrhs, int dtype) {
  int64_t rows = 0;
  for (size_t r = 0; r + 1 < gp.runs.size(); ++r) rows += gp.runs[r].out_rows;
  const size_t nr = gp.runs.size();
  return gr_al256((size_t)rows * nrhs * elem_bytes(dtype)) + gr_al256((size_t)gp.ngroups * nrhs * 4) +
         gr_al256(nr * sizeof(GroupedArgs)) + gr_al256((nr + 1) * 4);
}

int run_grouped_persist(Fact* F, int opC, int dtype, int64_t nrhs, const void* xt, void* yt, void* scratch,
                        cudaStream_t s, int cw_override, int mode) {
  const GroupedPlan& gp = F->gp[opC][dtype];
  if (!gp.ok) return fail(BF_EINTERNAL, "grouped apply not built");
  if (nrhs > INT32_MAX) return fail(BF_EINVAL, "too many right-hand sides");
  size_t smem = 0;
  const int CW = persist_cw(gp, nrhs, dtype, cw_override, &smem);
  if (CW < 1) return fail(BF_EINTERNAL, "persistent apply: a group does not fit");
  const size_t es = elem_bytes(dtype);
  const int slices = (int)((nrhs + CW - 1) / CW);
  const int nruns = (int)gp.runs.size();
  int64_t rows = 0;
  for (int r = 0; r + 1 < nruns; ++r) rows += gp.runs[r].out_rows;
  char* p = (char*)scratch;
  char* inter = p;
  int32_t* flags = (int32_t*)(p + gr_al256((size_t)rows * nrhs * es));
  char* argp = (char*)flags + gr_al256((size_t)gp.ngroups * nrhs * 4);
  int32_t* rg0 = (int32_t*)(argp + gr_al256(nruns * sizeof(GroupedArgs)));
  std::vector<GroupedArgs> args(nruns);
  std::vector<int32_t> g0(nruns + 1);
  int64_t row0 = 0;
  for (int r = 0; r < nruns; ++r) {
    const GroupedRun& run = gp.runs[r];
    GroupedArgs& a = args[r];
    a.img = gp.d_img + run.img_off;
    a.stride = run.img_stride;
    a.group0 = run.group0;
    a.N = (int)nrhs;
    a.CW = CW;
    // run r reads run r - 1's rows (x for the first) and writes its own (y for the last)
    a.x = r == 0 ? xt : (const void*)(inter + (size_t)(row0 - gp.runs[r - 1].out_rows) * nrhs * es);
    a.in_ld = run.in_ld;
    a.y = r + 1 == nruns ? yt : (void*)(inter + (size_t)row0 * nrhs * es);
    if (r + 1 < nruns) row0 += run.out_rows;
    g0[r] = run.group0;
  }
  g0[nruns] = gp.ngroups;
  if (mode != 2) {   // the per-run arguments (this call's buffers)
    BF_TRY(upload_async(argp, args.data(), nruns * sizeof(GroupedArgs), s));
    BF_TRY(upload_async(rg0, g0.data(), (nruns + 1) * sizeof(int32_t), s));
  }
  if (mode == 1) return BF_OK;
  BF_CUDA_TRY(cudaMemsetAsync(flags, 0, (size_t)gp.ngroups * slices * 4, s));
  GroupedPersistArgs pa{};
  pa.args = (const GroupedArgs*)argp;
  pa.run_group0 = rg0;
  pa.nruns = nruns;
  pa.ntasks = gp.ngroups * slices;
  pa.w.dep_ptr = gp.d_dep_ptr;
  pa.w.dep_idx = gp.d_dep_idx;
  pa.w.flags = flags;
  pa.w.status = tc_status_ptr();
  pa.w.limit_ns = 1000000000ull;
  pa.w.slices = slices;
  if (!pa.w.status) return fail(BF_ECUDA, "device status flag not found");
  const int NT = CW > 32 || dtype == BF_C128 ? 256 : 128;
  return launch_persist(pa, dtype, NT, smem, s);
}

// One task whose group (empty: no rows, no tiles) depends on itself, so its
// wait runs out after limit_ns, sets the status flag and the kernel returns.
int grouped_wait_probe(uint64_t limit_ns, cudaStream_t s) {
  DevBuf buf;
  BF_TRY(buf.alloc(nullptr, 4096, s));
  char* p = (char*)buf.p;
  GroupedGroup G{};
  const int32_t dep[3] = {0, 1, 0};   // dep_ptr {0, 1}, dep_idx {0}: the group reads itself
  GroupedArgs a{};
  a.img = (const uint8_t*)p;           // one image: the empty head
  a.stride = (int64_t)gr_align16(sizeof(GroupedGroup));
  a.N = 1;
  a.CW = 1;
  int rc = BF_OK;
  const int32_t g0[2] = {0, 1};
  if (cudaMemsetAsync(p, 0, 4096, s) != cudaSuccess ||
      cudaMemcpyAsync(p, &G, sizeof(G), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(p + 1024, dep, sizeof(dep), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(p + 2048, &a, sizeof(a), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(p + 3072, g0, sizeof(g0), cudaMemcpyHostToDevice, s) != cudaSuccess)
    rc = fail(BF_ECUDA, "probe set-up copy failed");
  GroupedPersistArgs pa{};
  pa.args = (const GroupedArgs*)(p + 2048);
  pa.run_group0 = (const int32_t*)(p + 3072);
  pa.nruns = 1;
  pa.ntasks = 1;
  pa.w.dep_ptr = (const int32_t*)(p + 1024);
  pa.w.dep_idx = (const int32_t*)(p + 1024) + 2;
  pa.w.flags = (int32_t*)(p + 1536);
  pa.w.status = tc_status_ptr();
  pa.w.limit_ns = limit_ns;
  pa.w.slices = 1;
  if (!rc && !pa.w.status) rc = fail(BF_ECUDA, "device status flag not found");
  if (!rc) rc = launch_persist(pa, BF_C64, 128, gr_smem_bytes(a.stride, 0, 1, 8), s);
  if (!rc && host_sync(s) != cudaSuccess) rc = fail(BF_ECUDA, "probe synchronisation failed");
  buf.release(s);
  return rc;
}

}  // namespace bf
