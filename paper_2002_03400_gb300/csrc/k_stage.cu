// Block-sparse stage products of the butterfly: one launch applies every
// block of one factor (V^0, W^j, B, R^j or U^L, or their adjoints) to a block
// of vectors.  The same kernel serves the apply (eq. hybrid_butterfly_mat),
// the peeling of already-recovered factors from the sketches (Alg. 2, the
// lines that project K(T_tau,S_nu)^T Gamma_tau and K(T_tau,S_nu) Omega_nu
// and form V^T Omega_nu) and the projection of the centre level.
//
// Each task is one output block:
//   out[M x N] = sum_t op_t(mat_t)[M x K_t] * in_t[K_t x N],  t < nterms <= 2
// Blocks have ranks ~10-60, far too small for a CTA each, and a stage is
// bound by memory latency (each block's entries and inputs are a few KB).
// Two kernel shapes compute the same sums (every output is one lane's
// sequential FMA chain over the terms and k, so they agree bit for bit and
// the result does not depend on N or on the lane layout):
//   variant 0: one warp per (task, column slice, group of RT rows) --
//     thousands of warps; each K step issues its KC input and RT x KC factor
//     loads together, so their latencies overlap;
//   variant 1: one warp per (task, column slice) keeping RT1 rows per lane
//     and walking K one element at a time -- fewer instructions per output;
//   variant 2: one warp per (task, column slice) that copies the factor
//     block whole into shared memory first (coalesced) and stages its inputs
//     KC2 rows at a time -- no factor-load latency inside the K loop;
//   variants 3-5: one warp per (task, 64-column slice, WFR = 8, 4 or 12
//     rows), two columns and WFR rows per lane (a register tile: WFR
//     broadcast factor loads and two input loads per k for 2 WFR complex
//     FMAs);
//   variants 6-7: one CTA per (task, 64-column slice, block of 16 or 32
//     rows) that stages each round of input rows and factor entries in
//     shared memory with asynchronous copies, all in flight at once, and
//     computes from there (one load latency per round, not per k).
// In variants 0-2 the warp's lanes cover CW columns x 32/CW rows, CW the
// smallest power of two >= N (at most 32), so small numbers of right-hand
// sides still use every lane.  The apply picks the variant per stage and column count
// as measured by the apply tuner, else by stage_variant_default.
// Operand layouts (per StageTerm/StageTask):
//   ld > 0: column-major, element (k, c) at off + k + c*ld
//   ld < 0: row-major,    element (k, c) at off + k*(-ld) + c
//   ld = 0: row-major with the launch's column count N: off is a row index,
//           element (k, c) at (off + k)*N + c  (apply intermediates)
// Row-major intermediates make the loads of one k and the stores of one
// output row contiguous across the lanes.
#include <atomic>

#include "bf_internal.h"
#include "cx.cuh"

namespace bf {

namespace {
constexpr int WARPS = 8, THREADS = 32 * WARPS;
constexpr int RT = 2;    // output rows per lane
constexpr int KC = 8;    // K per step: KC inputs and RT x KC factor entries loaded together

struct Strides {
  int64_t off, rs, cs;
};
__device__ __forceinline__ Strides strides(int64_t off, int64_t ld, int N) {
  if (ld > 0) return {off, 1, ld};
  if (ld < 0) return {off, -ld, 1};
  return {off * N, N, 1};
}

// Programmatic dependent launch: let the next stage's grid start, warm L2
// with this warp's first factor blocks (they do not depend on the previous
// stage), then wait until the previous grid has completed and its writes are
// visible.  Every read of a stage input and every write comes after the
// wait.  Without a programmatic dependency the wait returns at once.
template <typename V>
__device__ __forceinline__ void stage_prologue(const StageTask* __restrict__ tasks, int ti, int lane) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (ti >= 0) {
    const StageTask& tk = tasks[ti];
    for (int t = 0; t < tk.nterms; ++t) {
      const StageTerm& T = tk.t[t];
      const int64_t rows = T.conjT ? T.K : tk.M, cols = T.conjT ? tk.M : T.K;
      const int64_t bytes = ((cols - 1) * (int64_t)T.ldm + rows) * (int64_t)sizeof(V);
      for (int64_t off = (int64_t)lane * 128; off < bytes; off += 32 * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"((const char*)T.mat + off));
    }
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
}  // namespace

// Variant 0 ("mlp"): one warp per (task, column slice, RT-row group); K in
// steps of KC whose KC input and RT x KC factor loads are issued together.
template <typename R>
__global__ void __launch_bounds__(THREADS, 2)
stage_mlp_kernel(const StageTask* __restrict__ tasks, int ntasks, StageBases bases, int Noverride, int lcw,
                 int rgroups) {
  using V = typename Cx<R>::V;
  const int CW = 1 << lcw, RW = 32 >> lcw, GR = RW * RT;   // GR: rows per warp item
  const int lane = threadIdx.x & 31;
  const int ci = lane & (CW - 1), ri = lane >> lcw;
  const int nwarps = gridDim.x * WARPS;
  // work items: (task, column slice, row group); slices per task from the
  // launch's N, row groups from the launch's largest M (the host keeps the
  // item count below 2^31)
  const int Nl = Noverride;
  const int Nmax = Nl > 0 ? Nl : -Nl;   // Nl < 0: per-task N, -Nl the widest
  const int slices = Nmax > 0 ? (Nmax + CW - 1) / CW : 1;
  const int per_task = slices * rgroups;
  const int items = ntasks * per_task;
  {
    const int w0 = blockIdx.x * WARPS + (threadIdx.x >> 5);
    stage_prologue<V>(tasks, w0 < items ? w0 / per_task : -1, lane);
  }
  for (int w = blockIdx.x * WARPS + (threadIdx.x >> 5); w < items; w += nwarps) {
    const int ti = w / per_task, tw = w - ti * per_task;
    const int sl = tw / rgroups, rg = tw - sl * rgroups;
    const StageTask& tk = tasks[ti];
    const int M = tk.M, nterms = tk.nterms;
    const int i0 = rg * GR;
    if (i0 >= M) continue;
    const int N = Nl > 0 ? Nl : tk.N;
    const Strides so = strides(tk.out_off, tk.ldo, N);
    V* __restrict__ out = (V*)bases.p[tk.out_base] + so.off;
    // column slices of this warp: sl (fixed N) or all of them (per-task N)
    const int c_first = Nmax > 0 ? sl * CW : 0;
    const int c_last = Nl > 0 ? c_first + CW : (Nmax > 0 ? (c_first + CW < N ? c_first + CW : N) : N);
    bool rv[RT];
#pragma unroll
    for (int r = 0; r < RT; ++r) rv[r] = i0 + ri + r * RW < M;
    for (int c0 = c_first; c0 < c_last; c0 += CW) {
      const int c = c0 + ci;
      const bool cv = c < N;
      V acc[RT];
#pragma unroll
      for (int r = 0; r < RT; ++r) acc[r] = Cx<R>::make(0, 0);
      for (int term = 0; term < nterms; ++term) {
        const StageTerm& T = tk.t[term];
        const V* __restrict__ mat = (const V*)T.mat;
        const int K = T.K, ldm = T.ldm, cj = T.conjT;
        const Strides si = strides(T.in_off, T.ldi, N);
        const V* __restrict__ in = (const V*)bases.p[T.in_base] + si.off + (int64_t)c * si.cs;
        // element (i, k) of op(mat): mat[i + k ldm], or conj(mat[k + i ldm])
        const int istep = cj ? ldm : 1, kstep = cj ? 1 : ldm;   // blocks are small: 32-bit offsets
        const V* __restrict__ mrow = mat + (int64_t)(i0 + ri) * istep;
        for (int k0 = 0; k0 < K; k0 += KC) {
          V x[KC], a[RT][KC];
#pragma unroll
          for (int u = 0; u < KC; ++u) {
            const bool kv = k0 + u < K;
            x[u] = (cv && kv) ? in[(int64_t)(k0 + u) * si.rs] : Cx<R>::make(0, 0);
#pragma unroll
            for (int r = 0; r < RT; ++r)
              a[r][u] = (rv[r] && kv) ? mrow[r * RW * istep + (k0 + u) * kstep]
                                      : Cx<R>::make(0, 0);
          }
#pragma unroll
          for (int u = 0; u < KC; ++u)
#pragma unroll
            for (int r = 0; r < RT; ++r) {
              if (cj) a[r][u].y = -a[r][u].y;
              cmac(acc[r], a[r][u], x[u]);
            }
        }
      }
      if (cv) {
#pragma unroll
        for (int r = 0; r < RT; ++r)
          if (rv[r]) out[(int64_t)(i0 + ri + r * RW) * so.rs + (int64_t)c * so.cs] = acc[r];
      }
    }
  }
}

// Variant 1 ("rows"): one warp per (task, column slice); each lane keeps
// RT1 rows and walks K one element at a time (fewer, longer warps: cheaper
// per output when the number of columns is large).
constexpr int RT1 = 8;
template <typename R>
__global__ void __launch_bounds__(THREADS)
stage_rows_kernel(const StageTask* __restrict__ tasks, int ntasks, StageBases bases, int Noverride, int lcw) {
  using V = typename Cx<R>::V;
  const int CW = 1 << lcw, RW = 32 >> lcw;
  const int lane = threadIdx.x & 31;
  const int ci = lane & (CW - 1), ri = lane >> lcw;
  const int nwarps = gridDim.x * WARPS;
  const int Nl = Noverride;
  const int Nmax = Nl > 0 ? Nl : -Nl;   // Nl < 0: per-task N, -Nl the widest
  const int slices = Nmax > 0 ? (Nmax + CW - 1) / CW : 1;
  const int items = ntasks * slices;
  {
    const int w0 = blockIdx.x * WARPS + (threadIdx.x >> 5);
    stage_prologue<V>(tasks, w0 < items ? w0 / slices : -1, lane);
  }
  for (int w = blockIdx.x * WARPS + (threadIdx.x >> 5); w < items; w += nwarps) {
    const int ti = w / slices, sl = w - ti * slices;
    const StageTask& tk = tasks[ti];
    const int M = tk.M, nterms = tk.nterms;
    const int N = Nl > 0 ? Nl : tk.N;
    const Strides so = strides(tk.out_off, tk.ldo, N);
    V* __restrict__ out = (V*)bases.p[tk.out_base] + so.off;
    const int c_first = Nmax > 0 ? sl * CW : 0;
    const int c_last = Nl > 0 ? c_first + CW : (Nmax > 0 ? (c_first + CW < N ? c_first + CW : N) : N);
    for (int c0 = c_first; c0 < c_last; c0 += CW) {
      const int c = c0 + ci;
      const bool cv = c < N;
      for (int i0 = 0; i0 < M; i0 += RW * RT1) {
        V acc[RT1];
#pragma unroll
        for (int r = 0; r < RT1; ++r) acc[r] = Cx<R>::make(0, 0);
        for (int term = 0; term < nterms; ++term) {
          const StageTerm& T = tk.t[term];
          const V* __restrict__ mat = (const V*)T.mat;
          const int K = T.K, ldm = T.ldm, cj = T.conjT;
          const Strides si = strides(T.in_off, T.ldi, N);
          const V* __restrict__ in = (const V*)bases.p[T.in_base] + si.off + (int64_t)c * si.cs;
          const int istep = cj ? ldm : 1, kstep = cj ? 1 : ldm;
          const V* __restrict__ mrow = mat + (int64_t)(i0 + ri) * istep;
          for (int k = 0; k < K; ++k) {
            const V x = cv ? in[(int64_t)k * si.rs] : Cx<R>::make(0, 0);
            const V* __restrict__ mk = mrow + k * kstep;
#pragma unroll
            for (int r = 0; r < RT1; ++r)
              if (i0 + ri + r * RW < M) {
                V a = mk[r * RW * istep];
                if (cj) a.y = -a.y;
                cmac(acc[r], a, x);
              }
          }
        }
        if (cv) {
#pragma unroll
          for (int r = 0; r < RT1; ++r) {
            const int i = i0 + ri + r * RW;
            if (i < M) out[(int64_t)i * so.rs + (int64_t)c * so.cs] = acc[r];
          }
        }
      }
    }
  }
}

// Variant 2 ("block"): one warp per (task, column slice); each factor block
// (when it has at most FLAT entries) is copied whole into the warp's slice of
// shared memory, CB stored columns at a time with consecutive lanes on
// consecutive entries, the inputs follow KC2 rows at a time, and the
// products read shared memory (larger blocks: chunks of KC2 columns).
constexpr int RT2 = 16, KC2 = 8, PR2 = 64, FLAT2 = KC2 * PR2, CB2 = 8;
template <typename R>
constexpr size_t block_smem() {
  return sizeof(typename Cx<R>::V) * WARPS * KC2 * (32 + PR2);
}
template <typename R>
__global__ void __launch_bounds__(THREADS, 2)
stage_block_kernel(const StageTask* __restrict__ tasks, int ntasks, StageBases bases, int Noverride, int lcw) {
  using V = typename Cx<R>::V;
  extern __shared__ __align__(16) uint8_t stage_smem_raw[];
  const int CW = 1 << lcw, RW = 32 >> lcw;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ci = lane & (CW - 1), ri = lane >> lcw;
  const int prows = RT2 * RW < PR2 ? RT2 * RW : PR2;
  V (*xs)[32] = (V(*)[32])(stage_smem_raw + sizeof(V) * warp * KC2 * (32 + PR2));
  V (*ms)[PR2] = (V(*)[PR2])((uint8_t*)xs + sizeof(V) * KC2 * 32);
  V* __restrict__ fl = &ms[0][0];
  const int nwarps = gridDim.x * WARPS;
  const int Nl = Noverride;
  const int Nmax = Nl > 0 ? Nl : -Nl;   // Nl < 0: per-task N, -Nl the widest
  const int slices = Nmax > 0 ? (Nmax + CW - 1) / CW : 1;
  const int items = ntasks * slices;
  {
    const int w0 = blockIdx.x * WARPS + warp;
    stage_prologue<V>(tasks, w0 < items ? w0 / slices : -1, lane);
  }
  for (int w = blockIdx.x * WARPS + warp; w < items; w += nwarps) {
    const int ti = w / slices, sl = w - ti * slices;
    const StageTask& tk = tasks[ti];
    const int M = tk.M, nterms = tk.nterms;
    const int N = Nl > 0 ? Nl : tk.N;
    const Strides so = strides(tk.out_off, tk.ldo, N);
    V* __restrict__ out = (V*)bases.p[tk.out_base] + so.off;
    const int c_first = Nmax > 0 ? sl * CW : 0;
    const int c_last = Nl > 0 ? c_first + CW : (Nmax > 0 ? (c_first + CW < N ? c_first + CW : N) : N);
    for (int c0 = c_first; c0 < c_last; c0 += CW) {
      const int c = c0 + ci;
      const bool cv = c < N;
      for (int i0 = 0; i0 < M; i0 += prows) {
        const int mrows = M - i0 < prows ? M - i0 : prows;
        V acc[RT2];
#pragma unroll
        for (int r = 0; r < RT2; ++r) acc[r] = Cx<R>::make(0, 0);
        for (int term = 0; term < nterms; ++term) {
          const StageTerm& T = tk.t[term];
          const V* __restrict__ mat = (const V*)T.mat;
          const int K = T.K, ldm = T.ldm, cj = T.conjT;
          const Strides si = strides(T.in_off, T.ldi, N);
          const V* __restrict__ in = (const V*)bases.p[T.in_base] + si.off + (int64_t)c * si.cs;
          const bool whole = M * K <= FLAT2;
          if (whole) {
            // stored columns (length sl_, count sc) of M x K (or K x M, conj)
            __syncwarp();
            const int sl_ = cj ? K : M, sc = cj ? M : K;
            for (int e0 = 0; e0 < sl_; e0 += 32) {
              const int e = e0 + lane;
              for (int j0 = 0; j0 < sc; j0 += CB2) {
                V t[CB2];
#pragma unroll
                for (int u = 0; u < CB2; ++u)
                  t[u] = (e < sl_ && j0 + u < sc) ? mat[e + (int64_t)(j0 + u) * ldm] : Cx<R>::make(0, 0);
#pragma unroll
                for (int u = 0; u < CB2; ++u)
                  if (e < sl_ && j0 + u < sc) {
                    if (cj) t[u].y = -t[u].y;
                    fl[e + (j0 + u) * sl_] = t[u];
                  }
              }
            }
          }
          for (int k0 = 0; k0 < K; k0 += KC2) {
            const int kn = K - k0 < KC2 ? K - k0 : KC2;
            if (!whole) __syncwarp();
#pragma unroll
            for (int kk = 0; kk < KC2; ++kk)
              xs[kk][lane] = (cv && kk < kn) ? in[(int64_t)(k0 + kk) * si.rs] : Cx<R>::make(0, 0);
            if (!whole) {
#pragma unroll
              for (int j = 0; j < KC2 * PR2 / 32; ++j) {
                const int e = lane + 32 * j;
                const int i = cj ? e / KC2 : e % PR2, kk = cj ? e % KC2 : e / PR2;
                V a = Cx<R>::make(0, 0);
                if (i < mrows && kk < kn) {
                  a = cj ? mat[(k0 + kk) + (int64_t)(i0 + i) * ldm] : mat[(i0 + i) + (int64_t)(k0 + kk) * ldm];
                  if (cj) a.y = -a.y;
                }
                ms[kk][i] = a;
              }
            }
            __syncwarp();
            // element (i, kk) of the chunk: whole block fl[i + k M] / fl[k + i K],
            // chunk ms[kk][i - i0]
            const int fi = whole ? (cj ? K : 1) : 1, fk = whole ? (cj ? 1 : M) : PR2;
            const V* __restrict__ fb = whole ? fl + (i0 + ri) * fi + k0 * fk : &ms[0][ri];
#pragma unroll 2
            for (int kk = 0; kk < kn; ++kk) {
              const V x = xs[kk][lane];
              const V* __restrict__ fr = fb + kk * fk;
#pragma unroll
              for (int r = 0; r < RT2; ++r)
                if (ri + r * RW < mrows) cmac(acc[r], fr[r * RW * fi], x);
            }
            __syncwarp();
          }
        }
        if (cv) {
#pragma unroll
          for (int r = 0; r < RT2; ++r) {
            const int i = ri + r * RW;
            if (i < mrows) out[(int64_t)(i0 + i) * so.rs + (int64_t)c * so.cs] = acc[r];
          }
        }
      }
    }
  }
}

// Variants 3-5 ("wide"): one warp per (task, 64-column slice, group of WFR
// rows; WFR = 8, 4, 12: the tuner picks per stage); lane l takes columns 2l
// and 2l + 1 of the slice and all WFR rows,
// so per k the warp issues WFR factor loads (one address each, broadcast to
// all lanes) and two input loads (consecutive columns across the lanes) for
// 2 WFR complex FMAs per lane -- the register tile of a small GEMM.  Rows
// past the task's end and columns past N re-read a valid row / column and
// are not stored.
template <typename R, int WFR>
__global__ void __launch_bounds__(THREADS, 2)
stage_wide_kernel(const StageTask* __restrict__ tasks, int ntasks, StageBases bases, int Noverride, int rgroups) {
  using V = typename Cx<R>::V;
  const int lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * WARPS;
  const int Nl = Noverride;
  const int Nmax = Nl > 0 ? Nl : -Nl;   // Nl < 0: per-task N, -Nl the widest
  const int slices = Nmax > 0 ? (Nmax + 63) / 64 : 1;
  const int per_task = slices * rgroups;
  const int items = ntasks * per_task;
  {
    const int w0 = blockIdx.x * WARPS + (threadIdx.x >> 5);
    stage_prologue<V>(tasks, w0 < items ? w0 / per_task : -1, lane);
  }
  for (int w = blockIdx.x * WARPS + (threadIdx.x >> 5); w < items; w += nwarps) {
    const int ti = w / per_task, tw = w - ti * per_task;
    const int sl = tw / rgroups, rg = tw - sl * rgroups;
    const StageTask& tk = tasks[ti];
    const int M = tk.M, nterms = tk.nterms;
    const int i0 = rg * WFR;
    if (i0 >= M) continue;
    const int N = Nl > 0 ? Nl : tk.N;
    const int c = sl * 64 + 2 * lane;
    if (sl * 64 >= N) continue;
    const bool v0 = c < N, v1 = c + 1 < N;
    const int nr = min(WFR, M - i0);
    const Strides so = strides(tk.out_off, tk.ldo, N);
    V* __restrict__ out = (V*)bases.p[tk.out_base] + so.off;
    V acc[WFR][2];
#pragma unroll
    for (int r = 0; r < WFR; ++r) acc[r][0] = acc[r][1] = Cx<R>::make(0, 0);
    for (int term = 0; term < nterms; ++term) {
      const StageTerm& T = tk.t[term];
      const V* __restrict__ mat = (const V*)T.mat;
      const int K = T.K, ldm = T.ldm, cj = T.conjT;
      const Strides si = strides(T.in_off, T.ldi, N);
      const V* __restrict__ in = (const V*)bases.p[T.in_base] + si.off;
      const V* __restrict__ x0 = in + (int64_t)min(c, N - 1) * si.cs;
      const V* __restrict__ x1 = in + (int64_t)min(c + 1, N - 1) * si.cs;
      const int istep = cj ? ldm : 1, kstep = cj ? 1 : ldm;   // blocks are small: 32-bit offsets
      int mo[WFR];
#pragma unroll
      for (int r = 0; r < WFR; ++r) mo[r] = (i0 + min(r, nr - 1)) * istep;
#pragma unroll 2
      for (int k = 0; k < K; ++k) {
        const V a0 = x0[(int64_t)k * si.rs], a1 = x1[(int64_t)k * si.rs];
        V e[WFR];
#pragma unroll
        for (int r = 0; r < WFR; ++r) e[r] = mat[mo[r] + k * kstep];
#pragma unroll
        for (int r = 0; r < WFR; ++r) {
          if (cj) e[r].y = -e[r].y;
          cmac(acc[r][0], e[r], a0);
          cmac(acc[r][1], e[r], a1);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < WFR; ++r)
      if (r < nr) {
        V* o = out + (int64_t)(i0 + r) * so.rs;
        if (v0) o[(int64_t)c * so.cs] = acc[r][0];
        if (v1) o[(int64_t)(c + 1) * so.cs] = acc[r][1];
      }
  }
}

// Variants 6-7 ("staged"): one CTA per (task, 64-column slice, block of
// 8 SRR rows; SRR = 2 or 4).  The K range is walked in rounds of up to SKR
// rows: every thread issues its share of the round's asynchronous copies
// (the input rows of the slice, 16 bytes per copy where aligned, and the
// factor entries of the CTA's rows), all in flight together, then one wait;
// the products read shared memory.  Lane l holds columns 2l and 2l + 1,
// warp w rows w SRR .. w SRR + SRR - 1 of the block, so per k a lane reads
// one input pair and SRR factor entries (a broadcast) for 2 SRR complex
// FMAs.  Load latency is paid once per round instead of once per k step.
template <typename V>
__host__ __device__ constexpr int staged_kr() {
  return sizeof(V) == 8 ? 48 : 24;
}
template <typename V, int SRR>
__host__ __device__ constexpr size_t staged_smem() {
  return (size_t)staged_kr<V>() * (64 + 8 * SRR) * sizeof(V);
}

template <int BYTES>
__device__ __forceinline__ void cp_async_to_shared(void* dst, const void* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}

template <typename R, int SRR>
__global__ void __launch_bounds__(THREADS)
stage_staged_kernel(const StageTask* __restrict__ tasks, int ntasks, StageBases bases, int Noverride,
                    int rblocks) {
  using V = typename Cx<R>::V;
  constexpr int KR = staged_kr<V>(), RB = 8 * SRR;
  extern __shared__ __align__(16) uint8_t staged_smem_raw[];
  V* __restrict__ xs = (V*)staged_smem_raw;   // [KR][64]: input rows of the round
  V* __restrict__ fs = xs + KR * 64;          // [KR][RB]: factor entries (k, row)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Nl = Noverride;
  const int Nmax = Nl > 0 ? Nl : -Nl;   // Nl < 0: per-task N, -Nl the widest
  const int slices = Nmax > 0 ? (Nmax + 63) / 64 : 1;
  const int per_task = slices * rblocks;
  const int items = ntasks * per_task;
  stage_prologue<V>(tasks, warp == 0 && (int)blockIdx.x < items ? (int)blockIdx.x / per_task : -1, lane);
  for (int it = blockIdx.x; it < items; it += gridDim.x) {
    const int ti = it / per_task, tw = it - ti * per_task;
    const int sl = tw / rblocks, rb = tw - sl * rblocks;
    const StageTask& tk = tasks[ti];
    const int M = tk.M, nterms = tk.nterms;
    const int N = Nl > 0 ? Nl : tk.N;
    const int c0 = sl * 64, r0 = rb * RB;
    if (c0 >= N || r0 >= M) continue;   // uniform over the CTA
    const int cw = min(64, N - c0), mr = min(RB, M - r0);
    const int c = 2 * lane, i0 = warp * SRR;
    V acc[SRR][2];
#pragma unroll
    for (int r = 0; r < SRR; ++r) acc[r][0] = acc[r][1] = Cx<R>::make(0, 0);
    for (int term = 0; term < nterms; ++term) {
      const StageTerm& T = tk.t[term];
      const V* __restrict__ mat = (const V*)T.mat;
      const int K = T.K, ldm = T.ldm, cj = T.conjT;
      const Strides si = strides(T.in_off, T.ldi, N);
      const V* __restrict__ in = (const V*)bases.p[T.in_base] + si.off + c0 * si.cs;
      // pairs of columns in one 16-byte copy: row-major rows of even length
      // starting 16-byte aligned (complex128: every element)
      const bool pair16 = sizeof(V) == 16 || (si.cs == 1 && (si.rs & 1) == 0 && (cw & 1) == 0 &&
                                              ((uintptr_t)in & 15) == 0);
      for (int k0 = 0; k0 < K; k0 += KR) {
        const int kn = min(KR, K - k0);
        __syncthreads();   // the previous round's reads are done
        if (sizeof(V) == 8 && pair16) {
          const int pw = cw >> 1;   // column pairs per row
          for (int e = tid; e < kn * pw; e += THREADS) {
            const int k = e / pw, p = e - k * pw;
            cp_async_to_shared<16>(xs + k * 64 + 2 * p, in + (int64_t)(k0 + k) * si.rs + 2 * p);
          }
        } else {
          for (int e = tid; e < kn * cw; e += THREADS) {
            const int k = e / cw, cc = e - k * cw;
            cp_async_to_shared<sizeof(V)>(xs + k * 64 + cc, in + (int64_t)(k0 + k) * si.rs + (int64_t)cc * si.cs);
          }
        }
        // factor entry (row r0 + i, k0 + k) of op(mat): conj ? mat[i ldm + k] : mat[i + k ldm]
        if (cj) {
          for (int e = tid; e < mr * kn; e += THREADS) {
            const int i = e / kn, k = e - i * kn;
            cp_async_to_shared<sizeof(V)>(fs + k * RB + i, mat + (int64_t)(r0 + i) * ldm + k0 + k);
          }
        } else {
          for (int e = tid; e < mr * kn; e += THREADS) {
            const int k = e / mr, i = e - k * mr;
            cp_async_to_shared<sizeof(V)>(fs + k * RB + i, mat + (r0 + i) + (int64_t)(k0 + k) * ldm);
          }
        }
        asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        if (i0 < mr) {
          // rows past the block's end re-read its last row (never stored)
          int ro[SRR];
#pragma unroll
          for (int r = 0; r < SRR; ++r) ro[r] = min(i0 + r, mr - 1);
          const int cl = min(c, cw - 1), cr = min(c + 1, cw - 1);
#pragma unroll 4
          for (int k = 0; k < kn; ++k) {
            const V a0 = xs[k * 64 + cl], a1 = xs[k * 64 + cr];
#pragma unroll
            for (int r = 0; r < SRR; ++r) {
              V e = fs[k * RB + ro[r]];
              if (cj) e.y = -e.y;
              cmac(acc[r][0], e, a0);
              cmac(acc[r][1], e, a1);
            }
          }
        }
      }
    }
    if (i0 < mr) {
      const Strides so = strides(tk.out_off, tk.ldo, N);
      V* __restrict__ out = (V*)bases.p[tk.out_base] + so.off;
#pragma unroll
      for (int r = 0; r < SRR; ++r)
        if (i0 + r < mr) {
          V* o = out + (int64_t)(r0 + i0 + r) * so.rs;
          if (c < cw) o[(int64_t)(c0 + c) * so.cs] = acc[r][0];
          if (c + 1 < cw) o[(int64_t)(c0 + c + 1) * so.cs] = acc[r][1];
        }
    }
  }
}

// Untuned choice: the many-warp variant for up to 16 complex64 columns, the
// wide register-tile variant for more, the whole-block variant for
// complex128 (and for per-task column counts: peeling).
// Peel stages of Alg. 2's W and R steps (Sec. 4.2-4.3): a few thousand small
// products out (M x N) = sum_t A_t (M x K_t) in_t (K_t x N) with M, K of a
// block's rank and N up to k 2^(l-j) columns.  One CTA per (task, block of
// CB columns): the factor blocks A_t and the input block go to shared memory
// with coalesced loads (column-major inputs along K, row-major along N), the
// outputs are formed from shared memory and stored along the output's
// contiguous dimension.  Terms in order, K ascending (the stage kernels'
// order of the sum).
template <typename R>
__global__ void __launch_bounds__(256) peel_kernel(const StageTask* __restrict__ tasks, StageBases bases, int CB,
                                                   int MM, int KM) {
  using V = typename Cx<R>::V;
  extern __shared__ __align__(16) uint8_t peel_smem[];
  __shared__ StageTask tk;   // the task's descriptor, read once
  const int tid = threadIdx.x;
  if (tid == 0) tk = tasks[blockIdx.x];
  __syncthreads();
  const int M = tk.M, N = tk.N, nterms = tk.nterms;
  const int cb0 = blockIdx.y * CB;
  if (cb0 >= N) return;
  const int nc = N - cb0 < CB ? N - cb0 : CB;
  V* sA = (V*)peel_smem;               // [term][k][i], KM x MM each
  V* sX = sA + 2 * KM * MM;            // [term][k][c], KM x CB each
  for (int t = 0; t < nterms; ++t) {
    const StageTerm& T = tk.t[t];
    const V* __restrict__ mat = (const V*)T.mat;
    const int K = T.K, ldm = T.ldm;
    V* a = sA + t * KM * MM;
    if (T.conjT) {   // stored K x M: A(i, k) = conj(mat[k + i ldm])
      for (int e = tid; e < K * M; e += blockDim.x) {
        const int k = e % K, i = e / K;
        V v = mat[k + (int64_t)i * ldm];
        v.y = -v.y;
        a[k * MM + i] = v;
      }
    } else {         // stored M x K: A(i, k) = mat[i + k ldm]
      for (int e = tid; e < K * M; e += blockDim.x) {
        const int i = e % M, k = e / M;
        a[k * MM + i] = mat[i + (int64_t)k * ldm];
      }
    }
    const Strides si = strides(T.in_off, T.ldi, N);
    const V* __restrict__ in = (const V*)bases.p[T.in_base] + si.off;
    V* x = sX + t * KM * CB;
    if (si.rs == 1) {   // column-major: K contiguous per column
      for (int e = tid; e < K * nc; e += blockDim.x) {
        const int k = e % K, c = e / K;
        x[k * CB + c] = in[k + (int64_t)(cb0 + c) * si.cs];
      }
    } else {            // row-major: columns contiguous per row
      for (int e = tid; e < K * nc; e += blockDim.x) {
        const int c = e % nc, k = e / nc;
        x[k * CB + c] = in[(int64_t)k * si.rs + (cb0 + c) * si.cs];
      }
    }
  }
  __syncthreads();
  const Strides so = strides(tk.out_off, tk.ldo, N);
  V* __restrict__ out = (V*)bases.p[tk.out_base] + so.off;
  const bool colmajor = so.rs == 1;
  const int K0 = tk.t[0].K, K1 = nterms > 1 ? tk.t[1].K : 0;
  for (int e = tid; e < M * nc; e += blockDim.x) {
    const int i = colmajor ? e % M : e / nc, c = colmajor ? e / M : e % nc;
    V acc = Cx<R>::make(0, 0);
    for (int t = 0; t < nterms; ++t) {
      const int K = t == 0 ? K0 : K1;
      const V* a = sA + t * KM * MM + i;
      const V* x = sX + t * KM * CB + c;
      for (int k = 0; k < K; ++k) cmac(acc, a[k * MM], x[k * CB]);
    }
    out[(int64_t)i * so.rs + (int64_t)(cb0 + c) * so.cs] = acc;
  }
}

int launch_peel(const StageTask* d_tasks, int ntasks, int maxM, int maxN, int maxK, const StageBases& bases,
                int dtype, cudaStream_t s, bool* launched) {
  *launched = false;
  if (ntasks <= 0 || maxM <= 0 || maxN <= 0) {
    *launched = true;
    return BF_OK;
  }
  const size_t vs = dtype == BF_C128 ? sizeof(double2) : sizeof(float2);
  int CB = 128;
  auto bytes = [&](int cb) { return (size_t)2 * maxK * (maxM + cb) * vs; };
  while (CB > 32 && bytes(CB) > 64 * 1024) CB /= 2;
  if (bytes(CB) > 96 * 1024) return BF_OK;   // very large blocks: the stage kernels
  const dim3 grid((unsigned)ntasks, (unsigned)((maxN + CB - 1) / CB));
  note_launch();
  // the attribute is the kernel's largest size, not this launch's: launches
  // from two host threads (the two sides of a factorization) must not lower
  // it under each other
  if (dtype == BF_C128) {
    BF_CUDA_TRY(cudaFuncSetAttribute(peel_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
    peel_kernel<double><<<grid, 256, bytes(CB), s>>>(d_tasks, bases, CB, maxM, maxK);
  } else {
    BF_CUDA_TRY(cudaFuncSetAttribute(peel_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
    peel_kernel<float><<<grid, 256, bytes(CB), s>>>(d_tasks, bases, CB, maxM, maxK);
  }
  BF_CUDA_TRY(cudaGetLastError());
  *launched = true;
  return BF_OK;
}

static std::atomic<int> g_stage_variant{-1};
int set_stage_variant(int v) {
  if (v < -1 || v >= STAGE_VARIANTS) return fail(BF_EINVAL, "stage variant must be -1 .. 7");
  g_stage_variant.store(v);
  return BF_OK;
}

int stage_variant_default(int nrhs, int dtype) {
  if (dtype == BF_C64 && nrhs > 0) return nrhs <= 16 ? 0 : 3;
  return 2;
}

int launch_stage(const StageTask* d_tasks, int ntasks, int maxM, int maxN, int Noverride,
                 const StageBases& bases, int dtype, cudaStream_t s, int variant, bool pdl) {
  if (Noverride > 0) maxN = Noverride;
  if (ntasks <= 0 || maxM <= 0 || maxN <= 0) return BF_OK;
  if (Noverride > 0 && g_stage_variant.load() >= 0) variant = g_stage_variant.load();
  if (variant < 0) variant = stage_variant_default(Noverride, dtype);
  // lanes along columns: the smallest power of two >= N, at most 32 (per-task
  // N without an override: 32)
  int lcw = 5;
  if (Noverride > 0) {
    lcw = 0;
    while ((1 << lcw) < Noverride && lcw < 5) ++lcw;
  }
  const int64_t slices = Noverride != 0 ? ((Noverride > 0 ? Noverride : -Noverride) + (1 << lcw) - 1) >> lcw : 1;
  const int gr = (32 >> lcw) * RT;
  // wide variants: 8 (variant 3), 4 (variant 4) or 12 (variant 5) rows per warp
  const int wfr = variant == 4 ? 4 : variant == 5 ? 12 : 8;
  const bool wide_v = variant >= 3 && variant <= 5;
  // staged variants: blocks of 16 (variant 6) or 32 (variant 7) rows per CTA
  const bool staged_v = variant >= 6;
  const int srb = variant == 7 ? 32 : 16;
  const int rgroups = variant == 0 ? (maxM + gr - 1) / gr
                      : wide_v     ? (maxM + wfr - 1) / wfr
                      : staged_v   ? (maxM + srb - 1) / srb
                                   : 1;
  const int64_t wslices = Noverride != 0 ? ((Noverride > 0 ? Noverride : -Noverride) + 63) / 64 : 1;
  const int64_t warps = (int64_t)ntasks * (wide_v || staged_v ? wslices : slices) * rgroups;
  if (warps >= ((int64_t)1 << 31)) return fail(BF_EINVAL, "stage launch too large");
  int64_t blocks = staged_v ? warps : (warps + WARPS - 1) / WARPS;   // staged: one CTA per item
  if (blocks > 152 * 32) blocks = 152 * 32;
  // launch with a programmatic dependency on the previous kernel when asked
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(THREADS);
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  note_launch();
  cudaError_t e = cudaSuccess;
  if (variant == 0) {
    cfg.dynamicSmemBytes = 0;
    e = dtype == BF_C128
            ? cudaLaunchKernelEx(&cfg, stage_mlp_kernel<double>, d_tasks, ntasks, bases, Noverride, lcw, rgroups)
            : cudaLaunchKernelEx(&cfg, stage_mlp_kernel<float>, d_tasks, ntasks, bases, Noverride, lcw, rgroups);
  } else if (wide_v) {
    cfg.dynamicSmemBytes = 0;
    auto wide = [&](auto kd, auto kf) {
      return dtype == BF_C128 ? cudaLaunchKernelEx(&cfg, kd, d_tasks, ntasks, bases, Noverride, rgroups)
                              : cudaLaunchKernelEx(&cfg, kf, d_tasks, ntasks, bases, Noverride, rgroups);
    };
    switch (wfr) {
      case 4: e = wide(stage_wide_kernel<double, 4>, stage_wide_kernel<float, 4>); break;
      case 12: e = wide(stage_wide_kernel<double, 12>, stage_wide_kernel<float, 12>); break;
      default: e = wide(stage_wide_kernel<double, 8>, stage_wide_kernel<float, 8>); break;
    }
  } else if (staged_v) {
    auto staged = [&](auto kd, auto kf, size_t smd, size_t smf) {
      cfg.dynamicSmemBytes = dtype == BF_C128 ? smd : smf;
      return dtype == BF_C128 ? cudaLaunchKernelEx(&cfg, kd, d_tasks, ntasks, bases, Noverride, rgroups)
                              : cudaLaunchKernelEx(&cfg, kf, d_tasks, ntasks, bases, Noverride, rgroups);
    };
    e = variant == 7 ? staged(stage_staged_kernel<double, 4>, stage_staged_kernel<float, 4>,
                              staged_smem<double2, 4>(), staged_smem<float2, 4>())
                     : staged(stage_staged_kernel<double, 2>, stage_staged_kernel<float, 2>,
                              staged_smem<double2, 2>(), staged_smem<float2, 2>());
  } else if (variant == 1) {
    cfg.dynamicSmemBytes = 0;
    e = dtype == BF_C128 ? cudaLaunchKernelEx(&cfg, stage_rows_kernel<double>, d_tasks, ntasks, bases, Noverride, lcw)
                         : cudaLaunchKernelEx(&cfg, stage_rows_kernel<float>, d_tasks, ntasks, bases, Noverride, lcw);
  } else if (dtype == BF_C128) {
    constexpr size_t sm = block_smem<double>();
    BF_CUDA_TRY(cudaFuncSetAttribute(stage_block_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    cfg.dynamicSmemBytes = sm;
    e = cudaLaunchKernelEx(&cfg, stage_block_kernel<double>, d_tasks, ntasks, bases, Noverride, lcw);
  } else {
    constexpr size_t sm = block_smem<float>();
    BF_CUDA_TRY(cudaFuncSetAttribute(stage_block_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    cfg.dynamicSmemBytes = sm;
    e = cudaLaunchKernelEx(&cfg, stage_block_kernel<float>, d_tasks, ntasks, bases, Noverride, lcw);
  }
  if (e != cudaSuccess) return fail(BF_ECUDA, std::string("stage launch: ") + cudaGetErrorString(e));
  BF_CUDA_TRY(cudaGetLastError());
  return BF_OK;
}

}  // namespace bf
