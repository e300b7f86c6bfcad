// Mixed-precision sketch products on the 5th-generation tensor cores
// (tcgen05) with split-precision operands:
//   Y[:, g*k + c] = sum_{j in rows_g} A[:, j] X[j, c]   (or the adjoint form)
// for the built-in operators (Alg. 2 input, structured sketches of Sec. 4.1),
// computed as one real GEMM per 128-row tile:
//   [Yr | Yi] = [Ar | Ai] * [[Xr, Xi], [-Xi, Xr]].
// Operands are split into parts a = a0 + a1 (+ a2) and the products kept
// down to the FP32 level:
//   SPLIT 3 (default, kind::f16 with bf16 parts): the split is exact (8 + 8
//     + 8 significant bits); a0 b0 + a0 b1 + a1 b0 + a0 b2 + a1 b1 + a2 b0,
//     the dropped terms below 2^-24 |a b|;
//   SPLIT 2 (3xTF32, kind::tf32): a0 b0 + a0 b1 + a1 b0 (~2^-21 relative).
//
// Per CTA (one job, one group, 128 rows, one K range, all 2k real columns),
// K advances in chunks of 16 complex columns through an S-stage ring in
// shared memory, with one CTA barrier per chunk:
//   * every thread forms one row's entries for one or two 16-byte
//     core-matrix rows of the chunk (8 bf16 or 4 TF32 values each; the
//     float-float formulas of kentry.cuh on column points staged in shared
//     memory, or loads of a stored complex64 A), splits them and writes each
//     part with one 16-byte store into the K-major, no-swizzle core-matrix
//     layout (8 rows x 16 B per core matrix; 8 lanes fill one core matrix,
//     so stores are free of bank conflicts);
//   * the B operand [[Xr, Xi], [-Xi, Xr]] of the chunk is built from X rows
//     staged by cp.async two chunks ahead (column stride padded by 16 B so
//     the 16-byte loads of 8 lanes hit distinct banks);
//   * one thread waits (bounded) for the MMAs of chunk c-S+1, then after the
//     barrier issues this chunk's tcgen05.mma (M = 128, N = 2k, 32 bytes of
//     K each) and commits them to the stage's mbarrier; the a0*b0 products
//     accumulate in one of two tensor-memory main accumulators, the cross
//     terms (~2^-8 smaller or less) in a correction accumulator over the
//     whole K range;
//   * every 64 complex K the warps move the resting main accumulator into a
//     (hi, lo) pair kept in tensor memory with Knuth's TwoSum (so sums over
//     n = 16384 points keep FP32 accuracy) while the other accumulates; the
//     correction accumulator is added to lo once, at the end;
//   * launches with few row tiles split K across CTAs (decided per job);
//     partial (hi, lo) sums go to a workspace and a second kernel adds them
//     with TwoSum;
//   * a wait that exceeds 1 s of %globaltimer records a device flag
//     (reported as BF_ETIMEOUT), frees the tensor memory and returns.
#include <algorithm>

#include "bf_internal.h"
#include "cx.cuh"
#include "kentry.cuh"

namespace bf {

using namespace dev;

__device__ int g_tc_status;   // 1 once a bounded wait has given up
// limit of every bounded wait (1 s; lowered only by the wait probe below)
__device__ unsigned long long g_wait_limit_ns = 1000000000ull;

namespace {
constexpr int TM = 128;            // rows per CTA (MMA M)
constexpr int NWARP = 8;           // producer warps (entries, B operand, staging, drains)
constexpr int ISSUER_WARP = 0;     // 1: a ninth warp waits for and issues the MMAs; 0: thread 0 does
constexpr int THREADS = 32 * (NWARP + ISSUER_WARP);
constexpr int XS = 2;              // buffers of staged X rows and points (prefetch depth)
constexpr uint32_t CORE = 128;     // bytes of one 8 x 16 B core matrix
constexpr int NR_MAX = 96;         // widest tile: 48 complex columns

// entry kinds of a job
constexpr int EK_DENSE = 0, EK_H2D = 1, EK_H3D = 2, EK_DFT = 3;
__device__ __forceinline__ int point_arrays(int ek) { return ek == EK_H3D ? 6 : ek == EK_H2D ? 4 : ek == EK_DFT ? 2 : 0; }

struct TcTile {
  int32_t job, group;          // group of the output (segment 0)
  int64_t row0;
  int64_t k0, k1;              // K range of this CTA
  int64_t ws;                  // float4 offset of this (job, group, split) partial, or -1
  int64_t g1, ws1;             // the same for segment 1 of a two-level job
};
struct TcRegion {              // one (job, group) region to reduce
  int64_t ws, M, kcols, ldy, ycol0;
  int32_t nsplit, pad;
  float2* Y;
};

// tensor-memory columns: two main accumulators [0, NR) and [NR, 2NR) (the
// a0*b0 products of alternate groups of DR chunks, so one is drained while
// the other accumulates), the correction accumulator [2NR, 3NR) (the cross
// terms, ~2^-11 smaller, so their roundings do not reach the total), and
// the TwoSum pair hi [3NR, 4NR), lo [4NR, 5NR); a power of two with 16
// spare columns for the epilogue's last 16-column slice (it may pass the
// end of lo by 8)
__host__ __device__ constexpr int tmem_cols(int nr) {
  return 5 * nr + 16 <= 32 ? 32 : 5 * nr + 16 <= 64 ? 64 : 5 * nr + 16 <= 128 ? 128 : 5 * nr + 16 <= 256 ? 256 : 512;
}
static_assert(5 * NR_MAX + 16 <= 512, "accumulators of the widest tile fit in tensor memory");

// Shape of one tile configuration: K advances in chunks of KCH = 16 complex
// columns, operands in bf16 parts (three-way split) or TF32 parts (3xTF32);
// S stages of the A
// and B operands (the MMAs of a chunk may run while the next S-1 chunks are
// formed); XS buffers of staged X rows and column points.  Shared memory
// in byte offsets.
template <int NR, int SPLIT>
struct Cfg {
  static constexpr int EB = SPLIT == 3 ? 2 : 4;   // operand bytes: bf16 parts (exact split) or TF32 parts
  static constexpr int VS = 16 / EB;              // values per 16-byte core-matrix row
  static constexpr int KCH = 16;
  static constexpr int KR = 2 * KCH;           // real K per chunk: real parts of A, then imaginary parts
  static constexpr int KG = KR * EB / 16;      // core matrices along K
  static constexpr int G = KCH / VS;           // groups of VS columns per chunk (real or imaginary part)
  static constexpr int PT = G / 2;             // groups per thread per chunk
  static constexpr int KSTEPS = KR * EB / 32;  // MMAs along K per chunk (32 bytes of K each)
  static constexpr int DR = 64 / KCH;          // chunks between drains of a main accumulator (64 complex K)
  static constexpr int KP = NR / 2;
  static constexpr bool TWO = tmem_cols(NR) <= 256;   // two CTAs per SM fit in tensor memory
  static constexpr uint32_t XCOL = KCH * 8 + 16;      // bytes per staged X column (16 B pad)
  static constexpr uint32_t A_PART = TM * KR * EB, A_BUF = SPLIT * A_PART;
  static constexpr uint32_t B_PART = NR * KR * EB, B_BUF = SPLIT * B_PART;
  static constexpr uint32_t X_BUF = KP * XCOL, P_BUF = 6 * KCH * 4;
  static constexpr uint32_t LIMIT = TWO ? 112 * 1024 : 226 * 1024;   // per CTA, static part aside
  static constexpr uint32_t total(int s) { return s * (A_BUF + B_BUF) + XS * (X_BUF + P_BUF); }
  static constexpr int S = total(4) <= LIMIT ? 4 : total(3) <= LIMIT ? 3 : 2;
  static constexpr uint32_t A0 = 0, B0 = S * A_BUF, X0 = B0 + S * B_BUF, P0 = X0 + XS * X_BUF;
  static constexpr uint32_t TOTAL = P0 + XS * P_BUF;
  // one CTA per SM for wide tiles (their tensor memory is the SM's)
  static constexpr uint32_t LAUNCH_SMEM = TWO ? TOTAL : (TOTAL > 120 * 1024 ? TOTAL : 120 * 1024);
  static constexpr int IW = NR * KG / NWARP;   // B items per warp
  static constexpr int BIT = (IW + 31) / 32;
  static constexpr int XW = KP * KCH / NWARP;  // X copies per warp
  static constexpr int XIT = (XW + 31) / 32;
  static_assert(TOTAL <= LIMIT, "tile exceeds shared memory");
  static_assert(IW % 8 == 0 && S - 2 < DR, "B items by 8-lane groups; drains before reuse");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, LBO (K-adjacent core matrices),
// SBO (8-row groups), in 16-byte units; version 1 at bits 46-47; no swizzle
template <int KG>
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  constexpr uint32_t SBO = KG * CORE;
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((CORE >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((SBO >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor: D FP32 (bits 4-5 = 1), A and B TF32 (bits 7-9 and
// 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}
// the same for kind::f16 with bf16 A and B (type 1)
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// two floats -> bf16x2 (round to nearest even; x0 in the low half)
__device__ __forceinline__ uint32_t bf16x2_rn(float x0, float x1) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(x1), "f"(x0));
  return r;
}

// Operand parts of one 16-byte core-matrix row.
// SPLIT 2 (4 values, TF32): round-to-nearest parts, x - p0 - p1 ~ 2^-22 |x|.
// SPLIT 3 (8 values, bf16): x = p0 + p1 + p2 exactly -- each part rounds the
// remainder to 8 significant bits (x has 24; x - p0 has at most 16, its
// remainder at most 8), so the six products kept (i + j <= 2) miss only
// terms below 2^-24 |x y|.
template <int SPLIT, int V>
__device__ __forceinline__ void split_row(const float (&x)[V], uint4 (&p)[3]) {
  uint32_t a[4], b[4], c[4];
  if (SPLIT == 3) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      a[i] = bf16x2_rn(x[2 * i], x[2 * i + 1]);
      const float r0 = x[2 * i] - __uint_as_float(a[i] << 16), r1 = x[2 * i + 1] - __uint_as_float(a[i] & 0xFFFF0000u);
      b[i] = bf16x2_rn(r0, r1);
      c[i] = bf16x2_rn(r0 - __uint_as_float(b[i] << 16), r1 - __uint_as_float(b[i] & 0xFFFF0000u));
    }
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      a[j] = tf32_rna(x[j]);
      b[j] = tf32_rna(x[j] - __uint_as_float(a[j]));
      c[j] = 0u;
    }
  }
  p[0] = make_uint4(a[0], a[1], a[2], a[3]);
  p[1] = make_uint4(b[0], b[1], b[2], b[3]);
  p[2] = make_uint4(c[0], c[1], c[2], c[3]);
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint4 v) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}
__device__ __forceinline__ float4 ld_shared_v4(uint32_t addr) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr)
               : "memory");
  return v;
}

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_try(uint32_t addr, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(addr), "r"(parity)
      : "memory");
  return done != 0;
}
// the same, the thread suspended until the phase completes or about `ns`
// nanoseconds have passed (so a waiting warp takes no issue slots from the
// warps that share its scheduler)
__device__ __forceinline__ bool mbar_try_sleep(uint32_t addr, uint32_t parity, uint32_t ns) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(addr), "r"(parity), "r"(ns)
      : "memory");
  return done != 0;
}
// the bounded part of a wait, out of line so that the inlined fast path is
// one try_wait: false after g_wait_limit_ns (1 s), or as soon as *abort is set
__device__ __noinline__ bool mbar_wait_slow(uint32_t addr, uint32_t parity, const volatile int* abort) {
  const uint64_t t0 = now_ns();
  const uint64_t limit = *(const volatile unsigned long long*)&g_wait_limit_ns;
  for (;;) {
    if (mbar_try_sleep(addr, parity, 1000000u)) return true;
    if ((abort && *abort) || now_ns() - t0 > limit) return false;
  }
}
// waits for the phase of parity `parity` of the mbarrier at addr; the timer
// is read only once the phase is found incomplete; false after 1 s (or once
// *abort is set)
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity, const volatile int* abort = nullptr) {
  return mbar_try(addr, parity) || mbar_wait_slow(addr, parity, abort);
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// one MMA step: kind::tf32 for 4-byte operands, kind::f16 (bf16 A and B)
// for 2-byte ones
template <int EB>
__device__ __forceinline__ void mma_step(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if (EB == 2)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
            dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(
            dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// bytes (a multiple of 16, both addresses 16-byte aligned) from global memory
// into shared memory by the bulk-copy engine, completing on mbarrier bar
// (whose expected transaction count must cover them), with an L2
// eviction-priority policy (l2_evict_first / l2_evict_last)
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar), "l"(policy)
      : "memory");
}
// L2 policies: evict_first for data read once (entry images), evict_last
// for data every row tile re-reads (the per-launch B operand)
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// arrive on bar, adding `bytes` to its expected transaction count
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

}  // namespace

// This thread's row of the tile: its point (float-float, in registers), the
// wavenumber, the sign of imaginary parts (exp(-i k r) in 2D; conjugation
// for the adjoint) and, for stored operators, the matrix.
struct RowCtx {
  float rp[6];
  float kh, kl, isg;
  unsigned neg;   // sign bit when imaginary parts are negated (isg < 0)
  const float2* A;
  int64_t lda;
  int opN;
};

// entry kind of a job's formula (stored matrix or built-in kernel)
__device__ __forceinline__ int formula_kind(const SketchJob& J) {
  return J.kind == 0 ? EK_DENSE
         : J.ktype == BF_KERNEL_HELMHOLTZ_2D ? EK_H2D
         : J.ktype == BF_KERNEL_HELMHOLTZ_3D ? EK_H3D
                                             : EK_DFT;
}

__device__ __forceinline__ void row_ctx(const SketchJob& J, int ek, int64_t gi, bool rvalid, RowCtx& R) {
  const int opN = J.op == BF_OP_N;
  const int npt = point_arrays(ek);
  const float* rowp = opN ? J.tgtF : J.srcF;
  const int64_t rown = opN ? J.m : J.n;
#pragma unroll
  for (int d = 0; d < 6; ++d) R.rp[d] = (d < npt && rvalid) ? rowp[d * rown + gi] : 0.f;
  R.kh = J.kh;
  R.kl = J.kl;
  R.opN = opN;
  R.A = (const float2*)J.A;
  R.lda = J.lda;
  // imaginary sign: exp(-i k r) in 2D, then conjugation for the adjoint
  const float base = ek == EK_H2D ? -1.f : 1.f;
  R.isg = opN ? base : -base;
  R.neg = R.isg < 0.f ? 0x80000000u : 0u;
}

// Four entries of row gi at columns gk0 .. gk0+3 (kernel entries use the
// chunk's column points staged at pts: array d at pts + ps d bytes).
// Columns at or past kend are not read (their entries are zeroed by the caller).
__device__ __forceinline__ void form4(int ek, const RowCtx& R, uint32_t pts, uint32_t ps, int64_t gi,
                                      int64_t gk0, int64_t kend, float* re, float* im) {
  if (ek == EK_DENSE) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gk = gk0 + j < kend ? gk0 + j : kend - 1;
      const float2 v = R.opN ? R.A[gi + gk * R.lda] : R.A[gk + gi * R.lda];
      re[j] = v.x;
      im[j] = v.y * R.isg;
    }
    return;
  }
  const float4 xh = ld_shared_v4(pts), xl = ld_shared_v4(pts + ps);
  const float cxh[4] = {xh.x, xh.y, xh.z, xh.w}, cxl[4] = {xl.x, xl.y, xl.z, xl.w};
  if (ek == EK_DFT) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float2 v = dft_ff(R.rp[0], R.rp[1], cxh[j], cxl[j]);
      re[j] = v.x;
      im[j] = v.y * R.isg;
    }
    return;
  }
  const float4 yh = ld_shared_v4(pts + 2 * ps), yl = ld_shared_v4(pts + 3 * ps);
  const float cyh[4] = {yh.x, yh.y, yh.z, yh.w}, cyl[4] = {yl.x, yl.y, yl.z, yl.w};
  if (ek == EK_H2D) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float2 v = helmholtz_ff<false>(R.rp, cxh[j], cxl[j], cyh[j], cyl[j], 0.f, 0.f, R.kh, R.kl, R.neg);
      re[j] = v.x;
      im[j] = v.y;
    }
    return;
  }
  const float4 zh = ld_shared_v4(pts + 4 * ps), zl = ld_shared_v4(pts + 5 * ps);
  const float czh[4] = {zh.x, zh.y, zh.z, zh.w}, czl[4] = {zl.x, zl.y, zl.z, zl.w};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float2 v = helmholtz_ff<true>(R.rp, cxh[j], cxl[j], cyh[j], cyl[j], czh[j], czl[j], R.kh, R.kl, R.neg);
    re[j] = v.x;
    im[j] = v.y;
  }
}

// V (4 or 8) entries of row gi at columns gk0 .. gk0+V-1, four at a time.
template <int V>
__device__ __forceinline__ void form_row(int ek, const RowCtx& R, uint32_t pts, uint32_t ps, int64_t gi,
                                         int64_t gk0, int64_t kend, float (&re)[V], float (&im)[V]) {
#pragma unroll
  for (int h = 0; h < V / 4; ++h) form4(ek, R, pts + 16u * h, ps, gi, gk0 + 4 * h, kend, re + 4 * h, im + 4 * h);
}

// TwoSum the main accumulator at column moff into the pair (hi, lo) (and,
// at the end, add the correction accumulator to lo) for this warp's 32
// tensor-memory lanes; the warps sharing a lane quadrant take alternate
// 16-column slices.
template <int NR, bool CORR>
__device__ __forceinline__ void drain(uint32_t tq, int sub, uint32_t moff) {
#pragma unroll 1
  for (int s = sub; s < NR / 16; s += NWARP / 4) {
    uint32_t d[16], h[16], l[16], e[16];
    tmem_ld16(tq + moff + s * 16, d);
    tmem_ld16(tq + 3 * NR + s * 16, h);
    tmem_ld16(tq + 4 * NR + s * 16, l);
    if (CORR) tmem_ld16(tq + 2 * NR + s * 16, e);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const FF t = two_sum(__uint_as_float(h[i]), __uint_as_float(d[i]));
      h[i] = __float_as_uint(t.h);
      const float add = CORR ? t.l + __uint_as_float(e[i]) : t.l;
      l[i] = __float_as_uint(__uint_as_float(l[i]) + add);
    }
    tmem_st16(tq + 3 * NR + s * 16, h);
    tmem_st16(tq + 4 * NR + s * 16, l);
  }
  tmem_wait_st();
}

template <int NR, int SPLIT>
__global__ void __launch_bounds__(THREADS, 2)
sketch_tc_kernel(const SketchJob* __restrict__ jobs, const TcTile* __restrict__ tiles, float4* __restrict__ ws) {
  using C = Cfg<NR, SPLIT>;
  constexpr int S = C::S, KCH = C::KCH, KG = C::KG, G = C::G, DR = C::DR, KP = C::KP, VS = C::VS;
  constexpr int COLS = tmem_cols(NR);
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ SketchJob J;
  __shared__ TcTile T;
  __shared__ __align__(8) uint64_t mbar[S];   // MMA completion of chunks c with c % S = s
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    T = tiles[blockIdx.x];
    J = jobs[T.job];
    for (int s = 0; s < S; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[s])), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tm = tmem_slot;
  // tensor memory: warp w reaches lanes 32 (w % 4) .. + 31; the two warps of
  // a lane quadrant share its column slices
  const bool producer = warp < NWARP, issuer = tid == 32 * NWARP * ISSUER_WARP;
  const int quad = warp & 3, sub = warp >> 2;
  const uint32_t tq = tm + ((uint32_t)(quad * 32) << 16);
  if (producer) {
    uint32_t z[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) z[i] = 0u;
#pragma unroll 1
    for (int s = sub; s < 2 * NR / 16; s += 2) tmem_st16(tq + 3 * NR + s * 16, z);
    tmem_wait_st();
  }

  const int64_t row0 = T.row0, M = J.M, kcols = J.kcols, ygs = J.ygs;
  // K range: this CTA's split, or the whole group
  const int64_t k0 = T.k0 >= 0 ? T.k0 : (J.d_off ? J.d_off[T.group] : 0);
  const int64_t k1 = T.k0 >= 0 ? T.k1 : (J.d_off ? J.d_off[T.group + 1] : J.Ktot);
  const float2* __restrict__ X = (const float2*)J.X;
  const int64_t ldx = J.ldx;
  const int nch = (int)((k1 - k0 + KCH - 1) / KCH);
  const uint32_t sb = smem_u32(smem);

  // entry kind and this thread's row context
  const int opN = J.op == BF_OP_N;
  const int ek = formula_kind(J);
  const int npt = point_arrays(ek);
  // producer mapping: warp w forms rows 16w .. 16w+15; each 8-lane group
  // fills one core matrix (8 rows x 4 columns) per store; a thread's groups
  // of 4 columns are kg0, kg0 + 2, ...
  const int prow = 16 * warp + (lane & 7) + 8 * ((lane >> 4) & 1), kg0 = (lane >> 3) & 1;
  const int64_t gi = row0 + prow;
  const bool rvalid = producer && gi < M;
  const uint32_t a_st = (uint32_t)(prow >> 3) * KG * CORE + (uint32_t)(prow & 7) * 16;
  RowCtx R;
  row_ctx(J, ek, gi, rvalid, R);
  const float* colp = opN ? J.srcF : J.tgtF;
  const int64_t coln = opN ? J.n : J.m;

  // B operand items of this thread: item (nr, kg) = 4 consecutive K of row
  // nr; packed as B offset | X offset << 16 | (reads imaginary parts) << 30
  // | (negated) << 31; all-ones for none
  uint32_t bdesc[C::BIT];
#pragma unroll
  for (int q = 0; q < C::BIT; ++q) {
    const int li = lane + 32 * q, it = warp * C::IW + li;
    const int nr = ((it / (8 * KG)) << 3) | (it & 7), kg = (it >> 3) & (KG - 1);
    const int part = kg >= G ? 1 : 0;          // 0: rows of Ar, 1: rows of Ai
    const int kk0 = (kg & (G - 1)) * VS;
    const int col = nr % KP, blk = nr / KP;    // blk 0: a column of Yr, 1: of Yi
    // B = [[Xr, Xi], [-Xi, Xr]]: (part, blk) = (0,0) Xr, (0,1) Xi, (1,0) -Xi, (1,1) Xr
    const uint32_t im = (uint32_t)((part ^ blk) & 1), neg = (part == 1 && blk == 0) ? 1u : 0u;
    const uint32_t o = (uint32_t)(nr >> 3) * KG * CORE + (uint32_t)kg * CORE + (uint32_t)(nr & 7) * 16;
    const uint32_t xo = (uint32_t)col * C::XCOL + (uint32_t)kk0 * 8;
    bdesc[q] = li < C::IW ? (o | (xo << 16) | (im << 30) | (neg << 31)) : 0xFFFFFFFFu;
  }

  // rows kb .. kb+KCH-1 of X (columns < KP, zero filled) and of the column
  // point arrays into buffer c % XS; one cp.async group per chunk (empty
  // past the end), so that waiting for all but the newest XS-2 groups
  // completes the next chunk
  auto stage = [&](int c) {
    if (!producer || c >= nch) {
      cp_async_commit();
      return;
    }
    const int64_t kb = k0 + (int64_t)c * KCH;
    const uint32_t xb = sb + C::X0 + (uint32_t)(c % XS) * C::X_BUF;
#pragma unroll
    for (int q = 0; q < C::XIT; ++q) {
      const int li = lane + 32 * q;
      if (li >= C::XW) break;
      const int x = warp * C::XW + li, col = x / KCH, kk = x % KCH;
      const int64_t gk = kb + kk;
      const bool v = gk < k1 && col < kcols;
      cp_async8(xb + (uint32_t)col * C::XCOL + (uint32_t)kk * 8,
                v ? (const void*)(X + gk + (int64_t)col * ldx) : (const void*)X, v);
    }
    const int pidx = lane * NWARP + warp;
    if (pidx < npt * KCH) {
      const uint32_t pb = sb + C::P0 + (uint32_t)(c % XS) * C::P_BUF;
      const int d = pidx / KCH, kk = pidx % KCH;
      const int64_t gk = kb + kk;
      const bool v = gk < k1;
      cp_async4(pb + (uint32_t)(d * KCH + kk) * 4, v ? (const void*)(colp + d * coln + gk) : (const void*)colp, v);
    }
    cp_async_commit();
  };

  const uint32_t mb0 = smem_u32(&mbar[0]);   // mbar[s] at mb0 + 8 s
  constexpr uint32_t idesc = C::EB == 2 ? idesc_bf16(NR) : idesc_tf32(NR);
  uint32_t mph = 0;    // bit s: parity of the next phase of mbar[s] to wait for
  bool ok = true;
  int drained = 0;     // groups of DR chunks whose main accumulator is in (hi, lo)
  int issued = -1;     // last chunk whose MMAs were issued
#pragma unroll
  for (int c = 0; c < XS; ++c) stage(c);
  cp_async_wait<XS - 1>();
  __syncthreads();
  for (int c = 0; c < nch; ++c) {
    const uint32_t s = (uint32_t)(c % S), xbuf = (uint32_t)(c % XS);
    const int64_t kb = k0 + (int64_t)c * KCH;
    const uint32_t aB = sb + C::A0 + s * C::A_BUF, bB = sb + C::B0 + s * C::B_BUF;
    // 1. entries of chunk c into A[s] (its last reader, the MMAs of chunk
    //    c-S, completed before the previous barrier)
#pragma unroll
    for (int r = 0; r < C::PT; ++r) {
      if (!producer) break;
      const int kg = kg0 + 2 * r;
      float re[VS], im[VS];
      const int64_t gk0 = kb + VS * kg;
      form_row<VS>(ek, R, sb + C::P0 + xbuf * C::P_BUF + 4u * VS * (uint32_t)kg, KCH * 4, rvalid ? gi : row0, gk0,
                   k1, re, im);
      if (kb + KCH > k1) {   // ragged last chunk: columns past k1 are zero
#pragma unroll
        for (int j = 0; j < VS; ++j)
          if (gk0 + j >= k1) re[j] = 0.f, im[j] = 0.f;
      }
      uint4 pr[3], pm[3];
      split_row<SPLIT, VS>(re, pr);
      split_row<SPLIT, VS>(im, pm);
      const uint32_t ar = aB + a_st + (uint32_t)kg * CORE, ai = ar + (uint32_t)G * CORE;
#pragma unroll
      for (int q = 0; q < SPLIT; ++q) {
        st_shared_v4(ar + q * C::A_PART, pr[q]);
        st_shared_v4(ai + q * C::A_PART, pm[q]);
      }
    }
    // 2. B = [[Xr, Xi], [-Xi, Xr]] (N x K, K-major) of chunk c into B[s]
    {
      const uint32_t xb = sb + C::X0 + xbuf * C::X_BUF;
#pragma unroll
      for (int q = 0; q < C::BIT; ++q) {
        const uint32_t d = bdesc[q];
        if (!producer || d == 0xFFFFFFFFu) continue;
        const uint32_t xa = xb + ((d >> 16) & 0x3FFFu);
        const bool im = (d >> 30) & 1u;
        const uint32_t neg = d & 0x80000000u;
        float v[VS];
#pragma unroll
        for (int h = 0; h < VS / 2; ++h) {   // two complex X values per 16-byte load
          const float4 u = ld_shared_v4(xa + 16u * h);
          v[2 * h] = __uint_as_float(__float_as_uint(im ? u.y : u.x) ^ neg);
          v[2 * h + 1] = __uint_as_float(__float_as_uint(im ? u.w : u.z) ^ neg);
        }
        uint4 pv[3];
        split_row<SPLIT, VS>(v, pv);
#pragma unroll
        for (int p = 0; p < SPLIT; ++p) st_shared_v4(bB + p * C::B_PART + (d & 0xFFFFu), pv[p]);
      }
    }
    // 3. this thread's copies of chunk c+1 have landed
    cp_async_wait<XS - 2>();
    // 4. the MMAs of chunk c-S+1 have completed (chunk c+1 rewrites its A and B)
    const int cw = c - S + 1;
    bool gave_up = false;
    if (cw >= 0 && issuer) {
      const uint32_t sw = (uint32_t)(cw % S);
      gave_up = !mbar_wait(mb0 + 8u * sw, (mph >> sw) & 1u);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    if (__syncthreads_or(gave_up)) {
      ok = false;
      break;
    }
    if (cw >= 0) mph ^= 1u << (cw % S);
    tc_fence_after();
    // 5. a group of DR chunks whose MMAs have all completed moves into
    //    (hi, lo) while the other main accumulator takes the next group; it
    //    is drained before the MMAs of the group after next reuse it
    if (cw >= 0 && (drained + 1) * DR - 1 <= cw) {
      if (producer) drain<NR, false>(tq, sub, (uint32_t)(drained & 1) * NR);
      ++drained;
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
    }
    // 6. stage chunk c+XS into the X / point buffers chunk c has finished reading
    stage(c + XS);
    // 7. the issuing thread issues the chunk's MMAs and commits them to mbar[s]
    if (issuer) {
      // descriptors advance by (byte offset >> 4) in their start-address field
      const uint64_t dA = sdesc<KG>(aB), dB = sdesc<KG>(bB);
      constexpr uint64_t pa = C::A_PART >> 4, pb = C::B_PART >> 4;
      const uint32_t tmain = tm + (uint32_t)((c / DR) & 1) * NR, tcorr = tm + 2 * NR;
      const uint32_t carry = (c % DR) != 0 ? 1u : 0u;   // a main accumulator restarts with its group
      const uint32_t cacc = c > 0 ? 1u : 0u;             // the correction runs over all K
      constexpr int EB = C::EB;
#pragma unroll
      for (int ks = 0; ks < C::KSTEPS; ++ks) {
        const uint64_t o = (uint64_t)(ks * 2 * CORE) >> 4;
        mma_step<EB>(tmain, dA + o, dB + o, idesc, ks > 0 ? 1u : carry);           // a0 b0 -> main
        mma_step<EB>(tcorr, dA + o, dB + pb + o, idesc, ks > 0 ? 1u : cacc);       // cross terms -> correction
        mma_step<EB>(tcorr, dA + pa + o, dB + o, idesc, 1u);
        if (SPLIT == 3) {
          mma_step<EB>(tcorr, dA + o, dB + 2 * pb + o, idesc, 1u);
          mma_step<EB>(tcorr, dA + pa + o, dB + pb + o, idesc, 1u);
          mma_step<EB>(tcorr, dA + 2 * pa + o, dB + o, idesc, 1u);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       mb0 + 8u * s)
                   : "memory");
    }
    issued = c;
  }
  if (ok && nch > 0) {
    bool gave_up = false;
    if (issuer) {
      const uint32_t sl = (uint32_t)((nch - 1) % S);
      gave_up = !mbar_wait(mb0 + 8u * sl, (mph >> sl) & 1u);
    }
    if (__syncthreads_or(gave_up)) {
      ok = false;
    } else {
      tc_fence_after();
      const int ngroups = (nch + DR - 1) / DR;
      for (; drained < ngroups && producer; ++drained) {
        if (drained + 1 < ngroups)
          drain<NR, false>(tq, sub, (uint32_t)(drained & 1) * NR);
        else
          drain<NR, true>(tq, sub, (uint32_t)(drained & 1) * NR);
      }
    }
  }
  cp_async_wait_all();
  if (!ok) {
    if (issuer) {
      atomicExch(&g_tc_status, 1);
      if (issued >= 0) {   // bounded chance for the MMAs in flight
        const uint32_t sl = (uint32_t)(issued % S);
        mbar_wait(mb0 + 8u * sl, (mph >> sl) & 1u);
      }
    }
    __syncthreads();
  } else {
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const int64_t row = row0 + quad * 32 + lane;
#pragma unroll 1
    for (int s = sub; s < (KP + 15) / 16 && producer; s += NWARP / 4) {
      uint32_t hr[16], lr[16], hm[16], lm[16];
      // columns beyond KP read allocated but unused tensor memory; skipped below
      const int c0 = s * 16;
      tmem_ld16(tq + 3 * NR + c0, hr);
      tmem_ld16(tq + 4 * NR + c0, lr);
      tmem_ld16(tq + 3 * NR + KP + c0, hm);
      tmem_ld16(tq + 4 * NR + KP + c0, lm);
      tmem_wait_ld();
      if (row < M) {
        const int64_t kc0 = J.nseg == 2 ? J.kcols0 : kcols;   // columns of segment 0
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int col = c0 + i;
          if (col >= kcols || col >= KP) continue;
          const bool s1 = col >= kc0;
          const int64_t cl = s1 ? col - kc0 : col, wsx = s1 ? T.ws1 : T.ws;
          if (wsx < 0) {
            float2* __restrict__ Y = (float2*)(s1 ? J.Y1 : J.Y);
            const int64_t g = s1 ? T.g1 : T.group, gs = s1 ? J.ygs1 : ygs, ld = s1 ? J.ldy1 : J.ldy;
            Y[row + (g * gs + cl) * ld] = make_float2(__uint_as_float(hr[i]) + __uint_as_float(lr[i]),
                                                       __uint_as_float(hm[i]) + __uint_as_float(lm[i]));
          } else {
            ws[wsx + cl * M + row] = make_float4(__uint_as_float(hr[i]), __uint_as_float(lr[i]),
                                                 __uint_as_float(hm[i]), __uint_as_float(lm[i]));
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(COLS) : "memory");
  }
}

// Y = sum over splits of the partial (hi, lo) pairs, TwoSum in FP32.
__global__ void tc_reduce_kernel(const TcRegion* __restrict__ regs, int nreg, const float4* __restrict__ ws) {
  const TcRegion R = regs[blockIdx.y];
  const int64_t total = R.M * R.kcols;
  const int64_t stride = R.M * R.kcols;   // float4 entries per split
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = t % R.M, col = t / R.M;
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    for (int s = 0; s < R.nsplit; ++s) {
      const float4 p = ws[R.ws + s * stride + col * R.M + row];
      FF a = two_sum(rh, p.x);
      rh = a.h, rl += a.l + p.y;
      FF b = two_sum(ih, p.z);
      ih = b.h, il += b.l + p.w;
    }
    R.Y[row + (R.ycol0 + col) * R.ldy] = make_float2(rh + rl, ih + il);
  }
}

// ---------------------------------------------------------------------------
// Entry images and the image-fed sketch kernel
// ---------------------------------------------------------------------------
// An entry image holds one orientation of a built-in operator's entries in
// complex64, as the tiles the image-fed sketch kernel consumes: tile
// (row tile rt, 16-column chunk kc) at img + (rt * nchi + kc) * IMG_TILE,
// 128 rows of 128 bytes (16 complex entries, re/im interleaved); the 16-byte
// segment q (2 entries) of row r sits at position q ^ (r & 7) so that the
// eight rows a quarter-warp reads land in distinct bank groups.  Entries are
// those the on-the-fly producers form (same formula, same thread mapping);
// rows past M and columns past K are zero.
constexpr int IMG_CPB = 32;                    // chunks per CTA of the image kernel
constexpr uint32_t IMG_TILE = TM * 16 * 8;     // bytes of one tile

__device__ __forceinline__ uint32_t img_seg(int r, int q) { return (uint32_t)r * 128u + (uint32_t)((q ^ (r & 7)) * 16); }

// Both entry images in one pass (A for op N, A^H for op C): a CTA forms the
// entries of one 128-target tile x IMG_CPB 16-source chunks (the on-the-fly
// producers' formula and thread mapping) and writes them as A's tiles; every 4
// chunks (64 sources) the entries also go through shared memory
// (conflict-free row stride of 129 entries) and come back out transposed
// and conjugated as rows 64 h .. 64 h + 63 of the A^H tiles of those sources
// (the conjugate of A's entry is the op-C formula's value: the distance is
// computed sign-symmetrically).  A^H tiles past the m targets are skipped.
constexpr int IMG_PASS = 4;   // chunks (64 sources) per transpose pass
__global__ void __launch_bounds__(256) entry_images_kernel(const SketchJob J, uint8_t* __restrict__ imgN,
                                                           uint8_t* __restrict__ imgC, int64_t nchN,
                                                           int64_t nchC) {
  using C = Cfg<16, 3>;
  constexpr int KCH = C::KCH, VS = C::VS, LDS = TM + 1;
  __shared__ __align__(16) float pts[IMG_CPB * 6 * KCH];
  extern __shared__ __align__(16) float2 stage[];   // [IMG_PASS * KCH][LDS]: (source, target)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ek = formula_kind(J);
  const int npt = point_arrays(ek);
  const int64_t row0 = (int64_t)blockIdx.x * TM, M = J.M, K = J.Ktot;   // targets, sources
  const int prow = 16 * warp + (lane & 7) + 8 * ((lane >> 4) & 1), kg = (lane >> 3) & 1;
  const int64_t gi = row0 + prow;
  const bool rvalid = gi < M;
  RowCtx R;
  row_ctx(J, ek, gi, rvalid, R);
  const float* colp = J.srcF;
  const int64_t coln = J.n;
  const int64_t c0 = (int64_t)blockIdx.y * IMG_CPB;
  const int nc = (int)(nchN - c0 < IMG_CPB ? nchN - c0 : IMG_CPB);
  for (int idx = tid; idx < nc * npt * KCH; idx += 256) {
    const int c = idx / (npt * KCH), d = (idx / KCH) % npt, kk = idx % KCH;
    const int64_t gk = (c0 + c) * KCH + kk;
    pts[(c * 6 + d) * KCH + kk] = gk < K ? colp[d * coln + gk] : 0.f;
  }
  __syncthreads();
  const uint32_t pb = smem_u32(pts);
#pragma unroll 1
  for (int p0 = 0; p0 < nc; p0 += IMG_PASS) {
    const int np = nc - p0 < IMG_PASS ? nc - p0 : IMG_PASS;
#pragma unroll 1
    for (int c = p0; c < p0 + np; ++c) {
      const int64_t kb = (c0 + c) * KCH;
      float re[VS], im[VS];
      const int64_t gk0 = kb + VS * kg;
      form_row<VS>(ek, R, pb + (uint32_t)(c * 6 * KCH * 4) + 4u * VS * (uint32_t)kg, KCH * 4, rvalid ? gi : row0,
                   gk0, K, re, im);
      if (kb + KCH > K || !rvalid) {
#pragma unroll
        for (int j = 0; j < VS; ++j)
          if (!rvalid || gk0 + j >= K) re[j] = 0.f, im[j] = 0.f;
      }
      uint8_t* tile = imgN + ((int64_t)blockIdx.x * nchN + c0 + c) * IMG_TILE;
#pragma unroll
      for (int t = 0; t < VS / 2; ++t)
        *(float4*)(tile + img_seg(prow, 4 * kg + t)) = make_float4(re[2 * t], im[2 * t], re[2 * t + 1], im[2 * t + 1]);
      const int sl = (c - p0) * KCH + VS * kg;   // this thread's first source of the pass
#pragma unroll
      for (int j = 0; j < VS; ++j) stage[(sl + j) * LDS + prow] = make_float2(re[j], -im[j]);
    }
    __syncthreads();
    // A^H tiles: row = source, 16 targets per chunk; a thread writes 16-byte
    // segments (2 targets), 8 consecutive lanes one 128-byte row
    const int64_t s_first = (c0 + p0) * KCH;   // first source of the pass
    for (int e = tid; e < np * KCH * (TM / 2); e += 256) {
      const int q = e & 7, tc = (e >> 3) & 7, sl = e >> 6;   // segment, target chunk of the tile, source
      const int64_t sg = s_first + sl, kcC = (int64_t)blockIdx.x * (TM / KCH) + tc;
      if (kcC >= nchC) continue;
      const int tl = tc * KCH + 2 * q;   // first target of the segment within the tile
      const float2 a = stage[sl * LDS + tl], b = stage[sl * LDS + tl + 1];
      uint8_t* tile = imgC + ((sg / TM) * nchC + kcC) * IMG_TILE;
      *(float4*)(tile + img_seg((int)(sg % TM), q)) = make_float4(a.x, a.y, b.x, b.y);
    }
    __syncthreads();
  }
}

int launch_entry_images(const SketchJob& jn, void* imgN, void* imgC, cudaStream_t s) {
  if (jn.kind != 1 || jn.op != BF_OP_N || jn.M <= 0 || jn.Ktot <= 0 || !imgN || !imgC)
    return fail(BF_EINVAL, "entry images of a non-kernel job");
  const int64_t nchN = entry_image_chunks(jn.Ktot), nchC = entry_image_chunks(jn.M);
  const dim3 grid((unsigned)((jn.M + TM - 1) / TM), (unsigned)((nchN + IMG_CPB - 1) / IMG_CPB));
  const size_t smem = (size_t)IMG_PASS * 16 * (TM + 1) * sizeof(float2);
  BF_CUDA_TRY(cudaFuncSetAttribute(entry_images_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  note_launch();
  entry_images_kernel<<<grid, 256, smem, s>>>(jn, (uint8_t*)imgN, (uint8_t*)imgC, nchN, nchC);
  BF_CUDA_TRY(cudaGetLastError());
  return BF_OK;
}

size_t entry_image_bytes(int64_t M, int64_t K) {
  return (size_t)((M + TM - 1) / TM) * (size_t)entry_image_chunks(K) * IMG_TILE;
}
int64_t entry_image_chunks(int64_t K) { return (K + 15) / 16; }

bool entry_image_fits(const SketchJob& j) {
  constexpr int64_t KCH = 16;
  if (j.split != 3 || j.nseg == 2 || j.kind != 1) return false;
  if (j.groups == 1) return true;
  if (!j.h_off) return false;
  for (int g = 0; g < j.groups; ++g)
    if (j.h_off[g] % KCH != 0) return false;
  return j.h_off[j.groups] % KCH == 0 || j.h_off[j.groups] == j.Ktot;
}

// B operand images of image jobs: for every 16-row chunk kc of X (rows
// 16 kc ..), the bf16 parts of [[Xr, Xi], [-Xi, Xr]] exactly as
// sketch_tc_kernel's producers build them (zero past Ktot and kcols), at
// bimg + kc * B_BUF.  Grid: (chunks, jobs).
template <int NR>
__global__ void __launch_bounds__(256) bimage_kernel(const SketchJob* __restrict__ jobs) {
  using C = Cfg<NR, 3>;
  constexpr int KG = C::KG, G = C::G, VS = C::VS, KP = NR / 2, KCH = C::KCH;
  const SketchJob& J = jobs[blockIdx.y];
  const int64_t kc = blockIdx.x, K = J.Ktot, kcols = J.kcols;
  if (kc * KCH >= K) return;
  const float* __restrict__ Xf = (const float*)J.X;
  uint8_t* out = (uint8_t*)J.bimg + kc * C::B_BUF;
  for (int it = threadIdx.x; it < NR * KG; it += blockDim.x) {
    const int nr = ((it / (8 * KG)) << 3) | (it & 7), kgb = (it >> 3) & (KG - 1);
    const int part = kgb >= G ? 1 : 0;
    const int kk0 = (kgb & (G - 1)) * VS;
    const int col = nr % KP, blk = nr / KP;
    const int im = (part ^ blk) & 1;
    const uint32_t neg = (part == 1 && blk == 0) ? 0x80000000u : 0u;
    float v[VS];
#pragma unroll
    for (int t = 0; t < VS; ++t) {
      const int64_t gk = kc * KCH + kk0 + t;
      const float x = (gk < K && col < kcols) ? Xf[2 * (gk + (int64_t)col * J.ldx) + im] : 0.f;
      v[t] = __uint_as_float(__float_as_uint(x) ^ neg);
    }
    uint4 pv[3];
    split_row<3, VS>(v, pv);
    const uint32_t o = (uint32_t)(nr >> 3) * KG * CORE + (uint32_t)kgb * CORE + (uint32_t)(nr & 7) * 16;
#pragma unroll
    for (int p = 0; p < 3; ++p) *(uint4*)(out + p * C::B_PART + o) = pv[p];
  }
}

namespace {
// tensor-memory columns of a chunk's A parts (3 parts x 2 K steps x 8) and
// whether two such slots fit beside the accumulators of an NR-column tile
constexpr int IMG_ACOLS = 48;
__host__ __device__ constexpr bool img_tmem_a(int nr) { return 8 * nr + 2 * IMG_ACOLS <= 512; }

// Image-fed tile shape: one CTA per SM, 736 threads -- two groups of 8
// producer warps (even and odd chunks: bf16 split of the A tile), an MMA
// warp, a tile loader warp, a B loader warp and four drain warps (the
// accumulator sets into (hi, lo), then the epilogue), synchronised by
// mbarriers only.
// SF slots hold image tiles (freed once the producers have read them), SB
// slots the chunks' B operands (bf16 parts formed once per launch, freed by
// the MMAs), S slots the bf16 A parts (in tensor memory where they fit,
// else in shared memory).
template <int NR>
struct ICfg {
  using C = Cfg<NR, 3>;
  static constexpr int KP = NR / 2;
  static constexpr bool TA = img_tmem_a(NR);                            // A parts in tensor memory
  static constexpr uint32_t F_SLOT = IMG_TILE;                          // image tile
  static constexpr uint32_t B_SLOT = (C::B_BUF + 127) / 128 * 128;      // B operand (bf16 parts)
  static constexpr uint32_t O_SLOT = TA ? 0 : C::A_BUF;                 // bf16 A parts (shared memory)
  static constexpr int SF = TA ? 8 : 4, SB = TA ? 8 : 4;
  static constexpr uint32_t LIMIT = 220 * 1024;
  static constexpr uint32_t total(int s) { return SF * F_SLOT + SB * B_SLOT + s * O_SLOT; }
  static constexpr int S = TA ? 2 : total(4) <= LIMIT ? 4 : 2;
  static constexpr uint32_t F0 = 0, B0 = SF * F_SLOT, O0 = B0 + SB * B_SLOT, TOTAL = O0 + S * O_SLOT;
  static constexpr uint32_t ACOL = 8 * NR;                              // first A column in tensor memory
  static_assert(TOTAL <= LIMIT && C::PT == 1 && C::VS == 8, "image tile: shared memory, one 8-column group per thread");
  // a producer group waits on a slot's mbarrier by phase parity; with an
  // odd slot count, consecutive uses of a slot alternate between the two
  // groups, and a group could see the phase two back (same parity) and pass
  // early.  Slot counts that are multiples of the group count make every
  // group observe every phase of the slots it uses.
  static_assert(S % 2 == 0 && SF % 2 == 0, "slot counts must be multiples of the producer groups");
  static_assert(C::DR == 4, "accumulator sets alternate every 4 chunks");
};
constexpr int IPG = 2;                                // producer groups
constexpr int IDRAINW = 4;                            // drain warps (one per lane quarter)
constexpr int ITHREADS = 32 * (IPG * NWARP + 3 + IDRAINW);
constexpr int IMMA_WARP = IPG * NWARP, ILOAD_WARP = IPG * NWARP + 1, IBLOAD_WARP = IPG * NWARP + 2,
              IDRAIN_WARP = IPG * NWARP + 3;

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, uint4 v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w)
               : "memory");
}
// kind::f16 MMA with A in tensor memory (K-major, M = 128 lanes), B in shared memory
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(
          d),
      "r"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
               "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
// Tensor memory of the image kernel: two accumulator sets (alternate
// groups of DR chunks) of three NR-column blocks each -- main (a0 b0),
// c1 (a0 b1 + a1 b0), c2 (a0 b2 + a1 b1 + a2 b0), adjacent so that one MMA
// with the B parts stacked along N fills them -- then hi, lo, and where
// they fit two A slots of IMG_ACOLS columns: a chunk's three bf16 parts x
// two K steps, each K step 8 columns (row i in lane i, 16 K values packed
// in pairs, the even one in the low half).  With A in tensor memory the
// MMAs read only B from shared memory.
__host__ __device__ constexpr int img_cols(int nr) {
  return 8 * nr + (img_tmem_a(nr) ? 2 * IMG_ACOLS : 0) <= 128   ? 128
         : 8 * nr + (img_tmem_a(nr) ? 2 * IMG_ACOLS : 0) <= 256 ? 256
                                                                 : 512;
}
// hi, lo += the set at column `set` (TwoSum of main into hi; the error and
// the correction sums into lo), in 8-column slices
template <int NR>
__device__ __forceinline__ void drain_set(uint32_t tq, int first, int step, uint32_t set) {
#pragma unroll 1
  for (int s = first; s < NR / 8; s += step) {
    uint32_t d[8], c1[8], c2[8], h[8], l[8];
    tmem_ld8(tq + set + s * 8, d);
    tmem_ld8(tq + set + NR + s * 8, c1);
    tmem_ld8(tq + set + 2 * NR + s * 8, c2);
    tmem_ld8(tq + 6 * NR + s * 8, h);
    tmem_ld8(tq + 7 * NR + s * 8, l);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const FF t = two_sum(__uint_as_float(h[i]), __uint_as_float(d[i]));
      h[i] = __float_as_uint(t.h);
      l[i] = __float_as_uint(__uint_as_float(l[i]) + (t.l + (__uint_as_float(c1[i]) + __uint_as_float(c2[i]))));
    }
    tmem_st8(tq + 6 * NR + s * 8, h);
    tmem_st8(tq + 7 * NR + s * 8, l);
  }
  tmem_wait_st();
}
}  // namespace

// Sketch product of image jobs: the same tiles, chunks, bf16 parts and six
// products as sketch_tc_kernel, with the products of one A part issued as
// one MMA over the stacked B parts (3 MMAs per 16 K instead of 6: one
// thread issues an MMA no faster than every ~50 cycles, while M = 128, K =
// 16 costs the tensor pipe N/2 cycles) and the correction sums drained with
// each group -- equal to sketch_tc_kernel's results up to FP32 rounding
// order.  Per chunk c of a CTA's K range,
//   tile loader -- waits for tile slot c % SF to be free (read by the
//              producers of chunk c - SF) and bulk-copies the image tile
//              into it, completing on fullF;
//   B loader -- waits for B slot c % SB (read by the MMAs of chunk c - SB:
//              done) and bulk-copies the chunk's B operand into it,
//              completing on full;
//   producer group c % 2 -- waits for fullF and for A slot c % S (its MMAs
//              of chunk c - S done), reads the tile rows, releases the tile,
//              splits the entries into bf16 parts, writes A (tensor memory,
//              or shared memory fenced to the async proxy) and arrives on
//              full;
//   drain warps -- once the MMAs of group g (4 chunks) are complete (accF),
//              move its accumulator set into (hi, lo) and release it
//              (accE); after the last group, write the rows out;
//   MMA warp -- waits for full (the A parts and the B operand of the chunk;
//              at a group's first chunk also for the drain of the group two
//              back), issues the chunk's MMAs and commits them to done (and
//              to accF at a group's end).
// full and done are rings of NB = 8 barriers indexed by chunk (one wait and
// one commit per chunk for the MMA thread); a slot ring of S or SB slots
// reuses its slot after done of the chunk S or SB back.
// Every wait is bounded (1 s); a role that gives up raises the abort flag
// and the device status, and the others stop at their next wait.
template <int NR>
__global__ void __launch_bounds__(ITHREADS, 1)
sketch_img_kernel(const SketchJob* __restrict__ jobs, const TcTile* __restrict__ tiles, float4* __restrict__ ws) {
  using I = ICfg<NR>;
  using C = Cfg<NR, 3>;
  constexpr int S = I::S, SF = I::SF, KCH = C::KCH, KG = C::KG, G = C::G, DR = C::DR, KP = I::KP, VS = C::VS;
  constexpr int COLS = img_cols(NR);
  static_assert(8 * NR <= 512 && 3 * NR <= 256, "two accumulator sets and (hi, lo) in tensor memory; N <= 256");
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ SketchJob J;
  __shared__ TcTile T;
  constexpr int NB = 8;
  static_assert(NB % S == 0 && NB % I::SB == 0, "slot rings divide the barrier ring");
  __shared__ __align__(8) uint64_t bars[2 * SF + 2 * NB + 4];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t b0 = smem_u32(&bars[0]);
  // fullF[i] = b0 + 8 i, emptyF[i] = +8 (SF + i), full[j] = +8 (2 SF + j),
  // done[j] = +8 (2 SF + NB + j), accF[b] = +8 (2 SF + 2 NB + b), accE[b] = +8 (2 SF + 2 NB + 2 + b)
  const uint32_t fullF = b0, emptyF = b0 + 8u * SF, full = b0 + 16u * SF, done = full + 8u * NB,
                 accF = done + 8u * NB, accE = accF + 16u;
  if (tid == 0) {
    T = tiles[blockIdx.x];
    J = jobs[T.job];
    for (int i = 0; i < SF; ++i) {
      mbar_init(fullF + 8u * i, 1);        // the loader's expect_tx arrive
      mbar_init(emptyF + 8u * i, NWARP);   // the producer group's warps (tile read)
    }
    for (int j = 0; j < NB; ++j) {
      mbar_init(full + 8u * j, NWARP + 1);   // the producer group's warps + the B loader's expect_tx arrive
      mbar_init(done + 8u * j, 1);           // the MMA commit
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accF + 8u * b, 1);
      mbar_init(accE + 8u * b, IDRAINW);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tm = tmem_slot;
  const int pgrp = warp / NWARP, pw = warp % NWARP;   // producer group and warp within it
  const int quad = pw & 3, sub = (pw >> 2) & 1;
  const uint32_t tq = tm + ((uint32_t)(quad * 32) << 16);
  if (warp < NWARP) {   // group 0 zeroes (hi, lo)
    uint32_t z[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) z[i] = 0u;
#pragma unroll 1
    for (int s = sub; s < 2 * NR / 8; s += 2) tmem_st8(tq + 6 * NR + s * 8, z);
    tmem_wait_st();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  const int64_t row0 = T.row0, M = J.M, kcols = J.kcols, ygs = J.ygs;
  const int64_t k0 = T.k0 >= 0 ? T.k0 : (J.d_off ? J.d_off[T.group] : 0);
  const int64_t k1 = T.k0 >= 0 ? T.k1 : (J.d_off ? J.d_off[T.group + 1] : J.Ktot);
  const int nch = (int)((k1 - k0 + KCH - 1) / KCH);
  const int ngroups = (nch + DR - 1) / DR;
  const uint32_t sb = smem_u32(smem);
  bool ok = true;

  if (warp == ILOAD_WARP) {
    // ---------------------------------------------------------------- loader
    const uint8_t* imgp = (const uint8_t*)J.img + ((row0 / TM) * J.img_nch + k0 / KCH) * (int64_t)IMG_TILE;
    const uint64_t pol = l2_evict_first();
    int c = 0;
    for (; c < nch; ++c) {
      const int sf = c % SF;
      int free_ok = 1;
      if (c >= SF && lane == 0) free_ok = mbar_wait(emptyF + 8u * sf, (uint32_t)(((c / SF) - 1) & 1)) ? 1 : 0;
      free_ok = __shfl_sync(0xffffffffu, free_ok, 0);
      if (!free_ok || *(volatile int*)&abort_flag) {
        ok = free_ok != 0;
        break;
      }
      if (lane == 0) {
        mbar_expect_tx(fullF + 8u * sf, IMG_TILE);
        bulk_copy(sb + I::F0 + (uint32_t)sf * I::F_SLOT, imgp + (int64_t)c * IMG_TILE, IMG_TILE, fullF + 8u * sf,
                  pol);
      }
    }
    if (!ok && lane == 0) {
      *(volatile int*)&abort_flag = 1;
      atomicExch(&g_tc_status, 1);
    }
    // the loads still in flight complete before the CTA ends (bounded)
    if (lane == 0)
      for (int q = c - SF < 0 ? 0 : c - SF; q < c; ++q) mbar_wait(fullF + 8u * (q % SF), (uint32_t)((q / SF) & 1));
    __syncwarp();
  } else if (warp == IBLOAD_WARP) {
    // -------------------------------------------------------------- B loader
    if (lane == 0) {
      const uint8_t* bimp = (const uint8_t*)J.bimg + (k0 / KCH) * (int64_t)C::B_BUF;
      const uint64_t pol = l2_evict_last();
      int c = 0;
      for (; c < nch; ++c) {
        const int sbi = c % I::SB, j = c % NB;
        if (*(volatile int*)&abort_flag) break;
        if (c >= I::SB && !mbar_wait(done + 8u * ((c - I::SB) % NB), (uint32_t)(((c - I::SB) / NB) & 1))) {
          *(volatile int*)&abort_flag = 1;
          atomicExch(&g_tc_status, 1);
          break;
        }
        mbar_expect_tx(full + 8u * j, C::B_BUF);
        bulk_copy(sb + I::B0 + (uint32_t)sbi * I::B_SLOT, bimp + (int64_t)c * C::B_BUF, C::B_BUF, full + 8u * j, pol);
      }
      // the copies still in flight land before the CTA ends (bounded; after
      // an abort the producers' arrivals may be missing and each wait ends
      // at its limit)
      for (int q = c - I::SB < 0 ? 0 : c - I::SB; q < c; ++q) mbar_wait(full + 8u * (q % NB), (uint32_t)((q / NB) & 1));
    }
    __syncwarp();
  } else if (warp == IMMA_WARP) {
    // ------------------------------------------------------------- MMA warp
    // The chunk loop is unrolled over one period of the rings (8 chunks: S,
    // SB and DR divide it; the accumulator set alternates every DR), so every
    // slot, barrier and operand address is a compile-time offset and each
    // phase parity a constant or a bit of the loop counter: the issuing
    // thread then keeps pace with the tensor pipe (six MMAs, 288 cycles of
    // M = 128 work per chunk at NR = 48).
    if (lane == 0) {
      static_assert(NB == 8 && DR == 4, "one unrolled period of the rings");
      constexpr uint32_t idesc = idesc_bf16(NR), idesc2 = idesc_bf16(2 * NR), idesc3 = idesc_bf16(3 * NR);
      constexpr uint64_t pa = C::A_PART >> 4;
      const uint64_t dA0 = sdesc<KG>(sb + I::O0), dB0 = sdesc<KG>(sb + I::B0);
      const volatile int* abortp = &abort_flag;
      int issued = -1;
      for (int c8 = 0; c8 < nch && ok; c8 += 8) {
        const uint32_t accE_par = (uint32_t)(((c8 >> 3) + 1) & 1);   // phase of the group two back
        const uint32_t full_par = (uint32_t)((c8 >> 3) & 1);          // chunk c8 + u on full[u]
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int c = c8 + u;
          if (c >= nch) break;
          const int s = u % S, sbi = u % I::SB, set = (u / DR) & 1;
          if (u % DR == 0 && c >= 2 * DR && !mbar_wait(accE + 8u * set, accE_par, abortp)) {
            ok = false;
            break;
          }
          if (!mbar_wait(full + 8u * u, full_par, abortp)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t dA = dA0 + (uint64_t)((s * I::O_SLOT) >> 4), dB = dB0 + (uint64_t)((sbi * I::B_SLOT) >> 4);
          const uint32_t aT = tm + I::ACOL + (uint32_t)(s * IMG_ACOLS);   // part p, K step ks: + 16 p + 8 ks
          // set of this group: [main | c1 | c2]; a0 [b0; b1; b2] -> all three,
          // a1 [b0; b1] -> c1, c2, a2 b0 -> c2 (the B parts are consecutive
          // 8-row groups, so stacking them along N is a larger N)
          const uint32_t tset = tm + (uint32_t)(set * 3 * NR);
          const uint32_t carry = (u % DR) != 0 ? 1u : 0u;   // the set restarts with its group
#pragma unroll
          for (int ks = 0; ks < C::KSTEPS; ++ks) {
            const uint64_t o = (uint64_t)(ks * 2 * CORE) >> 4;
            if constexpr (I::TA) {
              mma_ts(tset, aT + 8 * ks, dB + o, idesc3, ks > 0 ? 1u : carry);
              mma_ts(tset + NR, aT + 16 + 8 * ks, dB + o, idesc2, 1u);
              mma_ts(tset + 2 * NR, aT + 32 + 8 * ks, dB + o, idesc, 1u);
            } else {
              mma_step<2>(tset, dA + o, dB + o, idesc3, ks > 0 ? 1u : carry);
              mma_step<2>(tset + NR, dA + pa + o, dB + o, idesc2, 1u);
              mma_step<2>(tset + 2 * NR, dA + 2 * pa + o, dB + o, idesc, 1u);
            }
          }
          tc_commit(done + 8u * u);
          if (u % DR == DR - 1 || c == nch - 1) tc_commit(accF + 8u * set);
          issued = c;
        }
      }
      if (!ok) {
        *(volatile int*)&abort_flag = 1;
        atomicExch(&g_tc_status, 1);
        if (issued >= 0) mbar_wait(done + 8u * (issued % NB), (uint32_t)((issued / NB) & 1));
      }
    }
    __syncwarp();
  } else if (warp >= IDRAIN_WARP) {
    // ------------------------------------------------------------- drainers
    // each warp owns the 32 rows of its lane quarter: once the MMAs of group
    // g are complete it moves set g & 1 into (hi, lo) and releases the set;
    // after the last group it writes its rows out
    const volatile int* abortp = &abort_flag;
    for (int g = 0; g < ngroups && ok; ++g) {
      if (!mbar_wait(accF + 8u * (g & 1), (uint32_t)((g / 2) & 1), abortp)) {
        ok = false;
        break;
      }
      tc_fence_after();
      drain_set<NR>(tq, 0, 1, (uint32_t)(g & 1) * 3 * NR);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(accE + 8u * (g & 1));
    }
    if (ok && nch > 0) {
      // epilogue: (hi, lo) pairs of this warp's lanes to Y or to the split workspace
      const int64_t row = row0 + quad * 32 + lane;
#pragma unroll 1
      for (int s = 0; s < (KP + 7) / 8; ++s) {
        uint32_t hr[8], lr[8], hm[8], lm[8];
        const int c0 = s * 8;
        tmem_ld8(tq + 6 * NR + c0, hr);
        tmem_ld8(tq + 7 * NR + c0, lr);
        tmem_ld8(tq + 6 * NR + KP + c0, hm);
        tmem_ld8(tq + 7 * NR + KP + c0, lm);
        tmem_wait_ld();
        if (row < M) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int col = c0 + i;
            if (col >= kcols || col >= KP) continue;
            if (T.ws < 0) {
              float2* __restrict__ Y = (float2*)J.Y;
              Y[row + (T.group * ygs + col) * J.ldy] = make_float2(
                  __uint_as_float(hr[i]) + __uint_as_float(lr[i]), __uint_as_float(hm[i]) + __uint_as_float(lm[i]));
            } else {
              ws[T.ws + col * M + row] = make_float4(__uint_as_float(hr[i]), __uint_as_float(lr[i]),
                                                     __uint_as_float(hm[i]), __uint_as_float(lm[i]));
            }
          }
        }
      }
    }
    if (!ok && lane == 0) {
      *(volatile int*)&abort_flag = 1;
      atomicExch(&g_tc_status, 1);
    }
  } else {
    // ------------------------------------------------------------ producers
    // with A in tensor memory a warp owns the 32 rows of its lane quarter
    // (half the chunk's columns each); else 16 rows in core-matrix order
    const int prow = I::TA ? 32 * quad + lane : 16 * pw + (lane & 7) + 8 * ((lane >> 4) & 1);
    const int kg = I::TA ? sub : (lane >> 3) & 1;
    const uint32_t a_st = (uint32_t)(prow >> 3) * KG * CORE + (uint32_t)(prow & 7) * 16;
    const volatile int* abortp = &abort_flag;
    for (int c = pgrp; c < nch && ok; c += IPG) {
      const int sf = c % SF, s = c % S;
      if (!mbar_wait(fullF + 8u * sf, (uint32_t)((c / SF) & 1), abortp) ||
          (c >= S && !mbar_wait(done + 8u * ((c - S) % NB), (uint32_t)(((c - S) / NB) & 1), abortp))) {
        ok = false;
        break;
      }
      if constexpr (I::TA) tc_fence_after();   // the MMAs that read A slot s are complete
      const uint32_t fb = sb + I::F0 + (uint32_t)sf * I::F_SLOT;
      float re[VS], im[VS];
#pragma unroll
      for (int t = 0; t < VS / 2; ++t) {
        const float4 u = ld_shared_v4(fb + img_seg(prow, 4 * kg + t));
        re[2 * t] = u.x, im[2 * t] = u.y, re[2 * t + 1] = u.z, im[2 * t + 1] = u.w;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(emptyF + 8u * sf);   // this warp is done with the image tile
      uint4 pr[3], pm[3];
      split_row<3, VS>(re, pr);
      split_row<3, VS>(im, pm);
      if constexpr (I::TA) {
        // part q: real parts at K step 0, imaginary at K step 1; this
        // thread's 8 values are columns 4 kg .. 4 kg + 3 of each
        const uint32_t ta = tq + I::ACOL + (uint32_t)s * IMG_ACOLS + 4u * kg;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          tmem_st4(ta + 16 * q, pr[q]);
          tmem_st4(ta + 16 * q + 8, pm[q]);
        }
        tmem_wait_st();
        tc_fence_before();
      } else {
        const uint32_t aB = sb + I::O0 + (uint32_t)s * I::O_SLOT;
        const uint32_t ar = aB + a_st + (uint32_t)kg * CORE, ai = ar + (uint32_t)G * CORE;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          st_shared_v4(ar + q * C::A_PART, pr[q]);
          st_shared_v4(ai + q * C::A_PART, pm[q]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(full + 8u * (c % NB));
    }
    if (!ok && lane == 0) {
      *(volatile int*)&abort_flag = 1;
      atomicExch(&g_tc_status, 1);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(COLS) : "memory");
  }
}

template <int NR>
static int launch_img_nr(const SketchJob* dj, const TcTile* dt, unsigned ntiles, float4* ws, cudaStream_t s) {
  constexpr size_t smem = ICfg<NR>::TOTAL;
  BF_CUDA_TRY(cudaFuncSetAttribute(sketch_img_kernel<NR>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   (int)cudaSharedmemCarveoutMaxShared));
  BF_CUDA_TRY(cudaFuncSetAttribute(sketch_img_kernel<NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  note_launch();
  sketch_img_kernel<NR><<<ntiles, ITHREADS, smem, s>>>(dj, dt, ws);
  BF_CUDA_TRY(cudaGetLastError());
  return BF_OK;
}

static int launch_bimages(int nr, const std::vector<SketchJob>& jobs, const SketchJob* dj, const DevBuf&,
                          cudaStream_t s) {
  int64_t mc = 0;
  for (const auto& j : jobs) mc = std::max<int64_t>(mc, entry_image_chunks(j.Ktot));
  if (mc == 0) return BF_OK;
  const dim3 grid((unsigned)mc, (unsigned)jobs.size());
  note_launch();
  switch (nr) {
    case 16: bimage_kernel<16><<<grid, 256, 0, s>>>(dj); break;
    case 32: bimage_kernel<32><<<grid, 256, 0, s>>>(dj); break;
    case 48: bimage_kernel<48><<<grid, 256, 0, s>>>(dj); break;
    default: bimage_kernel<64><<<grid, 256, 0, s>>>(dj); break;
  }
  BF_CUDA_TRY(cudaGetLastError());
  return BF_OK;
}

static int launch_img(int nr, const SketchJob* dj, const TcTile* dt, unsigned nt, float4* ws, cudaStream_t s) {
  switch (nr) {
    case 16: return launch_img_nr<16>(dj, dt, nt, ws, s);
    case 32: return launch_img_nr<32>(dj, dt, nt, ws, s);
    case 48: return launch_img_nr<48>(dj, dt, nt, ws, s);
    default: return launch_img_nr<64>(dj, dt, nt, ws, s);
  }
}

bool sketch_tc_applies(const std::vector<SketchJob>& jobs) {
  for (const auto& j : jobs)
    if (j.kcols < 1) return false;
  return true;
}

template <int NR, int SPLIT>
static int launch_nr(const SketchJob* dj, const TcTile* dt, unsigned ntiles, float4* ws, cudaStream_t s) {
  constexpr size_t smem = Cfg<NR, SPLIT>::LAUNCH_SMEM;
  BF_CUDA_TRY(cudaFuncSetAttribute(sketch_tc_kernel<NR, SPLIT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   (int)cudaSharedmemCarveoutMaxShared));
  BF_CUDA_TRY(cudaFuncSetAttribute(sketch_tc_kernel<NR, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
  note_launch();
  sketch_tc_kernel<NR, SPLIT><<<ntiles, THREADS, smem, s>>>(dj, dt, ws);
  BF_CUDA_TRY(cudaGetLastError());
  return BF_OK;
}

template <int SPLIT>
static int launch_split(int nr, const SketchJob* dj, const TcTile* dt, unsigned nt, float4* ws, cudaStream_t s) {
  switch (nr) {
    case 16: return launch_nr<16, SPLIT>(dj, dt, nt, ws, s);
    case 32: return launch_nr<32, SPLIT>(dj, dt, nt, ws, s);
    case 48: return launch_nr<48, SPLIT>(dj, dt, nt, ws, s);
    case 64: return launch_nr<64, SPLIT>(dj, dt, nt, ws, s);
    default: return launch_nr<96, SPLIT>(dj, dt, nt, ws, s);
  }
}

static int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      n = v;
    else
      n = 152;
  }
  return n;
}

// Split-K factor of one job: minimises (waves of CTAs) x (16-column K
// chunks per CTA + a fixed per-CTA cost) for the job alone, so a job sums
// in the same order whether it runs alone or in a batch.  per_sm: CTAs
// resident per SM (2 for sketch_tc_kernel, 1 for the image kernel).
static int job_splits(int64_t base_tiles, int64_t max_chunks, int per_sm) {
  const int64_t wave = (int64_t)sm_count() * per_sm;
  int best = 1;
  double best_cost = 1e300;
  for (int ns = 1; ns <= 32; ++ns) {
    if (ns > 1 && max_chunks < 4 * ns) break;
    const double waves = (double)((base_tiles * ns + wave - 1) / wave);
    const double cost = waves * (double)((max_chunks + ns - 1) / ns + 6);
    if (cost < best_cost * 0.999) best = ns, best_cost = cost;
  }
  return best;
}

int launch_sketch_jobs_tc(const std::vector<SketchJob>& jobs_in, MemTracker* mt, cudaStream_t s) {
  // jobs wider than the widest tile run as column slices (entries formed once
  // per slice); every job keeps its Y group stride
  std::vector<SketchJob> jobs;
  const int64_t WMAX = NR_MAX / 2;
  for (SketchJob j : jobs_in) {
    if (j.ygs == 0) j.ygs = j.kcols;
    if (j.nseg == 2) {   // two-level jobs are built within the widest tile
      if (j.kcols > WMAX || j.kcols0 < 1 || j.kcols0 >= j.kcols || !j.h_off1 || !j.h_off)
        return fail(BF_EINVAL, "two-level sketch job out of range");
      jobs.push_back(j);
      continue;
    }
    // image jobs run in slices of at most 32 columns (the image kernel's
    // widest tile), whatever they are batched with
    const int64_t kc = j.kcols, wmax = j.img ? 32 : WMAX;
    for (int64_t c0 = 0; c0 < kc; c0 += wmax) {
      SketchJob q = j;
      q.kcols = std::min(wmax, kc - c0);
      q.X = (const float2*)j.X + c0 * j.ldx;
      q.Y = (float2*)j.Y + c0 * j.ldy;
      jobs.push_back(q);
    }
  }
  int64_t maxk = 0;
  int split = 2;
  for (const auto& j : jobs) maxk = std::max(maxk, j.kcols), split = std::max(split, j.split);
  // jobs of both split depths: one launch per depth, so that every job's
  // arithmetic is the same as when it runs alone
  for (const auto& j : jobs)
    if (j.split != split) {
      std::vector<SketchJob> lo, hi;
      for (const auto& q : jobs) (q.split == split ? hi : lo).push_back(q);
      BF_TRY(launch_sketch_jobs_tc(lo, mt, s));
      return launch_sketch_jobs_tc(hi, mt, s);
    }
  // jobs that read entry images and jobs that form entries: one launch each
  {
    bool any = false, all = true;
    for (const auto& j : jobs) any = any || j.img != nullptr, all = all && j.img != nullptr;
    if (any && !all) {
      std::vector<SketchJob> a, b;
      for (const auto& q : jobs) (q.img ? a : b).push_back(q);
      BF_TRY(launch_sketch_jobs_tc(b, mt, s));
      return launch_sketch_jobs_tc(a, mt, s);
    }
  }
  const bool from_images = !jobs.empty() && jobs[0].img != nullptr;
  // real columns N = 2 x padded sketch width, one of the compiled tile widths
  const int kp = (int)((maxk + 7) / 8 * 8);
  const int nr = kp <= 8 ? 16 : kp <= 16 ? 32 : kp <= 24 ? 48 : kp <= 32 ? 64 : 96;
  if (from_images && nr > 64) return fail(BF_EINVAL, "image sketch job wider than 32 columns");
  const int kch = split == 3 ? Cfg<16, 3>::KCH : Cfg<16, 2>::KCH;   // complex K per chunk
  std::vector<TcTile> tiles;
  std::vector<TcRegion> regs;
  int64_t wsz = 0;
  for (size_t ji = 0; ji < jobs.size(); ++ji) {
    const SketchJob& j = jobs[ji];
    if (j.M <= 0 || j.kcols <= 0) continue;
    const int64_t rt = (j.M + TM - 1) / TM;
    if (j.nseg == 2) {
      // CTAs cover (row tile, fine node f at the second level, K split);
      // segment 0 (node f >> shift1) sums over all of a coarse node's fine
      // nodes and splits, segment 1 over the splits of f
      const int64_t G1 = j.groups1, sh = j.shift1, w0 = j.kcols0, w1 = j.kcols - j.kcols0;
      int64_t maxk_f = 0;
      for (int64_t f = 0; f < G1; ++f) maxk_f = std::max(maxk_f, j.h_off1[f + 1] - j.h_off1[f]);
      const int ns = job_splits(rt * G1, (maxk_f + 15) / 16, 2);
      const int64_t n0 = ((int64_t)1 << sh) * ns;   // partials per coarse node
      std::vector<int64_t> ws0(j.groups), ws1(G1, -1);
      for (int g = 0; g < j.groups; ++g) {
        ws0[g] = wsz;
        regs.push_back({wsz, j.M, w0, j.ldy, (int64_t)g * j.ygs, (int32_t)n0, 0, (float2*)j.Y});
        wsz += n0 * j.M * w0;
      }
      if (ns > 1)
        for (int64_t f = 0; f < G1; ++f) {
          ws1[f] = wsz;
          regs.push_back({wsz, j.M, w1, j.ldy1, f * j.ygs1, ns, 0, (float2*)j.Y1});
          wsz += (int64_t)ns * j.M * w1;
        }
      for (int64_t f = 0; f < G1; ++f) {
        const int64_t ga = j.h_off1[f], gb = j.h_off1[f + 1], g0 = f >> sh;
        const int64_t ks = ((gb - ga + ns - 1) / ns + kch - 1) / kch * kch;
        for (int sp = 0; sp < ns; ++sp) {
          const int64_t a = std::min<int64_t>(gb, ga + sp * ks), b = std::min<int64_t>(gb, a + ks);
          const int64_t p0 = ws0[g0] + ((f - (g0 << sh)) * ns + sp) * j.M * w0;
          const int64_t p1 = ns > 1 ? ws1[f] + (int64_t)sp * j.M * w1 : -1;
          for (int64_t r0 = 0; r0 < j.M; r0 += TM)
            tiles.push_back(TcTile{(int32_t)ji, (int32_t)g0, r0, a, b, p0, f, p1});
        }
      }
      continue;
    }
    // K ranges of the groups (host copy of the node boundaries when given)
    auto krange = [&](int g, int64_t& a, int64_t& b) {
      if (j.groups == 1) a = 0, b = j.Ktot;
      else if (j.h_off) a = j.h_off[g], b = j.h_off[g + 1];
      else a = -1, b = -1;
    };
    int64_t maxk_g = 0;
    bool known = true;
    for (int g = 0; g < j.groups; ++g) {
      int64_t a, b;
      krange(g, a, b);
      if (a < 0) known = false;
      else maxk_g = std::max(maxk_g, b - a);
    }
    const int ns = known ? job_splits(rt * j.groups, (maxk_g + 15) / 16, from_images ? 1 : 2) : 1;
    for (int g = 0; g < j.groups; ++g) {
      int64_t ga, gb;
      krange(g, ga, gb);
      int64_t ws0 = -1;
      if (ns > 1) {
        ws0 = wsz;
        regs.push_back({wsz, j.M, j.kcols, j.ldy, (int64_t)g * j.ygs, ns, 0, (float2*)j.Y});
        wsz += (int64_t)ns * j.M * j.kcols;
      }
      const int64_t ks = ns > 1 ? ((gb - ga + ns - 1) / ns + kch - 1) / kch * kch : 0;
      for (int sp = 0; sp < ns; ++sp) {
        int64_t a = -1, b = -1;   // whole group range, resolved on the device
        if (ns > 1) {
          a = std::min<int64_t>(gb, ga + sp * ks);
          b = std::min<int64_t>(gb, a + ks);
        }
        for (int64_t r0 = 0; r0 < j.M; r0 += TM)
          tiles.push_back(TcTile{(int32_t)ji, g, r0, a, b, ns > 1 ? ws0 + (int64_t)sp * j.M * j.kcols : -1, 0, -1});
      }
    }
  }
  if (tiles.empty()) return BF_OK;
  const size_t jb = jobs.size() * sizeof(SketchJob), tb = tiles.size() * sizeof(TcTile),
               rb = regs.size() * sizeof(TcRegion);
  DevBuf d, w, bi;
  if (from_images) {   // B operand images, one per job (bf16 parts of every 16-row chunk)
    const size_t bbuf = (size_t)3 * nr * 32 * 2;
    size_t tot = 0;
    for (const auto& j : jobs) tot += (size_t)entry_image_chunks(j.Ktot) * bbuf;
    BF_TRY(bi.alloc(mt, tot, s));
    size_t off = 0;
    for (auto& j : jobs) {
      j.bimg = (char*)bi.p + off;
      off += (size_t)entry_image_chunks(j.Ktot) * bbuf;
    }
  }
  BF_TRY(d.alloc(mt, jb + tb + rb + 16, s));
  if (wsz) BF_TRY(w.alloc(mt, wsz * sizeof(float4), s));
  int rc = BF_OK;
  char* p = (char*)d.p;
  if (upload_async(p, jobs.data(), jb, s) != BF_OK || upload_async(p + jb, tiles.data(), tb, s) != BF_OK ||
      (rb && upload_async(p + jb + tb, regs.data(), rb, s) != BF_OK))
    rc = fail(BF_ECUDA, "upload of sketch jobs failed");
  const SketchJob* dj = (const SketchJob*)p;
  const TcTile* dt = (const TcTile*)(p + jb);
  const unsigned nt = (unsigned)tiles.size();
  if (!rc && from_images) rc = launch_bimages(nr, jobs, dj, bi, s);
  if (!rc)
    rc = from_images   ? launch_img(nr, dj, dt, nt, (float4*)w.p, s)
         : split == 3 ? launch_split<3>(nr, dj, dt, nt, (float4*)w.p, s)
                      : launch_split<2>(nr, dj, dt, nt, (float4*)w.p, s);
  if (!rc && !regs.empty()) {
    dim3 grid(64, (unsigned)regs.size());
    note_launch();
    tc_reduce_kernel<<<grid, 256, 0, s>>>((const TcRegion*)(p + jb + tb), (int)regs.size(), (const float4*)w.p);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) rc = fail(BF_ECUDA, std::string("sketch reduce: ") + cudaGetErrorString(e));
  }
  w.release(s);
  d.release(s);
  bi.release(s);
  return rc;
}

// The failure path of the bounded waits, exercised without a fault: one
// warp waits on an mbarrier that nothing arrives at, through the kernels'
// own wait routine, with the limit lowered to limit_ns; the wait gives up,
// the device flag is set, the kernel returns and the host reads the status.
__global__ void wait_probe_kernel() {
  __shared__ __align__(8) unsigned long long bar;
  const uint32_t addr = smem_u32(&bar);
  if (threadIdx.x == 0) {
    mbar_init(addr, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(addr, 0)) atomicExch(&g_tc_status, 1);
}

int wait_probe(uint64_t limit_ns, cudaStream_t s) {
  if (limit_ns == 0 || limit_ns > 1000000000ull) return fail(BF_EINVAL, "limit_ns must be in (0, 1e9]");
  int before = 0;
  note_sync();
  BF_CUDA_TRY(cudaMemcpyFromSymbol(&before, g_tc_status, sizeof(int)));
  if (before) return fail(BF_ETIMEOUT, "an earlier tensor-core wait had already given up (device flag set)");
  const unsigned long long lim = limit_ns, def = 1000000000ull;
  BF_CUDA_TRY(cudaMemcpyToSymbolAsync(g_wait_limit_ns, &lim, sizeof(lim), 0, cudaMemcpyHostToDevice, s));
  note_launch();
  wait_probe_kernel<<<1, 32, 0, s>>>();
  const cudaError_t e = cudaGetLastError();
  const cudaError_t e2 = cudaMemcpyToSymbolAsync(g_wait_limit_ns, &def, sizeof(def), 0, cudaMemcpyHostToDevice, s);
  const cudaError_t e3 = host_sync(s);
  if (e != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess)
    return fail(BF_ECUDA, std::string("wait probe: ") +
                              cudaGetErrorString(e != cudaSuccess ? e : e2 != cudaSuccess ? e2 : e3));
  return tc_status(true);
}

int* tc_status_ptr() {
  void* p = nullptr;
  return cudaGetSymbolAddress(&p, g_tc_status) == cudaSuccess ? (int*)p : nullptr;
}

int tc_status_copy(int32_t* dst, cudaStream_t s) {
  BF_CUDA_TRY(cudaMemcpyFromSymbolAsync(dst, g_tc_status, sizeof(int), 0, cudaMemcpyDeviceToDevice, s));
  return BF_OK;
}

int tc_status_value(int v, bool reset) {
  if (v && reset) {
    const int z = 0;
    note_sync();
    BF_CUDA_TRY(cudaMemcpyToSymbol(g_tc_status, &z, sizeof(int)));
  }
  return v ? fail(BF_ETIMEOUT, "a tensor-core sketch wait gave up (device flag set)") : BF_OK;
}

int tc_status(bool reset) {
  int v = 0;
  note_sync();
  BF_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_tc_status, sizeof(int)));
  return tc_status_value(v, reset);
}

}  // namespace bf
