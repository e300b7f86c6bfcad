// Mixed-precision sketch products on the 5th-generation tensor cores
// (tcgen05, kind::tf32) with split-precision TF32 products:
//   Y[:, g*k + c] = sum_{j in rows_g} A[:, j] X[j, c]   (or the adjoint form)
// for the built-in operators (Alg. 2 input, structured sketches of Sec. 4.1),
// computed as one real GEMM per 128-row tile:
//   [Yr | Yi] = [Ar | Ai] * [[Xr, Xi], [-Xi, Xr]].
// Operands are split into TF32 parts a = a0 + a1 (+ a2) and the products
// kept down to the FP32 level:
//   SPLIT 2 (3xTF32):  a0 b0 + a0 b1 + a1 b0                 (~2^-21 relative)
//   SPLIT 3 (6 terms): ... + a0 b2 + a1 b1 + a2 b0, the split exact (~FP32)
//
// Per CTA (one job, one group, 128 rows, one K range, all 2k real columns):
//   * 16 warps form the entries of a K chunk (the float-float formulas of
//     kentry.cuh, or loads of a stored complex64 A) and write their TF32
//     parts straight into one of two shared-memory A buffers (K-major,
//     no-swizzle core-matrix layout: 8 rows x 16 B per core matrix, 128 B
//     between K-adjacent, 8*KCH B between 8-row groups) while the tensor
//     core works on the previous chunk;
//   * the next chunk's rows of X are staged with cp.async meanwhile;
//   * after the previous chunk's MMAs complete (mbarrier, bounded wait),
//     warps 0-3 move the FP32 accumulator from tensor memory into a
//     (hi, lo) pair kept in tensor memory with Knuth's TwoSum (so sums over
//     n = 16384 points keep FP32 accuracy), the B operand
//     [[Xr, Xi], [-Xi, Xr]] parts are built from the staged rows, and one
//     thread issues the chunk's tcgen05.mma (M = 128, N = 2k, K = 8) and
//     commits them to the mbarrier;
//   * launches with few row tiles split K across CTAs; partial (hi, lo)
//     sums go to a workspace and a second kernel adds them with TwoSum;
//   * a wait that exceeds 1 s of %globaltimer records a device flag
//     (reported as BF_ETIMEOUT), frees the tensor memory and returns.
#include <algorithm>

#include "bf_internal.h"
#include "cx.cuh"
#include "kentry.cuh"

namespace bf {

using namespace dev;

__device__ int g_tc_status;   // 1 once a bounded wait has given up

namespace {
constexpr int TM = 128;        // rows per CTA (MMA M)
constexpr int THREADS = 512;
constexpr uint32_t CORE = 128; // bytes of one 8 x 16 B core matrix

struct TcTile {
  int32_t job, group;
  int64_t row0;
  int64_t k0, k1;              // K range of this CTA
  int64_t ws;                  // float4 offset of this (job, group, split) partial, or -1
};
struct TcRegion {              // one (job, group) region to reduce
  int64_t ws, M, kcols, ldy, ycol0;
  int32_t nsplit, pad;
  float2* Y;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

template <int KR>
__device__ __forceinline__ uint32_t kmaj(int row, int kr) {
  return (uint32_t)((row >> 3) * (KR / 4) * CORE + (kr >> 2) * CORE + (row & 7) * 16 + (kr & 3) * 4);
}

// shared-memory matrix descriptor: start, LBO (K-adjacent core matrices),
// SBO (8-row groups), in 16-byte units; version 1 at bits 46-47; no swizzle
template <int KR>
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  constexpr uint32_t SBO = (KR / 4) * CORE;
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((CORE >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((SBO >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor: D FP32 (bits 4-5 = 1), A and B TF32 (bits 7-9 and
// 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ uint32_t tf32_bits(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

template <int SPLIT>
__device__ __forceinline__ void split_parts(float x, uint32_t (&p)[3]) {
  p[0] = tf32_bits(x);
  const float r1 = x - __uint_as_float(p[0]);
  p[1] = tf32_bits(r1);
  if (SPLIT == 3) p[2] = tf32_bits(r1 - __uint_as_float(p[1]));
}

__device__ __forceinline__ void st_shared(uint32_t addr, uint32_t v) {
  asm volatile("st.shared.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
  const uint64_t t0 = now_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (now_ns() - t0 > 1000000000ull) return false;
  }
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

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(
          dtmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;" ::: "memory");
}

// tensor-memory columns: main accumulator [0, NR) (the a0*b0 products),
// correction accumulator [NR, 2NR) (the cross terms, ~2^-11 smaller, so
// their roundings do not reach the total), and the TwoSum pair hi
// [2NR, 3NR), lo [3NR, 4NR); a power of two >= 32 with 16 spare columns for
// the epilogue's last 16-column slice (it may pass the end of lo by 8)
__host__ __device__ constexpr int tmem_cols(int nr) {
  return 4 * nr + 16 <= 32 ? 32 : 4 * nr + 16 <= 64 ? 64 : 4 * nr + 16 <= 128 ? 128 : 4 * nr + 16 <= 256 ? 256 : 512;
}
static_assert(4 * 128 + 8 <= 512 + 8, "epilogue reads stay inside 512 columns for NR = 128 (KP = 64)");

template <int SPLIT>
__host__ __device__ constexpr int kch() { return SPLIT == 3 ? 16 : 32; }   // complex K per chunk

template <int NR, int SPLIT>
constexpr size_t smem_bytes() {
  constexpr int KR = 2 * kch<SPLIT>();
  return 2 * (size_t)SPLIT * TM * KR * 4       // A, two buffers
         + (size_t)SPLIT * NR * KR * 4         // B
         + (size_t)kch<SPLIT>() * (NR / 2) * 8;// staged X rows
}
}  // namespace

// TwoSum the main accumulator into the pair (hi, lo) and add the correction
// accumulator to lo, for this warp's 32 lanes (warps 0-3 only).
template <int NR>
__device__ __forceinline__ void drain(uint32_t tlane) {
#pragma unroll 1
  for (int s = 0; s < NR / 16; ++s) {
    uint32_t d[16], e[16], h[16], l[16];
    tmem_ld16(tlane + s * 16, d);
    tmem_ld16(tlane + NR + s * 16, e);
    tmem_ld16(tlane + 2 * NR + s * 16, h);
    tmem_ld16(tlane + 3 * NR + s * 16, l);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const FF t = two_sum(__uint_as_float(h[i]), __uint_as_float(d[i]));
      h[i] = __float_as_uint(t.h);
      l[i] = __float_as_uint(__uint_as_float(l[i]) + (t.l + __uint_as_float(e[i])));
    }
    tmem_st16(tlane + 2 * NR + s * 16, h);
    tmem_st16(tlane + 3 * NR + s * 16, l);
  }
  tmem_wait_st();
}

template <int NR, int SPLIT>
__global__ void __launch_bounds__(THREADS, 1)
sketch_tc_kernel(const SketchJob* __restrict__ jobs, const TcTile* __restrict__ tiles, float4* __restrict__ ws) {
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr int KCH = kch<SPLIT>(), KR = 2 * KCH, KP = NR / 2;
  constexpr int COLS = tmem_cols(NR);
  constexpr uint32_t A_PART = TM * KR * 4, A_BUF = SPLIT * A_PART, B_PART = NR * KR * 4;
  constexpr int EPT = KCH * TM / THREADS;        // entries per thread per chunk
  __shared__ SketchJob J;
  __shared__ TcTile T;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    T = tiles[blockIdx.x];
    J = jobs[T.job];
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1) : "memory");
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
  const uint32_t tlane = tm + ((uint32_t)(warp & 3) * 32u << 16);
  if (warp < 4) {
    uint32_t z[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) z[i] = 0u;
#pragma unroll 1
    for (int s = 0; s < 2 * NR / 16; ++s) tmem_st16(tlane + 2 * NR + s * 16, z);
    tmem_wait_st();
  }

  const int64_t row0 = T.row0, M = J.M, kcols = J.kcols;
  // K range: this CTA's split, or the whole group
  const int64_t k0 = T.k0 >= 0 ? T.k0 : (J.d_off ? J.d_off[T.group] : 0);
  const int64_t k1 = T.k0 >= 0 ? T.k1 : (J.d_off ? J.d_off[T.group + 1] : J.Ktot);
  const float2* __restrict__ X = (const float2*)J.X;
  const int64_t ldx = J.ldx;
  const uint32_t aBase = smem_u32(smem), bBase = aBase + 2 * A_BUF, xBase = bBase + SPLIT * B_PART;
  const float2* xs = (const float2*)(smem + 2 * A_BUF + SPLIT * B_PART);
  constexpr uint32_t idesc = idesc_tf32(NR);
  const int nch = (int)((k1 - k0 + KCH - 1) / KCH);
  // entry mapping: warp w forms rows 8w..8w+7, lane l row 8w + l/4 at K
  // offsets 4j + l%4, so every store of a warp fills one 128-byte core
  // matrix (no shared-memory bank conflicts)
  const int r = 8 * warp + (lane >> 2), kq = lane & 3;
  const int64_t gi = row0 + r;
  const uint32_t a_off = (uint32_t)warp * (KR / 4) * CORE + (uint32_t)(lane >> 2) * 16 + (uint32_t)kq * 4;
  constexpr int DR = KCH >= 64 ? 1 : 64 / KCH;   // chunks between accumulator drains (64 complex K)
  Entry<float> en;   // this thread's row of every chunk, in registers
  en.init(J, gi, gi < M);

  auto stage_x = [&](int c) {   // rows k0 + c*KCH .. of X, KP columns, zero filled
    const int64_t kb = k0 + (int64_t)c * KCH;
    for (int idx = tid; idx < KCH * KP; idx += THREADS) {
      const int kk = idx % KCH, col = idx / KCH;
      const int64_t gk = kb + kk;
      const bool v = gk < k1 && col < kcols;
      cp_async8(xBase + (uint32_t)(kk * KP + col) * 8, v ? (const void*)(X + gk + (int64_t)col * ldx) : (const void*)X,
                v);
    }
  };

  uint32_t parity = 0;
  bool ok = true;
  if (nch > 0) stage_x(0);
  for (int c = 0; c < nch && ok; ++c) {
    const int64_t kb = k0 + (int64_t)c * KCH;
    const uint32_t aBuf = aBase + (uint32_t)(c & 1) * A_BUF;
    // entries of this chunk, straight into the free A buffer (its last
    // reader, the MMAs of chunk c-2, completed before chunk c-1 was issued)
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int kk = 4 * q + kq;
      const int64_t gk = kb + kk;
      const float2 e = (gi < M && gk < k1) ? en.get(gi, gk) : make_float2(0.f, 0.f);
      uint32_t pr[3], pm[3];
      split_parts<SPLIT>(e.x, pr);
      split_parts<SPLIT>(e.y, pm);
      const uint32_t ar = aBuf + a_off + (uint32_t)q * CORE;   // real part: K column kk
      const uint32_t ai = ar + (KCH / 4) * CORE;               // imaginary part: KCH + kk
#pragma unroll
      for (int s = 0; s < SPLIT; ++s) {
        st_shared(ar + s * A_PART, pr[s]);
        st_shared(ai + s * A_PART, pm[s]);
      }
    }
    static_assert(EPT == KCH / 4, "one K column group of four per entry step");
    if (c > 0) {
      const bool w = mbar_wait(smem_u32(&mbar), parity);
      if (__syncthreads_or(!w)) {
        ok = false;
        break;
      }
      parity ^= 1u;
      tc_fence_after();
      if (warp < 4 && c % DR == 0) drain<NR>(tlane);
    }
    cp_async_wait_all();
    __syncthreads();
    // B = [[Xr, Xi], [-Xi, Xr]] (N x K, K-major) from the staged rows; one
    // warp instruction per 8 x 4 core matrix
    constexpr int KC4 = KR / 4;
    for (int cell = warp; cell < (NR / 8) * KC4; cell += THREADS / 32) {
      const int nr = 8 * (cell / KC4) + (lane >> 2), kr = 4 * (cell % KC4) + kq;
      const int kk = kr % KCH, part = kr / KCH;
      const int col = nr % KP, blk = nr / KP;
      const float2 x = xs[kk * KP + col];
      const float v = part == 0 ? (blk == 0 ? x.x : x.y) : (blk == 0 ? -x.y : x.x);
      uint32_t pv[3];
      split_parts<SPLIT>(v, pv);
      const uint32_t o = (uint32_t)cell * CORE + (uint32_t)(lane >> 2) * 16 + (uint32_t)kq * 4;
#pragma unroll
      for (int s = 0; s < SPLIT; ++s) st_shared(bBase + s * B_PART + o, pv[s]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    if (c + 1 < nch) stage_x(c + 1);   // lands while the next entries are formed
    if (tid == 0) {
      tc_fence_after();
      // descriptors advance by (byte offset >> 4) in their start-address field
      const uint64_t dA = sdesc<KR>(aBuf), dB = sdesc<KR>(bBase);
      constexpr uint64_t pa = A_PART >> 4, pb = B_PART >> 4;
      // the accumulator restarts right after each drain
      const uint32_t carry = (c % DR) != 0 ? 1u : 0u;
#pragma unroll
      for (int ks = 0; ks < KR / 8; ++ks) {
        const uint64_t o = (uint64_t)(ks * 2 * CORE) >> 4;
        const uint32_t first = (ks > 0) ? 1u : carry;
        mma_tf32(tm, dA + o, dB + o, idesc, first);                // a0 b0 -> main
        mma_tf32(tm + NR, dA + o, dB + pb + o, idesc, first);      // cross terms -> correction
        mma_tf32(tm + NR, dA + pa + o, dB + o, idesc, 1u);
        if (SPLIT == 3) {
          mma_tf32(tm + NR, dA + o, dB + 2 * pb + o, idesc, 1u);
          mma_tf32(tm + NR, dA + pa + o, dB + pb + o, idesc, 1u);
          mma_tf32(tm + NR, dA + 2 * pa + o, dB + o, idesc, 1u);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar))
                   : "memory");
    }
  }
  if (ok && nch > 0) {
    const bool w = mbar_wait(smem_u32(&mbar), parity);
    if (__syncthreads_or(!w)) {
      ok = false;
    } else {
      tc_fence_after();
      if (warp < 4) drain<NR>(tlane);
    }
  }
  cp_async_wait_all();
  if (!ok) {
    if (tid == 0) atomicExch(&g_tc_status, 1);
    mbar_wait(smem_u32(&mbar), parity);   // bounded chance for MMAs in flight
  } else if (warp < 4) {
    const int64_t row = row0 + warp * 32 + lane;
#pragma unroll 1
    for (int s = 0; s < (KP + 15) / 16; ++s) {
      uint32_t hr[16], lr[16], hm[16], lm[16];
      // columns beyond KP read allocated but unused tensor memory; skipped below
      const int c0 = s * 16;
      tmem_ld16(tlane + 2 * NR + c0, hr);
      tmem_ld16(tlane + 3 * NR + c0, lr);
      tmem_ld16(tlane + 2 * NR + KP + c0, hm);
      tmem_ld16(tlane + 3 * NR + KP + c0, lm);
      tmem_wait_ld();
      if (row < M) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int col = c0 + i;
          if (col >= kcols || col >= KP) continue;
          if (T.ws < 0) {
            float2* __restrict__ Y = (float2*)J.Y;
            Y[row + ((int64_t)T.group * kcols + col) * J.ldy] =
                make_float2(__uint_as_float(hr[i]) + __uint_as_float(lr[i]),
                            __uint_as_float(hm[i]) + __uint_as_float(lm[i]));
          } else {
            ws[T.ws + (int64_t)col * M + row] = make_float4(__uint_as_float(hr[i]), __uint_as_float(lr[i]),
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

bool sketch_tc_applies(const std::vector<SketchJob>& jobs) {
  for (const auto& j : jobs)
    if (j.kcols > 64 || j.kcols < 1) return false;
  return true;
}

template <int NR, int SPLIT>
static int launch_nr(const SketchJob* dj, const TcTile* dt, unsigned ntiles, float4* ws, cudaStream_t s) {
  constexpr size_t smem = smem_bytes<NR, SPLIT>();
  static_assert(smem <= 220 * 1024, "sketch tile exceeds shared memory");
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
    case 80: return launch_nr<80, SPLIT>(dj, dt, nt, ws, s);
    case 96: return launch_nr<96, SPLIT>(dj, dt, nt, ws, s);
    case 112: return launch_nr<112, SPLIT>(dj, dt, nt, ws, s);
    default: return launch_nr<128, SPLIT>(dj, dt, nt, ws, s);
  }
}

int launch_sketch_jobs_tc(const std::vector<SketchJob>& jobs, MemTracker* mt, cudaStream_t s) {
  int64_t maxk = 0;
  int split = 2;
  for (const auto& j : jobs) maxk = std::max(maxk, j.kcols), split = std::max(split, j.split);
  const int kp = (int)((maxk + 7) / 8 * 8);   // padded width, multiple of 8
  const int nr = 2 * kp;                       // real columns, multiple of 16, <= 128
  const int KCH = split == 3 ? 16 : 32;
  // rows tiles without splitting K; split K until the launch fills the GPU
  int64_t base_tiles = 0;
  for (const auto& j : jobs)
    if (j.M > 0 && j.kcols > 0) base_tiles += (int64_t)j.groups * ((j.M + TM - 1) / TM);
  if (base_tiles == 0) return BF_OK;
  int nsplit = 1;
  while (base_tiles * nsplit < 2 * 152 && nsplit < 16) nsplit *= 2;
  std::vector<TcTile> tiles;
  std::vector<TcRegion> regs;
  int64_t wsz = 0;
  for (size_t ji = 0; ji < jobs.size(); ++ji) {
    const SketchJob& j = jobs[ji];
    if (j.M <= 0 || j.kcols <= 0) continue;
    for (int g = 0; g < j.groups; ++g) {
      // K range of the group (host copy of the node boundaries is not kept
      // here, so splits are decided per group from the job's total K)
      const int64_t ktot = j.groups == 1 ? j.Ktot : -1;
      int ns = nsplit;
      if (ktot >= 0 && ktot < (int64_t)KCH * 4 * ns) ns = 1;
      if (ktot < 0) ns = 1;   // grouped launches have enough tiles
      int64_t ws0 = -1;
      if (ns > 1) {
        ws0 = wsz;
        regs.push_back({wsz, j.M, j.kcols, j.ldy, (int64_t)g * j.kcols, ns, 0, (float2*)j.Y});
        wsz += (int64_t)ns * j.M * j.kcols;
      }
      const int64_t ks = ns > 1 ? ((ktot + ns - 1) / ns + KCH - 1) / KCH * KCH : 0;
      for (int sp = 0; sp < ns; ++sp) {
        int64_t a = 0, b = 0;
        if (ns > 1) {
          a = std::min<int64_t>(ktot, sp * ks);
          b = std::min<int64_t>(ktot, a + ks);
        }
        for (int64_t r0 = 0; r0 < j.M; r0 += TM) {
          TcTile t{(int32_t)ji, g, r0, a, b, ns > 1 ? ws0 + (int64_t)sp * j.M * j.kcols : -1};
          if (ns == 1) t.k0 = -1, t.k1 = -1;   // whole group range, resolved on the device
          tiles.push_back(t);
        }
      }
    }
  }
  const size_t jb = jobs.size() * sizeof(SketchJob), tb = tiles.size() * sizeof(TcTile),
               rb = regs.size() * sizeof(TcRegion);
  DevBuf d, w;
  BF_TRY(d.alloc(mt, jb + tb + rb + 16, s));
  if (wsz) BF_TRY(w.alloc(mt, wsz * sizeof(float4), s));
  int rc = BF_OK;
  char* p = (char*)d.p;
  if (cudaMemcpyAsync(p, jobs.data(), jb, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(p + jb, tiles.data(), tb, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      (rb && cudaMemcpyAsync(p + jb + tb, regs.data(), rb, cudaMemcpyHostToDevice, s) != cudaSuccess))
    rc = fail(BF_ECUDA, "upload of sketch jobs failed");
  const SketchJob* dj = (const SketchJob*)p;
  const TcTile* dt = (const TcTile*)(p + jb);
  const unsigned nt = (unsigned)tiles.size();
  if (!rc) rc = split == 3 ? launch_split<3>(nr, dj, dt, nt, (float4*)w.p, s) : launch_split<2>(nr, dj, dt, nt, (float4*)w.p, s);
  if (!rc && !regs.empty()) {
    dim3 grid(64, (unsigned)regs.size());
    note_launch();
    tc_reduce_kernel<<<grid, 256, 0, s>>>((const TcRegion*)(p + jb + tb), (int)regs.size(), (const float4*)w.p);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) rc = fail(BF_ECUDA, std::string("sketch reduce: ") + cudaGetErrorString(e));
  }
  w.release(s);
  d.release(s);
  return rc;
}

int tc_status(bool reset) {
  int v = 0;
  BF_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_tc_status, sizeof(int)));
  if (v && reset) {
    const int z = 0;
    BF_CUDA_TRY(cudaMemcpyToSymbol(g_tc_status, &z, sizeof(int)));
  }
  return v ? fail(BF_ETIMEOUT, "a tensor-core sketch wait gave up (device flag set)") : BF_OK;
}

}  // namespace bf
