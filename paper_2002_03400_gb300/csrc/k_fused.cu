// Fused apply of a finished factorization (eq. hybrid_butterfly_mat) in two
// launches instead of L + 3 stage launches plus a gather and a scatter.
//
// The hybrid factorization splits at the centre level l_m: every block of
// the factors on the input side of B depends on one subtree of the input
// tree, every block on the output side on one subtree of the output tree
// (the complementary structure behind the paper's hybrid distributed layout,
// Sec. 6.2).  So for y = F x:
//   kernel 1: one CTA per (subtree of T_S at level L - l_m, column slice)
//     gathers its rows of x (through the tree permutation) into shared
//     memory and applies V^0, W^1 .. W^(l_m) and B there, level after level
//     (a CTA barrier between levels), writing its blocks of the centre-level
//     vector to a global exchange buffer;
//   kernel 2: one CTA per (subtree of T_T at level l_m, column slice) reads
//     its blocks of that vector and applies R^(l_m) .. R^(L-1) and U^L in
//     shared memory, then scatters its rows of y.
// F^H x and F^T x run the same way with the trees' roles swapped (kernel 1
// over subtrees of T_T: U^H, R^H levels, B^H; kernel 2 over subtrees of T_S:
// W^H levels, V^0).  The kernel boundary is the one device-wide exchange.
//
// Task lists are the stage apply's (apply_tasks_host), regrouped per subtree
// with their offsets remapped to the subtree's shared-memory rows, so every
// output is the same sequential FMA chain (terms in order, k ascending) as
// in the stage kernels: results equal the stage apply's bit for bit.
// Intermediates are row-major with the CTA's column-slice width CS.
#include <algorithm>
#include <cstring>
#include <map>

#include "bf_internal.h"
#include "cx.cuh"

namespace bf {

namespace {
constexpr int FTHREADS = 256;
constexpr size_t FUSED_SMEM_MAX = 200 * 1024;

struct FusedArgs {
  const FusedGroup* groups;
  const FusedLevel* levels;
  const StageTask* tasks;
  const int32_t* rowmap;
  const void* x;        // kernel 1: the user's x (ld ldx);   kernel 2: the exchange buffer
  int64_t ldx;
  void* y;              // kernel 1: the exchange buffer;     kernel 2: the user's y (ld ldy)
  int64_t ldy;
  const int64_t* perm;  // kernel 1: input-side tree -> user rows; kernel 2: output side (null: identity)
  int conj;             // F^T: conjugate on the way in and out
  int nrhs, CS;
  int io_max, lvl_max;  // rows of the staged input/output block and of one intermediate (per CS columns)
  int tasks_max;        // tasks and row tiles of the largest level (shared-memory copies)
  int rows_max;
  const FusedChunk* chunks;
  const FusedSeg* segs;
};
}  // namespace

// each thread computes a tile of FRT rows x FCT columns of one task: per k,
// FRT factor entries and FCT inputs feed FRT * FCT complex FMAs
constexpr int FRT = 4, FCT = 2;
// shared-memory staging area for the factor blocks of one chunk: two
// buffers, so that the next chunk's copies run while this one computes
constexpr size_t FAC_BYTES = 24 * 1024;

__device__ __forceinline__ void cp_async_elem(void* dst, const void* src, int bytes) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  if (bytes == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}

// The row tiles of one chunk: items (tile of FRT rows of one task, NC
// columns); every output is its own FMA chain over the terms in order and k
// ascending.  FAST: factor entries from the staging area and inputs from
// shared memory (shared-memory loads); otherwise generic loads (unstaged
// entries in global memory, or kernel 2's first inputs in the exchange buffer).
template <typename R, int NC, bool FAST>
__device__ __forceinline__ void fused_tiles(const StageTask* stk, const int32_t* smap, const FusedChunk C,
                                            const typename Cx<R>::V* fac, const typename Cx<R>::V* in, int64_t in_rs,
                                            int64_t in_c0, typename Cx<R>::V* out, int64_t out_rs, int64_t out_c0,
                                            int cw, int tid) {
  using V = typename Cx<R>::V;
  const int nct = (cw + NC - 1) / NC;
  for (int idx = C.tile0 * nct + tid; idx < C.tile1 * nct; idx += FTHREADS) {
    const int tl = idx / nct, ct = idx - tl * nct;
    const int32_t m = smap[tl];
    const StageTask& tk = stk[m >> 16];
    const int i0 = m & 0xffff, cc = ct * NC;
    const int nr = min(FRT, tk.M - i0), ncl = min(NC, cw - cc);
    V acc[FRT][NC];
#pragma unroll
    for (int r = 0; r < FRT; ++r)
#pragma unroll
      for (int j = 0; j < NC; ++j) acc[r][j] = Cx<R>::make(0, 0);
    for (int q = 0; q < tk.nterms; ++q) {
      const StageTerm& T = tk.t[q];
      // staged terms hold the staging-area offset of their entries
      const V* __restrict__ mat = (FAST || T.pad) ? fac + (intptr_t)T.mat : (const V*)T.mat;
      const int K = T.K, ldm = T.ldm, cj = T.conjT;
      const int istep = cj ? ldm : 1, kstep = cj ? 1 : ldm;
      // rows past the tile's end re-read its last row (loaded, never stored)
      int mo[FRT];
#pragma unroll
      for (int r = 0; r < FRT; ++r) mo[r] = (i0 + min(r, nr - 1)) * istep;
      const V* xin = in + T.in_off * in_rs + in_c0 + cc;
      int xo[NC];
#pragma unroll
      for (int j = 0; j < NC; ++j) xo[j] = min(j, ncl - 1);
#pragma unroll 2
      for (int k = 0; k < K; ++k) {
        V e[FRT], xv[NC];
        const int mk = k * kstep;
        const int64_t xk = (int64_t)k * in_rs;
#pragma unroll
        for (int r = 0; r < FRT; ++r) e[r] = mat[mo[r] + mk];
#pragma unroll
        for (int j = 0; j < NC; ++j) xv[j] = xin[xk + xo[j]];
#pragma unroll
        for (int r = 0; r < FRT; ++r) {
          if (cj) e[r].y = -e[r].y;
#pragma unroll
          for (int j = 0; j < NC; ++j) cmac(acc[r][j], e[r], xv[j]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < FRT; ++r)
#pragma unroll
      for (int j = 0; j < NC; ++j)
        if (r < nr && j < ncl) out[(tk.out_off + i0 + r) * out_rs + out_c0 + cc + j] = acc[r][j];
  }
}

// FIRST: kernel 1 (stages rows of x, writes the exchange buffer); otherwise
// kernel 2 (reads the exchange buffer, stages rows of y).  Shared memory:
// the staged rows (io), two level buffers, the current level's task
// descriptors and tile map, and the staging area of the factor blocks.
// Per level: the descriptors are copied once; then per chunk the factor
// blocks it reads are copied with cp.async by all threads, and its tiles
// are computed from shared memory only.
template <typename R, bool FIRST>
__global__ void __launch_bounds__(FTHREADS) fused_half_kernel(const FusedArgs a) {
  using V = typename Cx<R>::V;
  extern __shared__ __align__(16) uint8_t fused_smem[];
  const FusedGroup G = a.groups[blockIdx.x];
  const int CS = a.CS;
  const int c0 = blockIdx.y * CS;
  const int cw = min(CS, a.nrhs - c0);   // columns of this slice
  V* io = (V*)fused_smem;
  V* buf0 = io + (int64_t)a.io_max * CS;
  V* buf1 = buf0 + (int64_t)a.lvl_max * CS;
  StageTask* stk =
      (StageTask*)(fused_smem + ((((int64_t)a.io_max + 2 * (int64_t)a.lvl_max) * CS * sizeof(V) + 15) & ~(int64_t)15));
  int32_t* smap = (int32_t*)(stk + a.tasks_max);
  V* fac = (V*)((uint8_t*)stk + (((int64_t)a.tasks_max * sizeof(StageTask) + (int64_t)a.rows_max * 4 + 15) & ~(int64_t)15));
  const int tid = threadIdx.x;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (FIRST) {
    const V* x = (const V*)a.x;
    for (int idx = tid; idx < G.io_rows * cw; idx += FTHREADS) {
      const int c = idx / G.io_rows, i = idx - c * G.io_rows;
      const int64_t row = G.io_row0 + i;
      V v = x[(a.perm ? a.perm[row] : row) + (int64_t)(c0 + c) * a.ldx];
      if (a.conj) v.y = -v.y;
      io[i * CS + c] = v;
    }
  } else {
    // the exchange buffer is complete once kernel 1 has finished; before
    // that, warm L2 with this subtree's first-chunk factor blocks
    const FusedLevel L0 = a.levels[G.lev0];
    if (L0.nchunks > 0) {
      const FusedChunk C0 = a.chunks[L0.chunk0];
      for (int g = tid >> 5; g < C0.nseg; g += FTHREADS / 32) {
        const FusedSeg sg = a.segs[C0.seg0 + g];
        const int64_t bytes = (int64_t)sg.count * sizeof(V);
        for (int64_t off = (int64_t)(tid & 31) * 128; off < bytes; off += 32 * 128)
          asm volatile("prefetch.global.L2 [%0];" ::"l"((const char*)sg.src + off));
      }
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
  }
  // all chunks of the subtree in order, level after level; chunk k + 1's
  // factor copies are issued before chunk k is computed
  const int lane = tid & 31, warp = tid >> 5;
  constexpr int FE = (int)(FAC_BYTES / sizeof(V));
  int par = 0;                                   // staging buffer of the current chunk
  int nlv = 0, nch = 0;                          // next chunk to issue
  auto advance = [&](int& l, int& c) {
    while (l < G.nlev && c >= a.levels[G.lev0 + l].nchunks) ++l, c = 0;
  };
  advance(nlv, nch);
  int issued_par = 0;
  auto issue_next = [&]() {
    if (nlv >= G.nlev) {
      asm volatile("cp.async.commit_group;" ::: "memory");   // keeps one group per chunk
      return;
    }
    const FusedLevel Lq = a.levels[G.lev0 + nlv];
    const FusedChunk C = a.chunks[Lq.chunk0 + nch];
    if (C.staged) {
      V* dst = fac + issued_par * FE;
      for (int g = warp; g < C.nseg; g += FTHREADS / 32) {
        const FusedSeg sg = a.segs[C.seg0 + g];
        if (lane < sg.count) cp_async_elem(dst + sg.dst + lane, (const V*)sg.src + lane, (int)sizeof(V));
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    issued_par ^= 1;
    ++nch;
    advance(nlv, nch);
  };
  issue_next();   // chunk 0
  for (int lv = 0; lv < G.nlev; ++lv) {
    const FusedLevel Lv = a.levels[G.lev0 + lv];
    // this level's task descriptors and tile map into shared memory (the
    // previous level's last chunk ended with a barrier)
    {
      const uint4* src = (const uint4*)(a.tasks + Lv.task0);
      uint4* dst = (uint4*)stk;
      const int nv = Lv.ntasks * (int)(sizeof(StageTask) / sizeof(uint4));
      for (int v = tid; v < nv; v += FTHREADS) dst[v] = src[v];
      for (int r = tid; r < Lv.tiles; r += FTHREADS) smap[r] = a.rowmap[Lv.map0 + r];
    }
    const bool first = lv == 0, last = lv == G.nlev - 1;
    const bool in_smem = !(first && !FIRST);       // kernel 2 reads the exchange buffer first
    // input rows: the staged x (kernel 1) or the exchange buffer (kernel 2)
    // at the first level, else the previous level's buffer
    const V* in;
    int64_t in_rs, in_c0;
    if (first) {
      if (FIRST) in = io, in_rs = CS, in_c0 = 0;
      else in = (const V*)a.x, in_rs = a.nrhs, in_c0 = c0;
    } else {
      in = (lv & 1) ? buf0 : buf1, in_rs = CS, in_c0 = 0;
    }
    V* out;
    int64_t out_rs, out_c0;
    if (last) {
      if (FIRST) out = (V*)a.y, out_rs = a.nrhs, out_c0 = c0;
      else out = io, out_rs = CS, out_c0 = 0;
    } else {
      out = (lv & 1) ? buf1 : buf0, out_rs = CS, out_c0 = 0;
    }
    for (int ch = 0; ch < Lv.nchunks; ++ch) {
      const FusedChunk C = a.chunks[Lv.chunk0 + ch];
      issue_next();                                  // the next chunk's copies
      asm volatile("cp.async.wait_group 1;" ::: "memory");   // this chunk's copies have landed
      __syncthreads();   // (also orders the descriptors, the staged x and the previous level's outputs)
      const V* fb = fac + par * FE;
      const bool fast = C.staged && in_smem;
      if (cw == 1) {
        if (fast) fused_tiles<R, 1, true>(stk, smap, C, fb, in, in_rs, in_c0, out, out_rs, out_c0, cw, tid);
        else fused_tiles<R, 1, false>(stk, smap, C, fb, in, in_rs, in_c0, out, out_rs, out_c0, cw, tid);
      } else {
        if (fast) fused_tiles<R, FCT, true>(stk, smap, C, fb, in, in_rs, in_c0, out, out_rs, out_c0, cw, tid);
        else fused_tiles<R, FCT, false>(stk, smap, C, fb, in, in_rs, in_c0, out, out_rs, out_c0, cw, tid);
      }
      par ^= 1;
      __syncthreads();   // this chunk's staging buffer and outputs are complete
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  if (!FIRST) {
    V* y = (V*)a.y;
    for (int idx = tid; idx < G.io_rows * cw; idx += FTHREADS) {
      const int c = idx / G.io_rows, i = idx - c * G.io_rows;
      const int64_t row = G.io_row0 + i;
      V v = io[i * CS + c];
      if (a.conj) v.y = -v.y;
      y[(a.perm ? a.perm[row] : row) + (int64_t)(c0 + c) * a.ldy] = v;
    }
  }
}

namespace {

// Regroups the stage apply's tasks of stages [s0, s1) into per-subtree
// levels.  forward: groups follow the data from the first stage's input
// rows (part = partition of those rows); otherwise they follow it back from
// the last stage's output rows.  Offsets become subtree-local rows except
// the exchange side (kernel 1's last outputs, kernel 2's first inputs).
// Locates the factor block that holds a term's entries: its first element
// and element count, or false.
struct BlockLocator {
  const Fact* F;
  int dtype;
  bool find(const void* p, const char** base, int64_t* count) const {
    const size_t es = elem_bytes(dtype);
    for (const Stage& S : F->st) {
      const char* b = (const char*)(dtype == BF_C128 ? S.d64.p : S.d32.p);
      if (!b || (const char*)p < b || (const char*)p >= b + S.total * (int64_t)es) continue;
      const int64_t e = ((const char*)p - b) / (int64_t)es;
      const int blk = (int)(std::upper_bound(S.off.begin(), S.off.end(), e) - S.off.begin()) - 1;
      if (blk < 0) return false;
      *base = b + S.off[blk] * (int64_t)es;
      *count = (int64_t)S.rows[blk] * S.cols[blk];
      return true;
    }
    return false;
  }
};

// Splits the tasks [t0, t1) of one level into chunks whose factor blocks fit
// the staging area together (a task whose blocks alone do not fit forms an
// unstaged chunk and reads global memory); rewrites the staged terms' entry
// pointers as staging-area offsets.
bool chunk_level(FusedHalf& H, FusedLevel& Lv, const BlockLocator& loc, int64_t fac_elems) {
  Lv.chunk0 = (int32_t)H.chunks.size();
  std::map<const char*, int64_t> placed;   // block -> staging offset in this chunk
  int64_t used = 0;
  FusedChunk cur{0, 0, (int32_t)H.segs.size(), 0, 1, 0};
  int tile = 0;
  auto close = [&]() {
    if (cur.tile1 > cur.tile0) H.chunks.push_back(cur);
    cur = FusedChunk{tile, tile, (int32_t)H.segs.size(), 0, 1, 0};
    placed.clear();
    used = 0;
  };
  const size_t es = elem_bytes(loc.dtype);
  for (int t = 0; t < Lv.ntasks; ++t) {
    StageTask& tk = H.tasks[Lv.task0 + t];
    const int tiles = (tk.M + FRT - 1) / FRT;
    const char* base[2] = {nullptr, nullptr};
    int64_t cnt[2] = {0, 0}, need = 0;
    for (int q = 0; q < tk.nterms; ++q) {
      if (!loc.find(tk.t[q].mat, &base[q], &cnt[q])) return false;
      const bool dup = q == 1 && base[1] == base[0];
      if (!placed.count(base[q]) && !dup) need += cnt[q];
    }
    int64_t alone = cnt[0] + (tk.nterms == 2 && base[1] != base[0] ? cnt[1] : 0);
    if (alone > fac_elems) {   // unstaged: its own chunk, entries from global memory
      close();
      cur.staged = 0;
      cur.tile1 = tile + tiles;
      tile += tiles;
      H.chunks.push_back(cur);
      cur = FusedChunk{tile, tile, (int32_t)H.segs.size(), 0, 1, 0};
      continue;
    }
    if (used + need > fac_elems) close();
    for (int q = 0; q < tk.nterms; ++q) {
      auto it = placed.find(base[q]);
      if (it == placed.end()) {
        it = placed.insert({base[q], used}).first;
        for (int64_t e = 0; e < cnt[q]; e += 32) {   // pieces of <= 32 elements: one warp copies one
          H.segs.push_back(FusedSeg{base[q] + e * (int64_t)es, (int32_t)(used + e),
                                    (int32_t)std::min<int64_t>(32, cnt[q] - e)});
          ++cur.nseg;
        }
        used += cnt[q];
      }
      const int64_t delta = ((const char*)tk.t[q].mat - base[q]) / (int64_t)es;
      tk.t[q].mat = (const void*)(intptr_t)(it->second + delta);
      tk.t[q].pad = 1;
    }
    cur.tile1 = tile + tiles;
    tile += tiles;
  }
  close();
  Lv.nchunks = (int32_t)(H.chunks.size() - Lv.chunk0);
  return tile == Lv.tiles;
}

bool build_half(const std::vector<StageTask>& all, const ApplyPlan& ap, int s0, int s1,
                const std::vector<int64_t>& part, bool forward, const BlockLocator& loc, FusedHalf& H) {
  const int ng = (int)part.size() - 1;
  const int ns = s1 - s0;
  auto part_of = [&](int64_t row) {
    const auto it = std::upper_bound(part.begin(), part.end(), row);
    return (int)(it - part.begin()) - 1;
  };
  // group of every task of every stage of the half
  std::vector<std::vector<int>> grp(ns);
  for (int s = 0; s < ns; ++s) grp[s].assign(ap.count[s0 + s], -1);
  auto task = [&](int s, int t) -> const StageTask& { return all[ap.first[s0 + s] + t]; };
  if (forward) {
    std::map<int64_t, int> owner;   // output row start of the previous stage -> group
    for (int s = 0; s < ns; ++s) {
      std::map<int64_t, int> next;
      for (int t = 0; t < ap.count[s0 + s]; ++t) {
        const StageTask& tk = task(s, t);
        int g = -1;
        for (int q = 0; q < tk.nterms; ++q) {
          int gq = -1;
          if (s == 0) {
            gq = part_of(tk.t[q].in_off);
          } else {
            const auto it = owner.find(tk.t[q].in_off);
            if (it == owner.end()) return false;
            gq = it->second;
          }
          if (gq < 0 || gq >= ng || (g >= 0 && gq != g)) return false;
          g = gq;
        }
        grp[s][t] = g;
        next[tk.out_off] = g;
      }
      owner.swap(next);
    }
  } else {
    std::map<int64_t, int> need;   // input row start of the next stage -> group
    for (int s = ns - 1; s >= 0; --s) {
      std::map<int64_t, int> prev;
      for (int t = 0; t < ap.count[s0 + s]; ++t) {
        const StageTask& tk = task(s, t);
        int g = -1;
        if (s == ns - 1) {
          g = part_of(tk.out_off);
        } else {
          const auto it = need.find(tk.out_off);
          if (it == need.end()) return false;
          g = it->second;
        }
        if (g < 0 || g >= ng) return false;
        grp[s][t] = g;
        for (int q = 0; q < tk.nterms; ++q) {
          const auto ins = prev.insert({tk.t[q].in_off, g});
          if (!ins.second && ins.first->second != g) return false;
        }
      }
      need.swap(prev);
    }
  }
  // per group: levels of its tasks with local rows
  H.groups.assign(ng, FusedGroup{});
  H.levels.clear();
  H.tasks.clear();
  H.rowmap.clear();
  H.chunks.clear();
  H.segs.clear();
  H.io_max = 0;
  H.lvl_max = 0;
  H.tasks_max = 0;
  H.rows_max = 0;
  for (int g = 0; g < ng; ++g) {
    FusedGroup& G = H.groups[g];
    G.lev0 = (int32_t)H.levels.size();
    G.nlev = ns;
    G.io_row0 = (int32_t)part[g];
    G.io_rows = (int32_t)(part[g + 1] - part[g]);
    H.io_max = std::max(H.io_max, G.io_rows);
    if (G.io_rows >= (1 << 26)) return false;
    std::map<int64_t, int64_t> local_prev, local_cur;   // global row start -> local row
    for (int s = 0; s < ns; ++s) {
      FusedLevel Lv{};
      Lv.task0 = (int32_t)H.tasks.size();
      Lv.map0 = (int32_t)H.rowmap.size();
      int64_t rows = 0;
      local_cur.clear();
      for (int t = 0; t < ap.count[s0 + s]; ++t) {
        if (grp[s][t] != g) continue;
        StageTask tk = task(s, t);
        const int li = (int)(H.tasks.size() - Lv.task0);
        if (li >= (1 << 15) || tk.M >= (1 << 16)) return false;
        for (int q = 0; q < tk.nterms; ++q) {
          StageTerm& T = tk.t[q];
          if (s == 0) {
            if (forward) T.in_off -= part[g];          // staged input rows
          } else {
            const auto it = local_prev.find(T.in_off);
            if (it == local_prev.end()) return false;
            T.in_off = it->second;
          }
        }
        const bool last = s == ns - 1;
        if (last && !forward) {
          tk.out_off -= part[g];                       // staged output rows
        } else if (!(last && forward)) {
          local_cur[tk.out_off] = rows;                 // intermediate rows of this subtree
          tk.out_off = rows;
        }
        for (int i = 0; i < tk.M; i += FRT) H.rowmap.push_back((int32_t)((li << 16) | i));
        rows += tk.M;
        H.tasks.push_back(tk);
      }
      Lv.ntasks = (int32_t)(H.tasks.size() - Lv.task0);
      Lv.rows = (int32_t)rows;
      Lv.tiles = (int32_t)(H.rowmap.size() - Lv.map0);
      H.tasks_max = std::max(H.tasks_max, (int)Lv.ntasks);
      H.rows_max = std::max<int64_t>(H.rows_max, Lv.tiles);
      const bool last = s == ns - 1;
      if (!last) H.lvl_max = std::max<int64_t>(H.lvl_max, rows);
      if (rows >= ((int64_t)1 << 26)) return false;
      if (!chunk_level(H, Lv, loc, (int64_t)(FAC_BYTES / elem_bytes(loc.dtype)))) return false;
      H.levels.push_back(Lv);
      local_prev.swap(local_cur);
    }
  }
  return true;
}

// Every access the kernel makes through the tables stays inside its buffer:
// first-level inputs inside the staged rows (kernel 1) or the exchange
// buffer (kernel 2), later inputs inside the previous level's rows, outputs
// inside the level's rows, the exchange buffer (kernel 1's last level) or
// the staged rows (kernel 2's last level); row maps name existing rows.
bool validate_half(const FusedHalf& H, bool first_half, int64_t ex_rows, int64_t fac_elems) {
  for (const FusedGroup& G : H.groups) {
    if (G.nlev < 1 || G.lev0 < 0 || G.lev0 + G.nlev > (int)H.levels.size() || G.io_rows < 0 ||
        G.io_rows > H.io_max)
      return false;
    int64_t prev_rows = 0;
    for (int lv = 0; lv < G.nlev; ++lv) {
      const FusedLevel& Lv = H.levels[G.lev0 + lv];
      const bool first = lv == 0, last = lv == G.nlev - 1;
      if (Lv.task0 < 0 || Lv.task0 + Lv.ntasks > (int)H.tasks.size() || Lv.map0 < 0) return false;
      if (!last && Lv.rows > H.lvl_max) return false;
      const int64_t in_lim = first ? (first_half ? G.io_rows : ex_rows) : prev_rows;
      const int64_t out_lim = last ? (first_half ? ex_rows : G.io_rows) : Lv.rows;
      for (int t = 0; t < Lv.ntasks; ++t) {
        const StageTask& tk = H.tasks[Lv.task0 + t];
        if (tk.M < 1 || tk.out_off < 0 || tk.out_off + tk.M > out_lim || tk.nterms < 1 || tk.nterms > 2) return false;
        for (int q = 0; q < tk.nterms; ++q) {
          const StageTerm& T = tk.t[q];
          if (T.K < 0 || T.in_off < 0 || T.in_off + T.K > in_lim || T.ldm < 1) return false;
          if (T.ldm < (T.conjT ? T.K : tk.M)) return false;
          if (T.pad) {   // staged: every entry read lies in the staging area
            const int64_t off = (int64_t)(intptr_t)T.mat;
            const int64_t last_e = T.conjT ? (int64_t)(T.K - 1) + (int64_t)(tk.M - 1) * T.ldm
                                           : (int64_t)(tk.M - 1) + (int64_t)(T.K - 1) * T.ldm;
            if (off < 0 || (T.K > 0 && off + last_e >= fac_elems)) return false;
          }
        }
      }
      if (Lv.map0 + (int64_t)Lv.tiles > (int64_t)H.rowmap.size() || Lv.tiles > H.rows_max) return false;
      int64_t covered = 0;
      for (int r = 0; r < Lv.tiles; ++r) {
        const int32_t m = H.rowmap[Lv.map0 + r];
        const int li = m >> 16, i = m & 0xffff;
        if (li < 0 || li >= Lv.ntasks || i >= H.tasks[Lv.task0 + li].M) return false;
        covered += std::min(FRT, H.tasks[Lv.task0 + li].M - i);
      }
      if (covered != Lv.rows) return false;
      if (Lv.chunk0 < 0 || Lv.chunk0 + Lv.nchunks > (int)H.chunks.size()) return false;
      int next_tile = 0;
      for (int c = 0; c < Lv.nchunks; ++c) {
        const FusedChunk& C = H.chunks[Lv.chunk0 + c];
        if (C.tile0 != next_tile || C.tile1 < C.tile0 || C.seg0 < 0 || C.seg0 + C.nseg > (int)H.segs.size())
          return false;
        for (int g = 0; g < C.nseg; ++g) {
          const FusedSeg& sg = H.segs[C.seg0 + g];
          if (sg.dst < 0 || sg.count < 0 || (int64_t)sg.dst + sg.count > fac_elems) return false;
        }
        for (int t = C.tile0; t < C.tile1; ++t) {   // unstaged chunks hold unstaged terms only
          const StageTask& tk = H.tasks[Lv.task0 + (H.rowmap[Lv.map0 + t] >> 16)];
          for (int q = 0; q < tk.nterms; ++q)
            if ((tk.t[q].pad != 0) != (C.staged != 0)) return false;
        }
        next_tile = C.tile1;
      }
      if (next_tile != Lv.tiles) return false;
      prev_rows = Lv.rows;
    }
  }
  return true;
}

static_assert(sizeof(StageTask) % 16 == 0, "task descriptors are copied as 16-byte vectors");
size_t half_smem(const FusedHalf& H, int CS, size_t es) {
  const size_t data = (((size_t)H.io_max + 2 * (size_t)H.lvl_max) * CS * es + 15) & ~(size_t)15;
  const size_t meta = ((size_t)H.tasks_max * sizeof(StageTask) + (size_t)H.rows_max * sizeof(int32_t) + 15) & ~(size_t)15;
  return data + meta + 2 * FAC_BYTES;
}

// 0: by the tuner's measurement, 1: stage launches only, 2: fused where it
// applies, 3: persistent where it applies, 4: grouped where it applies
int g_apply_engine = 0;

}  // namespace

int set_apply_engine(int e) {
  if (e < 0 || e > 4)
    return fail(BF_EINVAL, "apply engine must be 0 (tuned), 1 (stages), 2 (fused), 3 (persistent) or 4 (grouped)");
  g_apply_engine = e;
  return BF_OK;
}
int apply_engine() { return g_apply_engine; }

// Host half of build_fused: the regrouped, validated tables (fp.ok false
// when the grouping does not apply); no device work.
bool plan_fused(const Fact* F, int opC, int dtype, FusedPlan& fp) {
  const Plan* P = F->plan;
  const int L = F->L, lm = F->lm;
  ApplyPlan ap;
  std::vector<StageTask> all;
  apply_tasks_host(F, opC, dtype, ap, all);
  const int nst = (int)ap.first.size();
  const int s1 = opC ? (L - lm) + 2 : lm + 2;
  if (s1 < 1 || s1 >= nst) return false;
  const std::vector<int64_t>& p1 = opC ? P->offT[lm] : P->offS[L - lm];
  const std::vector<int64_t>& p2 = opC ? P->offS[L - lm] : P->offT[lm];
  const BlockLocator loc{F, dtype};
  if (!build_half(all, ap, 0, s1, p1, true, loc, fp.h[0]) || !build_half(all, ap, s1, nst, p2, false, loc, fp.h[1]))
    return false;
  fp.ex_rows = ap.level_rows_max;
  const int64_t fe = (int64_t)(FAC_BYTES / elem_bytes(dtype));
  return validate_half(fp.h[0], true, fp.ex_rows, fe) && validate_half(fp.h[1], false, fp.ex_rows, fe);
}

int build_fused(Fact* F, int opC, int dtype, cudaStream_t s) {
  FusedPlan& fp = F->fp[opC][dtype];
  if (fp.built) return BF_OK;
  fp = FusedPlan();
  fp.built = true;
  if (!plan_fused(F, opC, dtype, fp)) return BF_OK;   // not expressible per subtree: the stage apply serves
  const size_t es = elem_bytes(dtype);
  if (half_smem(fp.h[0], 1, es) > FUSED_SMEM_MAX || half_smem(fp.h[1], 1, es) > FUSED_SMEM_MAX) return BF_OK;
  for (int h = 0; h < 2; ++h) {
    FusedHalf& H = fp.h[h];
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t sz[6] = {H.groups.size() * sizeof(FusedGroup), H.levels.size() * sizeof(FusedLevel),
                          H.tasks.size() * sizeof(StageTask), H.rowmap.size() * sizeof(int32_t),
                          H.chunks.size() * sizeof(FusedChunk), H.segs.size() * sizeof(FusedSeg)};
    const void* src[6] = {H.groups.data(), H.levels.data(), H.tasks.data(), H.rowmap.data(), H.chunks.data(),
                          H.segs.data()};
    size_t off[6], tot = 0;
    for (int i = 0; i < 6; ++i) off[i] = tot, tot += al(sz[i]);
    BF_TRY(H.dev.alloc(&F->mem, tot + 256, nullptr));
    std::vector<char> host(tot);
    for (int i = 0; i < 6; ++i)
      if (sz[i]) memcpy(host.data() + off[i], src[i], sz[i]);
    char* p = (char*)H.dev.p;
    BF_CUDA_TRY(cudaMemcpyAsync(p, host.data(), host.size(), cudaMemcpyHostToDevice, s));
    BF_CUDA_TRY(host_sync(s));
    H.d_groups = (const FusedGroup*)(p + off[0]);
    H.d_levels = (const FusedLevel*)(p + off[1]);
    H.d_tasks = (const StageTask*)(p + off[2]);
    H.d_rowmap = (const int32_t*)(p + off[3]);
    H.d_chunks = (const FusedChunk*)(p + off[4]);
    H.d_segs = (const FusedSeg*)(p + off[5]);
  }
  fp.ok = true;
  return BF_OK;
}

// Column-slice width: the tuned one, else the widest power of two up to 16
// (complex64) / 8 (complex128) whose staged rows fit the shared-memory budget.
int fused_slice_width(const FusedPlan& fp, int64_t nrhs, int dtype) {
  const size_t es = elem_bytes(dtype);
  const int tuned = fp.cs[nrhs_class(nrhs)];
  int cs = tuned > 0 ? tuned : (dtype == BF_C64 ? 16 : 8);
  while (cs > 1 && cs / 2 >= nrhs) cs /= 2;
  while (cs > 1 && (half_smem(fp.h[0], cs, es) > 96 * 1024 || half_smem(fp.h[1], cs, es) > 96 * 1024)) cs /= 2;
  return cs;
}

int run_fused(Fact* F, int opC, int dtype, int64_t nrhs, const void* x, int64_t ldx, void* y, int64_t ldy, int conj,
              void* exch, cudaStream_t s, int cs_override) {
  const FusedPlan& fp = F->fp[opC][dtype];
  const Plan* P = F->plan;
  if (nrhs > (int64_t)INT32_MAX) return fail(BF_EINVAL, "nrhs too large");
  const int CS = cs_override > 0 ? cs_override : fused_slice_width(fp, nrhs, dtype);
  const size_t es = elem_bytes(dtype);
  const int64_t slices = (nrhs + CS - 1) / CS;
  if (slices > 65535) return fail(BF_EINVAL, "too many column slices for one launch");
  const int64_t* perm_in = (const int64_t*)(opC ? P->d_permT.p : P->d_permS.p);
  const int64_t* perm_out = (const int64_t*)(opC ? P->d_permS.p : P->d_permT.p);
  const bool id_in = opC ? P->identT : P->identS, id_out = opC ? P->identS : P->identT;
  for (int h = 0; h < 2; ++h) {
    const FusedHalf& H = fp.h[h];
    FusedArgs a{};
    a.groups = H.d_groups;
    a.levels = H.d_levels;
    a.tasks = H.d_tasks;
    a.rowmap = H.d_rowmap;
    a.x = h == 0 ? x : exch;
    a.ldx = ldx;
    a.y = h == 0 ? exch : y;
    a.ldy = ldy;
    a.perm = h == 0 ? (id_in ? nullptr : perm_in) : (id_out ? nullptr : perm_out);
    a.conj = conj;
    a.nrhs = (int)nrhs;
    a.CS = CS;
    a.io_max = H.io_max;
    a.lvl_max = (int)H.lvl_max;
    a.tasks_max = H.tasks_max;
    a.rows_max = (int)H.rows_max;
    a.chunks = H.d_chunks;
    a.segs = H.d_segs;
    const size_t smem = half_smem(H, CS, es);
    if (smem > FUSED_SMEM_MAX) return fail(BF_EINVAL, "column slice too wide for shared memory");
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)H.groups.size(), (unsigned)slices);
    cfg.blockDim = dim3(FTHREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = h == 1 ? 1 : 0;   // kernel 2 may start while kernel 1 runs; it waits before reading
    cudaError_t e = cudaSuccess;
    note_launch();
    if (dtype == BF_C128) {
      auto k = h == 0 ? fused_half_kernel<double, true> : fused_half_kernel<double, false>;
      BF_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FUSED_SMEM_MAX));
      e = cudaLaunchKernelEx(&cfg, k, a);
    } else {
      auto k = h == 0 ? fused_half_kernel<float, true> : fused_half_kernel<float, false>;
      BF_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FUSED_SMEM_MAX));
      e = cudaLaunchKernelEx(&cfg, k, a);
    }
    if (e != cudaSuccess) return fail(BF_ECUDA, std::string("fused apply launch: ") + cudaGetErrorString(e));
  }
  return BF_OK;
}

}  // namespace bf
