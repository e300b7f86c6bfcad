// Grouped apply of a finished factorization (eq. hybrid_butterfly_mat): the
// L + 3 stages in runs of `depth` consecutive stages, one launch per run.
//
// The apply's chain only ever reads the previous stage's output, and in a
// butterfly each block of level j + 1 reads two blocks of level j (W^j: the
// two children of a column-tree node; R^j and the adjoints likewise), so the
// tasks of a few consecutive stages fall into small connected groups (for
// the W levels with depth 3: 4 + 4 + 4 blocks whose inputs are 8 blocks of
// the level below).  One CTA per (group, column slice):
//   - copies the group's factor blocks into shared memory before waiting
//     for the previous launch (they do not depend on it; programmatic
//     dependent launch), then the group's input rows of the previous run's
//     output (or of x);
//   - computes the run's stages one after another, the inner stages' blocks
//     in shared memory, and writes only the last stage's blocks to global
//     memory (one of two level buffers, or y).
// So an apply takes ceil((L + 3) / depth) launches, each reading its inputs
// once and writing its outputs once.  Every output is the same FMA chain as
// in the stage kernels (terms in order, k ascending): results equal the
// stage apply's bit for bit.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>

#include "bf_internal.h"
#include "cx.cuh"

namespace bf {

namespace {
constexpr int GT = 256;
constexpr size_t GR_SMEM_LIMIT = 110 * 1024;   // two CTAs per SM
constexpr size_t GR_FAC_LIMIT = 40 * 1024;     // staged factor bytes per group (more: read in place)

struct GroupedArgs {
  const GroupedGroup* groups;
  const GroupedTask* tasks;
  const GroupedSpan* spans;
  const GroupedSeg* segs;
  const int32_t* chunks;
  int group0;           // the run's first group
  int N, CW;            // right-hand sides, column-slice width
  const void* x;        // the run's input (row-major N columns when in_ld == 0, else column-major)
  int64_t in_ld;
  void* y;              // the run's output base
  int tasks_max, chunks_max, fac_max;   // shared-memory layout of the run
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
static_assert(sizeof(GroupedTask) % 8 == 0, "task descriptors are copied in 8-byte words");

// columns c and c + 1 of one row (16-byte aligned for complex64)
__device__ __forceinline__ void gr_ld_pair(const float2* p, float2& a, float2& b) {
  const float4 v = *(const float4*)p;
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void gr_ld_pair(const double2* p, double2& a, double2& b) {
  a = p[0];
  b = p[1];
}

// shared-memory bytes of one CTA: task descriptors, row chunks, staged
// factor blocks, the rows of every region (CW columns each)
template <typename V>
__host__ __device__ size_t gr_smem_bytes(int tasks_max, int chunks_max, int fac_max, int rows_max, int CW) {
  return gr_align16((size_t)tasks_max * sizeof(GroupedTask)) + gr_align16((size_t)chunks_max * 4) +
         (size_t)fac_max * sizeof(V) + (size_t)rows_max * CW * sizeof(V);
}

// one work item: rows r0 .. r0 + nr - 1 of task T for columns cl, cr of
// the slice; terms in order, k ascending (the stage kernels' FMA chains)
template <typename R, bool PAIR>
__device__ __forceinline__ void gr_item(const GroupedTask& T, int r0, const typename Cx<R>::V* __restrict__ rsm,
                                        const typename Cx<R>::V* __restrict__ fsm, const int32_t* reg_row, int CW,
                                        int cl, int cr, typename Cx<R>::V (&acc)[GR_RB][2]) {
  using V = typename Cx<R>::V;
  const int nr = min(GR_RB, T.M - r0);
#pragma unroll
  for (int r = 0; r < GR_RB; ++r) acc[r][0] = acc[r][1] = Cx<R>::make(0, 0);
  for (int q = 0; q < T.nterms; ++q) {
    const GroupedTerm& Q = T.t[q];
    const V* __restrict__ in = rsm + (int64_t)(reg_row[Q.in_reg] + Q.in_row) * CW;
    const V* __restrict__ mat = Q.fac_off >= 0 ? fsm + Q.fac_off : (const V*)Q.mat;
    const int K = Q.K, ldm = Q.ldm;
    // rows past the task's end re-read its last row (never stored)
    int ro[GR_RB];
    if (Q.conjT) {
#pragma unroll
      for (int r = 0; r < GR_RB; ++r) ro[r] = (r0 + min(r, nr - 1)) * ldm;
#pragma unroll 2
      for (int kk = 0; kk < K; ++kk) {
        V x0, x1;
        if constexpr (PAIR) {
          gr_ld_pair(in + kk * CW + cl, x0, x1);
        } else {
          x0 = in[kk * CW + cl], x1 = in[kk * CW + cr];
        }
#pragma unroll
        for (int r = 0; r < GR_RB; ++r) {
          const V e = mat[ro[r] + kk];
          cmac_conj(acc[r][0], e, x0);
          cmac_conj(acc[r][1], e, x1);
        }
      }
    } else {
#pragma unroll
      for (int r = 0; r < GR_RB; ++r) ro[r] = r0 + min(r, nr - 1);
#pragma unroll 2
      for (int kk = 0; kk < K; ++kk) {
        V x0, x1;
        if constexpr (PAIR) {
          gr_ld_pair(in + kk * CW + cl, x0, x1);
        } else {
          x0 = in[kk * CW + cl], x1 = in[kk * CW + cr];
        }
        const V* __restrict__ mk = mat + (int64_t)kk * ldm;
#pragma unroll
        for (int r = 0; r < GR_RB; ++r) {
          const V e = mk[ro[r]];
          cmac(acc[r][0], e, x0);
          cmac(acc[r][1], e, x1);
        }
      }
    }
  }
}
}  // namespace

template <typename R>
__global__ void __launch_bounds__(GT) grouped_kernel(const GroupedArgs a) {
  using V = typename Cx<R>::V;
  extern __shared__ __align__(16) uint8_t gr_smem[];
  GroupedTask* __restrict__ stask = (GroupedTask*)gr_smem;
  int32_t* __restrict__ schunk = (int32_t*)(gr_smem + gr_align16((size_t)a.tasks_max * sizeof(GroupedTask)));
  V* __restrict__ fsm = (V*)((uint8_t*)schunk + gr_align16((size_t)a.chunks_max * 4));   // staged factor blocks
  V* __restrict__ rsm = fsm + a.fac_max;                                                 // rows, CW columns each
  const GroupedGroup& G = a.groups[a.group0 + blockIdx.x];
  const int tid = threadIdx.x;
  const int CW = a.CW, N = a.N;
  const int c0 = blockIdx.y * CW;
  const int cw = min(CW, N - c0);
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  // descriptors, row chunks and factor blocks: independent of the previous launch
  {
    const int nw = G.ntasks * (int)(sizeof(GroupedTask) / 8);
    const uint2* src = (const uint2*)(a.tasks + G.task0);
    uint2* dst = (uint2*)stask;
    for (int v = tid; v < nw; v += GT) dst[v] = src[v];
    const int nc = G.st_chunk[G.nst];
    for (int v = tid; v < nc; v += GT) schunk[v] = a.chunks[G.chunk0 + v];
  }
  for (int g = 0; g < G.nseg; ++g) {
    const GroupedSeg sg = a.segs[G.seg0 + g];
    for (int e = tid; e < sg.count; e += GT) gr_cp_async<sizeof(V)>(fsm + sg.dst + e, (const V*)sg.src + e);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  // the group's input rows (region 0)
  const V* __restrict__ x = (const V*)a.x;
  for (int sp = 0; sp < G.nspans; ++sp) {
    const GroupedSpan S = a.spans[G.span0 + sp];
    if (a.in_ld == 0) {
      for (int e = tid; e < S.rows * cw; e += GT) {
        const int i = e / cw, c = e - i * cw;
        gr_cp_async<sizeof(V)>(rsm + (int64_t)(S.l0 + i) * CW + c, x + (S.g0 + i) * N + c0 + c);
      }
    } else {
      for (int e = tid; e < S.rows * cw; e += GT) {
        const int c = e / S.rows, i = e - c * S.rows;
        gr_cp_async<sizeof(V)>(rsm + (int64_t)(S.l0 + i) * CW + c, x + (S.g0 + i) + (int64_t)(c0 + c) * a.in_ld);
      }
    }
  }
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  const int pairs = (cw + 1) >> 1;
  // 16-byte input pairs: complex64 with an even slice width
  const bool pair = sizeof(V) == 8 && (CW & 1) == 0;
  V* __restrict__ y = (V*)a.y;
  for (int k = 0; k < G.nst; ++k) {
    const int ch0 = G.st_chunk[k], items = (G.st_chunk[k + 1] - ch0) * pairs;
    for (int idx = tid; idx < items; idx += GT) {
      const int ch = idx / pairs, p = idx - ch * pairs;
      const int32_t cp = schunk[ch0 + ch];
      const GroupedTask& T = stask[cp & 0xffff];
      const int r0 = cp >> 16;
      const int cl = 2 * p, cr = min(2 * p + 1, cw - 1);
      V acc[GR_RB][2];
      if (pair) gr_item<R, true>(T, r0, rsm, fsm, G.reg_row, CW, cl, cr, acc);
      else gr_item<R, false>(T, r0, rsm, fsm, G.reg_row, CW, cl, cr, acc);
      const int nr = min(GR_RB, T.M - r0);
      if (T.out_reg > 0) {
        V* o = rsm + (int64_t)(G.reg_row[T.out_reg] + T.out_row + r0) * CW;
#pragma unroll
        for (int r = 0; r < GR_RB; ++r)
          if (r < nr) {
            o[r * CW + cl] = acc[r][0];
            if (cl + 1 < cw) o[r * CW + cl + 1] = acc[r][1];
          }
      } else {
        const int64_t rs = T.ldo > 0 ? 1 : N, cs = T.ldo > 0 ? T.ldo : 1;
        V* o = y + (T.ldo > 0 ? T.out_row : T.out_row * N) + (int64_t)r0 * rs;
#pragma unroll
        for (int r = 0; r < GR_RB; ++r)
          if (r < nr) {
            o[r * rs + (int64_t)(c0 + cl) * cs] = acc[r][0];
            if (cl + 1 < cw) o[r * rs + (int64_t)(c0 + cl + 1) * cs] = acc[r][1];
          }
      }
    }
    __syncthreads();   // this stage's blocks are complete
  }
}

// ------------------------------------------------------------------ host --
namespace {

size_t grouped_smem(const GroupedRun& run, int CW, size_t es) {
  return es == 16 ? gr_smem_bytes<double2>(run.tasks_max, run.chunks_max, run.fac_max, run.rows_max, CW)
                  : gr_smem_bytes<float2>(run.tasks_max, run.chunks_max, run.fac_max, run.rows_max, CW);
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

// the factor block (first element, element count) holding a term's entries
bool locate_block(const Fact* F, int dtype, const void* ptr, const char** base, int64_t* count) {
  const size_t es = elem_bytes(dtype);
  for (const Stage& S : F->st) {
    const char* b = (const char*)(dtype == BF_C128 ? S.d64.p : S.d32.p);
    if (!b || (const char*)ptr < b || (const char*)ptr >= b + S.total * (int64_t)es) continue;
    const int64_t e = ((const char*)ptr - b) / (int64_t)es;
    const int blk = (int)(std::upper_bound(S.off.begin(), S.off.end(), e) - S.off.begin()) - 1;
    if (blk < 0) return false;
    *base = b + S.off[blk] * (int64_t)es;
    *count = (int64_t)S.rows[blk] * S.cols[blk];
    return true;
  }
  return false;
}

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
};

// Builds the groups of stages [s0, s0 + d) into T; false when a group does
// not fit (then the caller retries with a shorter run).
bool build_run(const Fact* F, int dtype, const std::vector<StageTask>& all, const ApplyPlan& tmp, int s0, int d,
               GroupedRun& run, RunTables& T) {
  const size_t es = elem_bytes(dtype);
  // tasks of the run, local numbering
  std::vector<int> first(d + 1, 0);
  for (int k = 0; k < d; ++k) first[k + 1] = first[k] + tmp.count[s0 + k];
  const int nt = first[d];
  auto gidx = [&](int k, int j) { return tmp.first[s0 + k] + j; };
  DSU dsu(nt);
  // producers inside the run: stage k's terms read stage k - 1's outputs
  for (int k = 1; k < d; ++k) {
    std::vector<std::pair<int64_t, int>> outs;   // (out_off, local index) of stage k - 1
    for (int j = 0; j < tmp.count[s0 + k - 1]; ++j) outs.push_back({all[gidx(k - 1, j)].out_off, first[k - 1] + j});
    std::sort(outs.begin(), outs.end());
    for (int j = 0; j < tmp.count[s0 + k]; ++j) {
      const StageTask& tk = all[gidx(k, j)];
      for (int q = 0; q < tk.nterms; ++q) {
        const int64_t a = tk.t[q].in_off, b = a + tk.t[q].K;
        auto it = std::upper_bound(outs.begin(), outs.end(), std::make_pair(a, INT32_MAX));
        if (it != outs.begin()) --it;
        for (; it != outs.end() && it->first < b; ++it) {
          const StageTask& pr = all[tmp.first[s0 + k - 1] + (it->second - first[k - 1])];
          if (it->first + pr.M > a) dsu.join(first[k] + j, it->second);
        }
      }
    }
  }
  // components in order of their first task
  std::map<int, std::vector<int>> comp;
  for (int i = 0; i < nt; ++i) comp[dsu.find(i)].push_back(i);
  run.group0 = (int32_t)T.groups.size();
  run.ngroups = (int32_t)comp.size();
  run.fac_max = 0;
  run.rows_max = 0;
  run.tasks_max = 0;
  run.chunks_max = 0;
  for (auto& kv : comp) {
    const std::vector<int>& mem = kv.second;   // ascending: stage by stage
    GroupedGroup G{};
    G.task0 = (int32_t)T.tasks.size();
    G.span0 = (int32_t)T.spans.size();
    G.seg0 = (int32_t)T.segs.size();
    G.chunk0 = (int32_t)T.chunks.size();
    G.nst = d;
    std::vector<std::vector<int>> byst(d);
    for (int i : mem) {
      const int k = (int)(std::upper_bound(first.begin(), first.end(), i) - first.begin()) - 1;
      byst[k].push_back(i);
    }
    // regions: 0 = the stage-0 inputs, k = the outputs of stage k - 1
    std::vector<RowMap> reg(d);
    {
      std::vector<std::pair<int64_t, int64_t>> v;
      for (int i : byst[0]) {
        const StageTask& tk = all[gidx(0, i - first[0])];
        for (int q = 0; q < tk.nterms; ++q) v.push_back({tk.t[q].in_off, tk.t[q].in_off + tk.t[q].K});
      }
      reg[0].build(v);
    }
    for (int k = 1; k < d; ++k) {
      std::vector<std::pair<int64_t, int64_t>> v;
      for (int i : byst[k - 1]) {
        const StageTask& tk = all[gidx(k - 1, i - first[k - 1])];
        v.push_back({tk.out_off, tk.out_off + tk.M});
      }
      reg[k].build(v);
    }
    G.reg_row[0] = 0;
    for (int k = 0; k < d; ++k) G.reg_row[k + 1] = G.reg_row[k] + (int32_t)reg[k].rows();
    for (int k = d + 1; k <= GR_MAXD; ++k) G.reg_row[k] = G.reg_row[d];
    for (size_t sp = 0; sp < reg[0].r.size(); ++sp)
      T.spans.push_back({reg[0].r[sp].first, reg[0].l0[sp], (int32_t)(reg[0].r[sp].second - reg[0].r[sp].first)});
    G.nspans = (int32_t)reg[0].r.size();
    // factor blocks of the group (each once)
    std::map<const char*, int32_t> placed;
    std::vector<GroupedSeg> segs;
    int64_t fac = 0;
    std::vector<GroupedTask> gt;
    std::vector<int32_t> chunks;
    G.st_chunk[0] = 0;
    for (int k = 0; k < d; ++k) {
      for (int i : byst[k]) {
        const StageTask& tk = all[gidx(k, i - first[k])];
        GroupedTask g{};
        g.M = tk.M;
        g.nterms = tk.nterms;
        if (k < d - 1) {
          g.out_reg = (int16_t)(k + 1);
          g.out_row = reg[k + 1].at(tk.out_off);
          if (g.out_row < 0) return false;
          g.ldo = 0;
        } else {
          g.out_reg = 0;
          g.out_row = tk.out_off;
          g.ldo = tk.ldo;
        }
        for (int q = 0; q < tk.nterms; ++q) {
          const StageTerm& S = tk.t[q];
          GroupedTerm& Q = g.t[q];
          Q.mat = S.mat;
          Q.K = S.K;
          Q.ldm = S.ldm;
          Q.conjT = S.conjT;
          Q.in_reg = (int16_t)k;
          const int64_t lr = reg[k].at(S.in_off);
          if (S.K > 0 && (lr < 0 || reg[k].at(S.in_off + S.K - 1) != lr + S.K - 1)) return false;
          Q.in_row = (int32_t)std::max<int64_t>(lr, 0);
          const char* b = nullptr;
          int64_t cnt = 0;
          if (!locate_block(F, dtype, S.mat, &b, &cnt)) return false;
          auto it = placed.find(b);
          if (it == placed.end()) {
            it = placed.emplace(b, (int32_t)fac).first;
            segs.push_back({b, (int32_t)fac, (int32_t)cnt});
            fac += cnt + (cnt & 1);   // keep every block 16-byte aligned for complex64
          }
          Q.fac_off = it->second + (int32_t)(((const char*)S.mat - b) / (int64_t)es);
        }
        if (gt.size() >= 0x10000 || tk.M >= 0x8000) return false;
        for (int r0 = 0; r0 < tk.M; r0 += GR_RB) chunks.push_back((r0 << 16) | (int32_t)gt.size());
        gt.push_back(g);
      }
      G.st_chunk[k + 1] = (int32_t)chunks.size();
    }
    for (int k = d + 1; k <= GR_MAXD; ++k) G.st_chunk[k] = G.st_chunk[d];
    G.ntasks = (int32_t)gt.size();
    if ((size_t)fac * es > GR_FAC_LIMIT) {   // read the factors in place
      for (auto& g : gt)
        for (int q = 0; q < g.nterms; ++q) g.t[q].fac_off = -1;
      segs.clear();
      fac = 0;
    }
    G.fac_elems = (int32_t)fac;
    G.nseg = (int32_t)segs.size();
    T.segs.insert(T.segs.end(), segs.begin(), segs.end());
    T.tasks.insert(T.tasks.end(), gt.begin(), gt.end());
    T.chunks.insert(T.chunks.end(), chunks.begin(), chunks.end());
    T.groups.push_back(G);
    run.fac_max = std::max(run.fac_max, (int32_t)fac);
    run.rows_max = std::max(run.rows_max, G.reg_row[d]);
    run.tasks_max = std::max(run.tasks_max, G.ntasks);
    run.chunks_max = std::max(run.chunks_max, G.st_chunk[d]);
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

int build_grouped(Fact* F, int opC, int dtype, int depth, cudaStream_t s) {
  GroupedPlan& gp = F->gp[opC][dtype];
  if (gp.built && gp.depth == depth) return BF_OK;
  if (depth < 1 || depth > GR_MAXD) return fail(BF_EINVAL, "grouped apply depth must be 1 .. 4");
  const auto pick = gp.pick;
  const auto cws = gp.cw;
  gp.dev.release(s);
  gp = GroupedPlan();
  gp.built = true;
  gp.depth = depth;
  gp.pick = pick;
  gp.cw = cws;
  ApplyPlan tmp;
  std::vector<StageTask> all;
  apply_tasks_host(F, opC, dtype, tmp, all);
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
  RunTables T;
  int64_t lvl_max = 0;
  int buf = 1;
  for (int s0 = 0; s0 < nst;) {
    int d = std::min(depth, nst - s0);
    GroupedRun run{};
    for (;; --d) {
      RunTables trial = T;
      if (build_run(F, dtype, all, tmp, s0, d, run, trial)) {
        T = std::move(trial);
        break;
      }
      if (d == 1) return BF_OK;   // a single stage does not fit: not applicable
    }
    run.in_base = s0 == 0 ? 0 : (buf == 1 ? 2 : 1);
    run.in_ld = s0 == 0 ? in_ld0 : 0;
    const bool last = s0 + d == nst;
    run.out_base = last ? 3 : buf;
    if (!last) {
      for (int t = tmp.first[s0 + d - 1]; t < tmp.first[s0 + d - 1] + tmp.count[s0 + d - 1]; ++t)
        lvl_max = std::max(lvl_max, all[t].out_off + all[t].M);
      buf = 3 - buf;
    }
    gp.runs.push_back(run);
    s0 += d;
  }
  gp.level_rows_max = std::max<int64_t>(lvl_max, 1);
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t b0 = T.groups.size() * sizeof(GroupedGroup), b1 = T.tasks.size() * sizeof(GroupedTask),
               b2 = std::max<size_t>(1, T.spans.size()) * sizeof(GroupedSpan),
               b3 = std::max<size_t>(1, T.segs.size()) * sizeof(GroupedSeg),
               b4 = std::max<size_t>(1, T.chunks.size()) * sizeof(int32_t);
  std::vector<char> host(al(b0) + al(b1) + al(b2) + al(b3) + b4, 0);
  memcpy(host.data(), T.groups.data(), b0);
  memcpy(host.data() + al(b0), T.tasks.data(), b1);
  if (!T.spans.empty()) memcpy(host.data() + al(b0) + al(b1), T.spans.data(), T.spans.size() * sizeof(GroupedSpan));
  if (!T.segs.empty())
    memcpy(host.data() + al(b0) + al(b1) + al(b2), T.segs.data(), T.segs.size() * sizeof(GroupedSeg));
  if (!T.chunks.empty())
    memcpy(host.data() + al(b0) + al(b1) + al(b2) + al(b3), T.chunks.data(), T.chunks.size() * sizeof(int32_t));
  BF_TRY(gp.dev.alloc(&F->mem, host.size(), nullptr));
  BF_CUDA_TRY(cudaMemcpyAsync(gp.dev.p, host.data(), host.size(), cudaMemcpyHostToDevice, s));
  BF_CUDA_TRY(host_sync(s));
  char* p = (char*)gp.dev.p;
  gp.d_groups = (const GroupedGroup*)p;
  gp.d_tasks = (const GroupedTask*)(p + al(b0));
  gp.d_spans = (const GroupedSpan*)(p + al(b0) + al(b1));
  gp.d_segs = (const GroupedSeg*)(p + al(b0) + al(b1) + al(b2));
  gp.d_chunks = (const int32_t*)(p + al(b0) + al(b1) + al(b2) + al(b3));
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
    a.groups = gp.d_groups;
    a.tasks = gp.d_tasks;
    a.spans = gp.d_spans;
    a.segs = gp.d_segs;
    a.chunks = gp.d_chunks;
    a.tasks_max = run.tasks_max;
    a.chunks_max = run.chunks_max;
    a.group0 = run.group0;
    a.N = (int)nrhs;
    a.CW = CW;
    a.x = bases[run.in_base];
    a.in_ld = run.in_ld;
    a.y = bases[run.out_base];
    a.fac_max = run.fac_max;
    const int slices = (int)((nrhs + CW - 1) / CW);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)run.ngroups, (unsigned)slices);
    cfg.blockDim = dim3(GT);
    cfg.dynamicSmemBytes = bytes(CW);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = r > 0 ? 1 : 0;
    // the attribute is the kernel's largest size, set once per process
    // (never lowered under a launch of another host thread)
    static std::once_flag attr_once[2];
    static cudaError_t attr_err[2] = {cudaSuccess, cudaSuccess};
    const int di = dtype == BF_C128 ? 1 : 0;
    std::call_once(attr_once[di], [&] {
      attr_err[di] = di ? cudaFuncSetAttribute(grouped_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)GR_SMEM_LIMIT)
                        : cudaFuncSetAttribute(grouped_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)GR_SMEM_LIMIT);
    });
    BF_CUDA_TRY(attr_err[di]);
    note_launch();
    const cudaError_t e = dtype == BF_C128 ? cudaLaunchKernelEx(&cfg, grouped_kernel<double>, a)
                                           : cudaLaunchKernelEx(&cfg, grouped_kernel<float>, a);
    if (e != cudaSuccess) return fail(BF_ECUDA, std::string("grouped apply launch: ") + cudaGetErrorString(e));
    BF_CUDA_TRY(cudaGetLastError());
  }
  return BF_OK;
}

}  // namespace bf
