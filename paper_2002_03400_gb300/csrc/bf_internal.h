// Internal declarations shared by the CUDA translation units of libbutterfly.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include <cstdio>

#include "../../include/butterfly.h"

namespace bf {

// A named NVTX range over one scope (Alg. 2's phases, an apply and its
// engine, the tuner): profilers show them on the timeline; without a tool
// attached a push or pop costs a few nanoseconds.  Ranges are per host
// thread, so the two sides of a factorization nest separately.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  NvtxRange(const char* fmt, int v) {
    char buf[64];
    std::snprintf(buf, sizeof(buf), fmt, v);
    nvtxRangePushA(buf);
  }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};


// ---------------------------------------------------------------- errors --
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

#define BF_CUDA_TRY(expr)                                                     \
  do {                                                                        \
    cudaError_t e__ = (expr);                                                 \
    if (e__ != cudaSuccess)                                                   \
      return ::bf::fail(BF_ECUDA, std::string(#expr) + ": " +                 \
                                      cudaGetErrorString(e__));               \
  } while (0)

#define BF_TRY(expr)          \
  do {                        \
    int s__ = (expr);         \
    if (s__ != BF_OK) return s__; \
  } while (0)

// --------------------------------------------------------------- streams --
// A NULL stream at the C ABI is the legacy default stream; it is carried as
// cudaStreamLegacy inside the library so that scratch buffers are always
// stream-ordered (cudaMallocAsync), and handed back as NULL to callbacks.
inline cudaStream_t user_stream(void* s) { return s ? (cudaStream_t)s : cudaStreamLegacy; }
inline void* api_stream(cudaStream_t s) { return s == cudaStreamLegacy ? nullptr : (void*)s; }

// --------------------------------------------------------------- memory ---
// Device buffers owned by a handle; allocation counted against a cap.
struct MemTracker {
  size_t cap = 0, used = 0, peak = 0;
};
int dev_alloc(MemTracker* mt, void** p, size_t bytes, cudaStream_t s);
// host -> device copy of a host buffer (e.g. a task list) that returns at
// once: staged through pinned memory, ordered on s; src may be reused after
// the call returns
int upload_async(void* dst, const void* src, size_t bytes, cudaStream_t s);
void dev_free(MemTracker* mt, void* p, size_t bytes, cudaStream_t s);

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  MemTracker* mt = nullptr;
  bool async_ = false;          // stream-ordered allocation (cudaMallocAsync)
  cudaStream_t stream_ = nullptr;
  int alloc(MemTracker* t, size_t b, cudaStream_t s);
  // stream-ordered allocation on s (no device synchronisation) of storage
  // that outlives the stream's work: released with cudaFree
  int alloc_kept(MemTracker* t, size_t b, cudaStream_t s);
  void release(cudaStream_t s);
  // stream-ordered free on s of a pool allocation (alloc or alloc_kept)
  void release_on(cudaStream_t s);
};

// ------------------------------------------------------------- handles ----
enum HandleKind : uint32_t {
  KIND_PLAN = 0xB0F1A001u,
  KIND_FACT = 0xB0F1A002u,
  KIND_OP = 0xB0F1A003u,
  KIND_APPLIER = 0xB0F1A004u
};

struct Plan;
struct Fact;
struct Operator;
struct SketchJob;

}  // namespace bf

struct bf_plan_s {
  uint32_t kind;
  bf::Plan* impl;
};
struct bf_fact_s {
  uint32_t kind;
  bf::Fact* impl;
};
struct bf_operator_s {
  uint32_t kind;
  bf::Operator* impl;
};
namespace bf {
struct Applier;
}
struct bf_applier_s {
  uint32_t kind;
  bf::Applier* impl;
};

namespace bf {

struct Plan {
  int64_t n = 0, m = 0;
  int dim = 0;
  int L = 0, lm = 0, leaf = 0;
  double tol = 0;
  bf_options opt{};
  bf_kernel_desc kern{BF_KERNEL_NONE, 0.0};
  bool has_points = false;
  std::vector<int64_t> permS, permT;          // tree position -> user index
  std::vector<std::vector<int64_t>> offS, offT;  // per level, 2^l + 1
  std::vector<double> srcTree, tgtTree;       // tree-ordered points (dim-major rows)
  // device copies
  MemTracker mem;
  DevBuf d_permS, d_permT;                    // int64
  DevBuf d_src, d_tgt;                        // double, SoA: x[n], y[n], z[n]
  DevBuf d_srcF, d_tgtF;                      // float-float SoA: [x_hi, x_lo, y_hi, y_lo, z_hi, z_lo]
  float kh = 0.f, kl = 0.f;                   // wavenumber as float-float
  DevBuf d_offS, d_offT;                      // int64, all levels concatenated
  std::vector<int64_t> lvl_start;             // level l starts at lvl_start[l] in d_off*
  bool identS = true, identT = true;          // permutation is the identity
  const int64_t* offS_dev(int l) const { return (const int64_t*)d_offS.p + lvl_start[l]; }
  const int64_t* offT_dev(int l) const { return (const int64_t*)d_offT.p + lvl_start[l]; }
};

// A black-box operator.  apply() works in user order; apply_tree() in the
// tree order of `plan` (only for operators bound to a plan).
struct Operator {
  int64_t m = 0, n = 0;
  Plan* plan = nullptr;                // non-null: native tree order of this plan
  int64_t cols_N = 0, cols_T = 0;
  virtual ~Operator() {}
  // Y = op(A) X, user order. op in {N, T, C}.
  virtual int apply(int op, int64_t ncols, const void* X, int64_t ldx, void* Y,
                    int64_t ldy, int dtype, cudaStream_t s) = 0;
  // Tree order of `plan` (only when plan != nullptr); op in {N, C}.
  virtual int apply_tree(int op, int64_t ncols, const void* X, int64_t ldx,
                         void* Y, int64_t ldy, int dtype, cudaStream_t s) {
    return fail(BF_EUNSUPPORTED, "operator has no tree-order product");
  }
  // built-in kernel operator (its entries have a closed form)
  virtual bool builtin_kernel() const { return false; }
  // resident entry image of op (BF_OP_N or BF_OP_C) in the tensor-core
  // layout (see SketchJob::img), or null
  virtual const void* entry_image(int op) const { return nullptr; }
  // Structured sketch (Sec. 4.1), tree order: for each node g of `groups`
  // with rows [off[g], off[g+1]) of the input side, and compact random
  // matrix Om (rows = input side, k columns, ld ldo):
  //   op N: Y[:, g*k:(g+1)*k] = A[:, rows_g] Om[rows_g, :]
  //   op C: Y[:, g*k:(g+1)*k] = A[rows_g, :]^H Om[rows_g, :]
  virtual bool has_structured() const { return false; }
  // Describes the structured product as a SketchJob for a batched launch
  // (plan-bound operators whose stored dtype matches); counts its columns.
  // Returns false when the operator cannot run batched.
  virtual bool sketch_job(int op, int groups, const int64_t* d_off, int64_t k, const void* Om,
                          int64_t ldo, void* Y, int64_t ldy, int dtype, SketchJob* job) {
    return false;
  }
  virtual int apply_structured(int op, int groups, const int64_t* d_off,
                               int64_t k, const void* Om, int64_t ldo, void* Y,
                               int64_t ldy, int dtype, cudaStream_t s) {
    return fail(BF_EUNSUPPORTED, "operator has no structured product");
  }
};

// -------------------------------------------------------- stage products --
// One output block (or column slice of it) of a block-sparse product:
//   out[M x N] = sum_t op_t(mat_t)[M x K_t] * in_t[K_t x N]
// op_t = 0: mat_t is M x K_t (ld ldm);  op_t = 1: mat_t is stored K_t x M and
// conjugate-transposed.  `in` and `out` are element offsets into one of four
// base pointers given at launch (so a task list can be reused with fresh
// scratch buffers); `mat` is an absolute device pointer into factor storage.
struct StageTerm {
  int64_t in_off;
  const void* mat;
  int64_t ldi;
  int32_t ldm;
  int32_t K;
  int16_t conjT;
  int16_t in_base;
  int32_t pad;
};
struct StageTask {
  int64_t out_off;
  int64_t ldo;
  int32_t M, N;
  int16_t nterms;
  int16_t out_base;
  int32_t pad;
  StageTerm t[2];
};
// ---------------------------------------------------------------- factors --
// One stage of the factorization in apply order: 2^L blocks, column-major,
// block b has rows[b] x cols[b] with ld = rows[b] at element offset off[b].
struct Stage {
  std::vector<int32_t> rows, cols;
  std::vector<int64_t> off;
  int64_t total = 0;                 // elements
  DevBuf d64;                        // complex128 data
  DevBuf d32;                        // complex64 copy (mixed precision / c64 apply)
  bool have32 = false;
};

// Cached task lists of one apply direction and dtype (eq. hybrid_butterfly_mat):
// stage i reads bases[in_base[i]] and writes bases[out_base[i]].
constexpr int NRHS_CLASSES = 6;      // right-hand-side counts 1, 2-4, 5-16, 17-32, 33-64, >64
inline int nrhs_class(int64_t n) { return n <= 1 ? 0 : n <= 4 ? 1 : n <= 16 ? 2 : n <= 32 ? 3 : n <= 64 ? 4 : 5; }
struct ApplyPlan {
  bool built = false;
  DevBuf tasks;
  std::vector<int64_t> first;        // first task of each stage
  std::vector<int> count, maxM, maxN;
  int64_t level_rows_max = 0;        // rows of the largest stacked intermediate
  // stage-kernel variant per stage and right-hand-side class, -1 untuned
  std::vector<std::array<int8_t, NRHS_CLASSES>> variant;
  int variant_of(size_t stage, int64_t nrhs) const {
    const int v = stage < variant.size() ? variant[stage][nrhs_class(nrhs)] : -1;
    return v >= 0 ? v : -1;
  }
};

// Fused apply (k_fused.cu): the stage apply's tasks regrouped per subtree.
// A group is one subtree (one CTA per group and column slice); its levels
// are the stages of one half of the apply, their rows local to the group.
struct FusedGroup {
  int32_t lev0, nlev;        // levels [lev0, lev0 + nlev) of the half's level table
  int32_t io_row0, io_rows;  // tree-order rows of x (first half) / y (second half) of the subtree
};
struct FusedLevel {
  int32_t task0, ntasks;     // tasks [task0, task0 + ntasks)
  int32_t rows, map0;        // output rows; row tiles at rowmap[map0 ..]
  int32_t tiles;             // rowmap[map0 + t] = (task - task0) << 16 | first row of tile t
  int32_t chunk0, nchunks;   // chunks [chunk0, chunk0 + nchunks) of the half's chunk table
  int32_t pad;
};
// A chunk of a level: the row tiles [tile0, tile1) computed after copying
// the factor blocks they read (segments [seg0, seg0 + nseg)) into the
// shared-memory staging area (staged = 0: the tasks read global memory).
struct FusedChunk {
  int32_t tile0, tile1, seg0, nseg, staged, pad;
};
struct FusedSeg {
  const void* src;           // first element of a factor block in global memory
  int32_t dst, count;        // staging-area element offset and element count
};
struct FusedHalf {
  std::vector<FusedGroup> groups;
  std::vector<FusedLevel> levels;
  std::vector<StageTask> tasks;
  std::vector<int32_t> rowmap;
  std::vector<FusedChunk> chunks;
  std::vector<FusedSeg> segs;
  int io_max = 0;
  int64_t lvl_max = 0;       // rows of the largest intermediate level (shared-memory level buffers)
  int tasks_max = 0;         // tasks and row tiles of the largest level (descriptor and tile-map copies)
  int64_t rows_max = 0;
  DevBuf dev;                // device copies of the four tables
  const FusedGroup* d_groups = nullptr;
  const FusedLevel* d_levels = nullptr;
  const StageTask* d_tasks = nullptr;
  const int32_t* d_rowmap = nullptr;
  const FusedChunk* d_chunks = nullptr;
  const FusedSeg* d_segs = nullptr;
};
struct FusedPlan {
  bool built = false, ok = false;
  FusedHalf h[2];
  int64_t ex_rows = 0;       // rows of the centre-level exchange buffer
  // per right-hand-side class: tuned column-slice width (0: default) and
  // engine (-1 untuned: stage launches; 0 fused measured faster; 1 stages)
  std::array<int, NRHS_CLASSES> cs{{0, 0, 0, 0, 0, 0}};
  std::array<int, NRHS_CLASSES> engine{{-1, -1, -1, -1, -1, -1}};
};

// Grouped apply: the stages in runs of up to GR_MAXD, one launch per run.
// Within a run the tasks fall into groups (the connected components of
// "reads the output of"); one CTA per (group, column slice) computes all of
// its group's tasks, the run's inner stages in shared memory.
constexpr int GR_MAXD = 4;
struct GroupedTerm {
  const void* mat;          // factor entries in global memory (entry (i, k) at mat[i ldm + k] when conjT, else mat[i + k ldm])
  int32_t fac_off;          // staged tile: element offset, entry (i, k) at fac_off + k tld + i (-1: read mat)
  int32_t K, ldm, tld;      // tld: the tile's row pitch (M rounded up to even)
  int16_t conjT, in_reg;    // input: shared-memory region in_reg (0: the staged run inputs)
  int32_t in_row;           // first local row of the input in that region
};
struct GroupedTask {
  int32_t M;
  int16_t nterms, out_reg;  // out_reg > 0: shared-memory region; 0: global (the run's output)
  int64_t out_row;          // local row (out_reg > 0) or global row offset (out_reg == 0)
  int64_t ldo;              // global output: 0 row-major (N columns), > 0 column-major
  GroupedTerm t[2];
  int32_t out_loc;          // column-major output: the first row in the group's output staging area
  int32_t pad;
};
struct GroupedSpan {        // global input rows [g0, g0 + rows) -> region-0 rows [l0, l0 + rows)
  int64_t g0;
  int32_t l0, rows;
};
struct GroupedSeg {         // one term's entries packed as a tile (entry (i, k) -> dst + (k tld + i) elements)
  const void* src;          // entry (i, k) at src[i ldm + k] when conj, else src[i + k ldm]
  int64_t dst;              // byte offset in the group images
  int32_t M, K, ldm, tld, conj, pad;
};
constexpr int GR_BUILD_AFTER = 3;     // untuned applies of (F, op, dtype) before the grouped engine takes over
constexpr int GR_RB = 16;             // rows of a work item (a lane's register tile: up to GR_RB rows x 1 column)
struct GroupedGroup {                   // the head of a group's image
  int32_t task0, ntasks, span0, nspans, seg0, nseg, chunk0;   // host tables (absolute indices)
  int32_t fac_elems;                    // staged factor elements (0: none staged)
  int32_t nst;                          // stages of this run
  int32_t st_chunk[GR_MAXD + 1];        // row chunks of stage k: [st_chunk[k], st_chunk[k + 1]) of the image's chunks
  int32_t reg_row[GR_MAXD + 1];         // region r: local rows [reg_row[r], reg_row[r + 1])
  int32_t off_tasks, off_spans, off_chunks, off_fac;   // byte offsets of the image's parts
  // column-major x and y (the first and the last run): region 0 held
  // column by column with pitch in_pitch (odd), the last stage's outputs
  // staged column by column at rows [out_row0, out_row0 + out_pitch) with
  // pitch out_pitch (odd) and written out along columns from the image's
  // output spans; 0: row-major
  int32_t in_pitch, out_row0, out_pitch, off_ospans, nospans, ospan0;
  int32_t out_ld;                       // y's leading dimension (column-major output)
};
// A group's image -- the head, its task descriptors, input spans and row
// chunks, then its factor tiles, 16-byte aligned parts -- is what the CTA
// holds in shared memory; the images of a run sit at a fixed stride, so a
// CTA copies its own with one coalesced pass and no descriptor read first.
struct GroupedRun {
  int32_t group0, ngroups;
  int32_t in_base, out_base;            // StageBases indices
  int64_t in_ld;                        // 0: row-major intermediates; > 0: column-major (x)
  int64_t img_off, img_stride;          // the run's first image (bytes into the images) and the stride
  int32_t desc_max, rows_max;           // largest descriptor part (bytes) and row count over the run's groups
  int64_t out_rows;                     // rows of the run's output (its last stage's level)
};
struct GroupedPlan {
  bool built = false, ok = false;
  int depth = 0;                        // stages per run
  DevBuf dev;                           // images | dependency lists | tile list (packing)
  std::vector<GroupedRun> runs;
  const uint8_t* d_img = nullptr;       // every run's group images
  const int32_t* d_dep_ptr = nullptr;   // persistent launch: the groups a group reads (CSR over groups)
  const int32_t* d_dep_idx = nullptr;
  int32_t ngroups = 0;
  int64_t level_rows_max = 0;           // rows of the largest run output (the two level buffers)
  std::array<int16_t, NRHS_CLASSES> cw{{0, 0, 0, 0, 0, 0}};   // tuned column-slice width (0: default)
  std::array<int8_t, NRHS_CLASSES> pick{{0, 0, 0, 0, 0, 0}};    // 1: the tuner measured it fastest
  std::array<int8_t, NRHS_CLASSES> ppick{{0, 0, 0, 0, 0, 0}};   // 1: ... in one persistent launch
  std::array<int8_t, NRHS_CLASSES> tuned{{0, 0, 0, 0, 0, 0}};   // 1: the tuner has measured this class
  int tuned_depth = 0;                  // the depth the tuner measured fastest (0: none)
  int merge = 1;                        // the built plan's groups: at least this many last-stage blocks
  int tuned_merge = 0;                  // the merge the tuner measured fastest (0: none)
  int64_t untuned_uses = 0;             // applies that found no tuned choice (the plan is built from the
                                        // GR_BUILD_AFTER-th on: it costs ~1.5 ms of host time at n = 16384)
};

struct Fact {
  Plan* plan = nullptr;
  int L = 0, lm = 0;
  int64_t n = 0, m = 0;
  std::vector<Stage> st;             // L + 3 stages
  std::vector<std::vector<int32_t>> rV;  // levels 0..lm
  std::vector<std::vector<int32_t>> rU;  // index j - lm for levels lm..L
  int64_t cols_N = 0, cols_T = 0;
  double seconds = 0;
  int attempts = 1, r0_used = 0;     // a-posteriori acceptance record (bf_fact_accept)
  double accept_err = -1.0;
  MemTracker mem;
  ApplyPlan ap[2][2];                // [op N / C][dtype C64 / C128]
  FusedPlan fp[2][2];                // fused apply, same indexing
  GroupedPlan gp[2][2];              // grouped apply, same indexing
  int stage_V0() const { return 0; }
  int stage_W(int j) const { return j; }
  int stage_B() const { return lm + 1; }
  int stage_R(int j) const { return j + 2; }
  int stage_U() const { return L + 2; }
  int ensure32(cudaStream_t s);
};

struct StageBases {
  void* p[4];
};
// N of every task is replaced by Noverride when Noverride > 0; Noverride < 0:
// per-task N, each task cut into 32-column slices (-Noverride the widest N)
// so that wide tasks spread over many warps; 0: per-task N, one warp per
// task.  variant:
// kernel shape (0 .. STAGE_VARIANTS - 1, same results), -1 for the default for Noverride.
// pdl: launch with a programmatic dependency on the previous kernel in s
// (only when that kernel is itself a stage launch of the same chain).
int launch_stage(const StageTask* d_tasks, int ntasks, int maxM, int maxN, int Noverride,
                 const StageBases& bases, int dtype, cudaStream_t s, int variant = -1, bool pdl = false);
// Peel-stage launch (one CTA per task and 32-128-column block, blocks and
// inputs staged in shared memory); *launched false when the blocks are too
// large for it (then use launch_stage).
int launch_peel(const StageTask* d_tasks, int ntasks, int maxM, int maxN, int maxK, const StageBases& bases,
                int dtype, cudaStream_t s, bool* launched);
// Times every stage-kernel variant on each stage of F's apply (direction,
// dtype, nrhs) and keeps the fastest per stage for that right-hand-side
// class; returns the tuned apply time in *ms (device, one call).
int tune_apply(Fact* F, int op, int dtype, int64_t nrhs, cudaStream_t s, float* ms);

// Fused apply: builds F->fp[opC][dtype] once (ok stays false when the
// subtree grouping does not apply or does not fit in shared memory); runs
// y = op(F) x in two launches with a caller-provided exchange buffer of
// fp.ex_rows * nrhs elements (cs_override > 0: that column-slice width).
int build_fused(Fact* F, int opC, int dtype, cudaStream_t s);
bool plan_fused(const Fact* F, int opC, int dtype, FusedPlan& fp);
int fused_slice_width(const FusedPlan& fp, int64_t nrhs, int dtype);
int run_fused(Fact* F, int opC, int dtype, int64_t nrhs, const void* x, int64_t ldx, void* y, int64_t ldy, int conj,
              void* exch, cudaStream_t s, int cs_override = 0);
// Grouped apply: builds F->gp[opC][dtype] with runs of `depth` stages,
// independent groups merged until each holds `merge` blocks of its run's
// last stage (0: the forced or tuned choice, else GR_MERGE_MIN for
// complex64 factorizations whose ranks are <= 16, none otherwise; rebuilt
// when either changes; ok false: not applicable);
// run_grouped computes y = op(F) x on tree-order x and y with two level
// buffers of gp.level_rows_max * nrhs elements each.
constexpr int GR_MERGE_MIN = 4;
int build_grouped(Fact* F, int opC, int dtype, int depth, cudaStream_t s, int merge = 0);
int run_grouped(Fact* F, int opC, int dtype, int64_t nrhs, const void* xt, void* yt, void* ping, void* pong,
                cudaStream_t s, int cw_override = 0);
// The same runs in one cooperative launch: a (group, column slice) task
// starts once the groups it reads have written their rows (per-task flags,
// bounded waits); every run writes its own rows of scratch, which holds
// grouped_persist_scratch_bytes.
size_t grouped_persist_scratch_bytes(const GroupedPlan& gp, int64_t nrhs, int dtype);
// mode 0: upload the per-run arguments into scratch and launch; 1: upload
// only; 2: launch on arguments uploaded before (a graph capture, whose
// buffers never change, uploads once outside the capture)
int run_grouped_persist(Fact* F, int opC, int dtype, int64_t nrhs, const void* xt, void* yt, void* scratch,
                        cudaStream_t s, int cw_override = 0, int mode = 0);
// one bounded dependency wait of the persistent launch on a flag nothing
// sets (sets the status flag)
int grouped_wait_probe(uint64_t limit_ns, cudaStream_t s);
// 0: the tuned depth (untuned: set by the largest block rank); 1 .. GR_MAXD:
// that depth for every grouped apply
int set_grouped_depth(int depth);
// 0: the tuned group merging (untuned: GR_MERGE_MIN for complex64, none for
// complex128); 1 .. 16: groups merged until they hold that many last-stage
// blocks (1: unmerged) for every grouped plan built later
int set_grouped_merge(int merge);
int grouped_merge();
// the engine of an apply's stages on tree-order buffers (0 stage launches,
// 1 persistent, 2 grouped), built as needed
int pick_inner_engine(Fact* F, int opC, int dtype, int64_t nrhs, bool overlap, cudaStream_t s, int* out);
int grouped_depth();
// 0: the fastest engine the tuner measured for the right-hand-side class
// (default; untuned: grouped where it applies); 1: stage launches only; 2: fused
// wherever it applies; 3: persistent wherever it applies; 4: grouped
int set_apply_engine(int e);
int apply_engine();

// Graph-captured apply (bf_applier): the stage chain of one (F, op, dtype,
// nrhs) on internal buffers, captured once into a CUDA graph.
struct Applier {
  Fact* F = nullptr;
  int op = 0, opC = 0, dtype = 0;
  int64_t nrhs = 0, in_rows = 0, out_rows = 0;
  DevBuf scratch;                      // xt | yt | ping | pong
  void *xt = nullptr, *yt = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t done = nullptr;          // end of the last run: runs are serialised
  bool ran = false;
};
int applier_create(Fact* F, int op, int64_t nrhs, int dtype, Applier** out);
int applier_run(Applier* A, const void* x, int64_t ldx, void* y, int64_t ldy, cudaStream_t s);
void applier_destroy(Applier* A);
int stage_variant_default(int nrhs, int dtype);
// -1: tuned or default shapes; 0 .. STAGE_VARIANTS - 1: that shape for every
// launch with a fixed column count (the apply's)
int set_stage_variant(int v);
constexpr int STAGE_VARIANTS = 8;

// ------------------------------------------------------------------- QR --
struct QRTask {
  const void* in;     // s x k, ld ldi
  void* q;            // s x cap output, ld = s
  int64_t ldi;
  int32_t s, k;
  int32_t cap;        // columns available in q (>= min(s,k))
  int32_t pad;
  double eps;         // truncation tolerance of this block's factorization
};
// Truncated column-pivoted Householder QR (Alg. 1 step 3); ranks[i] out.
// in dtype: C128 (factored in FP64) or C64 (factored in float-float, or in
// FP64 when fp64 is set); q is complex128 either way.
// Both kernels give a block's column RG lanes, RG = qr_lanes(rows, ...): a block's
// arithmetic (the row striding of its partial sums) depends on its own size
// only if every launch holds blocks of one qr_lanes class, so that the
// result of a block does not depend on what else is in the launch (batched
// factorizations equal individual ones bit for bit).  launch_qr requires it.
int qr_lanes(int s, int in_dtype, bool fp64);
int launch_qr(const QRTask* d_tasks, int ntasks, int maxS, int maxK, int in_dtype, bool fp64,
              int32_t* d_ranks, void* d_work, size_t work_bytes, cudaStream_t s);
size_t qr_workspace_bytes(int ntasks, int maxS, int maxK, int in_dtype, bool fp64);

// ------------------------------------------------------------ B solve ----
struct LSQTask {
  const void* P;      // s x k stacked peeled sketch (ld s)
  const void* Q;      // s x rU   (R_{tau,nu}, complex128, ld s)
  const void* X;      // rV x k   (V^H Omega, ld rV)
  void* B;            // rU x rV  output (complex128, ld rU)
  int32_t s, k, rU, rV;
};
// X^H and C^H live in shared memory when they fit, else in d_work
// (lsq_workspace_bytes, 0 when not needed)
size_t lsq_workspace_bytes(int ntasks, int maxK, int maxR);
int launch_lsq(const LSQTask* d_tasks, int ntasks, int maxS, int maxK, int maxR,
               int in_dtype, void* d_work, size_t work_bytes, cudaStream_t s);

// ------------------------------------------------------------- sketches --
// Counter-based Gaussian generator (Philox-4x32-10 + Box-Muller).
int launch_gaussian(uint64_t seed, uint32_t stream_id, int64_t row0, int64_t rows,
                    int64_t col0, int64_t col1, void* out, int64_t ld, int dtype,
                    cudaStream_t s);

// One built-in operator's sketch product (tree order), a unit of a batched
// launch: for each group g (node of the input-side tree, rows
// [off[g], off[g+1]) or all rows when d_off is null)
//   op N: Y[:, g*kcols + c] = sum_{j in rows_g} A[:, j] X[j, c]     (M = m)
//   op C: Y[:, g*kcols + c] = sum_{i in rows_g} conj(A[i, :]) X[i, c] (M = n)
// with A a dense stored tree-order matrix (kind 0) or kernel entries formed
// from the plan's points (kind 1).
struct SketchJob {
  int32_t kind, op, ktype, groups;
  int32_t split;          // tensor-core path: 2 = 3xTF32, 3 = exact three-way bf16 split
  int32_t pad_;
  int64_t M, Ktot, kcols;
  const int64_t* d_off;
  const void* A;
  int64_t lda;
  const double* tgt;      // FP64 points, [x | y | z] blocks of length m
  const double* src;      //                                          n
  const float* tgtF;      // float-float points, 6 blocks of length m
  const float* srcF;      //                                        n
  int64_t m, n;
  double wn;
  float kh, kl;
  const void* X;
  int64_t ldx;
  void* Y;
  int64_t ldy;
  int64_t ygs;            // Y columns between groups (0: kcols); set when a job is split by columns
  const int64_t* h_off;   // host copy of d_off (groups + 1 entries) or null
  // Second output segment (tensor-core path, built-in operators): columns
  // [kcols0, kcols) of X are the random matrix of a finer level of the same
  // input-side tree (groups1 = groups << shift1 nodes, host offsets h_off1);
  // their products go to Y1 (ld ldy1, group stride ygs1).  nseg = 1: none.
  int32_t nseg, shift1;
  int64_t kcols0, groups1, ldy1, ygs1;
  void* Y1;
  const int64_t* h_off1;
  // Entry image (tensor-core path, split 3, built-in operators): the
  // complex64 entries of every (128-row tile rt, 16-column chunk kc),
  // preformed, at img + (rt * img_nch + kc) * 16384 bytes
  // (launch_entry_images); null: entries are formed on the fly.  Used only
  // when every K range of the job starts on a chunk boundary and ends on one
  // or at Ktot.
  const void* img;
  int64_t img_nch;
  void* bimg;   // set by the launch: this job's B operand image (bf16 parts per 16-row chunk)
};
// Runs all jobs (same dtype) in one launch: one CTA per (job, group, row tile,
// column tile).  Job and tile lists are uploaded to stream-ordered scratch.
int launch_sketch_jobs(const std::vector<SketchJob>& jobs, int dtype, MemTracker* mt,
                       cudaStream_t s);
int launch_sketch_jobs_simt(const std::vector<SketchJob>& jobs, int dtype, MemTracker* mt,
                            cudaStream_t s);
// tcgen05 3xTF32 path (complex64 jobs with sketch width <= 64)
bool sketch_tc_applies(const std::vector<SketchJob>& jobs);
int launch_sketch_jobs_tc(const std::vector<SketchJob>& jobs, MemTracker* mt, cudaStream_t s);
// BF_ETIMEOUT if a tensor-core kernel's bounded wait gave up since the last reset
int tc_status(bool reset);
// device address of the status flag (set by any bounded wait that gave up)
int* tc_status_ptr();
// enqueues a copy of the device wait flag into dst (device memory) on s
int tc_status_copy(int32_t* dst, cudaStream_t s);
// the status of a flag value read back by tc_status_copy (resets it if asked)
int tc_status_value(int v, bool reset);
// runs one bounded wait that nothing completes, with the limit lowered to
// limit_ns; BF_ETIMEOUT when it gave up and returned (the designed outcome)
int wait_probe(uint64_t limit_ns, cudaStream_t s);
// Entry images (see SketchJob::img): bytes for an M x K orientation, and the
// launch that fills both of kernel job jn (op N: M = m targets, Ktot = n
// sources; X, Y and groups ignored) in one pass: imgN (m x n,
// entry_image_bytes(m, n)) and imgC (the op-C image, n x m,
// entry_image_bytes(n, m)); device, 16-byte aligned.
size_t entry_image_bytes(int64_t M, int64_t K);
int64_t entry_image_chunks(int64_t K);
int launch_entry_images(const SketchJob& jn, void* imgN, void* imgC, cudaStream_t s);
// whether job j may read an image: split 3, one segment, and every K range
// (groups and their split-K parts) on chunk boundaries
bool entry_image_fits(const SketchJob& j);
// 1: factorizations of built-in operators in mixed precision form entry
// images when they fit in device memory (default); 0: never
int set_entry_images(int on);
int entry_images_enabled();
// Bounds checks of every stage task list before its launch: on when the
// library is built with -DBF_DEBUG or when BF_DEBUG=1 is in the environment
// as the library loads.
bool debug_checks();
// Every task's output rows and every term's input rows lie inside their
// buffers (ext: elements of StageBases p[0..3], 0 = unknown, skipped) for a
// launch of N columns (N <= 0: each task's own N), ranks and term counts are
// in range, and a term whose entries lie in one of F's factor stages stays
// inside its block; BF_EINTERNAL names the first task that breaks a bound.
int check_stage_tasks(const char* what, const std::vector<struct StageTask>& tasks, int64_t N, const int64_t ext[4],
                      const struct Fact* F, int dtype);
// check_stage_tasks for an apply's lists (built by apply_tasks_host into ap)
int check_apply_tasks(const struct Fact* F, int opC, int dtype, const struct ApplyPlan& ap,
                      const std::vector<struct StageTask>& all);
// counts one kernel launch of this library (bf_launch_count)
void note_launch();
unsigned long long launches_so_far();
// counts one host-blocking CUDA call of this library (bf_sync_count)
void note_sync();
unsigned long long syncs_so_far();
// cudaStreamSynchronize, counted by bf_sync_count
inline cudaError_t host_sync(cudaStream_t s) {
  note_sync();
  return cudaStreamSynchronize(s);
}
// 0: tensor-core sketch where it applies (default), 1: SIMT sketch only
int set_sketch_engine(int e);
struct GemmGroups;
SketchJob dense_job(int op, const void* A, int64_t lda, int64_t m, int64_t n, const GemmGroups& g,
                    const void* X, int64_t ldx, void* Y, int64_t ldy);
SketchJob kernel_job(const Plan* P, int op, const GemmGroups& g, const void* X, int64_t ldx, void* Y,
                     int64_t ldy);

// Complex GEMM variants for the built-in operators (tree order), one job each.
// op N: Y[m x N] = A[:, k-range] * X ; op C: Y[n x N] = A[k-range rows,:]^H X
struct GemmGroups {
  int groups;             // >= 1
  const int64_t* d_off;   // groups+1 boundaries of the K range per group (device), or null
  int64_t kcols;          // columns per group (structured) or total columns (groups == 1)
};
int launch_dense_gemm(int op, const void* A, int64_t lda, int64_t m, int64_t n,
                      const GemmGroups& g, const void* X, int64_t ldx, void* Y,
                      int64_t ldy, int dtype, cudaStream_t s);
// img: the operator's resident entry image for op, or null (complex64
// products of N and C read it when the job's K ranges allow)
int launch_kernel_gemm(const Plan* plan, int op, const GemmGroups& g,
                       const void* X, int64_t ldx, void* Y, int64_t ldy,
                       int dtype, cudaStream_t s, const void* img = nullptr);

// ---------------------------------------------------------------- misc ----
// out[i, c] = conj?(in[perm[i], c])  (perm may be null: identity)
int launch_gather_rows(const int64_t* d_perm, int64_t rows, int64_t cols,
                       const void* in, int64_t ldi, void* out, int64_t ldo,
                       int conj, int dtype, cudaStream_t s);
// out[perm[i], c] = conj?(in[i, c])
int launch_scatter_rows(const int64_t* d_perm, int64_t rows, int64_t cols,
                        const void* in, int64_t ldi, void* out, int64_t ldo,
                        int conj, int dtype, cudaStream_t s);
// Structured expansion: out (rows x groups*k, zeroed) gets
// out[off[g]:off[g+1], g*k:(g+1)*k] = in[off[g]:off[g+1], 0:k]
int launch_expand_structured(int groups, const int64_t* d_off, int64_t rows,
                             int64_t k, const void* in, int64_t ldi, void* out,
                             int64_t ldo, int dtype, cudaStream_t s);
// out[i + j*ldo] = in[rp[i] + cp[j]*ldi] converted to out_dtype (rp/cp may be null)
int launch_gather2d(const int64_t* d_rp, const int64_t* d_cp, int64_t rows, int64_t cols,
                    const void* in, int64_t ldi, int in_dtype, void* out, int64_t ldo,
                    int out_dtype, cudaStream_t s);
int launch_convert(const void* in, void* out, int64_t count, int in_dtype,
                   int out_dtype, cudaStream_t s);
int launch_conj_inplace(void* p, int64_t rows, int64_t cols, int64_t ld,
                        int dtype, cudaStream_t s);
// sums of |a-b|^2 and |a|^2 over rows x cols into d_out[0..1] (double)
int launch_diff_norms(const void* a, const void* b, int64_t rows, int64_t cols,
                      int64_t lda, int64_t ldb, int dtype, double* d_out,
                      cudaStream_t s);

inline size_t elem_bytes(int dtype) { return dtype == BF_C128 ? 16 : 8; }

// ------------------------------------------------------- driver entries --
void apply_tasks_host(const Fact* F, int opC, int dtype, ApplyPlan& ap, std::vector<StageTask>& all);
int apply_fact(Fact* F, int op, int64_t nrhs, const void* x, int64_t ldx,
               void* y, int64_t ldy, int dtype, cudaStream_t s, bool tree_order);
int factor(Plan* P, Operator* A, cudaStream_t s, Fact** out);
// 1 (default): the two sides of Alg. 2 on two host threads and streams; 0: one after the other
int set_parallel_sides(int on);
// factor() followed by the a-posteriori acceptance of bf_options.accept_retries
int factor_accepted(Plan* P, Operator* A, cudaStream_t s, Fact** out);
int sketch_error(Fact* f, Operator* A, int ncols, uint64_t seed, int dtype, cudaStream_t s, double* err);
void destroy_fact(Fact* F);
// Alg. 2 for `count` operators in lockstep (one launch per kernel per phase
// across all of them); all plans must share one precision.
int factor_batch(int count, Plan* const* P, Operator* const* A, cudaStream_t s, Fact** out);

}  // namespace bf
