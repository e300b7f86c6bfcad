// C ABI of libbutterfly (include/butterfly.h): handles, the plan (bisection
// trees of Sec. 3.1), the black-box operators of Alg. 2's input, the error
// metric of Sec. 7 and factor import/export.
#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <system_error>
#include <thread>

#include <cstdio>
#include <cstdlib>

#include "bf_internal.h"

namespace bf {

// ---------------------------------------------------------------- errors --
static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }
int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

// --------------------------------------------------------------- memory ---
// Stream-ordered allocations come from the device's default memory pool; its
// release threshold is raised once per device (per process) so that freed
// blocks stay cached instead of going back to the driver at every
// synchronisation.
static void keep_pool(cudaStream_t s) {
  static std::atomic<uint64_t> done{0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  if (done.load() & (1ull << dev)) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  done.fetch_or(1ull << dev);
  (void)s;
}

// ---- host-to-device uploads of task lists through pinned staging ----
// A host vector copied with cudaMemcpyAsync from pageable memory may make the
// driver wait for the stream to drain before staging it, which stalls the
// host behind the kernels already queued (and leaves the GPU idle while the
// host then enqueues the next ones).  Uploads go through a per-thread,
// per-device ring of pinned slots instead; a slot is reused once the copy
// that read it has completed (an event per slot).
namespace {
struct PinnedRing {
  static constexpr int SLOTS = 32;
  static constexpr size_t SLOT = 256 * 1024;
  char* buf = nullptr;
  cudaEvent_t ev[SLOTS] = {};
  bool used[SLOTS] = {};
  int next = 0;
  int state = 0;   // 0: not set up, 1: ready, -1: unavailable (pageable copies)
  ~PinnedRing() {
    if (state != 1) return;
    for (int i = 0; i < SLOTS; ++i) cudaEventDestroy(ev[i]);
    cudaFreeHost(buf);
  }
  bool ready() {
    if (state == 0) {
      state = -1;
      if (cudaMallocHost(&buf, SLOTS * SLOT) != cudaSuccess) {
        buf = nullptr;
        cudaGetLastError();
        return false;
      }
      for (int i = 0; i < SLOTS; ++i)
        if (cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess) {
          for (int j = 0; j < i; ++j) cudaEventDestroy(ev[j]);
          cudaFreeHost(buf);
          buf = nullptr;
          cudaGetLastError();
          return false;
        }
      state = 1;
    }
    return state == 1;
  }
};
thread_local std::map<int, PinnedRing> t_rings;   // by device
}  // namespace

int upload_async(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return BF_OK;
  int dev = 0;
  BF_CUDA_TRY(cudaGetDevice(&dev));
  PinnedRing& R = t_rings[dev];
  if (!R.ready()) {
    BF_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
    return BF_OK;
  }
  for (size_t off = 0; off < bytes; off += PinnedRing::SLOT) {
    const size_t n = std::min(PinnedRing::SLOT, bytes - off);
    const int i = R.next;
    R.next = (R.next + 1) % PinnedRing::SLOTS;
    if (R.used[i]) BF_CUDA_TRY(cudaEventSynchronize(R.ev[i]));
    char* slot = R.buf + (size_t)i * PinnedRing::SLOT;
    std::memcpy(slot, (const char*)src + off, n);
    BF_CUDA_TRY(cudaMemcpyAsync((char*)dst + off, slot, n, cudaMemcpyHostToDevice, s));
    BF_CUDA_TRY(cudaEventRecord(R.ev[i], s));
    R.used[i] = true;
  }
  return BF_OK;
}

// MemTracker counters may be updated from the two sides of a factorization
// running on two host threads (factor.cu)
static std::mutex g_mem_mu;

int dev_alloc(MemTracker* mt, void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  {
    std::lock_guard<std::mutex> lk(g_mem_mu);
    if (mt && mt->cap && mt->used + bytes > mt->cap)
      return fail(BF_ENOMEM, "allocation of " + std::to_string(bytes) + " bytes exceeds mem_cap");
  }
  if (s) keep_pool(s);
  cudaError_t e = s ? cudaMallocAsync(p, bytes, s) : cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(BF_ENOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
  }
  if (mt) {
    std::lock_guard<std::mutex> lk(g_mem_mu);
    mt->used += bytes;
    mt->peak = std::max(mt->peak, mt->used);
  }
  return BF_OK;
}

void dev_free(MemTracker* mt, void* p, size_t bytes, cudaStream_t s) {
  if (!p) return;
  if (s)
    cudaFreeAsync(p, s);
  else
    cudaFree(p);
  if (mt) {
    std::lock_guard<std::mutex> lk(g_mem_mu);
    mt->used -= std::min(mt->used, bytes);
  }
}

int DevBuf::alloc(MemTracker* t, size_t b, cudaStream_t s) {
  release(s);
  mt = t;
  bytes = b ? b : 16;
  int rc = dev_alloc(t, &p, bytes, s);
  if (rc) bytes = 0;
  async_ = s != nullptr;
  stream_ = s;
  return rc;
}

int DevBuf::alloc_kept(MemTracker* t, size_t b, cudaStream_t s) {
  const int rc = alloc(t, b, s);
  async_ = false;   // owned past the stream: freed with cudaFree
  return rc;
}

void DevBuf::release_on(cudaStream_t s) {
  if (!p) return;
  dev_free(mt, p, bytes, s);
  p = nullptr;
  bytes = 0;
}

void DevBuf::release(cudaStream_t s) {
  if (!p) return;
  dev_free(mt, p, bytes, async_ ? (s ? s : stream_) : nullptr);
  p = nullptr;
  bytes = 0;
}

// ---------------------------------------------------------------- trees ---
// Bisection (Sec. 3.1): ceil(s/2) / floor(s/2) split; with points, ordered by
// the coordinate of largest bounding-box extent (ties: lowest axis, then
// lowest index).
static void bisect(const double* pts, int64_t count, int dim, int L, std::vector<int64_t>& perm,
                   std::vector<std::vector<int64_t>>& off) {
  // One index array split in place, level by level.  A node's lower half
  // is the set of its ceil(s/2) smallest points under (coordinate on the
  // axis of largest extent, index) -- a strict total order -- so above the
  // last level a selection (nth_element) yields the same sets as a sort;
  // the last split sorts, which fixes the order inside every leaf.
  perm.resize(count);
  std::iota(perm.begin(), perm.end(), 0);
  off.assign(1, {0, count});
  for (int lev = 0; lev < L; ++lev) {
    const std::vector<int64_t> cur = off.back();
    std::vector<int64_t> o(2 * (cur.size() - 1) + 1, 0);
    for (size_t i = 0; i + 1 < cur.size(); ++i) {
      const int64_t a = cur[i], b = cur[i + 1], s = b - a, h = (s + 1) / 2;
      if (pts && s > 1) {
        int ax = 0;
        double best = -1.0;
        for (int d = 0; d < dim; ++d) {
          double lo = pts[perm[a] * dim + d], hi = lo;
          for (int64_t t = a; t < b; ++t) {
            const double v = pts[perm[t] * dim + d];
            lo = std::min(lo, v);
            hi = std::max(hi, v);
          }
          if (hi - lo > best) best = hi - lo, ax = d;
        }
        auto less = [&](int64_t x, int64_t y) {
          const double vx = pts[x * dim + ax], vy = pts[y * dim + ax];
          return vx < vy || (vx == vy && x < y);
        };
        if (lev == L - 1)
          std::sort(perm.begin() + a, perm.begin() + b, less);
        else
          std::nth_element(perm.begin() + a, perm.begin() + a + h, perm.begin() + b, less);
      }
      o[2 * i + 1] = a + h;
      o[2 * i + 2] = b;
    }
    off.push_back(std::move(o));
  }
}

// ------------------------------------------------------------ operators ---
namespace {

struct PlanOp : Operator {
  // tree-order products without counting
  virtual int tree_impl(int op, int64_t ncols, const void* X, int64_t ldx, void* Y, int64_t ldy,
                        int dtype, cudaStream_t s) = 0;
  virtual int struct_impl(int op, int groups, const int64_t* d_off, int64_t k, const void* Om,
                          int64_t ldo, void* Y, int64_t ldy, int dtype, cudaStream_t s) = 0;
  bool has_structured() const override { return true; }
  // this operator's structured product as a batched-launch job (no launch)
  virtual bool make_job(int op, const GemmGroups& g, const void* X, int64_t ldx, void* Y, int64_t ldy,
                        int dtype, SketchJob* job) = 0;
  bool sketch_job(int op, int groups, const int64_t* d_off, int64_t k, const void* Om, int64_t ldo,
                  void* Y, int64_t ldy, int dtype, SketchJob* job) override {
    if (!make_job(op, GemmGroups{groups, d_off, k}, Om, ldo, Y, ldy, dtype, job)) return false;
    (op == BF_OP_N ? cols_N : cols_T) += groups * k;
    return true;
  }
  int apply_tree(int op, int64_t ncols, const void* X, int64_t ldx, void* Y, int64_t ldy, int dtype,
                 cudaStream_t s) override {
    (op == BF_OP_N ? cols_N : cols_T) += ncols;
    return tree_impl(op, ncols, X, ldx, Y, ldy, dtype, s);
  }
  int apply_structured(int op, int groups, const int64_t* d_off, int64_t k, const void* Om,
                       int64_t ldo, void* Y, int64_t ldy, int dtype, cudaStream_t s) override {
    (op == BF_OP_N ? cols_N : cols_T) += groups * k;
    return struct_impl(op, groups, d_off, k, Om, ldo, Y, ldy, dtype, s);
  }
  // user order: permute to tree order, product, permute back; A^T X = conj(A^H conj X)
  int apply(int op, int64_t ncols, const void* X, int64_t ldx, void* Y, int64_t ldy, int dtype,
            cudaStream_t s) override {
    if (ncols <= 0) return BF_OK;
    (op == BF_OP_N ? cols_N : cols_T) += ncols;
    const bool opN = op == BF_OP_N;
    const int conj = op == BF_OP_T ? 1 : 0;
    const int64_t in_rows = opN ? n : m, out_rows = opN ? m : n;
    const int64_t* pin = (const int64_t*)(opN ? plan->d_permS.p : plan->d_permT.p);
    const int64_t* pout = (const int64_t*)(opN ? plan->d_permT.p : plan->d_permS.p);
    const size_t es = elem_bytes(dtype);
    DevBuf t;
    BF_TRY(t.alloc(&plan->mem, (in_rows + out_rows) * ncols * es, s));
    char* xi = (char*)t.p;
    char* yo = xi + in_rows * ncols * es;
    int rc = launch_gather_rows(pin, in_rows, ncols, X, ldx, xi, in_rows, conj, dtype, s);
    if (!rc) rc = tree_impl(opN ? BF_OP_N : BF_OP_C, ncols, xi, in_rows, yo, out_rows, dtype, s);
    if (!rc) rc = launch_scatter_rows(pout, out_rows, ncols, yo, out_rows, Y, ldy, conj, dtype, s);
    t.release(s);
    return rc;
  }
};

struct DenseOp : PlanOp {
  DevBuf A;   // tree order, m x n, ld m, dtype dt
  int dt = BF_C128;
  ~DenseOp() override { A.release(nullptr); }
  bool make_job(int op, const GemmGroups& g, const void* X, int64_t ldx, void* Y, int64_t ldy, int dtype,
                SketchJob* job) override {
    if (dtype != dt) return false;
    *job = dense_job(op, A.p, m, m, n, g, X, ldx, Y, ldy);
    return true;
  }
  int run(int op, const GemmGroups& g, const void* X, int64_t ldx, void* Y, int64_t ldy, int dtype,
          cudaStream_t s) {
    if (dtype == dt) return launch_dense_gemm(op, A.p, m, m, n, g, X, ldx, Y, ldy, dtype, s);
    // compute in the stored dtype, convert at the boundary
    const bool opN = op == BF_OP_N;
    const int64_t in_rows = opN ? n : m, out_rows = opN ? m : n;
    const int64_t xcols = g.d_off ? g.kcols : g.kcols;
    const int64_t ycols = g.kcols * g.groups;
    DevBuf t;
    BF_TRY(t.alloc(&plan->mem, (in_rows * xcols + out_rows * ycols) * elem_bytes(dt), s));
    char* xi = (char*)t.p;
    char* yo = xi + in_rows * xcols * elem_bytes(dt);
    int rc = launch_gather2d(nullptr, nullptr, in_rows, xcols, X, ldx, dtype, xi, in_rows, dt, s);
    if (!rc) rc = launch_dense_gemm(op, A.p, m, m, n, g, xi, in_rows, yo, out_rows, dt, s);
    if (!rc) rc = launch_gather2d(nullptr, nullptr, out_rows, ycols, yo, out_rows, dt, Y, ldy, dtype, s);
    t.release(s);
    return rc;
  }
  int tree_impl(int op, int64_t ncols, const void* X, int64_t ldx, void* Y, int64_t ldy, int dtype,
                cudaStream_t s) override {
    GemmGroups g{1, nullptr, ncols};
    return run(op, g, X, ldx, Y, ldy, dtype, s);
  }
  int struct_impl(int op, int groups, const int64_t* d_off, int64_t k, const void* Om, int64_t ldo,
                  void* Y, int64_t ldy, int dtype, cudaStream_t s) override {
    GemmGroups g{groups, d_off, k};
    return run(op, g, Om, ldo, Y, ldy, dtype, s);
  }
};

struct KernelOp : PlanOp {
  DevBuf imgN, imgC;   // resident entry images (bf_operator_kernel_cached), or empty
  ~KernelOp() override {
    imgN.release(nullptr);
    imgC.release(nullptr);
  }
  bool builtin_kernel() const override { return true; }
  const void* entry_image(int op) const override {
    return op == BF_OP_N ? imgN.p : op == BF_OP_C ? imgC.p : nullptr;
  }
  bool make_job(int op, const GemmGroups& g, const void* X, int64_t ldx, void* Y, int64_t ldy, int dtype,
                SketchJob* job) override {
    *job = kernel_job(plan, op, g, X, ldx, Y, ldy);
    return true;
  }
  int tree_impl(int op, int64_t ncols, const void* X, int64_t ldx, void* Y, int64_t ldy, int dtype,
                cudaStream_t s) override {
    GemmGroups g{1, nullptr, ncols};
    return launch_kernel_gemm(plan, op, g, X, ldx, Y, ldy, dtype, s, entry_image(op));
  }
  int struct_impl(int op, int groups, const int64_t* d_off, int64_t k, const void* Om, int64_t ldo,
                  void* Y, int64_t ldy, int dtype, cudaStream_t s) override {
    GemmGroups g{groups, d_off, k};
    return launch_kernel_gemm(plan, op, g, Om, ldo, Y, ldy, dtype, s, entry_image(op));
  }
};

struct FactOp : Operator {
  Fact* F = nullptr;
  int apply(int op, int64_t ncols, const void* X, int64_t ldx, void* Y, int64_t ldy, int dtype,
            cudaStream_t s) override {
    (op == BF_OP_N ? cols_N : cols_T) += ncols;
    return apply_fact(F, op, ncols, X, ldx, Y, ldy, dtype, s, false);
  }
};

struct ComposedOp : Operator {
  Operator* A1 = nullptr;
  Operator* A2 = nullptr;
  MemTracker mem;
  int apply(int op, int64_t ncols, const void* X, int64_t ldx, void* Y, int64_t ldy, int dtype,
            cudaStream_t s) override {
    if (ncols <= 0) return BF_OK;
    (op == BF_OP_N ? cols_N : cols_T) += ncols;
    const int64_t kk = A1->n;
    DevBuf t;
    BF_TRY(t.alloc(&mem, kk * ncols * elem_bytes(dtype), s));
    int rc;
    if (op == BF_OP_N) {
      rc = A2->apply(op, ncols, X, ldx, t.p, kk, dtype, s);
      if (!rc) rc = A1->apply(op, ncols, t.p, kk, Y, ldy, dtype, s);
    } else {
      rc = A1->apply(op, ncols, X, ldx, t.p, kk, dtype, s);
      if (!rc) rc = A2->apply(op, ncols, t.p, kk, Y, ldy, dtype, s);
    }
    t.release(s);
    return rc;
  }
};

struct CallbackOp : Operator {
  bf_matvec_fn fn = nullptr;
  void* ctx = nullptr;
  MemTracker mem;
  int apply(int op, int64_t ncols, const void* X, int64_t ldx, void* Y, int64_t ldy, int dtype,
            cudaStream_t s) override {
    if (ncols <= 0) return BF_OK;
    (op == BF_OP_N ? cols_N : cols_T) += ncols;
    if (op != BF_OP_C) {
      const int r = fn(ctx, op, ncols, X, ldx, Y, ldy, dtype, api_stream(s));
      return r ? fail(BF_ECALLBACK, "black-box callback returned " + std::to_string(r)) : BF_OK;
    }
    // A^H X = conj(A^T conj X)
    DevBuf t;
    BF_TRY(t.alloc(&mem, m * ncols * elem_bytes(dtype), s));
    int rc = launch_gather_rows(nullptr, m, ncols, X, ldx, t.p, m, 1, dtype, s);
    if (!rc) {
      const int r = fn(ctx, BF_OP_T, ncols, t.p, m, Y, ldy, dtype, api_stream(s));
      rc = r ? fail(BF_ECALLBACK, "black-box callback returned " + std::to_string(r)) : BF_OK;
    }
    if (!rc) rc = launch_conj_inplace(Y, n, ncols, ldy, dtype, s);
    t.release(s);
    return rc;
  }
};

template <typename H>
H* check(void* h, uint32_t kind) {
  if (!h) return nullptr;
  H* x = (H*)h;
  return x->kind == kind ? x : nullptr;
}

int upload(MemTracker* mt, DevBuf& b, const void* src, size_t bytes) {
  BF_TRY(b.alloc(mt, bytes, nullptr));
  note_sync();
  BF_CUDA_TRY(cudaMemcpy(b.p, src, bytes, cudaMemcpyHostToDevice));
  return BF_OK;
}

}  // namespace

static std::atomic<unsigned long long> g_launches{0}, g_syncs{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
unsigned long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
void note_sync() { g_syncs.fetch_add(1, std::memory_order_relaxed); }
bool debug_checks() {
#ifdef BF_DEBUG
  return true;
#else
  static const bool on = [] {
    const char* v = std::getenv("BF_DEBUG");
    return v && v[0] == '1';
  }();
  return on;
#endif
}
unsigned long long syncs_so_far() { return g_syncs.load(std::memory_order_relaxed); }
}  // namespace bf

using namespace bf;

namespace bf {

// Sketch error of Sec. 7 (eq. error): ||A W - F W||_F / ||A W||_F with W the
// counter-based Gaussian test matrix (stream 5 << 8, user-order rows).
int sketch_error(Fact* f, Operator* A, int ncols, uint64_t seed, int dtype, cudaStream_t s, double* err) {
  const int64_t n = f->n, m = f->m;
  const size_t es = elem_bytes(dtype);
  DevBuf buf;
  BF_TRY(buf.alloc(&f->mem, (n + 2 * m) * ncols * es + 16, s));
  char* W = (char*)buf.p;
  char* AW = W + n * ncols * es;
  char* FW = AW + m * ncols * es;
  double* red = (double*)(FW + m * ncols * es);
  int rc = launch_gaussian(seed, 5u << 8, 0, n, 0, ncols, W, n, dtype, s);
  if (!rc) rc = A->apply(BF_OP_N, ncols, W, n, AW, m, dtype, s);
  if (!rc) rc = apply_fact(f, BF_OP_N, ncols, W, n, FW, m, dtype, s, false);
  if (!rc) rc = launch_diff_norms(AW, FW, m, ncols, m, m, dtype, red, s);
  double h[2] = {0, 0};
  if (!rc && cudaMemcpyAsync(h, red, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess) rc = fail(BF_ECUDA, "copy");
  if (!rc && host_sync(s) != cudaSuccess) rc = fail(BF_ECUDA, "sync");
  buf.release(s);
  if (rc) return rc;
  *err = h[1] > 0 ? std::sqrt(h[0] / h[1]) : 0.0;
  return BF_OK;
}

void destroy_fact(Fact* F) {
  if (!F) return;
  note_sync();
  cudaDeviceSynchronize();
  for (auto& S : F->st) S.d64.release(nullptr), S.d32.release(nullptr);
  for (auto& a : F->ap)
    for (auto& b : a) b.tasks.release(nullptr);
  for (auto& a : F->fp)
    for (auto& b : a)
      for (auto& h : b.h) h.dev.release(nullptr);
  for (auto& a : F->gp)
    for (auto& b : a) b.dev.release(nullptr);
  delete F;
}

// Alg. 2, then (bf_options.accept_retries > 0) the a-posteriori acceptance:
// the sketch error with 16 fresh test columns (seed 1009 + attempt, in the
// factorization's working precision) must be within the Thm 5.3 bound
// 2 sqrt(L+2) tol; otherwise Alg. 2 is redone with r0 doubled.
int factor_accepted(Plan* P, Operator* A, cudaStream_t s, Fact** out) {
  *out = nullptr;
  const int retries = P->opt.accept_retries;
  const int r0 = P->opt.r0;
  const int dtype = P->opt.precision == BF_PREC_MIXED ? BF_C64 : BF_C128;
  const double bound = 2.0 * std::sqrt((double)P->L + 2.0) * P->tol;
  int r = r0;
  for (int t = 0;; ++t) {
    Fact* F = nullptr;
    P->opt.r0 = r;   // the plan is used by one thread at a time
    int rc = factor(P, A, s, &F);
    P->opt.r0 = r0;
    if (rc) return rc;
    F->attempts = t + 1;
    F->r0_used = r;
    if (retries <= 0) {
      *out = F;
      return BF_OK;
    }
    double e = 0.0;
    rc = sketch_error(F, A, 16, 1009ull + (uint64_t)t, dtype, s, &e);
    if (rc) {
      destroy_fact(F);
      return rc;
    }
    F->accept_err = e;
    if (e <= bound) {
      *out = F;
      return BF_OK;
    }
    destroy_fact(F);
    if (t >= retries || 2 * (int64_t)r > P->opt.r_max)
      return fail(BF_ENOTCONVERGED, "sketch error " + std::to_string(e) + " above the bound " + std::to_string(bound) +
                                        " after " + std::to_string(t + 1) + " factorizations (last r0 " +
                                        std::to_string(r) + ")");
    r *= 2;
  }
}

}  // namespace bf

extern "C" {

void bf_options_default(bf_options* o) {
  if (!o) return;
  o->p = 2;
  o->r0 = 4;
  o->r_max = 1024;
  o->seed = 0;
  o->precision = BF_PREC_FP64;
  o->mem_cap = 0;
  o->qr_fp64 = 0;
  o->hybrid_level = -1;
  o->accept_retries = 0;
  o->leaf_passes = 0;
}

const char* bf_last_error(void) { return g_err.c_str(); }

int bf_plan_create(const double* src, int64_t n, const double* tgt, int64_t m, int dim,
                   const bf_kernel_desc* kern, int leaf, double tol, const bf_options* opt,
                   bf_plan* out) {
  if (!out) return fail(BF_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || m < 1 || leaf < 1 || !(tol >= 0)) return fail(BF_EINVAL, "bad n, m, leaf or tol");
  const bool pts = src && tgt;
  if ((src == nullptr) != (tgt == nullptr)) return fail(BF_EINVAL, "give both point sets or neither");
  if (pts && (dim < 1 || dim > 3)) return fail(BF_EINVAL, "dim must be 1, 2 or 3");
  bf_options o;
  bf_options_default(&o);
  if (opt) o = *opt;
  if (o.p < 0 || o.r0 < 1 || o.r_max < o.r0) return fail(BF_EINVAL, "bad p, r0 or r_max");
  if (o.precision != BF_PREC_FP64 && o.precision != BF_PREC_MIXED) return fail(BF_EINVAL, "bad precision");
  if (o.qr_fp64 != 0 && o.qr_fp64 != 1) return fail(BF_EINVAL, "bad qr_fp64");
  if (o.accept_retries < 0 || o.accept_retries > 30 || o.leaf_passes < 0)
    return fail(BF_EINVAL, "bad accept_retries or leaf_passes");
  int L = 0;
  const int64_t mx = std::max(n, m);
  while ((mx + ((int64_t)1 << L) - 1) >> L > leaf) ++L;
  if (L < 1) return fail(BF_EINVAL, "Alg. 2 needs at least one level below the root (L >= 1)");
  if (L > 24) return fail(BF_EINVAL, "tree too deep");
  if (o.hybrid_level < -1 || o.hybrid_level > L - 1)
    return fail(BF_EINVAL, "hybrid_level must be -1 or in [0, L-1] (L = " + std::to_string(L) + ")");
  Plan* P = new Plan();
  P->n = n;
  P->m = m;
  P->dim = pts ? dim : 0;
  P->L = L;
  P->lm = o.hybrid_level < 0 ? L / 2 : o.hybrid_level;
  P->leaf = leaf;
  P->tol = tol;
  P->opt = o;
  P->mem.cap = o.mem_cap;
  if (kern) P->kern = *kern;
  P->has_points = pts;
  // the two trees are independent: for large point sets the target tree is
  // built on a second thread (serially if no thread can be started).  No
  // exception may cross the C ABI: any failure of the build (e.g. bad_alloc
  // on a large point set) frees the plan and returns a status.
  try {
    bool trees = false;
    if (pts && n + m >= 8192) {
      try {
        bool ok_T = false;
        std::thread tt([&] {
          try {
            bisect(tgt, m, dim, L, P->permT, P->offT);
            ok_T = true;
          } catch (...) {   // no exception may leave a thread: the serial path below redoes it
          }
        });
        try {
          bisect(src, n, dim, L, P->permS, P->offS);
        } catch (...) {
          tt.join();   // a joinable thread must not be destroyed
          throw;
        }
        tt.join();
        trees = ok_T;
      } catch (const std::system_error&) {
      }
    }
    if (!trees) {
      bisect(pts ? src : nullptr, n, dim, L, P->permS, P->offS);
      bisect(pts ? tgt : nullptr, m, dim, L, P->permT, P->offT);
    }
  } catch (const std::bad_alloc&) {
    delete P;
    return fail(BF_ENOMEM, "host memory exhausted while building the bisection trees");
  } catch (...) {
    delete P;
    return fail(BF_EINVAL, "the bisection trees could not be built");
  }
  for (int b = 0; b < (1 << L); ++b)
    if (P->offS[L][b + 1] == P->offS[L][b] || P->offT[L][b + 1] == P->offT[L][b]) {
      delete P;
      return fail(BF_EINVAL, "a leaf of the bisection tree is empty (too few points for the leaf size)");
    }
  for (int64_t i = 0; i < n; ++i) P->identS = P->identS && P->permS[i] == i;
  for (int64_t i = 0; i < m; ++i) P->identT = P->identT && P->permT[i] == i;
  int rc = upload(&P->mem, P->d_permS, P->permS.data(), n * 8);
  if (!rc) rc = upload(&P->mem, P->d_permT, P->permT.data(), m * 8);
  std::vector<int64_t> cS, cT;
  for (int l = 0; l <= L; ++l) {
    P->lvl_start.push_back((int64_t)cS.size());
    cS.insert(cS.end(), P->offS[l].begin(), P->offS[l].end());
    cT.insert(cT.end(), P->offT[l].begin(), P->offT[l].end());
  }
  if (!rc) rc = upload(&P->mem, P->d_offS, cS.data(), cS.size() * 8);
  if (!rc) rc = upload(&P->mem, P->d_offT, cT.data(), cT.size() * 8);
  if (!rc && pts) {
    std::vector<double> s3(3 * n, 0.0), t3(3 * m, 0.0);
    for (int64_t i = 0; i < n; ++i)
      for (int d = 0; d < dim; ++d) s3[d * n + i] = src[P->permS[i] * dim + d];
    for (int64_t i = 0; i < m; ++i)
      for (int d = 0; d < dim; ++d) t3[d * m + i] = tgt[P->permT[i] * dim + d];
    rc = upload(&P->mem, P->d_src, s3.data(), s3.size() * 8);
    if (!rc) rc = upload(&P->mem, P->d_tgt, t3.data(), t3.size() * 8);
    // float-float copies (hi = float(x), lo = float(x - hi)) for the mixed
    // path's entries: layout [x_hi, x_lo, y_hi, y_lo, z_hi, z_lo] x count
    auto split = [](const std::vector<double>& v, int64_t cnt) {
      std::vector<float> f(6 * cnt);
      for (int d = 0; d < 3; ++d)
        for (int64_t i = 0; i < cnt; ++i) {
          const double x = v[d * cnt + i];
          const float h = (float)x;
          f[(2 * d) * cnt + i] = h;
          f[(2 * d + 1) * cnt + i] = (float)(x - (double)h);
        }
      return f;
    };
    const std::vector<float> sf = split(s3, n), tf = split(t3, m);
    if (!rc) rc = upload(&P->mem, P->d_srcF, sf.data(), sf.size() * 4);
    if (!rc) rc = upload(&P->mem, P->d_tgtF, tf.data(), tf.size() * 4);
    P->kh = (float)P->kern.wavenumber;
    P->kl = (float)(P->kern.wavenumber - (double)P->kh);
  }
  if (rc) {
    P->d_permS.release(nullptr), P->d_permT.release(nullptr), P->d_offS.release(nullptr);
    P->d_offT.release(nullptr), P->d_src.release(nullptr), P->d_tgt.release(nullptr);
    P->d_srcF.release(nullptr), P->d_tgtF.release(nullptr);
    delete P;
    return rc;
  }
  bf_plan h = new bf_plan_s{KIND_PLAN, P};
  *out = h;
  return BF_OK;
}

int bf_bisect(const double* pts, int64_t count, int dim, int L, int64_t* perm, int64_t* off) {
  if (count < 1 || L < 0 || L > 24 || !perm || !off || (pts && (dim < 1 || dim > 3)))
    return fail(BF_EINVAL, "bad arguments");
  std::vector<int64_t> p;
  std::vector<std::vector<int64_t>> o;
  bisect(pts, count, dim, L, p, o);
  std::memcpy(perm, p.data(), count * 8);
  int64_t q = 0;
  for (int l = 0; l <= L; ++l) {
    std::memcpy(off + q, o[l].data(), o[l].size() * 8);
    q += (int64_t)o[l].size();
  }
  return BF_OK;
}

int bf_plan_info(bf_plan plan, int* L, int* lm, int64_t* n, int64_t* m) {
  auto* h = check<bf_plan_s>(plan, KIND_PLAN);
  if (!h) return fail(BF_EINVAL, "not a plan");
  if (L) *L = h->impl->L;
  if (lm) *lm = h->impl->lm;
  if (n) *n = h->impl->n;
  if (m) *m = h->impl->m;
  return BF_OK;
}

int bf_plan_trees(bf_plan plan, int64_t* permS, int64_t* permT, int64_t* offS, int64_t* offT) {
  auto* h = check<bf_plan_s>(plan, KIND_PLAN);
  if (!h) return fail(BF_EINVAL, "not a plan");
  Plan* P = h->impl;
  if (permS) std::memcpy(permS, P->permS.data(), P->n * 8);
  if (permT) std::memcpy(permT, P->permT.data(), P->m * 8);
  int64_t q = 0;
  for (int l = 0; l <= P->L; ++l) {
    if (offS) std::memcpy(offS + q, P->offS[l].data(), P->offS[l].size() * 8);
    if (offT) std::memcpy(offT + q, P->offT[l].data(), P->offT[l].size() * 8);
    q += (int64_t)P->offS[l].size();
  }
  return BF_OK;
}

int bf_operator_dense(bf_plan plan, const void* A, int64_t lda, int dtype, void* stream,
                      bf_operator* out) {
  if (!out) return fail(BF_EINVAL, "out is NULL");
  *out = nullptr;
  auto* h = check<bf_plan_s>(plan, KIND_PLAN);
  if (!h || !A) return fail(BF_EINVAL, "bad plan or matrix");
  Plan* P = h->impl;
  if (lda < P->m || (dtype != BF_C64 && dtype != BF_C128)) return fail(BF_EINVAL, "bad lda or dtype");
  auto* op = new DenseOp();
  op->plan = P;
  op->m = P->m;
  op->n = P->n;
  op->dt = P->opt.precision == BF_PREC_MIXED ? BF_C64 : BF_C128;
  int rc = op->A.alloc(&P->mem, P->m * P->n * elem_bytes(op->dt), nullptr);
  if (!rc)
    rc = launch_gather2d((const int64_t*)P->d_permT.p, (const int64_t*)P->d_permS.p, P->m, P->n, A, lda,
                         dtype, op->A.p, P->m, op->dt, user_stream(stream));
  if (!rc) {
    cudaError_t e = host_sync(user_stream(stream));
    if (e != cudaSuccess) rc = fail(BF_ECUDA, cudaGetErrorString(e));
  }
  if (rc) {
    delete op;
    return rc;
  }
  *out = new bf_operator_s{KIND_OP, op};
  return BF_OK;
}

int bf_operator_kernel(bf_plan plan, bf_operator* out) {
  if (!out) return fail(BF_EINVAL, "out is NULL");
  *out = nullptr;
  auto* h = check<bf_plan_s>(plan, KIND_PLAN);
  if (!h) return fail(BF_EINVAL, "not a plan");
  Plan* P = h->impl;
  if (!P->has_points || P->kern.type == BF_KERNEL_NONE) return fail(BF_EINVAL, "plan has no kernel or points");
  if (P->kern.type == BF_KERNEL_DFT && P->dim != 1) return fail(BF_EINVAL, "DFT kernel needs 1-D points");
  auto* op = new KernelOp();
  op->plan = P;
  op->m = P->m;
  op->n = P->n;
  *out = new bf_operator_s{KIND_OP, op};
  return BF_OK;
}

int bf_operator_kernel_cached(bf_plan plan, void* stream, bf_operator* out) {
  BF_TRY(bf_operator_kernel(plan, out));
  auto* op = (KernelOp*)(*out)->impl;
  Plan* P = op->plan;
  cudaStream_t s = user_stream(stream);
  int rc = op->imgN.alloc(&P->mem, entry_image_bytes(P->m, P->n), s);
  if (!rc) rc = op->imgC.alloc(&P->mem, entry_image_bytes(P->n, P->m), s);
  if (!rc) {
    const SketchJob j = kernel_job(P, BF_OP_N, GemmGroups{1, nullptr, 1}, nullptr, 0, nullptr, 0);
    rc = launch_entry_images(j, op->imgN.p, op->imgC.p, s);
  }
  if (rc) {
    bf_free(*out);
    *out = nullptr;
  }
  return rc;
}

int bf_operator_factored(bf_fact F, bf_operator* out) {
  if (!out) return fail(BF_EINVAL, "out is NULL");
  *out = nullptr;
  auto* h = check<bf_fact_s>(F, KIND_FACT);
  if (!h) return fail(BF_EINVAL, "not a factorization");
  auto* op = new FactOp();
  op->F = h->impl;
  op->m = h->impl->m;
  op->n = h->impl->n;
  *out = new bf_operator_s{KIND_OP, op};
  return BF_OK;
}

int bf_operator_composed(bf_operator A1, bf_operator A2, bf_operator* out) {
  if (!out) return fail(BF_EINVAL, "out is NULL");
  *out = nullptr;
  auto* h1 = check<bf_operator_s>(A1, KIND_OP);
  auto* h2 = check<bf_operator_s>(A2, KIND_OP);
  if (!h1 || !h2) return fail(BF_EINVAL, "not an operator");
  if (h1->impl->n != h2->impl->m) return fail(BF_EINVAL, "inner dimensions differ");
  auto* op = new ComposedOp();
  op->A1 = h1->impl;
  op->A2 = h2->impl;
  op->m = h1->impl->m;
  op->n = h2->impl->n;
  *out = new bf_operator_s{KIND_OP, op};
  return BF_OK;
}

int bf_operator_callback(int64_t m, int64_t n, bf_matvec_fn fn, void* ctx, bf_operator* out) {
  if (!out) return fail(BF_EINVAL, "out is NULL");
  *out = nullptr;
  if (m < 1 || n < 1 || !fn) return fail(BF_EINVAL, "bad size or callback");
  auto* op = new CallbackOp();
  op->m = m;
  op->n = n;
  op->fn = fn;
  op->ctx = ctx;
  *out = new bf_operator_s{KIND_OP, op};
  return BF_OK;
}

int bf_operator_apply(bf_operator A, int op, int64_t ncols, const void* X, int64_t ldx, void* Y,
                      int64_t ldy, int dtype, void* stream) {
  auto* h = check<bf_operator_s>(A, KIND_OP);
  if (!h) return fail(BF_EINVAL, "not an operator");
  if (op != BF_OP_N && op != BF_OP_T && op != BF_OP_C) return fail(BF_EINVAL, "bad op");
  if (dtype != BF_C64 && dtype != BF_C128) return fail(BF_EINVAL, "bad dtype");
  const int64_t in_rows = op == BF_OP_N ? h->impl->n : h->impl->m;
  const int64_t out_rows = op == BF_OP_N ? h->impl->m : h->impl->n;
  if (ncols < 0 || ldx < in_rows || ldy < out_rows) return fail(BF_EINVAL, "bad ncols or leading dimension");
  return h->impl->apply(op, ncols, X, ldx, Y, ldy, dtype, user_stream(stream));
}

int bf_operator_counts(bf_operator A, int64_t* cols_N, int64_t* cols_T) {
  auto* h = check<bf_operator_s>(A, KIND_OP);
  if (!h) return fail(BF_EINVAL, "not an operator");
  if (cols_N) *cols_N = h->impl->cols_N;
  if (cols_T) *cols_T = h->impl->cols_T;
  return BF_OK;
}

int bf_factor(bf_plan plan, bf_operator A, void* stream, bf_fact* out) {
  if (!out) return fail(BF_EINVAL, "out is NULL");
  *out = nullptr;
  auto* hp = check<bf_plan_s>(plan, KIND_PLAN);
  if (!hp) return fail(BF_EINVAL, "not a plan");
  Operator* op = nullptr;
  bf_operator tmp = nullptr;
  if (A) {
    auto* ho = check<bf_operator_s>(A, KIND_OP);
    if (!ho) return fail(BF_EINVAL, "not an operator");
    op = ho->impl;
  } else {
    BF_TRY(bf_operator_kernel(plan, &tmp));
    op = tmp->impl;
  }
  Fact* F = nullptr;
  const int rc = factor_accepted(hp->impl, op, user_stream(stream), &F);
  if (tmp) bf_free(tmp);
  if (rc) return rc;
  *out = new bf_fact_s{KIND_FACT, F};
  return BF_OK;
}

int bf_set_sketch_engine(int engine) { return set_sketch_engine(engine); }
int bf_set_entry_images(int on) { return set_entry_images(on); }
int bf_set_apply_engine(int engine) { return set_apply_engine(engine); }
int bf_set_stage_variant(int v) { return set_stage_variant(v); }
int bf_set_grouped_depth(int depth) { return set_grouped_depth(depth); }
int bf_set_grouped_merge(int merge) { return set_grouped_merge(merge); }
int bf_set_parallel_sides(int on) { return set_parallel_sides(on); }

unsigned long long bf_launch_count(void) { return bf::launches_so_far(); }
unsigned long long bf_sync_count(void) { return bf::syncs_so_far(); }

int bf_factor_batch(int count, const bf_plan* plans, const bf_operator* ops, void* stream, bf_fact* out) {
  if (!out || !plans || count < 1) return fail(BF_EINVAL, "bad batch arguments");
  for (int i = 0; i < count; ++i) out[i] = nullptr;
  std::vector<Plan*> P(count);
  std::vector<Operator*> A(count);
  std::vector<bf_operator> tmp;
  int rc = BF_OK;
  for (int i = 0; i < count && !rc; ++i) {
    auto* hp = check<bf_plan_s>(plans[i], KIND_PLAN);
    if (!hp) {
      rc = fail(BF_EINVAL, "batch entry " + std::to_string(i) + " is not a plan");
      break;
    }
    P[i] = hp->impl;
    if (ops && ops[i]) {
      auto* ho = check<bf_operator_s>(ops[i], KIND_OP);
      if (!ho) {
        rc = fail(BF_EINVAL, "batch entry " + std::to_string(i) + " is not an operator");
        break;
      }
      A[i] = ho->impl;
    } else {
      bf_operator t = nullptr;
      rc = bf_operator_kernel(plans[i], &t);
      if (!rc) tmp.push_back(t), A[i] = t->impl;
    }
  }
  std::vector<Fact*> F(count, nullptr);
  if (!rc) rc = factor_batch(count, P.data(), A.data(), user_stream(stream), F.data());
  for (auto t : tmp) bf_free(t);
  if (rc) return rc;
  for (int i = 0; i < count; ++i) out[i] = new bf_fact_s{KIND_FACT, F[i]};
  return BF_OK;
}

int bf_apply(bf_fact F, int64_t nrhs, const void* x, int64_t ldx, void* y, int64_t ldy, int dtype,
             void* stream) {
  auto* h = check<bf_fact_s>(F, KIND_FACT);
  if (!h) return fail(BF_EINVAL, "not a factorization");
  if (nrhs < 0) return fail(BF_EINVAL, "nrhs < 0");
  return apply_fact(h->impl, BF_OP_N, nrhs, x, ldx, y, ldy, dtype, user_stream(stream), false);
}

int bf_applier_create(bf_fact F, int op, int64_t nrhs, int dtype, bf_applier* out) {
  auto* h = check<bf_fact_s>(F, KIND_FACT);
  if (!h || !out) return fail(BF_EINVAL, "not a factorization");
  *out = nullptr;
  Applier* A = nullptr;
  BF_TRY(applier_create(h->impl, op, nrhs, dtype, &A));
  *out = new bf_applier_s{KIND_APPLIER, A};
  return BF_OK;
}

int bf_applier_run(bf_applier A, const void* x, int64_t ldx, void* y, int64_t ldy, void* stream) {
  auto* h = check<bf_applier_s>(A, KIND_APPLIER);
  if (!h) return fail(BF_EINVAL, "not an applier");
  return applier_run(h->impl, x, ldx, y, ldy, user_stream(stream));
}

int bf_apply_tune(bf_fact F, int op, int64_t nrhs, int dtype, void* stream, float* ms_out) {
  auto* h = check<bf_fact_s>(F, KIND_FACT);
  if (!h) return fail(BF_EINVAL, "not a factorization");
  return tune_apply(h->impl, op, dtype, nrhs, user_stream(stream), ms_out);
}

int bf_apply_T(bf_fact F, int op, int64_t nrhs, const void* x, int64_t ldx, void* y, int64_t ldy,
               int dtype, void* stream) {
  auto* h = check<bf_fact_s>(F, KIND_FACT);
  if (!h) return fail(BF_EINVAL, "not a factorization");
  if (op != BF_OP_T && op != BF_OP_C) return fail(BF_EINVAL, "op must be BF_OP_T or BF_OP_C");
  if (nrhs < 0) return fail(BF_EINVAL, "nrhs < 0");
  return apply_fact(h->impl, op, nrhs, x, ldx, y, ldy, dtype, user_stream(stream), false);
}

int bf_ranks(bf_fact F, int side, int level, int32_t* out) {
  auto* h = check<bf_fact_s>(F, KIND_FACT);
  if (!h || !out) return fail(BF_EINVAL, "bad factorization or output");
  Fact* f = h->impl;
  const std::vector<int32_t>* r = nullptr;
  if (side == 0 && level >= 0 && level <= f->lm) r = &f->rV[level];
  if (side == 1 && level >= f->lm && level <= f->L) r = &f->rU[level - f->lm];
  if (!r) return fail(BF_EINVAL, "level out of range for this side");
  std::memcpy(out, r->data(), r->size() * 4);
  return BF_OK;
}

int bf_fact_info(bf_fact F, int64_t* stored, int64_t* cols_N, int64_t* cols_T, double* secs) {
  auto* h = check<bf_fact_s>(F, KIND_FACT);
  if (!h) return fail(BF_EINVAL, "not a factorization");
  Fact* f = h->impl;
  if (stored) {
    int64_t s = 0;
    for (const auto& S : f->st)
      for (size_t b = 0; b < S.rows.size(); ++b) s += (int64_t)S.rows[b] * S.cols[b];
    *stored = s;
  }
  if (cols_N) *cols_N = f->cols_N;
  if (cols_T) *cols_T = f->cols_T;
  if (secs) *secs = f->seconds;
  return BF_OK;
}

int bf_fact_import(bf_plan plan, const int32_t* rV, const int32_t* rU, const void* const* blocks,
                   int dtype, bf_fact* out) {
  if (!out) return fail(BF_EINVAL, "out is NULL");
  *out = nullptr;
  auto* hp = check<bf_plan_s>(plan, KIND_PLAN);
  if (!hp || !rV || !rU || !blocks) return fail(BF_EINVAL, "bad arguments");
  if (dtype != BF_C128) return fail(BF_EINVAL, "import takes complex128 blocks");
  Plan* P = hp->impl;
  const int L = P->L, lm = P->lm, nb = 1 << L;
  Fact* F = new Fact();
  F->plan = P;
  F->L = L;
  F->lm = lm;
  F->n = P->n;
  F->m = P->m;
  F->mem.cap = P->opt.mem_cap;
  F->st.resize(L + 3);
  F->rV.assign(lm + 1, std::vector<int32_t>(nb));
  F->rU.assign(L - lm + 1, std::vector<int32_t>(nb));
  for (int j = 0; j <= lm; ++j) std::memcpy(F->rV[j].data(), rV + (int64_t)j * nb, nb * 4);
  for (int j = 0; j <= L - lm; ++j) std::memcpy(F->rU[j].data(), rU + (int64_t)j * nb, nb * 4);
  auto shape = [&](int s, int b, int& rows, int& cols) {
    if (s == 0) {
      rows = (int)(P->offS[L][b + 1] - P->offS[L][b]), cols = F->rV[0][b];
    } else if (s <= lm) {
      const int j = s, nn = 1 << (L - j), sg = b / nn, mu = b % nn;
      const int p0 = (sg >> 1) * (2 * nn) + 2 * mu;
      rows = F->rV[j - 1][p0] + F->rV[j - 1][p0 + 1], cols = F->rV[j][b];
    } else if (s == lm + 1) {
      rows = F->rU[0][b], cols = F->rV[lm][b];
    } else if (s <= L + 1) {
      const int j = s - 2, nn = 1 << (L - j), nn1 = nn >> 1, tau = b / nn, nu = b % nn;
      rows = F->rU[j + 1 - lm][(2 * tau) * nn1 + (nu >> 1)] + F->rU[j + 1 - lm][(2 * tau + 1) * nn1 + (nu >> 1)];
      cols = F->rU[j - lm][b];
    } else {
      rows = (int)(P->offT[L][b + 1] - P->offT[L][b]), cols = F->rU[L - lm][b];
    }
  };
  int rc = BF_OK;
  for (int s = 0; s < L + 3 && !rc; ++s) {
    Stage& S = F->st[s];
    S.rows.resize(nb);
    S.cols.resize(nb);
    S.off.resize(nb);
    int64_t tot = 0;
    for (int b = 0; b < nb; ++b) {
      int r, c;
      shape(s, b, r, c);
      if (r < 1 || c < 1) rc = fail(BF_EINVAL, "ranks must be >= 1");
      S.rows[b] = r;
      S.cols[b] = c;
      S.off[b] = tot;
      tot += (int64_t)r * c;
    }
    S.total = tot;
    if (!rc) rc = S.d64.alloc(&F->mem, tot * 16, nullptr);
    if (!rc) note_sync();
    if (!rc && cudaMemcpy(S.d64.p, blocks[s], tot * 16, cudaMemcpyHostToDevice) != cudaSuccess)
      rc = fail(BF_ECUDA, "copy of imported blocks failed");
  }
  if (rc) {
    for (auto& S : F->st) S.d64.release(nullptr);
    delete F;
    return rc;
  }
  *out = new bf_fact_s{KIND_FACT, F};
  return BF_OK;
}

// ---- checkpoint files: a factorization's ranks, block shapes and factor
// entries (complex128, and the complex64 copy where it exists, so that a
// reloaded factorization applies bit for bit as the saved one) ----
namespace {
struct FactFileHeader {
  char magic[8];          // "BFFACT01"
  int32_t version, L, lm, nstages, nb, have32;
  int64_t n, m, cols_N, cols_T;
  double seconds;
};
constexpr int FACT_FILE_VERSION = 1;

struct FileCloser {
  FILE* f;
  ~FileCloser() {
    if (f) std::fclose(f);
  }
};
}  // namespace

int bf_fact_save(bf_fact F, const char* path) {
  auto* h = check<bf_fact_s>(F, KIND_FACT);
  if (!h || !path) return fail(BF_EINVAL, "bad arguments");
  Fact* f = h->impl;
  const int nb = 1 << f->L;
  bool have32 = true;
  for (const Stage& S : f->st) have32 = have32 && S.have32;
  FactFileHeader hd{};
  std::memcpy(hd.magic, "BFFACT01", 8);
  hd.version = FACT_FILE_VERSION;
  hd.L = f->L;
  hd.lm = f->lm;
  hd.nstages = (int32_t)f->st.size();
  hd.nb = nb;
  hd.have32 = have32 ? 1 : 0;
  hd.n = f->n;
  hd.m = f->m;
  hd.cols_N = f->cols_N;
  hd.cols_T = f->cols_T;
  hd.seconds = f->seconds;
  FileCloser fc{std::fopen(path, "wb")};
  if (!fc.f) return fail(BF_EINVAL, std::string("cannot open ") + path + " for writing");
  bool ok = std::fwrite(&hd, sizeof(hd), 1, fc.f) == 1;
  for (const auto& v : f->rV) ok = ok && std::fwrite(v.data(), 4, nb, fc.f) == (size_t)nb;
  for (const auto& v : f->rU) ok = ok && std::fwrite(v.data(), 4, nb, fc.f) == (size_t)nb;
  std::vector<char> buf;
  for (const Stage& S : f->st) {
    ok = ok && std::fwrite(S.rows.data(), 4, nb, fc.f) == (size_t)nb &&
         std::fwrite(S.cols.data(), 4, nb, fc.f) == (size_t)nb && std::fwrite(S.off.data(), 8, nb, fc.f) == (size_t)nb &&
         std::fwrite(&S.total, 8, 1, fc.f) == 1;
    for (int w = 0; w < (have32 ? 2 : 1) && ok; ++w) {
      const size_t bytes = (size_t)S.total * (w ? 8 : 16);
      buf.resize(bytes);
      note_sync();
      if (bytes && cudaMemcpy(buf.data(), w ? S.d32.p : S.d64.p, bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(BF_ECUDA, "copy of the factors to the host failed");
      ok = std::fwrite(buf.data(), 1, bytes, fc.f) == bytes;
    }
  }
  if (!ok) return fail(BF_EINVAL, std::string("write to ") + path + " failed");
  return std::fclose(fc.f) == 0 ? (fc.f = nullptr, BF_OK) : (fc.f = nullptr, fail(BF_EINVAL, "close failed"));
}

int bf_fact_load(bf_plan plan, const char* path, bf_fact* out) {
  if (!out) return fail(BF_EINVAL, "out is NULL");
  *out = nullptr;
  auto* hp = check<bf_plan_s>(plan, KIND_PLAN);
  if (!hp || !path) return fail(BF_EINVAL, "bad arguments");
  Plan* P = hp->impl;
  FileCloser fc{std::fopen(path, "rb")};
  if (!fc.f) return fail(BF_EINVAL, std::string("cannot open ") + path);
  FactFileHeader hd{};
  if (std::fread(&hd, sizeof(hd), 1, fc.f) != 1 || std::memcmp(hd.magic, "BFFACT01", 8) != 0 ||
      hd.version != FACT_FILE_VERSION)
    return fail(BF_EINVAL, std::string(path) + " is not a factorization file of this version");
  if (hd.n != P->n || hd.m != P->m || hd.L != P->L || hd.lm != P->lm || hd.nb != (1 << P->L) ||
      hd.nstages != P->L + 3)
    return fail(BF_EINVAL, "the file's factorization does not match the plan (n, m, L or l_m)");
  const int nb = hd.nb;
  Fact* F = new Fact();
  F->plan = P;
  F->L = hd.L;
  F->lm = hd.lm;
  F->n = hd.n;
  F->m = hd.m;
  F->cols_N = hd.cols_N;
  F->cols_T = hd.cols_T;
  F->seconds = hd.seconds;
  F->mem.cap = P->opt.mem_cap;
  F->st.resize(hd.nstages);
  F->rV.assign(hd.lm + 1, std::vector<int32_t>(nb));
  F->rU.assign(hd.L - hd.lm + 1, std::vector<int32_t>(nb));
  int rc = BF_OK;
  bool ok = true;
  for (auto& v : F->rV) ok = ok && std::fread(v.data(), 4, nb, fc.f) == (size_t)nb;
  for (auto& v : F->rU) ok = ok && std::fread(v.data(), 4, nb, fc.f) == (size_t)nb;
  std::vector<char> buf;
  for (Stage& S : F->st) {
    if (!ok || rc) break;
    S.rows.resize(nb);
    S.cols.resize(nb);
    S.off.resize(nb);
    ok = std::fread(S.rows.data(), 4, nb, fc.f) == (size_t)nb && std::fread(S.cols.data(), 4, nb, fc.f) == (size_t)nb &&
         std::fread(S.off.data(), 8, nb, fc.f) == (size_t)nb && std::fread(&S.total, 8, 1, fc.f) == 1;
    // blocks in order, inside the stage, not overlapping (a block may be
    // laid out at a capacity above its final rank, leaving a gap)
    int64_t end = 0;
    for (int b = 0; ok && b < nb; ++b) {
      ok = S.rows[b] >= 0 && S.cols[b] >= 0 && S.off[b] >= end;
      end = S.off[b] + (int64_t)S.rows[b] * S.cols[b];
    }
    ok = ok && end <= S.total;
    for (int w = 0; w < (hd.have32 ? 2 : 1) && ok && !rc; ++w) {
      const size_t bytes = (size_t)S.total * (w ? 8 : 16);
      buf.resize(bytes);
      ok = std::fread(buf.data(), 1, bytes, fc.f) == bytes;
      DevBuf& d = w ? S.d32 : S.d64;
      if (ok) rc = d.alloc(&F->mem, bytes ? bytes : 16, nullptr);
      if (ok && !rc) note_sync();
      if (ok && !rc && bytes && cudaMemcpy(d.p, buf.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = fail(BF_ECUDA, "copy of the loaded factors failed");
      if (w) S.have32 = true;
    }
  }
  if (!rc && !ok) rc = fail(BF_EINVAL, std::string(path) + " is truncated or inconsistent");
  if (rc) {
    destroy_fact(F);
    return rc;
  }
  *out = new bf_fact_s{KIND_FACT, F};
  return BF_OK;
}

int bf_fact_export(bf_fact F, int stage, void* host_out, size_t* bytes) {
  auto* h = check<bf_fact_s>(F, KIND_FACT);
  if (!h || !bytes) return fail(BF_EINVAL, "bad arguments");
  Fact* f = h->impl;
  if (stage < 0 || stage >= (int)f->st.size()) return fail(BF_EINVAL, "stage out of range");
  const Stage& S = f->st[stage];
  size_t need = 0;
  for (size_t b = 0; b < S.rows.size(); ++b) need += (size_t)S.rows[b] * S.cols[b] * 16;
  if (!host_out || *bytes < need) {
    *bytes = need;
    return host_out ? fail(BF_EINVAL, "output buffer too small") : BF_OK;
  }
  char* o = (char*)host_out;
  for (size_t b = 0; b < S.rows.size(); ++b) {
    const size_t sz = (size_t)S.rows[b] * S.cols[b] * 16;
    note_sync();
    BF_CUDA_TRY(cudaMemcpy(o, (const char*)S.d64.p + S.off[b] * 16, sz, cudaMemcpyDeviceToHost));
    o += sz;
  }
  *bytes = need;
  return BF_OK;
}

int bf_gaussian(uint64_t seed, uint32_t stream_id, int64_t row0, int64_t rows, int64_t col0, int64_t col1,
                void* out, int64_t ld, int dtype, void* stream) {
  if (!out || rows < 0 || ld < rows || col1 < col0 || row0 < 0) return fail(BF_EINVAL, "bad arguments");
  if (dtype != BF_C64 && dtype != BF_C128) return fail(BF_EINVAL, "bad dtype");
  return launch_gaussian(seed, stream_id, row0, rows, col0, col1, out, ld, dtype, user_stream(stream));
}

int bf_error(bf_fact F, bf_operator A, int ncols, uint64_t seed, int dtype, void* stream, double* err) {
  auto* hf = check<bf_fact_s>(F, KIND_FACT);
  auto* ho = check<bf_operator_s>(A, KIND_OP);
  if (!hf || !ho || !err || ncols < 1) return fail(BF_EINVAL, "bad arguments");
  if (dtype != BF_C64 && dtype != BF_C128) return fail(BF_EINVAL, "bad dtype");
  return sketch_error(hf->impl, ho->impl, ncols, seed, dtype, user_stream(stream), err);
}

int bf_fact_accept(bf_fact F, int* attempts, int* r0_used, double* err) {
  auto* h = check<bf_fact_s>(F, KIND_FACT);
  if (!h) return fail(BF_EINVAL, "not a factorization");
  if (attempts) *attempts = h->impl->attempts;
  if (r0_used) *r0_used = h->impl->r0_used;
  if (err) *err = h->impl->accept_err;
  return BF_OK;
}

int bf_debug_wait_timeout(uint64_t limit_ns, void* stream) {
  const cudaStream_t s = user_stream(stream);
  int rc = wait_probe(limit_ns, s);
  if (rc != BF_ETIMEOUT) return rc;
  // the persistent apply's dependency wait, on a flag nothing sets
  rc = grouped_wait_probe(limit_ns, s);
  if (rc) return rc;
  rc = tc_status(true);
  if (rc == BF_OK) return fail(BF_EINTERNAL, "the apply's dependency wait did not give up");
  return rc;
}

void bf_free(void* handle) {
  if (!handle) return;
  const uint32_t kind = *(uint32_t*)handle;
  if (kind == KIND_PLAN) {
    auto* h = (bf_plan_s*)handle;
    Plan* P = h->impl;
    note_sync();
    cudaDeviceSynchronize();
    P->d_permS.release(nullptr), P->d_permT.release(nullptr), P->d_offS.release(nullptr);
    P->d_offT.release(nullptr), P->d_src.release(nullptr), P->d_tgt.release(nullptr);
    P->d_srcF.release(nullptr), P->d_tgtF.release(nullptr);
    delete P;
    h->kind = 0;
    delete h;
  } else if (kind == KIND_FACT) {
    auto* h = (bf_fact_s*)handle;
    destroy_fact(h->impl);
    h->kind = 0;
    delete h;
  } else if (kind == KIND_APPLIER) {
    auto* h = (bf_applier_s*)handle;
    applier_destroy(h->impl);
    h->kind = 0;
    delete h;
  } else if (kind == KIND_OP) {
    auto* h = (bf_operator_s*)handle;
    note_sync();
    cudaDeviceSynchronize();
    delete h->impl;
    h->kind = 0;
    delete h;
  }
}

}  // extern "C"
