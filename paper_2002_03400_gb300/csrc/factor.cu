// Alg. 2 -- adaptive randomized hybrid butterfly factorization -- as a host
// scheduler over the device kernels, for a batch of operators in lockstep.
//
// Phases (each one launch per kernel for every operator of the batch):
//   V^0 leaf loop (Alg. 2 loop "V"), U^L leaf loop (loop "U"): draw the new
//     random columns, one black-box sketch, batched truncated QR per leaf,
//     ranks to the host, double r where not converged;
//   W^l, l = 1, 2, ...: structured sketch Y = A^H Gamma-bar of level l (Sec.
//     4.1), peeling of V^0, W^1..W^(l-1) along the ancestor paths (one stage
//     launch per tree level), batched QR -> W^l (Sec. 4.3);
//   R^l, l = L-1, L-2, ...: structured sketch Z = A Omega-bar, peeling of
//     U^L, R^(L-1)..R^(l+1), batched QR -> R^l (Sec. 4.2); at the centre
//     level l_m also X = V^H Omega and the B least squares (eq. Bij).
// Operators with different tree depths take part in the phases that exist
// for them (W step t runs level t where t <= l_m; R step t runs level L - t
// where L - t >= l_m).  Per-phase buffers of all operators live in shared
// arenas so that one task list addresses every operator.  Ranks come back to
// the host once per phase to size the next sketch (width max(r1 + r2) + p).
//
// Readings (shared with the oracle): r restarts at r0 for each leaf loop;
// each leaf pass appends r new random columns; a leaf loop also stops once
// r + p reaches the largest leaf; one sketch width per level; at l_m the
// width also covers max r^V + p; B = (U^H K Omega)(V^H Omega)^+.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <memory>
#include <string>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <system_error>
#include <thread>

#include "bf_internal.h"

namespace bf {

namespace {

enum { STAGE_V0 = 1, STAGE_U0 = 2, STAGE_W = 3, STAGE_R = 4 };
inline uint32_t sid(int stage, int level) { return (uint32_t)((stage << 8) | level); }

// RAII stream-ordered scratch
struct Scratch {
  DevBuf b;
  cudaStream_t s;
  explicit Scratch(cudaStream_t st) : s(st) {}
  Scratch(const Scratch&) = delete;
  ~Scratch() { b.release(s); }
  int alloc(MemTracker* mt, size_t bytes) { return b.alloc(mt, bytes ? bytes : 16, s); }
  char* p() const { return (char*)b.p; }
};

struct OpState {
  Plan* P;
  Operator* A;
  Fact* F;
  int L, lm, nb;
  // leaf loops
  int r = 0, k = 0, passes = 0;
  int64_t kcap = 0;
  bool done = false;
  DevBuf Y;
  std::vector<int32_t> ranks;
  // level phases
  int l = 0;
  std::vector<int32_t> Ps;
  std::vector<int64_t> Poff;
  int64_t goff = 0, yoff = 0, poff = 0, soff = 0, xoff = 0;   // element offsets into arenas
  std::vector<int64_t> prev, cur;                              // peel block offsets
  int in_base = -1;
  // entry images of a built-in operator for this factorization (op N:
  // m x n, op C: n x m): the operator's resident ones, or formed here
  DevBuf imgN, imgC;
  const void* img_n = nullptr;
  const void* img_c = nullptr;
};

struct Batch {
  std::vector<OpState> ops;
  cudaStream_t s;
  int dt;
  size_t es;
  MemTracker mem;   // shared arenas

  const void* fblk(OpState& o, int stage, int b, int row = 0) const {
    const Stage& S = o.F->st[stage];
    const char* base = (const char*)(dt == BF_C128 ? S.d64.p : S.d32.p);
    return base + (S.off[b] + row) * (int64_t)es;
  }
};

StageTask task(int out_base, int64_t out_off, int64_t ldo, int M, int N) {
  StageTask t{};
  t.out_base = (int16_t)out_base;
  t.out_off = out_off;
  t.ldo = ldo;
  t.M = M;
  t.N = N;
  return t;
}
void term(StageTask& t, int in_base, int64_t in_off, int64_t ldi, const void* mat, int ldm, int K,
          int conjT) {
  StageTerm& T = t.t[t.nterms++];
  T.in_base = (int16_t)in_base;
  T.in_off = in_off;
  T.ldi = ldi;
  T.mat = mat;
  T.ldm = ldm;
  T.K = K;
  T.conjT = (int16_t)conjT;
}

// One stage launch of a phase's block products on bases {b0, b1, b2, b3}.
int run_tasks(Batch& B, const std::vector<StageTask>& tasks, const Scratch& b0, const Scratch& b1,
              const Scratch& b2, const Scratch& b3) {
  if (tasks.empty()) return BF_OK;
  const StageBases bases{{b0.p(), b1.p(), b2.p(), b3.p()}};
  if (debug_checks()) {
    const int64_t es = (int64_t)B.es;
    const int64_t ext[4] = {(int64_t)b0.b.bytes / es, (int64_t)b1.b.bytes / es, (int64_t)b2.b.bytes / es,
                            (int64_t)b3.b.bytes / es};
    BF_TRY(check_stage_tasks("factorization task list", tasks, 0, ext, nullptr, B.dt));
  }
  Scratch d(B.s);
  BF_TRY(d.alloc(&B.mem, tasks.size() * sizeof(StageTask)));
  BF_TRY(upload_async(d.p(), tasks.data(), tasks.size() * sizeof(StageTask), B.s));
  int mM = 0, mN = 0, mK = 0;
  for (const auto& t : tasks) {
    mM = std::max(mM, t.M), mN = std::max(mN, t.N);
    for (int q = 0; q < t.nterms; ++q) mK = std::max(mK, t.t[q].K);
  }
  bool done = false;
  BF_TRY(launch_peel((const StageTask*)d.p(), (int)tasks.size(), mM, mN, mK, bases, B.dt, B.s, &done));
  if (done) return BF_OK;
  // per-task N in 32-column slices: the first peel stages of a level carry
  // k 2^(l-j) columns per block
  return launch_stage((const StageTask*)d.p(), (int)tasks.size(), mM, mN, -mN, bases, B.dt, B.s);
}

// One structured sketch request (Sec. 4.1): Y = op(A) Omega-bar for the
// block-diagonal expansion over the nodes at `level` of the input-side tree
// of the compact random matrix Om (input rows x k).  Tree order.
struct SketchReq {
  OpState* o;
  int op, level;
  int64_t k;
  const void* Om;
  void* Y;
};

// Products that cannot run batched (user callbacks, factored or composed
// operators, dtype mismatch): expand Omega-bar and call the black box.
int sketch_one(Batch& B, const SketchReq& q) {
  Plan* P = q.o->P;
  Operator* A = q.o->A;
  const bool opN = q.op == BF_OP_N;
  const int groups = 1 << q.level;
  const int64_t in_rows = opN ? P->n : P->m, out_rows = opN ? P->m : P->n;
  const int64_t* d_off = opN ? P->offS_dev(q.level) : P->offT_dev(q.level);
  const int64_t ncols = groups * q.k;
  if (A->plan == P && A->has_structured())
    return A->apply_structured(q.op, groups, d_off, q.k, q.Om, in_rows, q.Y, out_rows, B.dt, B.s);
  Scratch ex(B.s);
  BF_TRY(ex.alloc(&q.o->F->mem, in_rows * ncols * B.es));
  BF_TRY(launch_expand_structured(groups, d_off, in_rows, q.k, q.Om, in_rows, ex.p(), in_rows, B.dt, B.s));
  if (A->plan == P) return A->apply_tree(q.op, ncols, ex.p(), in_rows, q.Y, out_rows, B.dt, B.s);
  Scratch u(B.s);
  BF_TRY(u.alloc(&q.o->F->mem, (in_rows + out_rows) * ncols * B.es));
  char* ui = u.p();
  char* uo = u.p() + in_rows * ncols * B.es;
  const int64_t* pin = (const int64_t*)(opN ? P->d_permS.p : P->d_permT.p);
  const int64_t* pout = (const int64_t*)(opN ? P->d_permT.p : P->d_permS.p);
  BF_TRY(launch_scatter_rows(pin, in_rows, ncols, ex.p(), in_rows, ui, in_rows, 0, B.dt, B.s));
  BF_TRY(A->apply(q.op, ncols, ui, in_rows, uo, out_rows, B.dt, B.s));
  return launch_gather_rows(pout, out_rows, ncols, uo, out_rows, q.Y, out_rows, 0, B.dt, B.s);
}

// All requests of a phase: built-in operators in one batched launch, the
// rest one by one.
int sketch_all(Batch& B, const std::vector<SketchReq>& reqs) {
  std::vector<SketchJob> jobs;
  for (const auto& q : reqs) {
    Plan* P = q.o->P;
    const bool opN = q.op == BF_OP_N;
    const int groups = 1 << q.level;
    const int64_t in_rows = opN ? P->n : P->m, out_rows = opN ? P->m : P->n;
    const int64_t* d_off = opN ? P->offS_dev(q.level) : P->offT_dev(q.level);
    SketchJob j{};
    if (q.o->A->plan == P && q.o->A->sketch_job(q.op, groups, d_off, q.k, q.Om, in_rows, q.Y, out_rows, B.dt, &j)) {
      // tensor-core products: the exact three-way bf16 split (FP32-level
      // products) at every tolerance -- on this GPU it is also faster than
      // 3xTF32 (half the operand bytes and MMA instructions), which stays
      // selectable through bf_set_sketch_engine
      j.split = 3;
      j.h_off = (opN ? P->offS[q.level] : P->offT[q.level]).data();
      const void* img = opN ? q.o->img_n : q.o->img_c;
      if ((q.op == BF_OP_N || q.op == BF_OP_C) && img && entry_image_fits(j)) {
        j.img = img;
        j.img_nch = entry_image_chunks(j.Ktot);
      }
      jobs.push_back(j);
    } else
      BF_TRY(sketch_one(B, q));
  }
  return launch_sketch_jobs(jobs, B.dt, &B.mem, B.s);
}

// Entry images (mixed precision, built-in operators): every sketch of the
// factorization streams its entries (complex64 tiles) instead of forming
// m x n kernel entries per sketch.  Both orientations are formed once, here;
// operators are served in batch order while the images fit in half of the
// free device memory and, under a memory cap, in half of what the cap
// leaves (the rest is for the factorization); the others form entries on
// the fly.
int make_images(Batch& B) {
  NvtxRange nv("entry images");
  if (B.dt != BF_C64 || !entry_images_enabled()) return BF_OK;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return BF_OK;
  size_t budget = free_b / 2;
  for (auto& o : B.ops) {
    Plan* P = o.P;
    if (o.A->plan != P || !o.A->builtin_kernel()) continue;
    if (o.A->entry_image(BF_OP_N) && o.A->entry_image(BF_OP_C)) {   // resident in the operator
      o.img_n = o.A->entry_image(BF_OP_N);
      o.img_c = o.A->entry_image(BF_OP_C);
      continue;
    }
    const size_t bN = entry_image_bytes(P->m, P->n), bC = entry_image_bytes(P->n, P->m);
    if (bN + bC > budget) continue;
    if (B.mem.cap && (B.mem.used >= B.mem.cap || bN + bC > (B.mem.cap - B.mem.used) / 2)) continue;
    if (o.imgN.alloc(&B.mem, bN, B.s) != BF_OK || o.imgC.alloc(&B.mem, bC, B.s) != BF_OK) {
      o.imgN.release(B.s);
      o.imgC.release(B.s);
      continue;
    }
    budget -= bN + bC;
    const SketchJob j = kernel_job(P, BF_OP_N, GemmGroups{1, nullptr, 1}, nullptr, 0, nullptr, 0);
    BF_TRY(launch_entry_images(j, o.imgN.p, o.imgC.p, B.s));
    o.img_n = o.imgN.p;
    o.img_c = o.imgC.p;
  }
  return BF_OK;
}

// Lays out a stage: rows[b] x cap[b] blocks, allocates complex128 storage.
int layout_stage(Batch& B, OpState& o, Stage& S, const std::vector<int32_t>& rows, const std::vector<int32_t>& cap) {
  S.d64.release_on(B.s);   // an earlier layout of this stage (leaf passes): pool storage
  S.d32.release_on(B.s);
  S.have32 = false;
  const size_t nb = rows.size();
  S.rows = rows;
  S.cols.assign(nb, 0);
  S.off.assign(nb, 0);
  int64_t tot = 0;
  for (size_t b = 0; b < nb; ++b) {
    S.off[b] = tot;
    tot += (int64_t)rows[b] * cap[b];
  }
  S.total = tot;
  return S.d64.alloc_kept(&o.F->mem, std::max<int64_t>(tot, 1) * 16, B.s);
}

int make32(Batch& B, OpState& o, Stage& S) {
  if (B.dt != BF_C64) return BF_OK;
  BF_TRY(S.d32.alloc_kept(&o.F->mem, std::max<int64_t>(S.total, 1) * 8, B.s));
  BF_TRY(launch_convert(S.d64.p, S.d32.p, S.total, BF_C128, BF_C64, B.s));
  S.have32 = true;
  return BF_OK;
}

// One batched truncated QR over blocks of several operators.
struct QRJob {
  OpState* o;
  Stage* S;
  std::vector<const void*> in;
  std::vector<int64_t> ld;
  int k;
  std::vector<int32_t>* ranks;
};
int qr_all(Batch& B, std::vector<QRJob>& jobs) {
  std::vector<QRTask> tasks;
  for (auto& J : jobs) {
    const int nb = (int)J.S->rows.size();
    for (int b = 0; b < nb; ++b) {
      QRTask t{};
      t.in = J.in[b];
      t.ldi = J.ld[b];
      t.s = J.S->rows[b];
      t.k = J.k;
      t.cap = std::min(J.S->rows[b], J.k);
      t.q = (char*)J.S->d64.p + J.S->off[b] * 16;
      t.eps = J.o->P->tol;
      tasks.push_back(t);
    }
  }
  if (tasks.empty()) return BF_OK;
  const int nt = (int)tasks.size();
  const bool fp64 = B.ops[0].P->opt.qr_fp64 != 0;
  // one launch per lane class (qr_lanes of the block's rows), so that each
  // block is factored with the same arithmetic alone and in a batch
  std::vector<int> order(nt);
  for (int i = 0; i < nt; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return qr_lanes(tasks[a].s, B.dt, fp64) < qr_lanes(tasks[b].s, B.dt, fp64); });
  std::vector<QRTask> sorted(nt);
  for (int i = 0; i < nt; ++i) sorted[i] = tasks[order[i]];
  struct Range {
    int a, b, maxS, maxK;
  };
  std::vector<Range> ranges;
  size_t wbytes = 0;
  for (int i = 0; i < nt;) {
    const int cls = qr_lanes(sorted[i].s, B.dt, fp64);
    Range r{i, i, 1, 1};
    while (r.b < nt && qr_lanes(sorted[r.b].s, B.dt, fp64) == cls) {
      r.maxS = std::max(r.maxS, (int)sorted[r.b].s);
      r.maxK = std::max(r.maxK, (int)sorted[r.b].k);
      ++r.b;
    }
    wbytes = std::max(wbytes, qr_workspace_bytes(r.b - r.a, r.maxS, r.maxK, B.dt, fp64));
    ranges.push_back(r);
    i = r.b;
  }
  Scratch d(B.s), w(B.s);
  // the ranks, then the tensor-core wait flag: one read-back, one host wait
  BF_TRY(d.alloc(&B.mem, nt * sizeof(QRTask) + (nt + 1) * sizeof(int32_t)));
  BF_TRY(upload_async(d.p(), sorted.data(), nt * sizeof(QRTask), B.s));
  int32_t* d_r = (int32_t*)(d.p() + nt * sizeof(QRTask));
  if (wbytes) BF_TRY(w.alloc(&B.mem, wbytes));
  for (const Range& r : ranges)
    BF_TRY(launch_qr((const QRTask*)d.p() + r.a, r.b - r.a, r.maxS, r.maxK, B.dt, fp64, d_r + r.a, w.p(), wbytes,
                     B.s));
  BF_TRY(tc_status_copy(d_r + nt, B.s));
  std::vector<int32_t> hs(nt + 1), h(nt);
  BF_CUDA_TRY(cudaMemcpyAsync(hs.data(), d_r, (nt + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, B.s));
  BF_CUDA_TRY(host_sync(B.s));
  for (int i = 0; i < nt; ++i) h[order[i]] = hs[i];
  BF_TRY(tc_status_value(hs[nt], true));
  size_t q = 0;
  for (auto& J : jobs) {
    const size_t nb = J.S->rows.size();
    J.ranks->assign(h.begin() + q, h.begin() + q + nb);
    J.S->cols = *J.ranks;
    q += nb;
    BF_TRY(make32(B, *J.o, *J.S));
  }
  return BF_OK;
}

// Adaptive leaf loops (Alg. 2 loops "V" and "U") for all operators.  Vside:
// Y = A^H Gamma_t, leaves of T_S; else Z = A Omega_s, leaves of T_T.
int leaf_phase(Batch& B, bool Vside) {
  NvtxRange nv(Vside ? "Alg. 2 leaf bases V0 (loop V)" : "Alg. 2 leaf bases UL (loop U)");
  for (auto& o : B.ops) {
    o.r = o.P->opt.r0;
    o.kcap = 0;
    o.passes = 0;
    o.done = false;
  }
  int rc = BF_OK;
  for (;;) {
    std::vector<OpState*> act;
    for (auto& o : B.ops)
      if (!o.done) act.push_back(&o);
    if (act.empty()) break;
    {
      std::vector<SketchReq> reqs;
      std::vector<std::unique_ptr<Scratch>> G;
      for (OpState* o : act) {
        Plan* P = o->P;
        const int64_t in_rows = Vside ? P->m : P->n, out_rows = Vside ? P->n : P->m;
        o->k = o->r + P->opt.p;
        if (o->k <= o->kcap) continue;
        DevBuf Yn;
        BF_TRY(Yn.alloc(&o->F->mem, out_rows * o->k * B.es, B.s));
        if (o->kcap > 0)
          BF_CUDA_TRY(cudaMemcpyAsync(Yn.p, o->Y.p, out_rows * o->kcap * B.es, cudaMemcpyDeviceToDevice, B.s));
        o->Y.release(B.s);
        o->Y = Yn;
        G.emplace_back(new Scratch(B.s));
        BF_TRY(G.back()->alloc(&o->F->mem, in_rows * (o->k - o->kcap) * B.es));
        BF_TRY(launch_gaussian(P->opt.seed, sid(Vside ? STAGE_V0 : STAGE_U0, 0), 0, in_rows, o->kcap, o->k,
                               G.back()->p(), in_rows, B.dt, B.s));
        reqs.push_back({o, Vside ? BF_OP_C : BF_OP_N, 0, o->k - o->kcap, G.back()->p(),
                        (char*)o->Y.p + out_rows * o->kcap * B.es});
        o->kcap = o->k;
      }
      BF_TRY(sketch_all(B, reqs));
    }
    std::vector<QRJob> jobs;
    for (OpState* o : act) {
      Plan* P = o->P;
      const int L = P->L, nb = 1 << L;
      const int64_t out_rows = Vside ? P->n : P->m;
      const auto& off = Vside ? P->offS[L] : P->offT[L];
      Stage& S = o->F->st[Vside ? o->F->stage_V0() : o->F->stage_U()];
      std::vector<int32_t> rows(nb), cap(nb);
      for (int b = 0; b < nb; ++b) rows[b] = (int32_t)(off[b + 1] - off[b]), cap[b] = std::min(rows[b], o->k);
      BF_TRY(layout_stage(B, *o, S, rows, cap));
      QRJob J{o, &S, std::vector<const void*>(nb), std::vector<int64_t>(nb, out_rows), o->k, &o->ranks};
      for (int b = 0; b < nb; ++b) J.in[b] = (const char*)o->Y.p + off[b] * B.es;
      jobs.push_back(std::move(J));
    }
    BF_TRY(qr_all(B, jobs));
    for (OpState* o : act) {
      Plan* P = o->P;
      const int L = P->L, nb = 1 << L;
      const auto& off = Vside ? P->offS[L] : P->offT[L];
      int maxleaf = 0;
      for (int b = 0; b < nb; ++b) maxleaf = std::max<int>(maxleaf, (int)(off[b + 1] - off[b]));
      const int maxr = *std::max_element(o->ranks.begin(), o->ranks.end());
      ++o->passes;
      const bool capped = P->opt.leaf_passes > 0 && o->passes >= P->opt.leaf_passes;
      if (o->r > maxr || o->k >= maxleaf || capped) {
        o->done = true;
        o->Y.release(B.s);
        if (Vside)
          o->F->rV[0] = o->ranks;
        else
          o->F->rU[o->L - o->lm] = o->ranks;
        continue;
      }
      o->r *= 2;
      if (o->r > P->opt.r_max) rc = fail(BF_ENOTCONVERGED, "adaptive leaf rank exceeds r_max");
    }
    if (rc) return rc;
  }
  return BF_OK;
}

// W^l for every operator with l_m >= t (l = t).
int w_phase(Batch& B, int t) {
  NvtxRange nv("Alg. 2 W step %d", t);
  std::vector<OpState*> act;
  for (auto& o : B.ops)
    if (o.lm >= t) act.push_back(&o);
  if (act.empty()) return BF_OK;
  const int l = t;
  int64_t gtot = 0, ytot = 0, ptot = 0, stot = 0;
  for (OpState* o : act) {
    Plan* P = o->P;
    const int L = o->L, nb = o->nb, nt = 1 << l, nn = 1 << (L - l);
    const auto& prev = o->F->rV[l - 1];
    o->l = l;
    o->Ps.assign(nb, 0);
    int k = 0;
    for (int tau = 0; tau < nt; ++tau)
      for (int nu = 0; nu < nn; ++nu) {
        const int base = (tau >> 1) * (2 * nn);
        o->Ps[tau * nn + nu] = prev[base + 2 * nu] + prev[base + 2 * nu + 1];
        k = std::max(k, o->Ps[tau * nn + nu]);
      }
    o->k = k + P->opt.p;
    o->Poff.assign(nb + 1, 0);
    for (int b = 0; b < nb; ++b) o->Poff[b + 1] = o->Poff[b] + (int64_t)o->Ps[b] * o->k;
    o->goff = gtot, gtot += P->m * (int64_t)o->k;
    o->yoff = ytot, ytot += P->n * (int64_t)nt * o->k;
    o->poff = ptot, ptot += o->Poff[nb];
    int64_t mx = 0;   // largest non-final peel level of this operator
    for (int j = 0; j < l - 1; ++j) {
      int64_t tot = 0;
      for (int b = 0; b < nb; ++b) tot += (int64_t)o->F->rV[j][b] * ((int64_t)o->k << (l - j));
      mx = std::max(mx, tot);
    }
    o->soff = stot, stot += mx;
  }
  Scratch G(B.s), Y(B.s), Pb(B.s), SA(B.s), SB(B.s);
  BF_TRY(G.alloc(&B.mem, gtot * B.es));
  BF_TRY(Y.alloc(&B.mem, ytot * B.es));
  BF_TRY(Pb.alloc(&B.mem, ptot * B.es));
  BF_TRY(SA.alloc(&B.mem, stot * B.es));
  BF_TRY(SB.alloc(&B.mem, stot * B.es));
  std::vector<SketchReq> reqs;
  for (OpState* o : act) {
    BF_TRY(launch_gaussian(o->P->opt.seed, sid(STAGE_W, l), 0, o->P->m, 0, o->k, G.p() + o->goff * B.es, o->P->m,
                           B.dt, B.s));
    reqs.push_back({o, BF_OP_C, l, o->k, G.p() + o->goff * B.es, Y.p() + o->yoff * B.es});
  }
  BF_TRY(sketch_all(B, reqs));

  // peel V_{p tau, nu'}^H off Y into P_{tau,nu} = [V^H Y_tau(S_2nu); V^H Y_tau(S_2nu+1)]
  for (OpState* o : act) o->in_base = 0;
  for (int j = 0; j < l; ++j) {
    const bool fin = (j == l - 1);
    std::vector<StageTask> tasks;
    for (OpState* o : act) {
      Plan* P = o->P;
      Fact* F = o->F;
      const int L = o->L, nb = o->nb, nn = 1 << (L - l);
      const int64_t ncols = (int64_t)o->k << (l - j);
      const int outb = fin ? 3 : (o->in_base == 1 ? 2 : 1);
      const int nmu = 1 << (L - j);
      const auto& offS = P->offS[L];
      o->cur.assign(nb + 1, 0);
      for (int b = 0; b < nb; ++b) o->cur[b + 1] = o->cur[b] + (int64_t)F->rV[j][b] * ncols;
      for (int sg = 0; sg < (1 << j); ++sg)
        for (int mu = 0; mu < nmu; ++mu) {
          const int b = sg * nmu + mu;
          const int M = F->rV[j][b];
          auto add_terms = [&](StageTask& tk, int64_t colo) {
            if (j == 0) {
              const int sz = (int)(offS[mu + 1] - offS[mu]);
              term(tk, 0, o->yoff + offS[mu] + colo * P->n, P->n, B.fblk(*o, F->stage_V0(), mu), sz, sz, 1);
            } else {
              // level j-1 blocks are row-major with 2*ncols columns
              const int p0 = (sg >> 1) * (2 * nmu) + 2 * mu, p1 = p0 + 1;
              const int k0 = F->rV[j - 1][p0], k1 = F->rV[j - 1][p1];
              const int ldm = F->st[F->stage_W(j)].rows[b];
              const int64_t c0 = (sg & 1) * ncols + colo;
              term(tk, o->in_base, o->soff + o->prev[p0] + c0, -2 * ncols, B.fblk(*o, F->stage_W(j), b), ldm, k0, 1);
              term(tk, o->in_base, o->soff + o->prev[p1] + c0, -2 * ncols, B.fblk(*o, F->stage_W(j), b, k0), ldm,
                   k1, 1);
            }
          };
          if (!fin) {
            StageTask tk = task(outb, o->soff + o->cur[b], -ncols, M, (int)ncols);
            add_terms(tk, 0);
            tasks.push_back(tk);
          } else {
            const int nu = mu >> 1;
            const int rowoff = (mu & 1) ? F->rV[l - 1][sg * (2 * nn) + (mu & ~1)] : 0;
            for (int a = 0; a < 2; ++a) {
              const int bp = (2 * sg + a) * nn + nu;
              StageTask tk = task(3, o->poff + o->Poff[bp] + rowoff, o->Ps[bp], M, o->k);
              add_terms(tk, (int64_t)a * o->k);
              tasks.push_back(tk);
            }
          }
        }
      o->prev.swap(o->cur);
      o->in_base = outb;
    }
    BF_TRY(run_tasks(B, tasks, Y, SA, SB, Pb));
  }
  std::vector<QRJob> jobs;
  for (OpState* o : act) {
    Stage& S = o->F->st[o->F->stage_W(l)];
    std::vector<int32_t> cap(o->nb);
    for (int b = 0; b < o->nb; ++b) cap[b] = std::min(o->Ps[b], o->k);
    BF_TRY(layout_stage(B, *o, S, o->Ps, cap));
    QRJob J{o, &S, std::vector<const void*>(o->nb), std::vector<int64_t>(o->nb), o->k, &o->F->rV[l]};
    for (int b = 0; b < o->nb; ++b) J.in[b] = Pb.p() + (o->poff + o->Poff[b]) * B.es, J.ld[b] = o->Ps[b];
    jobs.push_back(std::move(J));
  }
  return qr_all(B, jobs);
}

// R^l for every operator with L - t >= l_m (l = L - t); X and B at l_m.
int r_phase(Batch& B, int t) {
  NvtxRange nv("Alg. 2 R step %d (centre level at the last)", t);
  std::vector<OpState*> act;
  for (auto& o : B.ops)
    if (o.L - t >= o.lm) act.push_back(&o);
  if (act.empty()) return BF_OK;
  int64_t gtot = 0, ztot = 0, ptot = 0, stot = 0;
  for (OpState* o : act) {
    Plan* P = o->P;
    const int L = o->L, lm = o->lm, nb = o->nb, l = L - t, nt = 1 << l, nn = 1 << (L - l), nn1 = nn >> 1;
    const auto& nxt = o->F->rU[l + 1 - lm];
    o->l = l;
    o->Ps.assign(nb, 0);
    int k = 0;
    for (int tau = 0; tau < nt; ++tau)
      for (int nu = 0; nu < nn; ++nu) {
        o->Ps[tau * nn + nu] = nxt[(2 * tau) * nn1 + (nu >> 1)] + nxt[(2 * tau + 1) * nn1 + (nu >> 1)];
        k = std::max(k, o->Ps[tau * nn + nu]);
      }
    if (l == lm) k = std::max(k, *std::max_element(o->F->rV[lm].begin(), o->F->rV[lm].end()));
    o->k = k + P->opt.p;
    o->Poff.assign(nb + 1, 0);
    for (int b = 0; b < nb; ++b) o->Poff[b + 1] = o->Poff[b] + (int64_t)o->Ps[b] * o->k;
    o->goff = gtot, gtot += P->n * (int64_t)o->k;
    o->yoff = ztot, ztot += P->m * (int64_t)nn * o->k;
    o->poff = ptot, ptot += o->Poff[nb];
    int64_t mx = 0;
    for (int j = L; j > l + 1; --j) {
      int64_t tot = 0;
      for (int b = 0; b < nb; ++b) tot += (int64_t)o->F->rU[j - lm][b] * ((int64_t)o->k << (j - l));
      mx = std::max(mx, tot);
    }
    if (l == lm)   // project_X intermediates (k columns per block)
      for (int j = 0; j < lm; ++j) {
        int64_t tot = 0;
        for (int b = 0; b < nb; ++b) tot += (int64_t)o->F->rV[j][b] * o->k;
        mx = std::max(mx, tot);
      }
    o->soff = stot, stot += mx;
  }
  Scratch G(B.s), Z(B.s), Pb(B.s), SA(B.s), SB(B.s);
  BF_TRY(G.alloc(&B.mem, gtot * B.es));
  BF_TRY(Z.alloc(&B.mem, ztot * B.es));
  BF_TRY(Pb.alloc(&B.mem, ptot * B.es));
  BF_TRY(SA.alloc(&B.mem, stot * B.es));
  BF_TRY(SB.alloc(&B.mem, stot * B.es));
  std::vector<SketchReq> reqs;
  for (OpState* o : act) {
    BF_TRY(launch_gaussian(o->P->opt.seed, sid(STAGE_R, o->l), 0, o->P->n, 0, o->k, G.p() + o->goff * B.es,
                           o->P->n, B.dt, B.s));
    reqs.push_back({o, BF_OP_N, o->L - o->l, o->k, G.p() + o->goff * B.es, Z.p() + o->yoff * B.es});
  }
  BF_TRY(sketch_all(B, reqs));

  // peel U_{tau', p nu}^H off Z into P_{tau,nu} = [U^H Z_nu(T_2tau); U^H Z_nu(T_2tau+1)]
  for (OpState* o : act) o->in_base = 0;
  for (int st = 0; st < t; ++st) {
    std::vector<StageTask> tasks;
    for (OpState* o : act) {
      Plan* P = o->P;
      Fact* F = o->F;
      const int L = o->L, lm = o->lm, nb = o->nb, l = o->l, nn = 1 << (L - l);
      const int j = L - st;
      const bool fin = (j == l + 1);
      auto ru = [&](int jj, int b) { return F->rU[jj - lm][b]; };
      const int64_t ncols = (int64_t)o->k << (j - l);
      const int outb = fin ? 3 : (o->in_base == 1 ? 2 : 1);
      const int nmu = 1 << (L - j);
      const auto& offT = P->offT[L];
      o->cur.assign(nb + 1, 0);
      for (int b = 0; b < nb; ++b) o->cur[b + 1] = o->cur[b] + (int64_t)ru(j, b) * ncols;
      for (int sg = 0; sg < (1 << j); ++sg)
        for (int mu = 0; mu < nmu; ++mu) {
          const int b = sg * nmu + mu;
          const int M = ru(j, b);
          auto add_terms = [&](StageTask& tk, int64_t colo) {
            if (j == L) {
              const int sz = (int)(offT[sg + 1] - offT[sg]);
              term(tk, 0, o->yoff + offT[sg] + colo * P->m, P->m, B.fblk(*o, F->stage_U(), sg), sz, sz, 1);
            } else {
              // level j+1 blocks are row-major with 2*ncols columns
              const int nm1 = nmu >> 1;
              const int c0i = (2 * sg) * nm1 + (mu >> 1), c1i = (2 * sg + 1) * nm1 + (mu >> 1);
              const int k0 = ru(j + 1, c0i), k1 = ru(j + 1, c1i);
              const int ldm = F->st[F->stage_R(j)].rows[b];
              const int64_t cc = (mu & 1) * ncols + colo;
              term(tk, o->in_base, o->soff + o->prev[c0i] + cc, -2 * ncols, B.fblk(*o, F->stage_R(j), b), ldm, k0, 1);
              term(tk, o->in_base, o->soff + o->prev[c1i] + cc, -2 * ncols, B.fblk(*o, F->stage_R(j), b, k0), ldm,
                   k1, 1);
            }
          };
          if (!fin) {
            StageTask tk = task(outb, o->soff + o->cur[b], -ncols, M, (int)ncols);
            add_terms(tk, 0);
            tasks.push_back(tk);
          } else {
            const int tau = sg >> 1;
            const int rowoff = (sg & 1) ? ru(l + 1, (sg & ~1) * nmu + mu) : 0;
            for (int cc = 0; cc < 2; ++cc) {
              const int bp = tau * nn + 2 * mu + cc;
              StageTask tk = task(3, o->poff + o->Poff[bp] + rowoff, o->Ps[bp], M, o->k);
              add_terms(tk, (int64_t)cc * o->k);
              tasks.push_back(tk);
            }
          }
        }
      o->prev.swap(o->cur);
      o->in_base = outb;
    }
    BF_TRY(run_tasks(B, tasks, Z, SA, SB, Pb));
  }
  std::vector<QRJob> jobs;
  for (OpState* o : act) {
    Stage& S = o->F->st[o->F->stage_R(o->l)];
    std::vector<int32_t> cap(o->nb);
    for (int b = 0; b < o->nb; ++b) cap[b] = std::min(o->Ps[b], o->k);
    BF_TRY(layout_stage(B, *o, S, o->Ps, cap));
    QRJob J{o, &S, std::vector<const void*>(o->nb), std::vector<int64_t>(o->nb), o->k, &o->F->rU[o->l - o->lm]};
    for (int b = 0; b < o->nb; ++b) J.in[b] = Pb.p() + (o->poff + o->Poff[b]) * B.es, J.ld[b] = o->Ps[b];
    jobs.push_back(std::move(J));
  }
  BF_TRY(qr_all(B, jobs));

  // centre level: X_{tau,nu} = V_{tau,nu}^H Omega_nu through V^0, W^1..W^(l_m)
  std::vector<OpState*> ctr;
  for (OpState* o : act)
    if (o->l == o->lm) ctr.push_back(o);
  if (ctr.empty()) return BF_OK;
  int64_t xtot = 0, jmax = 0;
  for (OpState* o : ctr) {
    int64_t x = 0;
    for (int b = 0; b < o->nb; ++b) x += (int64_t)o->F->rV[o->lm][b] * o->k;
    o->xoff = xtot, xtot += x;
    jmax = std::max<int64_t>(jmax, o->lm);
    o->in_base = 0;
  }
  Scratch Xb(B.s);
  BF_TRY(Xb.alloc(&B.mem, xtot * B.es));
  for (int j = 0; j <= jmax; ++j) {
    std::vector<StageTask> tasks;
    for (OpState* o : ctr) {
      if (j > o->lm) continue;
      Plan* P = o->P;
      Fact* F = o->F;
      const int L = o->L, nb = o->nb, k = o->k;
      const bool fin = j == o->lm;
      const int outb = fin ? 3 : (o->in_base == 1 ? 2 : 1);
      const int nmu = 1 << (L - j);
      const auto& offS = P->offS[L];
      o->cur.assign(nb + 1, 0);
      for (int b = 0; b < nb; ++b) o->cur[b + 1] = o->cur[b] + (int64_t)F->rV[j][b] * k;
      const int64_t obase = fin ? o->xoff : o->soff;
      for (int sg = 0; sg < (1 << j); ++sg)
        for (int mu = 0; mu < nmu; ++mu) {
          const int b = sg * nmu + mu;
          const int M = F->rV[j][b];
          // intermediates row-major; the final X blocks column-major (ld r^V) for the solve
          StageTask tk = task(outb, obase + o->cur[b], fin ? M : -k, M, k);
          if (j == 0) {
            const int sz = (int)(offS[mu + 1] - offS[mu]);
            term(tk, 0, o->goff + offS[mu], P->n, B.fblk(*o, F->stage_V0(), mu), sz, sz, 1);
          } else {
            const int p0 = (sg >> 1) * (2 * nmu) + 2 * mu, p1 = p0 + 1;
            const int k0 = F->rV[j - 1][p0], k1 = F->rV[j - 1][p1];
            const int ldm = F->st[F->stage_W(j)].rows[b];
            term(tk, o->in_base, o->soff + o->prev[p0], -k, B.fblk(*o, F->stage_W(j), b), ldm, k0, 1);
            term(tk, o->in_base, o->soff + o->prev[p1], -k, B.fblk(*o, F->stage_W(j), b, k0), ldm, k1, 1);
          }
          tasks.push_back(tk);
        }
      o->prev.swap(o->cur);
      o->in_base = outb;
    }
    BF_TRY(run_tasks(B, tasks, G, SA, SB, Xb));
  }
  // B = argmin ||C - B X||_F, C = R^H P (eq. Bij)
  std::vector<LSQTask> lt;
  int maxR = 1, maxS = 1, maxK = 1;
  for (OpState* o : ctr) {
    Fact* F = o->F;
    const int lm = o->lm, nb = o->nb;
    Stage& S = F->st[F->stage_R(lm)];
    Stage& SBs = F->st[F->stage_B()];
    std::vector<int32_t> rows(nb), cols(nb);
    for (int b = 0; b < nb; ++b) {
      rows[b] = F->rU[0][b];
      cols[b] = F->rV[lm][b];
      maxR = std::max({maxR, rows[b], cols[b]});
      maxS = std::max(maxS, o->Ps[b]);
    }
    maxK = std::max(maxK, o->k);
    BF_TRY(layout_stage(B, *o, SBs, rows, cols));
    SBs.cols = cols;
    for (int b = 0; b < nb; ++b) {
      LSQTask tk{};
      tk.P = Pb.p() + (o->poff + o->Poff[b]) * B.es;
      tk.Q = (const char*)S.d64.p + S.off[b] * 16;
      tk.X = Xb.p() + (o->xoff + o->prev[b]) * B.es;
      tk.B = (char*)SBs.d64.p + SBs.off[b] * 16;
      tk.s = o->Ps[b];
      tk.k = o->k;
      tk.rU = rows[b];
      tk.rV = cols[b];
      lt.push_back(tk);
    }
  }
  Scratch d(B.s), lw(B.s);
  BF_TRY(d.alloc(&B.mem, lt.size() * sizeof(LSQTask)));
  BF_TRY(upload_async(d.p(), lt.data(), lt.size() * sizeof(LSQTask), B.s));
  const size_t lwb = lsq_workspace_bytes((int)lt.size(), maxK, maxR);
  if (lwb) BF_TRY(lw.alloc(&B.mem, lwb));
  BF_TRY(launch_lsq((const LSQTask*)d.p(), (int)lt.size(), maxS, maxK, maxR, B.dt, lw.p(), lwb, B.s));
  for (OpState* o : ctr) BF_TRY(make32(B, *o, o->F->st[o->F->stage_B()]));
  BF_CUDA_TRY(host_sync(B.s));
  return BF_OK;
}

// A side's own copy of the batch: the same operators, plans and
// factorizations, its own stream, phase state and arenas (the entry images
// stay owned by the original batch; their device pointers are shared).
Batch side_copy(const Batch& B, cudaStream_t s) {
  Batch S;
  S.s = s;
  S.dt = B.dt;
  S.es = B.es;
  S.mem.cap = B.mem.cap;
  S.ops.resize(B.ops.size());
  for (size_t i = 0; i < B.ops.size(); ++i) {
    const OpState& o = B.ops[i];
    OpState& q = S.ops[i];
    q.P = o.P;
    q.A = o.A;
    q.F = o.F;
    q.L = o.L;
    q.lm = o.lm;
    q.nb = o.nb;
    q.img_n = o.img_n;
    q.img_c = o.img_c;
  }
  return S;
}

std::atomic<int> g_parallel_sides{1};

// One persistent host thread for the W side of factorizations (its pinned
// upload ring and CUDA state stay set up between calls); one factorization
// uses it at a time, others run their sides sequentially.
class SideWorker {
 public:
  static SideWorker* get() {
    static SideWorker* w = make();
    return w;
  }
  std::mutex use;   // held by the factorization whose W side runs here
  void submit(std::function<void()> f) {
    std::lock_guard<std::mutex> lk(mu_);
    job_ = std::move(f);
    has_ = true;
    done_ = false;
    cv_.notify_one();
  }
  void wait() {
    std::unique_lock<std::mutex> lk(mu_);
    done_cv_.wait(lk, [&] { return done_; });
  }

 private:
  static SideWorker* make() {
    SideWorker* w = new SideWorker();   // lives until the process exits
    try {
      std::thread([w] { w->loop(); }).detach();
    } catch (const std::system_error&) {
      delete w;
      return nullptr;
    }
    return w;
  }
  void loop() {
    for (;;) {
      std::function<void()> f;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return has_; });
        f = std::move(job_);
        has_ = false;
      }
      f();
      {
        std::lock_guard<std::mutex> lk(mu_);
        done_ = true;
      }
      done_cv_.notify_all();
    }
  }
  std::mutex mu_;
  std::condition_variable cv_, done_cv_;
  std::function<void()> job_;
  bool has_ = false, done_ = true;
};

// Alg. 2's loops for all operators.  The row-basis side (loop "V", then the
// W levels) and the column-basis side (loop "U", then the R levels above
// the centre) do not depend on each other (Sec. 4.2-4.3); only the centre
// level (R at l_m, X = V^H Omega, the B solve) needs both.  So the W side
// runs on a second host thread and stream while this thread runs the R
// side, and joins it before the first centre level: each side's host
// synchronisations and latency-bound phases (QR, peeling) overlap the other
// side's sketches.  The launches of every phase are the same as when the
// sides run one after the other, so the results are identical.  Operators
// not bound to the plan (callbacks, factored and composed operators, whose
// products may share state) and memory-capped batches run sequentially.
int run_sides(Batch& B, int maxlm, int maxr) {
  bool parallel = g_parallel_sides.load() != 0 && B.mem.cap == 0;
  for (const auto& o : B.ops) parallel = parallel && o.A->plan == o.P && o.F->mem.cap == 0;
  if (!parallel) {
    int rc = leaf_phase(B, true);
    if (!rc) rc = leaf_phase(B, false);
    for (int t = 1; !rc && t <= maxlm; ++t) rc = w_phase(B, t);
    for (int t = 1; !rc && t <= maxr; ++t) rc = r_phase(B, t);
    return rc;
  }
  cudaStream_t sw = nullptr;
  cudaEvent_t ev = nullptr;
  BF_CUDA_TRY(cudaStreamCreateWithFlags(&sw, cudaStreamNonBlocking));
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess || cudaEventRecord(ev, B.s) != cudaSuccess ||
      cudaStreamWaitEvent(sw, ev, 0) != cudaSuccess) {   // the W side starts after the entry images
    if (ev) cudaEventDestroy(ev);
    cudaStreamDestroy(sw);
    return fail(BF_ECUDA, "side stream set-up failed");
  }
  Batch BW = side_copy(B, sw), BR = side_copy(B, B.s);
  int rcw = BF_OK;
  std::string errw;
  int dev = 0;
  cudaGetDevice(&dev);
  auto w_side = [&]() {
    int rc = cudaSetDevice(dev) == cudaSuccess ? BF_OK : fail(BF_ECUDA, "W side: cudaSetDevice failed");
    try {
      if (!rc) rc = leaf_phase(BW, true);
      for (int t = 1; !rc && t <= maxlm; ++t) rc = w_phase(BW, t);
    } catch (...) {   // no exception may leave the worker
      rc = fail(BF_ENOMEM, "host allocation failed on the W side");
    }
    const cudaError_t e = host_sync(sw);   // (the last factor copies)
    if (!rc && e != cudaSuccess) rc = fail(BF_ECUDA, std::string("W side: ") + cudaGetErrorString(e));
    if (rc) errw = bf_last_error();
    rcw = rc;
  };
  SideWorker* worker = SideWorker::get();
  std::unique_lock<std::mutex> held;
  if (worker) held = std::unique_lock<std::mutex>(worker->use, std::try_to_lock);
  const bool threaded = worker && held.owns_lock();
  if (threaded)
    worker->submit(w_side);
  else
    w_side();   // no worker free: the W side first, here
  bool joined = !threaded;
  auto join = [&]() {
    if (!joined) worker->wait(), joined = true;
  };
  int rc = BF_OK;
  try {
    rc = leaf_phase(BR, false);
    for (int t = 1; !rc && t <= maxr; ++t) {
      bool centre = false;
      for (const auto& o : BR.ops) centre = centre || o.L - t == o.lm;
      if (centre) {
        join();
        if (rcw) break;
      }
      rc = r_phase(BR, t);
    }
  } catch (...) {
    rc = fail(BF_ENOMEM, "host allocation failed on the R side");
  }
  join();
  for (auto& o : BW.ops) o.Y.release(sw);
  for (auto& o : BR.ops) o.Y.release(B.s);
  host_sync(sw);
  cudaEventDestroy(ev);
  cudaStreamDestroy(sw);
  if (rcw) {
    set_error(errw);
    return rcw;
  }
  return rc;
}

void destroy(Fact* F) {
  for (auto& S : F->st) S.d64.release(nullptr), S.d32.release(nullptr);
  delete F;
}

}  // namespace

int factor_batch(int count, Plan* const* P, Operator* const* A, cudaStream_t s, Fact** out) {
  NvtxRange nv("bf_factor (Alg. 2), operators: %d", count);
  for (int i = 0; i < count; ++i) out[i] = nullptr;
  if (count < 1) return fail(BF_EINVAL, "empty batch");
  const int prec = P[0]->opt.precision;
  for (int i = 0; i < count; ++i) {
    if (A[i]->m != P[i]->m || A[i]->n != P[i]->n)
      return fail(BF_EINVAL, "operator shape does not match its plan (batch entry " + std::to_string(i) + ")");
    if (P[i]->opt.precision != prec) return fail(BF_EINVAL, "all plans of a batch must share one precision");
    if (P[i]->opt.qr_fp64 != P[0]->opt.qr_fp64) return fail(BF_EINVAL, "all plans of a batch must share qr_fp64");
    if (P[i]->opt.accept_retries > 0 && count > 1)
      return fail(BF_EUNSUPPORTED, "a-posteriori acceptance (accept_retries) is a bf_factor option");
  }
  const auto t0 = std::chrono::steady_clock::now();
  Batch B;
  B.s = s;
  B.dt = prec == BF_PREC_MIXED ? BF_C64 : BF_C128;
  B.es = elem_bytes(B.dt);
  size_t cap = 0;
  bool capped = true;
  for (int i = 0; i < count; ++i) capped = capped && P[i]->opt.mem_cap > 0, cap += P[i]->opt.mem_cap;
  B.mem.cap = capped ? cap : 0;
  B.ops.resize(count);
  std::vector<int64_t> n0(count), t0c(count);
  int maxlm = 0, maxr = 0;
  for (int i = 0; i < count; ++i) {
    OpState& o = B.ops[i];
    o.P = P[i];
    o.A = A[i];
    o.L = P[i]->L;
    o.lm = P[i]->lm;
    o.nb = 1 << o.L;
    Fact* F = new Fact();
    F->plan = P[i];
    F->L = o.L;
    F->lm = o.lm;
    F->n = P[i]->n;
    F->m = P[i]->m;
    F->mem.cap = P[i]->opt.mem_cap;
    F->st.resize(o.L + 3);
    F->rV.assign(o.lm + 1, {});
    F->rU.assign(o.L - o.lm + 1, {});
    o.F = F;
    n0[i] = A[i]->cols_N;
    t0c[i] = A[i]->cols_T;
    maxlm = std::max(maxlm, o.lm);
    maxr = std::max(maxr, o.L - o.lm);
  }
  int rc = make_images(B);
  if (!rc) rc = run_sides(B, maxlm, maxr);
  if (!rc) {
    const cudaError_t e = host_sync(s);
    if (e != cudaSuccess) rc = fail(BF_ECUDA, cudaGetErrorString(e));
  }
  for (auto& o : B.ops) {
    o.Y.release(s);
    o.imgN.release(s);
    o.imgC.release(s);
  }
  if (rc) {
    for (auto& o : B.ops) destroy(o.F);
    return rc;
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int i = 0; i < count; ++i) {
    Fact* F = B.ops[i].F;
    F->cols_N = A[i]->cols_N - n0[i];
    F->cols_T = A[i]->cols_T - t0c[i];
    F->seconds = secs;
    out[i] = F;
  }
  return BF_OK;
}

int set_parallel_sides(int on) {
  if (on != 0 && on != 1) return fail(BF_EINVAL, "parallel sides: 0 or 1");
  g_parallel_sides.store(on);
  return BF_OK;
}

int factor(Plan* P, Operator* A, cudaStream_t s, Fact** out) {
  *out = nullptr;
  return factor_batch(1, &P, &A, s, out);
}

}  // namespace bf
