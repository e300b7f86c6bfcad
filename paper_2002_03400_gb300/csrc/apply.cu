// Apply of a finished hybrid butterfly factorization (eq. hybrid_butterfly_mat):
//   F x  = U^L R^(L-1) ... R^(l_m) B^(l_m) W^(l_m) ... W^1 V^0 x
//   F^H x = V^0^H W^1^H ... B^H ... R^(L-1)^H U^L^H x,   F^T x = conj(F^H conj x)
// as L + 3 block-sparse stage launches.  Intermediates of one level are
// stored as one stacked matrix (rows = sum of the level's block ranks,
// ld = that sum), so the task lists do not depend on the number of
// right-hand sides and are built once per factorization, direction and dtype.
#include <algorithm>

#include "bf_internal.h"

namespace bf {

namespace {

void prefix(const std::vector<int32_t>& r, std::vector<int64_t>& off) {
  off.assign(r.size() + 1, 0);
  for (size_t i = 0; i < r.size(); ++i) off[i + 1] = off[i] + r[i];
}

struct Builder {
  std::vector<StageTask> all;
  ApplyPlan* ap;
  int cur_first = 0;
  void begin() { cur_first = (int)all.size(); }
  void end() {
    int mM = 0, mN = 0;
    for (size_t i = cur_first; i < all.size(); ++i) {
      mM = std::max(mM, all[i].M);
      mN = std::max(mN, all[i].N);
    }
    ap->first.push_back(cur_first);
    ap->count.push_back((int)all.size() - cur_first);
    ap->maxM.push_back(mM);
    ap->maxN.push_back(mN);
  }
};

StageTask mk(int out_base, int64_t out_off, int64_t ldo, int M) {
  StageTask t{};
  t.out_base = (int16_t)out_base;
  t.out_off = out_off;
  t.ldo = ldo;
  t.M = M;
  t.N = 0;
  t.nterms = 0;
  return t;
}
void add_term(StageTask& t, int in_base, int64_t in_off, int64_t ldi, const void* mat, int ldm,
              int K, int conjT) {
  StageTerm& T = t.t[t.nterms++];
  T.in_base = (int16_t)in_base;
  T.in_off = in_off;
  T.ldi = ldi;
  T.mat = mat;
  T.ldm = ldm;
  T.K = K;
  T.conjT = (int16_t)conjT;
}

}  // namespace

// Factor block pointer in the requested dtype (complex128 data or its
// complex64 copy), optionally advanced by `row` rows.
static const void* blk(const Fact* F, int stage, int b, int dtype, int row = 0) {
  const Stage& S = F->st[stage];
  const char* base = (const char*)(dtype == BF_C128 ? S.d64.p : S.d32.p);
  return base + (S.off[b] + row) * (int64_t)elem_bytes(dtype);
}

// Host half of the task lists: fills ap's stage metadata and `all`.
void apply_tasks_host(const Fact* F, int opC, int dtype, ApplyPlan& ap, std::vector<StageTask>& all) {
  const Plan* P = F->plan;
  const int L = F->L, lm = F->lm, nb = 1 << L;
  std::vector<std::vector<int64_t>> rowV(lm + 1), rowU(L - lm + 1);
  for (int j = 0; j <= lm; ++j) prefix(F->rV[j], rowV[j]);
  for (int j = lm; j <= L; ++j) prefix(F->rU[j - lm], rowU[j - lm]);
  // stacked level intermediates are row-major with the launch's column
  // count: ld = 0 and the offsets below are row indices
  auto RV = [&](int) { return (int64_t)0; };
  auto RU = [&](int) { return (int64_t)0; };
  auto rv = [&](int j, int b) { return F->rV[j][b]; };
  auto ru = [&](int j, int b) { return F->rU[j - lm][b]; };
  int64_t rows_max = 0;
  for (int j = 0; j <= lm; ++j) rows_max = std::max(rows_max, rowV[j][nb]);
  for (int j = lm; j <= L; ++j) rows_max = std::max(rows_max, rowU[j - lm][nb]);
  ap.level_rows_max = rows_max;
  const auto& offS = P->offS[L];
  const auto& offT = P->offT[L];
  Builder B;
  B.ap = &ap;
  int cur = 1;
  auto flip = [&]() { cur = 3 - cur; };
  if (!opC) {
    // V^0: leaf projections V_{t,nu}^H x(S_nu)
    B.begin();
    for (int nu = 0; nu < nb; ++nu) {
      StageTask t = mk(cur, rowV[0][nu], RV(0), rv(0, nu));
      const int sz = (int)(offS[nu + 1] - offS[nu]);
      add_term(t, 0, offS[nu], P->n, blk(F, F->stage_V0(), nu, dtype), sz, sz, 1);
      B.all.push_back(t);
    }
    B.end();
    // W^j: x_j(s,mu) = W^H [x_{j-1}(s/2, 2mu); x_{j-1}(s/2, 2mu+1)]
    for (int j = 1; j <= lm; ++j) {
      const int in = cur;
      flip();
      B.begin();
      const int nn = 1 << (L - j);
      for (int sg = 0; sg < (1 << j); ++sg)
        for (int mu = 0; mu < nn; ++mu) {
          const int b = sg * nn + mu;
          const int p0 = (sg >> 1) * (2 * nn) + 2 * mu, p1 = p0 + 1;
          StageTask t = mk(cur, rowV[j][b], RV(j), rv(j, b));
          const int ldm = F->st[F->stage_W(j)].rows[b];
          add_term(t, in, rowV[j - 1][p0], RV(j - 1), blk(F, F->stage_W(j), b, dtype), ldm, rv(j - 1, p0), 1);
          add_term(t, in, rowV[j - 1][p1], RV(j - 1), blk(F, F->stage_W(j), b, dtype, rv(j - 1, p0)), ldm,
                   rv(j - 1, p1), 1);
          B.all.push_back(t);
        }
      B.end();
    }
    // B^(l_m)
    {
      const int in = cur;
      flip();
      B.begin();
      for (int b = 0; b < nb; ++b) {
        StageTask t = mk(cur, rowU[0][b], RU(lm), ru(lm, b));
        add_term(t, in, rowV[lm][b], RV(lm), blk(F, F->stage_B(), b, dtype), ru(lm, b), rv(lm, b), 0);
        B.all.push_back(t);
      }
      B.end();
    }
    // R^j: level j -> j+1, u_{j+1}(s', mu') = sum_c R_{s'/2, 2mu'+c}[rows of s'] u_j(s'/2, 2mu'+c)
    for (int j = lm; j < L; ++j) {
      const int in = cur;
      flip();
      B.begin();
      const int nn = 1 << (L - j), nn1 = nn >> 1;
      for (int sp = 0; sp < (1 << (j + 1)); ++sp)
        for (int mp = 0; mp < nn1; ++mp) {
          const int bo = sp * nn1 + mp;
          StageTask t = mk(cur, rowU[j + 1 - lm][bo], RU(j + 1), ru(j + 1, bo));
          const int rowoff = (sp & 1) ? ru(j + 1, (sp & ~1) * nn1 + mp) : 0;
          for (int c = 0; c < 2; ++c) {
            const int b = (sp >> 1) * nn + 2 * mp + c;
            add_term(t, in, rowU[j - lm][b], RU(j), blk(F, F->stage_R(j), b, dtype, rowoff),
                     F->st[F->stage_R(j)].rows[b], ru(j, b), 0);
          }
          B.all.push_back(t);
        }
      B.end();
    }
    // U^L: y(T_tau) = U_{tau,s} u_L(tau)
    {
      const int in = cur;
      B.begin();
      for (int tau = 0; tau < nb; ++tau) {
        const int sz = (int)(offT[tau + 1] - offT[tau]);
        StageTask t = mk(3, offT[tau], P->m, sz);
        add_term(t, in, rowU[L - lm][tau], RU(L), blk(F, F->stage_U(), tau, dtype), sz, ru(L, tau), 0);
        B.all.push_back(t);
      }
      B.end();
    }
  } else {
    // U^H
    B.begin();
    for (int tau = 0; tau < nb; ++tau) {
      const int sz = (int)(offT[tau + 1] - offT[tau]);
      StageTask t = mk(cur, rowU[L - lm][tau], RU(L), ru(L, tau));
      add_term(t, 0, offT[tau], P->m, blk(F, F->stage_U(), tau, dtype), sz, sz, 1);
      B.all.push_back(t);
    }
    B.end();
    // R^j^H: level j+1 -> j
    for (int j = L - 1; j >= lm; --j) {
      const int in = cur;
      flip();
      B.begin();
      const int nn = 1 << (L - j), nn1 = nn >> 1;
      for (int tau = 0; tau < (1 << j); ++tau)
        for (int nu = 0; nu < nn; ++nu) {
          const int b = tau * nn + nu;
          const int c0 = (2 * tau) * nn1 + (nu >> 1), c1 = (2 * tau + 1) * nn1 + (nu >> 1);
          StageTask t = mk(cur, rowU[j - lm][b], RU(j), ru(j, b));
          const int ldm = F->st[F->stage_R(j)].rows[b];
          add_term(t, in, rowU[j + 1 - lm][c0], RU(j + 1), blk(F, F->stage_R(j), b, dtype), ldm, ru(j + 1, c0), 1);
          add_term(t, in, rowU[j + 1 - lm][c1], RU(j + 1), blk(F, F->stage_R(j), b, dtype, ru(j + 1, c0)), ldm,
                   ru(j + 1, c1), 1);
          B.all.push_back(t);
        }
      B.end();
    }
    // B^H
    {
      const int in = cur;
      flip();
      B.begin();
      for (int b = 0; b < nb; ++b) {
        StageTask t = mk(cur, rowV[lm][b], RV(lm), rv(lm, b));
        add_term(t, in, rowU[0][b], RU(lm), blk(F, F->stage_B(), b, dtype), ru(lm, b), ru(lm, b), 1);
        B.all.push_back(t);
      }
      B.end();
    }
    // W^j^H: level j -> j-1
    for (int j = lm; j >= 1; --j) {
      const int in = cur;
      flip();
      B.begin();
      const int nn = 1 << (L - j);
      for (int rho = 0; rho < (1 << (j - 1)); ++rho)
        for (int kap = 0; kap < 2 * nn; ++kap) {
          const int bo = rho * (2 * nn) + kap;
          StageTask t = mk(cur, rowV[j - 1][bo], RV(j - 1), rv(j - 1, bo));
          const int rowoff = (kap & 1) ? rv(j - 1, rho * (2 * nn) + (kap & ~1)) : 0;
          for (int a = 0; a < 2; ++a) {
            const int b = (2 * rho + a) * nn + (kap >> 1);
            add_term(t, in, rowV[j][b], RV(j), blk(F, F->stage_W(j), b, dtype, rowoff),
                     F->st[F->stage_W(j)].rows[b], rv(j, b), 0);
          }
          B.all.push_back(t);
        }
      B.end();
    }
    // V^0: y(S_nu) = V_{t,nu} x_0(nu)
    {
      const int in = cur;
      B.begin();
      for (int nu = 0; nu < nb; ++nu) {
        const int sz = (int)(offS[nu + 1] - offS[nu]);
        StageTask t = mk(3, offS[nu], P->n, sz);
        add_term(t, in, rowV[0][nu], RV(0), blk(F, F->stage_V0(), nu, dtype), sz, rv(0, nu), 0);
        B.all.push_back(t);
      }
      B.end();
    }
  }
  all.swap(B.all);
}

// Bounds of an apply's task lists for one column (the row-major level
// buffers' rows scale with the column count, a column-major operand's rows
// do not depend on it): x, the two level buffers, y.
int check_apply_tasks(const Fact* F, int opC, int dtype, const ApplyPlan& ap, const std::vector<StageTask>& all) {
  const Plan* P = F->plan;
  const int64_t ext[4] = {opC ? P->m : P->n, ap.level_rows_max, ap.level_rows_max, opC ? P->n : P->m};
  return check_stage_tasks("apply task list", all, 1, ext, F, dtype);
}

static int build_apply(Fact* F, int opC, int dtype, cudaStream_t s) {
  ApplyPlan& ap = F->ap[opC][dtype];
  ap = ApplyPlan();
  std::vector<StageTask> all;
  apply_tasks_host(F, opC, dtype, ap, all);
  if (debug_checks()) BF_TRY(check_apply_tasks(F, opC, dtype, ap, all));
  BF_TRY(ap.tasks.alloc(&F->mem, all.size() * sizeof(StageTask), nullptr));
  BF_CUDA_TRY(cudaMemcpyAsync(ap.tasks.p, all.data(), all.size() * sizeof(StageTask),
                              cudaMemcpyHostToDevice, s));
  BF_CUDA_TRY(host_sync(s));
  ap.variant.assign(ap.first.size(), std::array<int8_t, NRHS_CLASSES>{-1, -1, -1, -1, -1, -1});
  ap.built = true;
  return BF_OK;
}

int Fact::ensure32(cudaStream_t s) {
  for (auto& S : st) {
    if (S.have32) continue;
    BF_TRY(S.d32.alloc(&mem, S.total * 8, nullptr));
    BF_TRY(launch_convert(S.d64.p, S.d32.p, S.total, BF_C128, BF_C64, s));
    S.have32 = true;
  }
  return BF_OK;
}

int check_stage_tasks(const char* what, const std::vector<StageTask>& tasks, int64_t N, const int64_t ext[4],
                      const Fact* F, int dtype) {
  const size_t es = elem_bytes(dtype);
  // first and last element an operand of `rows` rows and n columns touches
  auto span = [](int64_t off, int64_t ld, int64_t rows, int64_t n, int64_t* lo, int64_t* hi) {
    if (ld > 0) *lo = off, *hi = off + (rows - 1) + (n - 1) * ld;
    else if (ld < 0) *lo = off, *hi = off + (rows - 1) * (-ld) + (n - 1);
    else *lo = off * n, *hi = (off + rows - 1) * n + n - 1;
  };
  auto bad = [&](size_t i, const std::string& why) {
    return fail(BF_EINTERNAL, std::string(what) + ": task " + std::to_string(i) + " " + why);
  };
  for (size_t i = 0; i < tasks.size(); ++i) {
    const StageTask& t = tasks[i];
    const int64_t n = N > 0 ? N : t.N;
    if (t.M < 0 || t.nterms < 0 || t.nterms > 2 || n < 0) return bad(i, "has a negative size or too many terms");
    if (t.M == 0 || n == 0) continue;
    if (t.out_base < 0 || t.out_base > 3) return bad(i, "writes an unknown buffer");
    int64_t lo, hi;
    span(t.out_off, t.ldo, t.M, n, &lo, &hi);
    if (lo < 0 || (ext[t.out_base] > 0 && hi >= ext[t.out_base]))
      return bad(i, "writes outside buffer " + std::to_string(t.out_base));
    for (int q = 0; q < t.nterms; ++q) {
      const StageTerm& T = t.t[q];
      if (T.K < 0 || T.in_base < 0 || T.in_base > 3) return bad(i, "has a bad term");
      if (T.K == 0) continue;
      span(T.in_off, T.ldi, T.K, n, &lo, &hi);
      if (lo < 0 || (ext[T.in_base] > 0 && hi >= ext[T.in_base]))
        return bad(i, "reads outside buffer " + std::to_string(T.in_base));
      // entry (i, k) of op(mat): mat[i ldm + k] (adjoint) or mat[i + k ldm]
      if (T.ldm < (T.conjT ? T.K : t.M)) return bad(i, "has a leading dimension below its block's");
      if (!F) continue;
      const int64_t last = T.conjT ? (int64_t)(t.M - 1) * T.ldm + T.K - 1 : (t.M - 1) + (int64_t)(T.K - 1) * T.ldm;
      for (const Stage& S : F->st) {
        const char* b = (const char*)(dtype == BF_C128 ? S.d64.p : S.d32.p);
        if (!b || (const char*)T.mat < b || (const char*)T.mat >= b + S.total * (int64_t)es) continue;
        const int64_t e = ((const char*)T.mat - b) / (int64_t)es;
        const int blk = (int)(std::upper_bound(S.off.begin(), S.off.end(), e) - S.off.begin()) - 1;
        if (blk < 0 || e + last >= S.off[blk] + (int64_t)S.rows[blk] * S.cols[blk])
          return bad(i, "reads past its factor block");
        break;
      }
    }
  }
  return BF_OK;
}

// Runs the cached stages on bases {xt, ping, pong, yt}.
int run_apply_stages(Fact* F, int opC, int dtype, int64_t nrhs, void* xt, void* ping, void* pong,
                     void* yt, cudaStream_t s) {
  ApplyPlan& ap = F->ap[opC][dtype];
  StageBases bases{{xt, ping, pong, yt}};
  for (size_t i = 0; i < ap.first.size(); ++i) {
    const StageTask* d = (const StageTask*)ap.tasks.p + ap.first[i];
    // complex64 stages after the first overlap their start with the previous
    // stage (PDL); measured: -8..13% per apply for complex64, but slower for
    // complex128 with few columns (its longer stages run several waves and
    // the early-resident dependent CTAs take their slots)
    BF_TRY(launch_stage(d, ap.count[i], ap.maxM[i], (int)nrhs, (int)nrhs, bases, dtype, s, ap.variant_of(i, nrhs),
                        i > 0 && dtype == BF_C64));
  }
  return BF_OK;
}

// The engine for the stages of one apply on tree-order buffers: 0 the stage
// launches, 1 the persistent launch, 2 the grouped launches.  Forced by
// bf_set_apply_engine (3, 4), else the tuner's measurement for the
// right-hand-side class, else (untuned) the grouped engine, which is faster
// than the stage launches for every column count measured on the 2-D line
// pair and from 16 columns on for the 3-D caps (at default_grouped_depth)
// -- from the GR_BUILD_AFTER-th untuned apply
// of (F, op, dtype) on: its plan costs more host time to build than a few
// applies save, so a factorization applied once or twice keeps the stage
// launches.  Builds what it picks; falls back to the stage launches where
// an engine does not apply.  overlap: x and y share memory (the persistent
// engine's stages overlap in time, and a grouped apply of one run reads x
// and writes y in the same launch).
// Untuned run depth of the grouped engine from the factorization's largest
// block rank: small blocks (the 2-D line pair, ranks ~10) gain most from
// keeping three stages in shared memory; with ranks ~55 (3-D caps) a group
// of two or three stages no longer fits in shared memory with wide column
// slices, and one stage per launch (staged tiles, one warp per row chunk)
// is fastest (measured 1.4-2x faster than the stage launches there, two to
// three stages 1.1-3x slower).
static int default_grouped_depth(const Fact* F, int dtype) {
  int rmax = 0;
  for (const auto& v : F->rV)
    for (int r : v) rmax = std::max(rmax, r);
  for (const auto& v : F->rU)
    for (int r : v) rmax = std::max(rmax, r);
  if (rmax <= 16) return dtype == BF_C128 ? 2 : 3;
  return rmax <= 32 ? 2 : 1;
}

int pick_inner_engine(Fact* F, int opC, int dtype, int64_t nrhs, bool overlap, cudaStream_t s, int* out) {
  *out = 0;
  const int cls = nrhs_class(nrhs), eng = apply_engine();
  if (eng == 1 || eng == 2) return BF_OK;
  GroupedPlan& gp = F->gp[opC][dtype];
  const int depth = grouped_depth() > 0   ? grouped_depth()
                    : gp.tuned_depth > 0 ? gp.tuned_depth
                                         : default_grouped_depth(F, dtype);
  if (!overlap && (eng == 3 || (eng == 0 && gp.ppick[cls]))) {
    BF_TRY(build_grouped(F, opC, dtype, depth, s));
    if (gp.ok) {
      *out = 1;
      return BF_OK;
    }
  }
  bool want = eng == 4 || (eng == 0 && gp.pick[cls]);
  if (eng == 0 && !gp.tuned[cls]) want = ++gp.untuned_uses >= GR_BUILD_AFTER;
  if (want) {
    BF_TRY(build_grouped(F, opC, dtype, depth, s));
    if (gp.ok && !(overlap && gp.runs.size() < 2)) *out = 2;
  }
  return BF_OK;
}

int prepare_apply(Fact* F, int opC, int dtype, cudaStream_t s) {
  if (dtype == BF_C64) BF_TRY(F->ensure32(s));
  if (!F->ap[opC][dtype].built) BF_TRY(build_apply(F, opC, dtype, s));
  return BF_OK;
}

int apply_fact(Fact* F, int op, int64_t nrhs, const void* x, int64_t ldx, void* y, int64_t ldy,
               int dtype, cudaStream_t s, bool tree_order) {
  if (nrhs <= 0) return BF_OK;
  if (dtype != BF_C64 && dtype != BF_C128) return fail(BF_EINVAL, "dtype must be BF_C64 or BF_C128");
  if (op != BF_OP_N && op != BF_OP_T && op != BF_OP_C) return fail(BF_EINVAL, "bad op");
  const int opC = op == BF_OP_N ? 0 : 1;
  // the stage launches' device task lists are built below only when they run
  if (dtype == BF_C64) BF_TRY(F->ensure32(s));
  const Plan* P = F->plan;
  const int64_t in_rows = opC ? P->m : P->n, out_rows = opC ? P->n : P->m;
  if (ldx < in_rows || ldy < out_rows) return fail(BF_EINVAL, "leading dimension too small");
  const int64_t* perm_in = (const int64_t*)(opC ? P->d_permT.p : P->d_permS.p);
  const int64_t* perm_out = (const int64_t*)(opC ? P->d_permS.p : P->d_permT.p);
  const bool id_in = tree_order || (opC ? P->identT : P->identS);
  const bool id_out = tree_order || (opC ? P->identS : P->identT);
  const int conj = op == BF_OP_T ? 1 : 0;
  const size_t es = elem_bytes(dtype);
  // the fused apply (two launches): always where it applies (engine 2), or
  // where the tuner measured it faster than the stage launches for this
  // right-hand-side class (engine 0)
  if (!tree_order && apply_engine() == 2) BF_TRY(build_fused(F, opC, dtype, s));
  if (!tree_order && F->fp[opC][dtype].ok &&
      (apply_engine() == 2 || (apply_engine() == 0 && F->fp[opC][dtype].engine[nrhs_class(nrhs)] == 0))) {
    const FusedPlan& fp = F->fp[opC][dtype];
    {
      DevBuf ex;
      BF_TRY(ex.alloc(&F->mem, (size_t)fp.ex_rows * nrhs * es, s));
      const int rc = run_fused(F, opC, dtype, nrhs, x, ldx, y, ldy, conj, ex.p, s);
      ex.release(s);
      return rc;
    }
  }
  const bool direct_in = id_in && !conj && ldx == in_rows;
  const bool direct_out = id_out && !conj && ldy == out_rows;
  // the engine of the stages (pick_inner_engine); x and y overlapping rule
  // out the engines whose stages overlap in time
  bool overlap = false;
  if (direct_in && direct_out) {
    const char *xa = (const char*)x, *ya = (const char*)y;
    const char* xb = xa + (size_t)(ldx * (nrhs - 1) + in_rows) * es;
    const char* yb = ya + (size_t)(ldy * (nrhs - 1) + out_rows) * es;
    overlap = !(xb <= ya || yb <= xa);
  }
  int engine = 0;
  BF_TRY(pick_inner_engine(F, opC, dtype, nrhs, overlap, s, &engine));
  const bool flow = engine == 1, grouped = engine == 2;
  NvtxRange nv(flow ? "bf_apply: persistent launch, columns: %d" : grouped ? "bf_apply: grouped launches, columns: %d"
                                                                          : "bf_apply: stage launches, columns: %d",
               (int)std::min<int64_t>(nrhs, INT32_MAX));
  if (!flow && !grouped) BF_TRY(prepare_apply(F, opC, dtype, s));
  GroupedPlan& gp = F->gp[opC][dtype];
  const int64_t lvl = (grouped ? gp.level_rows_max : F->ap[opC][dtype].level_rows_max) * nrhs;
  const size_t inner = flow ? grouped_persist_scratch_bytes(gp, nrhs, dtype) : (size_t)(2 * lvl) * es;
  const size_t bytes = inner + ((direct_in ? 0 : in_rows * nrhs) + (direct_out ? 0 : out_rows * nrhs)) * es;
  DevBuf scratch;
  BF_TRY(scratch.alloc(&F->mem, bytes, s));
  char* p = (char*)scratch.p;
  void* ping = p;
  void* pong = p + lvl * es;
  char* q = p + inner;
  void* xt = direct_in ? const_cast<void*>(x) : (void*)q;
  if (!direct_in) q += in_rows * nrhs * es;
  void* yt = direct_out ? y : (void*)q;
  int rc = BF_OK;
  if (!direct_in)
    rc = launch_gather_rows(id_in ? nullptr : perm_in, in_rows, nrhs, x, ldx, xt, in_rows, conj, dtype, s);
  if (rc == BF_OK)
    rc = flow      ? run_grouped_persist(F, opC, dtype, nrhs, xt, yt, p, s)
         : grouped ? run_grouped(F, opC, dtype, nrhs, xt, yt, ping, pong, s)
                   : run_apply_stages(F, opC, dtype, nrhs, xt, ping, pong, yt, s);
  if (rc == BF_OK && !direct_out)
    rc = launch_scatter_rows(id_out ? nullptr : perm_out, out_rows, nrhs, yt, out_rows, y, ldy, conj, dtype, s);
  scratch.release(s);
  return rc;
}

// Apply tuner: each stage of the cached task lists, each stage-kernel
// variant, a warm-up launch and three timed launches on scratch operands
// (the variants compute identical sums, so timing on any data is timing on
// all data); the fastest variant per stage is kept for this right-hand-side
// class.  Synchronises the stream.
int tune_apply(Fact* F, int op, int dtype, int64_t nrhs, cudaStream_t s, float* ms) {
  NvtxRange nv("bf_apply_tune, columns: %d", (int)std::min<int64_t>(nrhs, INT32_MAX));
  if (nrhs <= 0) return fail(BF_EINVAL, "nrhs must be positive");
  if (dtype != BF_C64 && dtype != BF_C128) return fail(BF_EINVAL, "dtype must be BF_C64 or BF_C128");
  if (op != BF_OP_N && op != BF_OP_T && op != BF_OP_C) return fail(BF_EINVAL, "bad op");
  const int opC = op == BF_OP_N ? 0 : 1;
  BF_TRY(prepare_apply(F, opC, dtype, s));
  ApplyPlan& ap = F->ap[opC][dtype];
  const Plan* P = F->plan;
  const size_t es = elem_bytes(dtype);
  const int64_t rows = std::max(P->n, P->m), lvl = ap.level_rows_max * nrhs;
  DevBuf scratch;
  BF_TRY(scratch.alloc(&F->mem, (2 * lvl + 2 * rows * nrhs) * es, s));
  char* p = (char*)scratch.p;
  BF_CUDA_TRY(cudaMemsetAsync(p, 0, (2 * lvl + 2 * rows * nrhs) * es, s));
  StageBases bases{{p + 2 * lvl * es, p, p + lvl * es, p + 2 * lvl * es + rows * nrhs * es}};
  cudaEvent_t e[2];
  BF_CUDA_TRY(cudaEventCreate(&e[0]));
  BF_CUDA_TRY(cudaEventCreate(&e[1]));
  int rc = BF_OK;
  float total = 0.f;
  const int cls = nrhs_class(nrhs);
  for (size_t i = 0; i < ap.first.size() && !rc; ++i) {
    const StageTask* d = (const StageTask*)ap.tasks.p + ap.first[i];
    float best = 1e30f;
    int bv = stage_variant_default((int)nrhs, dtype);
    for (int v = 0; v < STAGE_VARIANTS && !rc; ++v) {
      rc = launch_stage(d, ap.count[i], ap.maxM[i], (int)nrhs, (int)nrhs, bases, dtype, s, v);
      if (!rc && cudaEventRecord(e[0], s) != cudaSuccess) rc = fail(BF_ECUDA, "event record failed");
      for (int r = 0; r < 3 && !rc; ++r) rc = launch_stage(d, ap.count[i], ap.maxM[i], (int)nrhs, (int)nrhs, bases, dtype, s, v);
      if (!rc) note_sync();
      if (!rc && (cudaEventRecord(e[1], s) != cudaSuccess || cudaEventSynchronize(e[1]) != cudaSuccess))
        rc = fail(BF_ECUDA, "event timing failed");
      float t = 0.f;
      if (!rc && cudaEventElapsedTime(&t, e[0], e[1]) != cudaSuccess) rc = fail(BF_ECUDA, "event timing failed");
      if (!rc && t < best) best = t, bv = v;
    }
    if (!rc) {
      ap.variant[i][cls] = (int8_t)bv;
      total += best / 3.f;
    }
  }
  // the fused apply: every column-slice width that fits, on the same
  // scratch operands (x = the input rows, y = the output rows of the
  // scratch, exchange = the two level buffers); keep the fastest width and
  // the faster of the two engines for this class
  float fused_best = 1e30f;
  if (!rc && apply_engine() != 1) rc = build_fused(F, opC, dtype, s);
  FusedPlan& fp = F->fp[opC][dtype];
  if (!rc && apply_engine() != 1 && fp.ok && 2 * lvl >= fp.ex_rows * nrhs) {
    int best_cs = 0;
    const int conj = op == BF_OP_T ? 1 : 0;
    char* xs = p + 2 * lvl * es;
    char* ys = xs + rows * nrhs * es;
    const int64_t in_rows = opC ? P->m : P->n, out_rows = opC ? P->n : P->m;
    for (int cs = 1; cs <= 32 && !rc; cs *= 2) {
      if (cs > 1 && cs / 2 >= nrhs) break;
      rc = run_fused(F, opC, dtype, nrhs, xs, in_rows, ys, out_rows, conj, p, s, cs);
      if (rc) {   // a width whose shared memory does not fit is skipped
        rc = BF_OK;
        set_error("");
        continue;
      }
      if (cudaEventRecord(e[0], s) != cudaSuccess) rc = fail(BF_ECUDA, "event record failed");
      for (int r = 0; r < 3 && !rc; ++r) rc = run_fused(F, opC, dtype, nrhs, xs, in_rows, ys, out_rows, conj, p, s, cs);
      if (!rc) note_sync();
      if (!rc && (cudaEventRecord(e[1], s) != cudaSuccess || cudaEventSynchronize(e[1]) != cudaSuccess))
        rc = fail(BF_ECUDA, "event timing failed");
      float t = 0.f;
      if (!rc && cudaEventElapsedTime(&t, e[0], e[1]) != cudaSuccess) rc = fail(BF_ECUDA, "event timing failed");
      if (!rc && t / 3.f < fused_best) fused_best = t / 3.f, best_cs = cs;
    }
    if (!rc && best_cs > 0) fp.cs[cls] = best_cs;
  }
  // the grouped apply at each run depth (1-4), group merging (complex64:
  // merged up to GR_MERGE_MIN last-stage blocks, or not) and slice width, as
  // launches per run (own level buffers) and as one persistent launch (own
  // scratch); the plan keeps the fastest depth and merging
  float grouped_best = 1e30f, persist_best = 1e30f;
  GroupedPlan& gp = F->gp[opC][dtype];
  if (!rc && (apply_engine() == 0 || apply_engine() == 3 || apply_engine() == 4)) {
    // tags: depth * 8 + merge
    int best_tag = 0, best_cw = 0, pbest_tag = 0, pbest_cw = 0;
    auto time3 = [&](auto&& run_once, float* best, int tag, int cw, int* bt, int* bc) {
      rc = run_once();
      if (!rc && cudaEventRecord(e[0], s) != cudaSuccess) rc = fail(BF_ECUDA, "event record failed");
      for (int r = 0; r < 3 && !rc; ++r) rc = run_once();
      if (!rc) note_sync();
      if (!rc && (cudaEventRecord(e[1], s) != cudaSuccess || cudaEventSynchronize(e[1]) != cudaSuccess))
        rc = fail(BF_ECUDA, "event timing failed");
      float t = 0.f;
      if (!rc && cudaEventElapsedTime(&t, e[0], e[1]) != cudaSuccess) rc = fail(BF_ECUDA, "event timing failed");
      if (!rc && t / 3.f < *best) *best = t / 3.f, *bt = tag, *bc = cw;
    };
    char* xs = p + 2 * lvl * es;
    char* ys = xs + rows * nrhs * es;
    const int merges[2] = {dtype == BF_C64 ? GR_MERGE_MIN : 1, 1};
    for (int v = 0; v < 2 * GR_MAXD && !rc; ++v) {
      const int depth = 1 + v / 2, merge = merges[v % 2];
      if (v % 2 == 1 && merge == merges[0]) continue;   // complex128: no merged variant
      rc = build_grouped(F, opC, dtype, depth, s, merge);
      if (rc) break;
      if (!gp.ok) continue;
      const int tag = depth * 8 + merge;
      DevBuf lb;
      rc = lb.alloc(&F->mem, (size_t)2 * gp.level_rows_max * nrhs * es, s);
      char* lp = (char*)lb.p;
      char* lq = lp + gp.level_rows_max * nrhs * es;
      DevBuf ps;
      if (!rc) rc = ps.alloc(&F->mem, grouped_persist_scratch_bytes(gp, nrhs, dtype), s);
      for (int cw = 16; cw <= 64 && !rc; cw *= 2) {
        if (cw > 16 && cw / 2 >= nrhs) break;   // wider slices than the columns change nothing
        time3([&] { return run_grouped(F, opC, dtype, nrhs, xs, ys, lp, lq, s, cw); }, &grouped_best, tag, cw,
              &best_tag, &best_cw);
        if (!rc)
          time3([&] { return run_grouped_persist(F, opC, dtype, nrhs, xs, ys, ps.p, s, cw); }, &persist_best, tag,
                cw, &pbest_tag, &pbest_cw);
      }
      if (!rc) rc = tc_status(true);   // a persistent wait that gave up (never expected)
      ps.release(s);
      lb.release(s);
    }
    const bool pw = persist_best < grouped_best;
    const int bt = pw ? pbest_tag : best_tag, bc = pw ? pbest_cw : best_cw;
    if (!rc && bt > 0) {
      rc = build_grouped(F, opC, dtype, bt / 8, s, bt % 8);
      gp.cw[cls] = (int16_t)bc;
      gp.tuned_depth = bt / 8;
      gp.tuned_merge = bt % 8;
    }
  }
  // the fastest engine serves this class from now on
  if (!rc) {
    const float best = std::min(std::min(total, fused_best), std::min(persist_best, grouped_best));
    gp.ppick[cls] = persist_best == best && best < total ? 1 : 0;
    gp.pick[cls] = !gp.ppick[cls] && grouped_best == best && best < total ? 1 : 0;
    gp.tuned[cls] = 1;
    if (fused_best < 1e30f) fp.engine[cls] = !gp.ppick[cls] && !gp.pick[cls] && fused_best <= total ? 0 : 1;
  }
  cudaEventDestroy(e[0]);
  cudaEventDestroy(e[1]);
  scratch.release(s);
  if (ms) *ms = std::min(std::min(total, fused_best), std::min(persist_best, grouped_best));
  return rc;
}

// ------------------------------------------------------- graph applier --
// The stage chain of an apply (eq. hybrid_butterfly_mat) never touches user
// memory when it runs on internal input/output buffers, so it is captured
// once into a CUDA graph; a run is then a gather of x into the internal input
// (user order -> tree order, conjugation for F^T), one graph launch, and a
// scatter of the internal output into y.
int applier_create(Fact* F, int op, int64_t nrhs, int dtype, Applier** out) {
  *out = nullptr;
  if (nrhs <= 0) return fail(BF_EINVAL, "nrhs must be positive");
  if (dtype != BF_C64 && dtype != BF_C128) return fail(BF_EINVAL, "dtype must be BF_C64 or BF_C128");
  if (op != BF_OP_N && op != BF_OP_T && op != BF_OP_C) return fail(BF_EINVAL, "bad op");
  Applier* A = new Applier();
  A->F = F;
  A->op = op;
  A->opC = op == BF_OP_N ? 0 : 1;
  A->dtype = dtype;
  A->nrhs = nrhs;
  const Plan* P = F->plan;
  A->in_rows = A->opC ? P->m : P->n;
  A->out_rows = A->opC ? P->n : P->m;
  cudaStream_t cs = nullptr;
  int rc = BF_OK;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) rc = fail(BF_ECUDA, "stream create failed");
  if (!rc) rc = prepare_apply(F, A->opC, dtype, cs);
  const size_t es = elem_bytes(dtype);
  // the engine bf_apply would use for this column count (internal x and y
  // never overlap)
  int inner = 0;
  if (!rc) rc = pick_inner_engine(F, A->opC, dtype, nrhs, false, cs, &inner);
  const int64_t lvl = rc ? 0
                         : (inner == 2 ? F->gp[A->opC][dtype].level_rows_max
                                       : F->ap[A->opC][dtype].level_rows_max) * nrhs;
  const size_t inner_bytes =
      inner == 1 ? grouped_persist_scratch_bytes(F->gp[A->opC][dtype], nrhs, dtype) : (size_t)(2 * lvl) * es;
  if (!rc) rc = A->scratch.alloc(&F->mem, (size_t)(A->in_rows * nrhs + A->out_rows * nrhs) * es + inner_bytes, nullptr);
  if (!rc) {
    char* p = (char*)A->scratch.p;
    A->xt = p;
    A->yt = p + A->in_rows * nrhs * es;
    char* ping = p + (A->in_rows + A->out_rows) * nrhs * es;
    char* pong = ping + lvl * es;
    // the persistent launch's arguments name the applier's own buffers:
    // uploaded once, before the capture
    if (inner == 1) rc = run_grouped_persist(F, A->opC, dtype, nrhs, A->xt, A->yt, ping, cs, 0, 1);
    if (!rc && (host_sync(cs) != cudaSuccess ||
                cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess)) {
      rc = fail(BF_ECUDA, "graph capture could not start");
    } else if (!rc) {
      rc = inner == 1   ? run_grouped_persist(F, A->opC, dtype, nrhs, A->xt, A->yt, ping, cs, 0, 2)
           : inner == 2 ? run_grouped(F, A->opC, dtype, nrhs, A->xt, A->yt, ping, pong, cs)
                        : run_apply_stages(F, A->opC, dtype, nrhs, A->xt, ping, pong, A->yt, cs);
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(cs, &g);
      if (!rc && e != cudaSuccess) rc = fail(BF_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      A->graph = g;
      if (!rc && cudaGraphInstantiate(&A->exec, g, 0) != cudaSuccess) rc = fail(BF_ECUDA, "graph instantiate failed");
    }
  }
  if (!rc && cudaEventCreateWithFlags(&A->done, cudaEventDisableTiming) != cudaSuccess)
    rc = fail(BF_ECUDA, "event create failed");
  if (cs) cudaStreamDestroy(cs);
  if (rc) {
    applier_destroy(A);
    return rc;
  }
  *out = A;
  return BF_OK;
}

int applier_run(Applier* A, const void* x, int64_t ldx, void* y, int64_t ldy, cudaStream_t s) {
  if (ldx < A->in_rows || ldy < A->out_rows) return fail(BF_EINVAL, "leading dimension too small");
  const Plan* P = A->F->plan;
  const int64_t* perm_in = (const int64_t*)(A->opC ? P->d_permT.p : P->d_permS.p);
  const int64_t* perm_out = (const int64_t*)(A->opC ? P->d_permS.p : P->d_permT.p);
  const bool id_in = A->opC ? P->identT : P->identS, id_out = A->opC ? P->identS : P->identT;
  const int conj = A->op == BF_OP_T ? 1 : 0;
  if (A->ran) BF_CUDA_TRY(cudaStreamWaitEvent(s, A->done, 0));
  BF_TRY(launch_gather_rows(id_in ? nullptr : perm_in, A->in_rows, A->nrhs, x, ldx, A->xt, A->in_rows, conj, A->dtype,
                            s));
  BF_CUDA_TRY(cudaGraphLaunch(A->exec, s));
  BF_TRY(launch_scatter_rows(id_out ? nullptr : perm_out, A->out_rows, A->nrhs, A->yt, A->out_rows, y, ldy, conj,
                             A->dtype, s));
  BF_CUDA_TRY(cudaEventRecord(A->done, s));
  A->ran = true;
  return BF_OK;
}

void applier_destroy(Applier* A) {
  if (!A) return;
  note_sync();
  cudaDeviceSynchronize();
  if (A->exec) cudaGraphExecDestroy(A->exec);
  if (A->graph) cudaGraphDestroy(A->graph);
  if (A->done) cudaEventDestroy(A->done);
  A->scratch.release(nullptr);
  delete A;
}

}  // namespace bf
