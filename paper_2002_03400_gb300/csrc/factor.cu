// Alg. 2 -- adaptive randomized hybrid butterfly factorization -- as a host
// scheduler over the device kernels.  Per level: draw the compact random
// matrix (counter-based generator), one black-box product for all blocks of
// the level (structured sketch, Sec. 4.1), peel the recovered factors along
// the ancestor paths (one stage launch per tree level), batched truncated
// pivoted QR (Alg. 1 step 3) and, at l_m, X = V^H Omega and the B least
// squares (eq. Bij).  Ranks return to the host once per level to size the
// next sketch (its width is max(r1 + r2) + p over the level's blocks).
//
// Readings (shared with the oracle): r restarts at r0 for each leaf loop;
// each leaf pass appends r new random columns; a leaf loop also stops once
// r + p reaches the largest leaf; one sketch width per level; at l_m the
// width also covers max r^V + p; B = (U^H K Omega)(V^H Omega)^+.
#include <algorithm>
#include <chrono>

#include "bf_internal.h"

namespace bf {

namespace {

enum { STAGE_V0 = 1, STAGE_U0 = 2, STAGE_W = 3, STAGE_R = 4 };
inline uint32_t sid(int stage, int level) { return (uint32_t)((stage << 8) | level); }

struct Ctx {
  Plan* P;
  Operator* A;
  Fact* F;
  cudaStream_t s;
  int dt;
  size_t es;
};

// RAII scratch (stream-ordered)
struct Scratch {
  DevBuf b;
  cudaStream_t s;
  explicit Scratch(cudaStream_t st) : s(st) {}
  ~Scratch() { b.release(s); }
  int alloc(MemTracker* mt, size_t bytes) { return b.alloc(mt, bytes, s); }
  char* p() const { return (char*)b.p; }
};

int upload_tasks(Ctx& c, const std::vector<StageTask>& tasks, Scratch& buf) {
  BF_TRY(buf.alloc(&c.F->mem, std::max<size_t>(1, tasks.size()) * sizeof(StageTask)));
  BF_CUDA_TRY(cudaMemcpyAsync(buf.p(), tasks.data(), tasks.size() * sizeof(StageTask),
                              cudaMemcpyHostToDevice, c.s));
  return BF_OK;
}

int run_tasks(Ctx& c, const std::vector<StageTask>& tasks, const StageBases& bases) {
  if (tasks.empty()) return BF_OK;
  Scratch d(c.s);
  BF_TRY(upload_tasks(c, tasks, d));
  int mM = 0, mN = 0;
  for (const auto& t : tasks) mM = std::max(mM, t.M), mN = std::max(mN, t.N);
  return launch_stage((const StageTask*)d.p(), (int)tasks.size(), mM, mN, 0, bases, c.dt, c.s);
}

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

// factor block in the sketch dtype
const void* fblk(Ctx& c, int stage, int b, int row = 0) {
  const Stage& S = c.F->st[stage];
  const char* base = (const char*)(c.dt == BF_C128 ? S.d64.p : S.d32.p);
  return base + (S.off[b] + row) * (int64_t)c.es;
}

// Sketch of Sec. 4.1: Y = op(A) Omega-bar with Omega-bar the block-diagonal
// expansion over the nodes at `level` of the input-side tree of the compact
// random matrix Om (input rows x k).  Tree order in and out.
int sketch(Ctx& c, int op, int level, int64_t k, const void* Om, void* Y) {
  Plan* P = c.P;
  Operator* A = c.A;
  const bool opN = op == BF_OP_N;
  const int groups = 1 << level;
  const int64_t in_rows = opN ? P->n : P->m, out_rows = opN ? P->m : P->n;
  const int64_t* d_off = opN ? P->offS_dev(level) : P->offT_dev(level);
  const int64_t ncols = groups * k;
  if (A->plan == P && A->has_structured())
    return A->apply_structured(op, groups, d_off, k, Om, in_rows, Y, out_rows, c.dt, c.s);
  Scratch ex(c.s);
  BF_TRY(ex.alloc(&c.F->mem, in_rows * ncols * c.es));
  BF_TRY(launch_expand_structured(groups, d_off, in_rows, k, Om, in_rows, ex.p(), in_rows, c.dt, c.s));
  if (A->plan == P) return A->apply_tree(op, ncols, ex.p(), in_rows, Y, out_rows, c.dt, c.s);
  // user-order black box
  Scratch u(c.s);
  BF_TRY(u.alloc(&c.F->mem, (in_rows + out_rows) * ncols * c.es));
  char* ui = u.p();
  char* uo = u.p() + in_rows * ncols * c.es;
  const int64_t* pin = (const int64_t*)(opN ? P->d_permS.p : P->d_permT.p);
  const int64_t* pout = (const int64_t*)(opN ? P->d_permT.p : P->d_permS.p);
  BF_TRY(launch_scatter_rows(pin, in_rows, ncols, ex.p(), in_rows, ui, in_rows, 0, c.dt, c.s));
  BF_TRY(A->apply(op, ncols, ui, in_rows, uo, out_rows, c.dt, c.s));
  return launch_gather_rows(pout, out_rows, ncols, uo, out_rows, Y, out_rows, 0, c.dt, c.s);
}

// Lays out a stage: rows[b] x cap[b] blocks, allocates complex128 storage.
int layout_stage(Ctx& c, Stage& S, const std::vector<int32_t>& rows, const std::vector<int32_t>& cap) {
  S.d64.release(nullptr);
  S.d32.release(nullptr);
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
  return S.d64.alloc(&c.F->mem, std::max<int64_t>(tot, 1) * 16, nullptr);
}

int make32(Ctx& c, Stage& S) {
  if (c.dt != BF_C64) return BF_OK;
  BF_TRY(S.d32.alloc(&c.F->mem, std::max<int64_t>(S.total, 1) * 8, nullptr));
  BF_TRY(launch_convert(S.d64.p, S.d32.p, S.total, BF_C128, BF_C64, c.s));
  S.have32 = true;
  return BF_OK;
}

// Batched truncated QR of blocks in[b] (rows[b] x k, ld ldin[b]) into stage S.
int qr_into(Ctx& c, Stage& S, const std::vector<const void*>& in, const std::vector<int64_t>& ldin,
            int k, std::vector<int32_t>& ranks) {
  const int nb = (int)S.rows.size();
  std::vector<QRTask> tasks(nb);
  int maxS = 1;
  for (int b = 0; b < nb; ++b) {
    QRTask& t = tasks[b];
    t.in = in[b];
    t.ldi = ldin[b];
    t.s = S.rows[b];
    t.k = k;
    t.cap = std::min(S.rows[b], k);
    t.q = (char*)S.d64.p + S.off[b] * 16;
    maxS = std::max(maxS, S.rows[b]);
  }
  const size_t wbytes = qr_workspace_bytes(nb, maxS, k);
  Scratch d(c.s), w(c.s);
  BF_TRY(d.alloc(&c.F->mem, nb * sizeof(QRTask) + nb * sizeof(int32_t)));
  BF_CUDA_TRY(cudaMemcpyAsync(d.p(), tasks.data(), nb * sizeof(QRTask), cudaMemcpyHostToDevice, c.s));
  int32_t* d_r = (int32_t*)(d.p() + nb * sizeof(QRTask));
  if (wbytes) BF_TRY(w.alloc(&c.F->mem, wbytes));
  BF_TRY(launch_qr((const QRTask*)d.p(), nb, maxS, k, c.P->tol, c.dt, d_r, w.p(), wbytes, c.s));
  ranks.assign(nb, 0);
  BF_CUDA_TRY(cudaMemcpyAsync(ranks.data(), d_r, nb * sizeof(int32_t), cudaMemcpyDeviceToHost, c.s));
  BF_CUDA_TRY(cudaStreamSynchronize(c.s));
  S.cols = ranks;
  return make32(c, S);
}

// Adaptive leaf loop (Alg. 2 loops "V" and "U").  Vside: Y = A^H Gamma_t,
// leaves of T_S; else Z = A Omega_s, leaves of T_T.
int leaf_loop(Ctx& c, bool Vside) {
  Plan* P = c.P;
  Fact* F = c.F;
  const int L = P->L, nb = 1 << L;
  const int op = Vside ? BF_OP_C : BF_OP_N;
  const int64_t in_rows = Vside ? P->m : P->n, out_rows = Vside ? P->n : P->m;
  const auto& off = Vside ? P->offS[L] : P->offT[L];
  Stage& S = F->st[Vside ? F->stage_V0() : F->stage_U()];
  const uint32_t id = sid(Vside ? STAGE_V0 : STAGE_U0, 0);
  int maxleaf = 0;
  std::vector<int32_t> rows(nb);
  for (int b = 0; b < nb; ++b) rows[b] = (int32_t)(off[b + 1] - off[b]), maxleaf = std::max(maxleaf, rows[b]);
  int r = P->opt.r0;
  int64_t kcap = 0;
  DevBuf Y;
  int rc = BF_OK;
  std::vector<int32_t> ranks;
  int k = 0;
  for (;;) {
    k = r + P->opt.p;
    if (k > kcap) {
      DevBuf Yn;
      rc = Yn.alloc(&F->mem, out_rows * k * c.es, c.s);
      if (rc) break;
      if (kcap > 0) {
        cudaError_t e = cudaMemcpyAsync(Yn.p, Y.p, out_rows * kcap * c.es, cudaMemcpyDeviceToDevice, c.s);
        if (e != cudaSuccess) {
          Yn.release(c.s);
          rc = fail(BF_ECUDA, cudaGetErrorString(e));
          break;
        }
      }
      {
        Scratch G(c.s);
        rc = G.alloc(&F->mem, in_rows * (k - kcap) * c.es);
        if (!rc) rc = launch_gaussian(P->opt.seed, id, 0, in_rows, kcap, k, G.p(), in_rows, c.dt, c.s);
        if (!rc) rc = sketch(c, op, 0, k - kcap, G.p(), (char*)Yn.p + out_rows * kcap * c.es);
      }
      Y.release(c.s);
      Y = Yn;
      kcap = k;
      if (rc) break;
    }
    std::vector<int32_t> cap(nb);
    for (int b = 0; b < nb; ++b) cap[b] = std::min(rows[b], k);
    rc = layout_stage(c, S, rows, cap);
    if (rc) break;
    std::vector<const void*> in(nb);
    std::vector<int64_t> ld(nb, out_rows);
    for (int b = 0; b < nb; ++b) in[b] = (const char*)Y.p + off[b] * c.es;
    rc = qr_into(c, S, in, ld, k, ranks);
    if (rc) break;
    const int maxr = *std::max_element(ranks.begin(), ranks.end());
    if (r > maxr || k >= maxleaf) break;
    r *= 2;
    if (r > P->opt.r_max) {
      rc = fail(BF_ENOTCONVERGED, "adaptive leaf rank exceeds r_max");
      break;
    }
  }
  Y.release(c.s);
  if (rc) return rc;
  if (Vside)
    F->rV[0] = ranks;
  else
    F->rU[L - F->lm] = ranks;
  return BF_OK;
}

// Peels V_{p tau, nu'}^H off the W-side sketch Y (n x 2^l k) into the QR
// inputs P_{tau,nu} = [V_{p tau,2nu}^H Y_tau(S_2nu); V_{p tau,2nu+1}^H Y_tau(S_2nu+1)].
int peel_V(Ctx& c, int l, int k, const void* Y, char* Pbuf, const std::vector<int64_t>& Poff,
           const std::vector<int32_t>& Ps) {
  Plan* P = c.P;
  Fact* F = c.F;
  const int L = P->L, nb = 1 << L, nn = 1 << (L - l);
  const auto& offS = P->offS[L];
  Scratch bufA(c.s), bufB(c.s);
  std::vector<int64_t> xoff_prev, xoff(nb + 1);
  int cur = -1;
  size_t maxbytes = 0;
  for (int j = 0; j < l - 1; ++j) {
    int64_t tot = 0;
    for (int b = 0; b < nb; ++b) tot += (int64_t)F->rV[j][b] * ((int64_t)k << (l - j));
    maxbytes = std::max(maxbytes, (size_t)tot * c.es);
  }
  if (maxbytes) {
    BF_TRY(bufA.alloc(&F->mem, maxbytes));
    BF_TRY(bufB.alloc(&F->mem, maxbytes));
  }
  for (int j = 0; j < l; ++j) {
    const int64_t ncols = (int64_t)k << (l - j);
    const bool fin = (j == l - 1);
    const int outb = fin ? 3 : (cur == 1 ? 2 : 1);
    const int nmu = 1 << (L - j);
    xoff[0] = 0;
    for (int b = 0; b < nb; ++b) xoff[b + 1] = xoff[b] + (int64_t)F->rV[j][b] * ncols;
    std::vector<StageTask> tasks;
    for (int sg = 0; sg < (1 << j); ++sg)
      for (int mu = 0; mu < nmu; ++mu) {
        const int b = sg * nmu + mu;
        const int M = F->rV[j][b];
        auto add_terms = [&](StageTask& t, int64_t colo) {
          if (j == 0) {
            const int sz = (int)(offS[mu + 1] - offS[mu]);
            term(t, 0, offS[mu] + colo * P->n, P->n, fblk(c, F->stage_V0(), mu), sz, sz, 1);
          } else {
            const int p0 = (sg >> 1) * (2 * nmu) + 2 * mu, p1 = p0 + 1;
            const int k0 = F->rV[j - 1][p0], k1 = F->rV[j - 1][p1];
            const int ldm = F->st[F->stage_W(j)].rows[b];
            const int64_t c0 = (sg & 1) * ncols + colo;
            // level j-1 blocks are row-major with 2*ncols columns
            term(t, cur, xoff_prev[p0] + c0, -2 * ncols, fblk(c, F->stage_W(j), b), ldm, k0, 1);
            term(t, cur, xoff_prev[p1] + c0, -2 * ncols, fblk(c, F->stage_W(j), b, k0), ldm, k1, 1);
          }
        };
        if (!fin) {
          StageTask t = task(outb, xoff[b], -ncols, M, (int)ncols);
          add_terms(t, 0);
          tasks.push_back(t);
        } else {
          const int nu = mu >> 1;
          const int rowoff = (mu & 1) ? F->rV[l - 1][sg * (2 * nn) + (mu & ~1)] : 0;
          for (int a = 0; a < 2; ++a) {
            const int bp = (2 * sg + a) * nn + nu;
            StageTask t = task(3, Poff[bp] + rowoff, Ps[bp], M, k);
            add_terms(t, (int64_t)a * k);
            tasks.push_back(t);
          }
        }
      }
    StageBases bases{{const_cast<void*>(Y), bufA.p(), bufB.p(), Pbuf}};
    BF_TRY(run_tasks(c, tasks, bases));
    xoff_prev = xoff;
    cur = outb;
  }
  return BF_OK;
}

// Peels U_{tau', p nu}^H off the R-side sketch Z (m x 2^(L-l) k) into
// P_{tau,nu} = [U_{2tau,p nu}^H Z_nu(T_2tau); U_{2tau+1,p nu}^H Z_nu(T_2tau+1)].
int peel_U(Ctx& c, int l, int k, const void* Z, char* Pbuf, const std::vector<int64_t>& Poff,
           const std::vector<int32_t>& Ps) {
  Plan* P = c.P;
  Fact* F = c.F;
  const int L = P->L, lm = F->lm, nb = 1 << L, nn = 1 << (L - l);
  const auto& offT = P->offT[L];
  auto ru = [&](int j, int b) { return F->rU[j - lm][b]; };
  Scratch bufA(c.s), bufB(c.s);
  std::vector<int64_t> yoff_prev, yoff(nb + 1);
  int cur = -1;
  size_t maxbytes = 0;
  for (int j = L; j > l + 1; --j) {
    int64_t tot = 0;
    for (int b = 0; b < nb; ++b) tot += (int64_t)ru(j, b) * ((int64_t)k << (j - l));
    maxbytes = std::max(maxbytes, (size_t)tot * c.es);
  }
  if (maxbytes) {
    BF_TRY(bufA.alloc(&F->mem, maxbytes));
    BF_TRY(bufB.alloc(&F->mem, maxbytes));
  }
  for (int j = L; j >= l + 1; --j) {
    const int64_t ncols = (int64_t)k << (j - l);
    const bool fin = (j == l + 1);
    const int outb = fin ? 3 : (cur == 1 ? 2 : 1);
    const int nmu = 1 << (L - j);
    yoff[0] = 0;
    for (int b = 0; b < nb; ++b) yoff[b + 1] = yoff[b] + (int64_t)ru(j, b) * ncols;
    std::vector<StageTask> tasks;
    for (int sg = 0; sg < (1 << j); ++sg)
      for (int mu = 0; mu < nmu; ++mu) {
        const int b = sg * nmu + mu;
        const int M = ru(j, b);
        auto add_terms = [&](StageTask& t, int64_t colo) {
          if (j == L) {
            const int sz = (int)(offT[sg + 1] - offT[sg]);
            term(t, 0, offT[sg] + colo * P->m, P->m, fblk(c, F->stage_U(), sg), sz, sz, 1);
          } else {
            const int nm1 = nmu >> 1;
            const int c0i = (2 * sg) * nm1 + (mu >> 1), c1i = (2 * sg + 1) * nm1 + (mu >> 1);
            const int k0 = ru(j + 1, c0i), k1 = ru(j + 1, c1i);
            const int ldm = F->st[F->stage_R(j)].rows[b];
            const int64_t cc = (mu & 1) * ncols + colo;
            // level j+1 blocks are row-major with 2*ncols columns
            term(t, cur, yoff_prev[c0i] + cc, -2 * ncols, fblk(c, F->stage_R(j), b), ldm, k0, 1);
            term(t, cur, yoff_prev[c1i] + cc, -2 * ncols, fblk(c, F->stage_R(j), b, k0), ldm, k1, 1);
          }
        };
        if (!fin) {
          StageTask t = task(outb, yoff[b], -ncols, M, (int)ncols);
          add_terms(t, 0);
          tasks.push_back(t);
        } else {
          const int tau = sg >> 1;
          const int rowoff = (sg & 1) ? ru(l + 1, (sg & ~1) * nmu + mu) : 0;
          for (int cc = 0; cc < 2; ++cc) {
            const int bp = tau * nn + 2 * mu + cc;
            StageTask t = task(3, Poff[bp] + rowoff, Ps[bp], M, k);
            add_terms(t, (int64_t)cc * k);
            tasks.push_back(t);
          }
        }
      }
    StageBases bases{{const_cast<void*>(Z), bufA.p(), bufB.p(), Pbuf}};
    BF_TRY(run_tasks(c, tasks, bases));
    yoff_prev = yoff;
    cur = outb;
  }
  return BF_OK;
}

// X_{tau,nu} = V_{tau,nu}^H Omega_nu at level l_m for every block, through
// V^0, W^1 .. W^(l_m) with the block-diagonal input (k columns per block).
int project_X(Ctx& c, int k, const void* Om, char* Xbuf, std::vector<int64_t>& xfin) {
  Plan* P = c.P;
  Fact* F = c.F;
  const int L = P->L, lm = F->lm, nb = 1 << L;
  const auto& offS = P->offS[L];
  Scratch bufA(c.s), bufB(c.s);
  size_t maxbytes = 0;
  for (int j = 0; j < lm; ++j) {
    int64_t tot = 0;
    for (int b = 0; b < nb; ++b) tot += (int64_t)F->rV[j][b] * k;
    maxbytes = std::max(maxbytes, (size_t)tot * c.es);
  }
  if (maxbytes) {
    BF_TRY(bufA.alloc(&F->mem, maxbytes));
    BF_TRY(bufB.alloc(&F->mem, maxbytes));
  }
  std::vector<int64_t> xprev, xo(nb + 1);
  int cur = -1;
  for (int j = 0; j <= lm; ++j) {
    const bool fin = j == lm;
    const int outb = fin ? 3 : (cur == 1 ? 2 : 1);
    const int nmu = 1 << (L - j);
    xo[0] = 0;
    for (int b = 0; b < nb; ++b) xo[b + 1] = xo[b] + (int64_t)F->rV[j][b] * k;
    std::vector<StageTask> tasks;
    for (int sg = 0; sg < (1 << j); ++sg)
      for (int mu = 0; mu < nmu; ++mu) {
        const int b = sg * nmu + mu;
        const int M = F->rV[j][b];
        // intermediates row-major; the final X blocks column-major (ld r^V) for the solve
        StageTask t = task(outb, xo[b], fin ? M : -k, M, k);
        if (j == 0) {
          const int sz = (int)(offS[mu + 1] - offS[mu]);
          term(t, 0, offS[mu], P->n, fblk(c, F->stage_V0(), mu), sz, sz, 1);
        } else {
          const int p0 = (sg >> 1) * (2 * nmu) + 2 * mu, p1 = p0 + 1;
          const int k0 = F->rV[j - 1][p0], k1 = F->rV[j - 1][p1];
          const int ldm = F->st[F->stage_W(j)].rows[b];
          term(t, cur, xprev[p0], -k, fblk(c, F->stage_W(j), b), ldm, k0, 1);
          term(t, cur, xprev[p1], -k, fblk(c, F->stage_W(j), b, k0), ldm, k1, 1);
        }
        tasks.push_back(t);
      }
    StageBases bases{{const_cast<void*>(Om), bufA.p(), bufB.p(), Xbuf}};
    BF_TRY(run_tasks(c, tasks, bases));
    xprev = xo;
    cur = outb;
  }
  xfin = xprev;
  return BF_OK;
}

int w_level(Ctx& c, int l) {
  Plan* P = c.P;
  Fact* F = c.F;
  const int L = P->L, nb = 1 << L, nt = 1 << l, nn = 1 << (L - l);
  const auto& prev = F->rV[l - 1];
  std::vector<int32_t> Ps(nb);
  int k = 0;
  for (int tau = 0; tau < nt; ++tau)
    for (int nu = 0; nu < nn; ++nu) {
      const int base = (tau >> 1) * (2 * nn);
      Ps[tau * nn + nu] = prev[base + 2 * nu] + prev[base + 2 * nu + 1];
      k = std::max(k, Ps[tau * nn + nu]);
    }
  k += P->opt.p;
  std::vector<int64_t> Poff(nb + 1, 0);
  for (int b = 0; b < nb; ++b) Poff[b + 1] = Poff[b] + (int64_t)Ps[b] * k;
  Scratch G(c.s), Y(c.s), Pb(c.s);
  BF_TRY(G.alloc(&F->mem, P->m * (int64_t)k * c.es));
  BF_TRY(launch_gaussian(P->opt.seed, sid(STAGE_W, l), 0, P->m, 0, k, G.p(), P->m, c.dt, c.s));
  BF_TRY(Y.alloc(&F->mem, P->n * (int64_t)nt * k * c.es));
  BF_TRY(sketch(c, BF_OP_C, l, k, G.p(), Y.p()));
  BF_TRY(Pb.alloc(&F->mem, Poff[nb] * c.es));
  BF_TRY(peel_V(c, l, k, Y.p(), Pb.p(), Poff, Ps));
  Stage& S = F->st[F->stage_W(l)];
  std::vector<int32_t> cap(nb);
  for (int b = 0; b < nb; ++b) cap[b] = std::min(Ps[b], k);
  BF_TRY(layout_stage(c, S, Ps, cap));
  std::vector<const void*> in(nb);
  std::vector<int64_t> ld(nb);
  for (int b = 0; b < nb; ++b) in[b] = Pb.p() + Poff[b] * c.es, ld[b] = Ps[b];
  return qr_into(c, S, in, ld, k, F->rV[l]);
}

int r_level(Ctx& c, int l) {
  Plan* P = c.P;
  Fact* F = c.F;
  const int L = P->L, lm = F->lm, nb = 1 << L, nt = 1 << l, nn = 1 << (L - l), nn1 = nn >> 1;
  const auto& nxt = F->rU[l + 1 - lm];
  std::vector<int32_t> Ps(nb);
  int k = 0;
  for (int tau = 0; tau < nt; ++tau)
    for (int nu = 0; nu < nn; ++nu) {
      Ps[tau * nn + nu] = nxt[(2 * tau) * nn1 + (nu >> 1)] + nxt[(2 * tau + 1) * nn1 + (nu >> 1)];
      k = std::max(k, Ps[tau * nn + nu]);
    }
  if (l == lm) k = std::max(k, *std::max_element(F->rV[lm].begin(), F->rV[lm].end()));
  k += P->opt.p;
  std::vector<int64_t> Poff(nb + 1, 0);
  for (int b = 0; b < nb; ++b) Poff[b + 1] = Poff[b] + (int64_t)Ps[b] * k;
  Scratch G(c.s), Z(c.s), Pb(c.s);
  BF_TRY(G.alloc(&F->mem, P->n * (int64_t)k * c.es));
  BF_TRY(launch_gaussian(P->opt.seed, sid(STAGE_R, l), 0, P->n, 0, k, G.p(), P->n, c.dt, c.s));
  BF_TRY(Z.alloc(&F->mem, P->m * (int64_t)nn * k * c.es));
  BF_TRY(sketch(c, BF_OP_N, L - l, k, G.p(), Z.p()));
  BF_TRY(Pb.alloc(&F->mem, Poff[nb] * c.es));
  BF_TRY(peel_U(c, l, k, Z.p(), Pb.p(), Poff, Ps));
  Stage& S = F->st[F->stage_R(l)];
  std::vector<int32_t> cap(nb);
  for (int b = 0; b < nb; ++b) cap[b] = std::min(Ps[b], k);
  BF_TRY(layout_stage(c, S, Ps, cap));
  std::vector<const void*> in(nb);
  std::vector<int64_t> ld(nb);
  for (int b = 0; b < nb; ++b) in[b] = Pb.p() + Poff[b] * c.es, ld[b] = Ps[b];
  BF_TRY(qr_into(c, S, in, ld, k, F->rU[l - lm]));
  if (l != lm) return BF_OK;

  // centre level: X = V^H Omega, then B (eq. Bij)
  Scratch Xb(c.s);
  int64_t xtot = 0;
  for (int b = 0; b < nb; ++b) xtot += (int64_t)F->rV[lm][b] * k;
  BF_TRY(Xb.alloc(&F->mem, xtot * c.es));
  std::vector<int64_t> xo;
  BF_TRY(project_X(c, k, G.p(), Xb.p(), xo));
  Stage& SB = F->st[F->stage_B()];
  std::vector<int32_t> rows(nb), cols(nb);
  int maxR = 1, maxS = 1;
  for (int b = 0; b < nb; ++b) {
    rows[b] = F->rU[0][b];
    cols[b] = F->rV[lm][b];
    maxR = std::max({maxR, rows[b], cols[b]});
    maxS = std::max(maxS, Ps[b]);
  }
  BF_TRY(layout_stage(c, SB, rows, cols));
  SB.cols = cols;
  std::vector<LSQTask> lt(nb);
  for (int b = 0; b < nb; ++b) {
    LSQTask& t = lt[b];
    t.P = Pb.p() + Poff[b] * c.es;
    t.Q = (const char*)S.d64.p + S.off[b] * 16;
    t.X = Xb.p() + xo[b] * c.es;
    t.B = (char*)SB.d64.p + SB.off[b] * 16;
    t.s = Ps[b];
    t.k = k;
    t.rU = rows[b];
    t.rV = cols[b];
  }
  Scratch d(c.s);
  BF_TRY(d.alloc(&F->mem, nb * sizeof(LSQTask)));
  BF_CUDA_TRY(cudaMemcpyAsync(d.p(), lt.data(), nb * sizeof(LSQTask), cudaMemcpyHostToDevice, c.s));
  BF_TRY(launch_lsq((const LSQTask*)d.p(), nb, maxS, k, maxR, c.dt, c.s));
  BF_TRY(make32(c, SB));
  BF_CUDA_TRY(cudaStreamSynchronize(c.s));
  return BF_OK;
}

}  // namespace

int factor(Plan* P, Operator* A, cudaStream_t s, Fact** out) {
  *out = nullptr;
  if (A->m != P->m || A->n != P->n) return fail(BF_EINVAL, "operator shape does not match the plan");
  const auto t0 = std::chrono::steady_clock::now();
  Fact* F = new Fact();
  F->plan = P;
  F->L = P->L;
  F->lm = P->lm;
  F->n = P->n;
  F->m = P->m;
  F->mem.cap = P->opt.mem_cap;
  F->st.resize(P->L + 3);
  F->rV.assign(P->lm + 1, {});
  F->rU.assign(P->L - P->lm + 1, {});
  Ctx c{P, A, F, s, P->opt.precision == BF_PREC_MIXED ? BF_C64 : BF_C128, 0};
  c.es = elem_bytes(c.dt);
  const int64_t n0 = A->cols_N, t0c = A->cols_T;
  int rc = leaf_loop(c, true);
  if (!rc) rc = leaf_loop(c, false);
  for (int l = 1; !rc && l <= P->lm; ++l) rc = w_level(c, l);
  for (int l = P->L - 1; !rc && l >= P->lm; --l) rc = r_level(c, l);
  if (!rc) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = fail(BF_ECUDA, cudaGetErrorString(e));
  }
  if (rc) {
    for (auto& S : F->st) S.d64.release(nullptr), S.d32.release(nullptr);
    delete F;
    return rc;
  }
  F->cols_N = A->cols_N - n0;
  F->cols_T = A->cols_T - t0c;
  F->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  *out = F;
  return BF_OK;
}

}  // namespace bf
