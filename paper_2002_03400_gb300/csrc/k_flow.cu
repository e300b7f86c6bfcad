// Persistent apply of a finished factorization (eq. hybrid_butterfly_mat):
// all L + 3 stages of y = op(F) x in one cooperative launch, each output
// block started as soon as the blocks it reads are written, instead of one
// launch (and one device-wide dependency) per stage.
//
// The stage lists of the stage apply (apply_tasks_host) are rewritten once
// per factorization, direction and dtype:
//   - every stage writes its own row range of one stacked buffer (no
//     ping-pong reuse, so a block is never overwritten while it is read);
//   - each task (one output block) lists the tasks whose outputs it reads
//     (for W^j: the two child blocks of level j - 1; for B and R^j: the
//     blocks of the level below; in general every producer whose rows meet
//     one of its input ranges).
// Tasks are numbered in stage order and CTA c takes tasks c, c + G, c + 2G,
// ...; with all G CTAs resident (a cooperative launch), the lowest
// unfinished task never waits, so every wait ends.  A task's thread 0 waits
// for its producers' flags (acquire; bounded by a time limit, after which
// the kernel sets the device status flag and the CTA returns), the factor
// entries of the task's first round are copied before that wait (they do not
// depend on it), and after the task's stores the CTA releases its flag.
// Intermediate rows are read around L1 (cp.async.cg, ld.global.cg): another
// SM wrote them during this launch.
//
// Per task the products are those of the staged stage kernel: one FMA chain
// per output, terms in order and k ascending, so results equal the stage
// apply's bit for bit.
#include <algorithm>
#include <cstring>

#include "bf_internal.h"
#include "cx.cuh"

namespace bf {

namespace {
constexpr int FL_THREADS = 256;
constexpr int FL_SRR = 2;   // rows per thread: blocks of 8 * FL_SRR rows

template <typename V>
__host__ __device__ constexpr int flow_kr() {
  return sizeof(V) == 8 ? 48 : 24;
}
template <typename V>
__host__ __device__ constexpr size_t flow_smem() {
  return (size_t)flow_kr<V>() * (64 + 8 * FL_SRR) * sizeof(V);
}

struct FlowArgs {
  const StageTask* tasks;
  const int32_t* dep_ptr;   // ntasks + 1
  const int32_t* dep_idx;
  int ntasks, N;            // N: right-hand sides (row-major intermediates of N columns)
  StageBases bases;         // 0: x (tree order), 1: stacked intermediates, 3: y (tree order)
  int32_t* flags;           // one per task, zero at launch
  int* status;              // device status flag: set when a wait gave up
  unsigned long long limit_ns;
};

struct Strides2 {
  int64_t off, rs, cs;
};
__device__ __forceinline__ Strides2 strides2(int64_t off, int64_t ld, int N) {
  if (ld > 0) return {off, 1, ld};
  if (ld < 0) return {off, -ld, 1};
  return {off * N, N, 1};
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int ld_acquire(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int32_t* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// true once *flag is set; false when the time limit passed or another CTA
// has already given up (the status flag), so one failure ends every wait
__device__ bool wait_flag(const int32_t* flag, const int* status, unsigned long long limit_ns) {
  if (ld_acquire(flag)) return true;
  const unsigned long long t0 = now_ns();
  for (unsigned it = 0;; ++it) {
    if (ld_acquire(flag)) return true;
    if ((it & 15) == 15) {
      if (ld_acquire(status)) return false;
      if (now_ns() - t0 > limit_ns) return false;
    }
    __nanosleep(32);
  }
}

template <int BYTES>
__device__ __forceinline__ void cp_async_cg(void* dst, const void* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ float2 ld_cg(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ double2 ld_cg(const double2* p) { return __ldcg(p); }

// factor entries (row r0 + i, k0 + k) of op(mat) for i < mr, k < kn into
// fs[k][i] (row stride RB)
template <typename V, int RB>
__device__ __forceinline__ void copy_factor(V* fs, const V* mat, int ldm, int cj, int r0, int mr, int k0, int kn,
                                            int tid) {
  if (cj) {
    for (int e = tid; e < mr * kn; e += FL_THREADS) {
      const int i = e / kn, k = e - i * kn;
      cp_async_cg<sizeof(V)>(fs + k * RB + i, mat + (int64_t)(r0 + i) * ldm + k0 + k);
    }
  } else {
    for (int e = tid; e < mr * kn; e += FL_THREADS) {
      const int k = e / mr, i = e - k * mr;
      cp_async_cg<sizeof(V)>(fs + k * RB + i, mat + (r0 + i) + (int64_t)(k0 + k) * ldm);
    }
  }
}
}  // namespace

template <typename R>
__global__ void __launch_bounds__(FL_THREADS) flow_kernel(const FlowArgs a) {
  using V = typename Cx<R>::V;
  constexpr int KR = flow_kr<V>(), RB = 8 * FL_SRR;
  extern __shared__ __align__(16) uint8_t flow_smem_raw[];
  V* __restrict__ xs = (V*)flow_smem_raw;   // [KR][64]
  V* __restrict__ fs = xs + KR * 64;        // [KR][RB]
  __shared__ int s_abort;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int N = a.N;
  const int slices = (N + 63) / 64;
  for (int t = blockIdx.x; t < a.ntasks; t += gridDim.x) {
    const StageTask& tk = a.tasks[t];
    const int M = tk.M, nterms = tk.nterms;
    const int rblocks = (M + RB - 1) / RB;
    // the first round's factor entries do not depend on other tasks
    bool pre = false;
    if (nterms > 0 && M > 0) {
      const StageTerm& T0 = tk.t[0];
      if (T0.K > 0) {
        __syncthreads();   // the previous task's reads of fs are done
        copy_factor<V, RB>(fs, (const V*)T0.mat, T0.ldm, T0.conjT, 0, min(RB, M), 0, min(KR, T0.K), tid);
        pre = true;
      }
    }
    if (tid == 0) {
      bool ok = true;
      for (int q = a.dep_ptr[t]; q < a.dep_ptr[t + 1] && ok; ++q)
        ok = wait_flag(a.flags + a.dep_idx[q], a.status, a.limit_ns);
      if (!ok) atomicExch(a.status, 1);
      s_abort = ok ? 0 : 1;
    }
    __syncthreads();
    if (s_abort) {
      asm volatile("cp.async.wait_all;" ::: "memory");
      return;
    }
    for (int sub = 0; sub < rblocks * slices; ++sub) {
      const int rb = sub / slices, sl = sub - rb * slices;
      const int c0 = sl * 64, r0 = rb * RB;
      const int cw = min(64, N - c0), mr = min(RB, M - r0);
      const int c = 2 * lane, i0 = warp * FL_SRR;
      V acc[FL_SRR][2];
#pragma unroll
      for (int r = 0; r < FL_SRR; ++r) acc[r][0] = acc[r][1] = Cx<R>::make(0, 0);
      for (int term = 0; term < nterms; ++term) {
        const StageTerm& T = tk.t[term];
        const V* __restrict__ mat = (const V*)T.mat;
        const int K = T.K, ldm = T.ldm, cj = T.conjT;
        const Strides2 si = strides2(T.in_off, T.ldi, N);
        const V* __restrict__ in = (const V*)a.bases.p[T.in_base] + si.off + c0 * si.cs;
        const bool pair16 = sizeof(V) == 16 || (si.cs == 1 && (si.rs & 1) == 0 && (cw & 1) == 0 &&
                                                ((uintptr_t)in & 15) == 0);
        for (int k0 = 0; k0 < K; k0 += KR) {
          const int kn = min(KR, K - k0);
          const bool first = pre && sub == 0 && term == 0 && k0 == 0;
          if (!first) {
            __syncthreads();   // the previous round's reads are done
            copy_factor<V, RB>(fs, mat, ldm, cj, r0, mr, k0, kn, tid);
          }
          if (sizeof(V) == 16 || pair16) {
            const int pw = sizeof(V) == 16 ? cw : cw >> 1;   // 16-byte units per row
            const int step = sizeof(V) == 16 ? 1 : 2;
            for (int e = tid; e < kn * pw; e += FL_THREADS) {
              const int k = e / pw, p = e - k * pw;
              cp_async_cg<16>(xs + k * 64 + step * p, in + (int64_t)(k0 + k) * si.rs + (int64_t)(step * p) * si.cs);
            }
          } else {
            // 8-byte elements one at a time, read around L1 into shared memory
            for (int e = tid; e < kn * cw; e += FL_THREADS) {
              const int k = e / cw, cc = e - k * cw;
              xs[k * 64 + cc] = ld_cg(in + (int64_t)(k0 + k) * si.rs + (int64_t)cc * si.cs);
            }
          }
          asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
          __syncthreads();
          if (i0 < mr) {
            int ro[FL_SRR];
#pragma unroll
            for (int r = 0; r < FL_SRR; ++r) ro[r] = min(i0 + r, mr - 1);
            const int cl = min(c, cw - 1), cr = min(c + 1, cw - 1);
#pragma unroll 4
            for (int k = 0; k < kn; ++k) {
              const V a0 = xs[k * 64 + cl], a1 = xs[k * 64 + cr];
#pragma unroll
              for (int r = 0; r < FL_SRR; ++r) {
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
        const Strides2 so = strides2(tk.out_off, tk.ldo, N);
        V* __restrict__ out = (V*)a.bases.p[tk.out_base] + so.off;
#pragma unroll
        for (int r = 0; r < FL_SRR; ++r)
          if (i0 + r < mr) {
            V* o = out + (int64_t)(r0 + i0 + r) * so.rs;
            if (c < cw) o[(int64_t)(c0 + c) * so.cs] = acc[r][0];
            if (c + 1 < cw) o[(int64_t)(c0 + c + 1) * so.cs] = acc[r][1];
          }
      }
    }
    __syncthreads();   // every store of the task is issued
    if (tid == 0) {
      __threadfence();
      st_release(a.flags + t, 1);
    }
  }
}

// ------------------------------------------------------------------ host --

// Rewrites the stage lists of (F, opC, dtype) for the persistent apply.
// ok stays false (the stage apply is used) when a list reads y or writes x,
// which the stage apply never does.
int build_flow(Fact* F, int opC, int dtype, cudaStream_t s) {
  FlowPlan& fl = F->fl[opC][dtype];
  if (fl.built) return BF_OK;
  fl = FlowPlan();
  fl.built = true;
  ApplyPlan tmp;
  std::vector<StageTask> all;
  apply_tasks_host(F, opC, dtype, tmp, all);
  const int nst = (int)tmp.first.size();
  // rows of each stage's output among the stacked intermediates
  std::vector<int64_t> rows(nst, 0), base(nst + 1, 0);
  for (int i = 0; i < nst; ++i)
    for (int t = tmp.first[i]; t < tmp.first[i] + tmp.count[i]; ++t) {
      const StageTask& tk = all[t];
      if (tk.out_base == 0) return BF_OK;
      if (tk.out_base == 1 || tk.out_base == 2) {
        if (tk.ldo != 0) return BF_OK;
        rows[i] = std::max(rows[i], tk.out_off + tk.M);
      }
    }
  for (int i = 0; i < nst; ++i) base[i + 1] = base[i] + rows[i];
  // producers of each intermediate row range: per stage, (first row, end, task)
  struct Span {
    int64_t a, b;
    int32_t task;
  };
  std::vector<std::vector<Span>> spans(nst);
  int last_writer[4] = {-1, -1, -1, -1};
  std::vector<int32_t> dep_ptr(all.size() + 1, 0), dep_idx;
  for (int i = 0; i < nst; ++i) {
    for (int t = tmp.first[i]; t < tmp.first[i] + tmp.count[i]; ++t) {
      StageTask& tk = all[t];
      std::vector<int32_t> d;
      for (int q = 0; q < tk.nterms; ++q) {
        StageTerm& T = tk.t[q];
        if (T.in_base == 3) return BF_OK;
        if (T.in_base == 1 || T.in_base == 2) {
          const int p = last_writer[T.in_base];
          if (p < 0 || T.ldi != 0) return BF_OK;
          T.in_off += base[p];
          T.in_base = 1;
          for (const Span& sp : spans[p])
            if (sp.a < T.in_off + T.K && T.in_off < sp.b) d.push_back(sp.task);
        }
      }
      std::sort(d.begin(), d.end());
      d.erase(std::unique(d.begin(), d.end()), d.end());
      for (int32_t x : d)
        if (x >= t) return fail(BF_EINTERNAL, "persistent apply: a task depends on a later task");
      dep_idx.insert(dep_idx.end(), d.begin(), d.end());
      dep_ptr[t + 1] = (int32_t)dep_idx.size();
    }
    // this stage's outputs (after its inputs were resolved: a stage reads
    // the previous writer of a buffer, never itself)
    for (int t = tmp.first[i]; t < tmp.first[i] + tmp.count[i]; ++t) {
      StageTask& tk = all[t];
      if (tk.out_base == 1 || tk.out_base == 2) {
        last_writer[tk.out_base] = i;
        tk.out_off += base[i];
        tk.out_base = 1;
        spans[i].push_back({tk.out_off, tk.out_off + tk.M, (int32_t)t});
      }
    }
  }
  fl.ntasks = (int)all.size();
  fl.inter_rows = base[nst];
  const size_t tb = all.size() * sizeof(StageTask), pb = dep_ptr.size() * sizeof(int32_t),
               ib = std::max<size_t>(1, dep_idx.size()) * sizeof(int32_t);
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  std::vector<char> host(al(tb) + al(pb) + ib, 0);
  memcpy(host.data(), all.data(), tb);
  memcpy(host.data() + al(tb), dep_ptr.data(), pb);
  if (!dep_idx.empty()) memcpy(host.data() + al(tb) + al(pb), dep_idx.data(), dep_idx.size() * sizeof(int32_t));
  BF_TRY(fl.dev.alloc(&F->mem, host.size(), nullptr));
  BF_CUDA_TRY(cudaMemcpyAsync(fl.dev.p, host.data(), host.size(), cudaMemcpyHostToDevice, s));
  BF_CUDA_TRY(host_sync(s));
  char* p = (char*)fl.dev.p;
  fl.d_tasks = (const StageTask*)p;
  fl.d_dep_ptr = (const int32_t*)(p + al(tb));
  fl.d_dep_idx = (const int32_t*)(p + al(tb) + al(pb));
  fl.ok = true;
  return BF_OK;
}

namespace {
template <typename R>
int launch_flow_kernel(const FlowArgs& a, cudaStream_t s) {
  using V = typename Cx<R>::V;
  constexpr size_t sm = flow_smem<V>();
  static int per_sm = -1, sms = 0;   // co-resident CTAs (kernel and device fixed per process)
  if (per_sm < 0) {
    int dev = 0, b = 0;
    BF_CUDA_TRY(cudaGetDevice(&dev));
    BF_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    BF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, flow_kernel<R>, FL_THREADS, sm));
    per_sm = b;
  }
  if (per_sm < 1) return fail(BF_ECUDA, "persistent apply: no CTA fits on an SM");
  const int grid = std::max(1, std::min(a.ntasks, per_sm * sms));
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(FL_THREADS);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  note_launch();
  const cudaError_t e = cudaLaunchKernelEx(&cfg, flow_kernel<R>, a);
  if (e != cudaSuccess) return fail(BF_ECUDA, std::string("persistent apply launch: ") + cudaGetErrorString(e));
  BF_CUDA_TRY(cudaGetLastError());
  return BF_OK;
}
}  // namespace

size_t flow_scratch_bytes(const FlowPlan& fl, int64_t nrhs, int dtype) {
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  return al((size_t)fl.inter_rows * nrhs * elem_bytes(dtype)) + al((size_t)fl.ntasks * sizeof(int32_t));
}

int run_flow(Fact* F, int opC, int dtype, int64_t nrhs, const void* xt, void* yt, void* scratch,
             cudaStream_t s) {
  const FlowPlan& fl = F->fl[opC][dtype];
  if (!fl.ok) return fail(BF_EINTERNAL, "persistent apply not built");
  if (nrhs > INT32_MAX) return fail(BF_EINVAL, "too many right-hand sides");
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  char* p = (char*)scratch;
  int32_t* flags = (int32_t*)(p + al((size_t)fl.inter_rows * nrhs * elem_bytes(dtype)));
  BF_CUDA_TRY(cudaMemsetAsync(flags, 0, (size_t)fl.ntasks * sizeof(int32_t), s));
  FlowArgs a{};
  a.tasks = fl.d_tasks;
  a.dep_ptr = fl.d_dep_ptr;
  a.dep_idx = fl.d_dep_idx;
  a.ntasks = fl.ntasks;
  a.N = (int)nrhs;
  a.bases = StageBases{{const_cast<void*>(xt), p, nullptr, yt}};
  a.flags = flags;
  a.status = tc_status_ptr();
  a.limit_ns = 1000000000ull;
  if (!a.status) return fail(BF_ECUDA, "device status flag not found");
  return dtype == BF_C128 ? launch_flow_kernel<double>(a, s) : launch_flow_kernel<float>(a, s);
}

// One task that waits for its own flag (which nothing sets) for limit_ns:
// the wait gives up, sets the device status flag and the kernel returns.
int flow_wait_probe(uint64_t limit_ns, cudaStream_t s) {
  DevBuf buf;
  BF_TRY(buf.alloc(nullptr, 256 + sizeof(StageTask), s));
  char* p = (char*)buf.p;
  int32_t* hdr = (int32_t*)p;   // flag | dep_ptr[2] | dep_idx[1]
  const int32_t h[4] = {0, 0, 1, 0};
  StageTask tk{};
  tk.out_base = 3;
  tk.M = 0;
  tk.nterms = 0;
  int rc = BF_OK;
  if (cudaMemcpyAsync(hdr, h, sizeof(h), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(p + 256, &tk, sizeof(tk), cudaMemcpyHostToDevice, s) != cudaSuccess)
    rc = fail(BF_ECUDA, "probe set-up copy failed");
  FlowArgs a{};
  a.tasks = (const StageTask*)(p + 256);
  a.dep_ptr = hdr + 1;
  a.dep_idx = hdr + 3;
  a.ntasks = 1;
  a.N = 1;
  a.bases = StageBases{{nullptr, nullptr, nullptr, nullptr}};
  a.flags = hdr;
  a.status = tc_status_ptr();
  a.limit_ns = limit_ns;
  if (!rc && !a.status) rc = fail(BF_ECUDA, "device status flag not found");
  if (!rc) rc = launch_flow_kernel<float>(a, s);
  if (!rc && host_sync(s) != cudaSuccess) rc = fail(BF_ECUDA, "probe synchronisation failed");
  buf.release(s);
  return rc;
}

}  // namespace bf
