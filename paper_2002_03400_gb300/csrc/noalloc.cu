// bf_apply_noalloc: the apply of a finished factorization without any device
// allocation, for callers that may not allocate while they run (see the
// declaration in include/butterfly.h).  All scratch lives in one file-scope
// device array of BF_NOALLOC_SCRATCH_BYTES, shared by every call on a device.
#include <algorithm>
#include <climits>
#include <mutex>

#include "bf_internal.h"

namespace bf {

// The array itself.  Host code must not use this name as an address: on the
// host it is only a stand-in for the symbol, so its device address is looked
// up once per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[BF_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 256;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the array on the current device (set-up on first use).
int scratch_address(void** out) {
  int dev = 0;
  BF_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(BF_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return fail(BF_ECUDA, std::string("cudaGetSymbolAddress of the no-alloc scratch failed: ") +
                                cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return BF_OK;
}

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }
}  // namespace

}  // namespace bf

using namespace bf;

extern "C" int bf_apply_noalloc(bf_fact Fh, int op, int64_t nrhs, const void* x, int64_t ldx, void* y,
                                int64_t ldy, int dtype, void* stream) {
  if (!Fh || ((bf_fact_s*)Fh)->kind != KIND_FACT) return fail(BF_EINVAL, "not a factorization");
  Fact* F = ((bf_fact_s*)Fh)->impl;
  if (op != BF_OP_N && op != BF_OP_T && op != BF_OP_C) return fail(BF_EINVAL, "bad op");
  if (dtype != BF_C64 && dtype != BF_C128) return fail(BF_EINVAL, "dtype must be BF_C64 or BF_C128");
  if (nrhs < 0) return fail(BF_EINVAL, "nrhs < 0");
  if (nrhs == 0) return BF_OK;
  const Plan* P = F->plan;
  const int opC = op == BF_OP_N ? 0 : 1;
  const int64_t in_rows = opC ? P->m : P->n, out_rows = opC ? P->n : P->m;
  if (!x || !y || ldx < in_rows || ldy < out_rows) return fail(BF_EINVAL, "bad pointer or leading dimension");
  if (dtype == BF_C64)
    for (const auto& S : F->st)
      if (!S.have32)
        return fail(BF_EINVAL,
                    "BF_C64 needs the factorization's complex64 copy: factor with BF_PREC_MIXED or call "
                    "bf_apply once with BF_C64 first");
  cudaStream_t s = user_stream(stream);
  const size_t es = elem_bytes(dtype);

  // task lists: the factorization's cached device copy if bf_apply built it,
  // else built on the host and copied into the head of the scratch array
  const ApplyPlan& cached = F->ap[opC][dtype];
  ApplyPlan local;
  std::vector<StageTask> host_tasks;
  const ApplyPlan* ap = &cached;
  size_t task_bytes = 0;
  if (!cached.built) {
    apply_tasks_host(F, opC, dtype, local, host_tasks);
    ap = &local;
    task_bytes = round256(host_tasks.size() * sizeof(StageTask));
  }
  const int conj = op == BF_OP_T ? 1 : 0;
  const bool direct_in = (opC ? P->identT : P->identS) && !conj && ldx == in_rows;
  const bool direct_out = (opC ? P->identS : P->identT) && !conj && ldy == out_rows;
  // Sizes in a form that cannot wrap: every factor is checked against the
  // array's size before it is multiplied, so a huge nrhs is refused here and
  // never reaches a kernel (whose column count is an int).
  const size_t cap = (size_t)BF_NOALLOC_SCRATCH_BYTES;
  const size_t rows_max = std::max<size_t>({(size_t)ap->level_rows_max, (size_t)in_rows, (size_t)out_rows, 1});
  size_t need = 0, lvl = 0, xb = 0, yb = 0;
  bool over = nrhs > (int64_t)INT32_MAX || (uint64_t)nrhs > cap / (es * rows_max);
  if (!over) {
    lvl = round256((size_t)ap->level_rows_max * (size_t)nrhs * es);
    xb = direct_in ? 0 : round256((size_t)in_rows * (size_t)nrhs * es);
    yb = direct_out ? 0 : round256((size_t)out_rows * (size_t)nrhs * es);
    need = task_bytes + 2 * lvl + xb + yb;
    over = need > cap;
  }
  if (over)
    return fail(BF_EINVAL, "bf_apply_noalloc needs " + (need ? std::to_string(need) : std::string("more")) +
                               " bytes of scratch for nrhs=" + std::to_string(nrhs) +
                               ", above BF_NOALLOC_SCRATCH_BYTES (" + std::to_string(cap) +
                               "); use fewer columns per call");
  // Without cached task lists the call copies them from host memory that
  // lives only for this call; a stream capture would record a copy from
  // memory that is gone when the graph runs, so that case is refused.
  if (!cached.built) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    BF_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone)
      return fail(BF_EINVAL,
                  "bf_apply_noalloc during stream capture needs this factorization's task lists for the op and "
                  "dtype on the device: run bf_apply once with them first");
  }

  void* base = nullptr;
  BF_TRY(scratch_address(&base));
  char* p = (char*)base;
  const StageTask* d_tasks = (const StageTask*)cached.tasks.p;
  if (!cached.built) {
    BF_CUDA_TRY(cudaMemcpyAsync(p, host_tasks.data(), host_tasks.size() * sizeof(StageTask),
                                cudaMemcpyHostToDevice, s));
    d_tasks = (const StageTask*)p;
  }
  char* q = p + task_bytes;
  void* ping = q;
  void* pong = q + lvl;
  q += 2 * lvl;
  void* xt = direct_in ? const_cast<void*>(x) : (void*)q;
  q += xb;
  void* yt = direct_out ? y : (void*)q;
  const int64_t* perm_in = (const int64_t*)(opC ? P->d_permT.p : P->d_permS.p);
  const int64_t* perm_out = (const int64_t*)(opC ? P->d_permS.p : P->d_permT.p);
  const bool id_in = opC ? P->identT : P->identS;
  const bool id_out = opC ? P->identS : P->identT;

  // Every scratch element read below is written earlier in this call (the
  // gather fills xt, each stage writes all rows of its output level for all
  // nrhs columns), so nothing needs clearing between calls.
  if (!direct_in)
    BF_TRY(launch_gather_rows(id_in ? nullptr : perm_in, in_rows, nrhs, x, ldx, xt, in_rows, conj, dtype, s));
  StageBases bases{{xt, ping, pong, yt}};
  for (size_t i = 0; i < ap->first.size(); ++i)
    BF_TRY(launch_stage(d_tasks + ap->first[i], ap->count[i], ap->maxM[i], (int)nrhs, (int)nrhs, bases, dtype, s,
                        ap->variant_of(i, nrhs), i > 0 && dtype == BF_C64));
  if (!direct_out)
    BF_TRY(launch_scatter_rows(id_out ? nullptr : perm_out, out_rows, nrhs, yt, out_rows, y, ldy, conj, dtype, s));
  return BF_OK;
}
