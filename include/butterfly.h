/*
 * butterfly.h -- C ABI of the GB300-native adaptive randomized butterfly
 * factorization (Liu, Xing, Guo, Michielssen, Ghysels, Li, "Butterfly
 * factorization via randomized matrix-vector multiplications",
 * arXiv:2002.03400).
 *
 * The library computes the hybrid butterfly factorization
 *     A ~= (U^L R^(L-1) ... R^(l_m)) B^(l_m) (W^(l_m) ... W^1 V^0),  l_m = floor(L/2)
 * (eq. hybrid_butterfly_mat, Sec. 3.3.3) of an m x n complex operator A given
 * only as a black box that multiplies A and A^T by blocks of vectors
 * (Alg. 2, Sec. 4), and applies the result in O(n log n) (Sec. 1).
 *
 * Conventions for every entry point:
 *   - Status: each call returns BF_OK (0) or a negative bf_status code; on
 *     error every out-handle is set to NULL, nothing leaks, and
 *     bf_last_error() returns a one-line reason (thread-local).
 *   - Complex data is interleaved (re, im): BF_C128 = two doubles per entry,
 *     BF_C64 = two floats.  Matrices are column-major with a leading
 *     dimension in elements.
 *   - "Device" pointers are CUDA global-memory addresses on the current
 *     device; "host" pointers are ordinary CPU memory.  Vectors passed to
 *     bf_apply and bf_operator_apply are in the caller's original point
 *     order; the library permutes to tree order itself.
 *   - Streams are cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are stream-ordered unless stated otherwise; calls that
 *     return ranks or errors to the host synchronize the stream.
 *   - Handles (bf_plan, bf_fact, bf_operator) are used by one host thread at
 *     a time; concurrent bf_apply calls on one bf_fact from different
 *     streams are allowed (factors are read-only after bf_factor returns).
 *   - Debug checks: with BF_DEBUG=1 in the environment when the library
 *     loads (or a build with -DBF_DEBUG), every block product's task list
 *     is checked on the host before its launch -- every block offset inside
 *     its buffer, ranks and term counts in range, factor entries inside
 *     their block -- and a violation returns BF_EINTERNAL naming the task.
 *     Results do not change.  Off by default (a few microseconds per list).
 *   - Memory: device memory is taken with cudaMallocAsync on the call's
 *     stream (or cudaMalloc) and is counted against bf_options.mem_cap;
 *     exceeding the cap returns BF_ENOMEM before any allocation.
 */
#ifndef BUTTERFLY_H
#define BUTTERFLY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bf_plan_s* bf_plan;          /* trees + parameters           */
typedef struct bf_fact_s* bf_fact;          /* resident factorization       */
typedef struct bf_operator_s* bf_operator;  /* black-box A (and A^T)        */

typedef enum {
  BF_OK = 0,
  BF_EINVAL = -1,          /* bad argument or size                          */
  BF_ENOMEM = -2,          /* device allocation failed or over mem_cap      */
  BF_ECALLBACK = -3,       /* a user black-box callback returned non-zero   */
  BF_ENOTCONVERGED = -4,   /* adaptive leaf rank exceeded r_max             */
  BF_ECUDA = -5,           /* a CUDA runtime call failed                    */
  BF_ETIMEOUT = -6,        /* a bounded device wait gave up                 */
  BF_EUNSUPPORTED = -7,    /* combination not built                         */
  BF_EINTERNAL = -8        /* an internal consistency check failed          */
} bf_status;

typedef enum { BF_C64 = 0, BF_C128 = 1 } bf_dtype;
/* op selects A (N), A^T (T) or A^H (C). */
typedef enum { BF_OP_N = 0, BF_OP_T = 1, BF_OP_C = 2 } bf_op;
/* FP64: every product in complex128.  MIXED: sketch products, peeling and
 * the factor copies used by them in complex64 (FP32 arithmetic); the B least
 * squares in FP64; pivoted QR and truncation in float-float (~2^-46, on the
 * FP32 pipe), or in FP64 when bf_options.qr_fp64 is set. */
typedef enum { BF_PREC_FP64 = 0, BF_PREC_MIXED = 1 } bf_precision;

typedef enum {
  BF_KERNEL_NONE = 0,
  BF_KERNEL_HELMHOLTZ_2D = 1,   /* exp(-i k r) / r                         */
  BF_KERNEL_HELMHOLTZ_3D = 2,   /* exp(+i k r) / (4 pi r)  (eq. 3dkernel)  */
  BF_KERNEL_DFT = 3             /* exp(-2 pi i t s), 1-D points            */
} bf_kernel_type;

typedef struct {
  int type;            /* bf_kernel_type                                  */
  double wavenumber;   /* k (ignored by BF_KERNEL_DFT)                    */
} bf_kernel_desc;

/* Parameters of Alg. 2 (its "Input" line) plus build options. */
typedef struct {
  int p;               /* oversampling (default 2)                          */
  int r0;              /* initial rank guess of the leaf loops (default 4)  */
  int r_max;           /* leaf-loop rank cap -> BF_ENOTCONVERGED (1024)     */
  uint64_t seed;       /* seed of the counter-based sketch generator        */
  int precision;       /* bf_precision (default BF_PREC_FP64)               */
  size_t mem_cap;      /* device-byte cap per handle, 0 = none              */
  int qr_fp64;         /* MIXED only: 1 = pivoted QR and truncation in FP64
                          instead of float-float (default 0)                */
  int hybrid_level;    /* level l of B in eq. hybrid_butterfly_mat: -1 (default)
                          = l_m = floor(L/2), Alg. 2's hybrid form; any
                          0 <= l <= L-1 runs the same loops with W levels
                          1..l and R levels L-1..l.  l = 0 is the
                          column-wise factorization of Sec. 3.3.1 (its outer
                          factor kept as B^0 V^0^H); the row-wise one of
                          Sec. 3.3.2 is l = 0 applied to A^T            */
  int accept_retries;  /* a-posteriori acceptance instead of trusting the
                          heuristic stop of the leaf loops (Sec. 4.2): 0
                          (default) = off; t > 0: after Alg. 2 the sketch
                          error of Sec. 7 (16 fresh test columns, seed
                          1009 + attempt) must be <= 2 sqrt(L+2) tol, else
                          the factorization is redone with r0 doubled, at
                          most t times, then BF_ENOTCONVERGED            */
  int leaf_passes;     /* cap on the passes of each adaptive leaf loop: 0
                          (default) = none; after that many passes the loop
                          stops as if converged (bounds the black-box work
                          of the leaf loops; accept_retries then decides) */
} bf_options;

/* Fills *opt with the defaults above. */
void bf_options_default(bf_options* opt);

/* Black-box callback (Alg. 2 input: products with A and with A^T).
 * op is BF_OP_N (Y = A X, X n x ncols, Y m x ncols) or BF_OP_T
 * (Y = A^T X, X m x ncols, Y n x ncols); X and Y are device pointers in
 * user point order, valid only during the call; dtype is a bf_dtype; work
 * must be enqueued on `stream`.  Return 0 on success, non-zero on failure
 * (the library then returns BF_ECALLBACK). */
typedef int (*bf_matvec_fn)(void* ctx, int op, int64_t ncols, const void* X,
                            int64_t ldx, void* Y, int64_t ldy, int dtype,
                            void* stream);

/* ---------------------------------------------------------------- plan -- */
/* Builds the bisection trees T_S (sources, n points) and T_T (targets, m
 * points) of depth L = smallest L with ceil(max(n,m)/2^L) <= leaf (Sec. 3.1).
 * src/tgt: host, row-major n x dim / m x dim doubles, or NULL for index order
 * (then dim is ignored).  A node of s points splits into ceil(s/2) and
 * floor(s/2): points are ordered by the coordinate of largest bounding-box
 * extent (ties: lowest axis, then lowest index).  kern may be NULL (no
 * built-in kernel operator).  tol is the truncation tolerance eps of Alg. 1.
 * opt may be NULL (defaults).  The plan copies everything it needs to the
 * device.  Errors: BF_EINVAL if n, m < 1, leaf < 1, L < 1 (Alg. 2 needs a
 * centre level below the leaves), an empty leaf, dim not in {1,2,3}, or
 * tol < 0. */
int bf_plan_create(const double* src, int64_t n, const double* tgt, int64_t m,
                   int dim, const bf_kernel_desc* kern, int leaf, double tol,
                   const bf_options* opt, bf_plan* out);

/* Tree depth L, centre level l_m, n, m (any pointer may be NULL). */
int bf_plan_info(bf_plan plan, int* L, int* lm, int64_t* n, int64_t* m);

/* Host copies: permS[i] / permT[i] = original index of tree position i
 * (length n / m); offS / offT (may be NULL) receive the node boundaries of
 * every level, level l at offset 2^l - 1 + l ... i.e. concatenated arrays
 * of 2^l + 1 entries for l = 0..L. */
int bf_plan_trees(bf_plan plan, int64_t* permS, int64_t* permT, int64_t* offS,
                  int64_t* offT);

/* Host-only bisection of one point set (the tree half of bf_plan_create;
 * needs no GPU).  pts: row-major count x dim doubles or NULL (index order).
 * perm (count int64) and off (sum over l=0..L of 2^l + 1 int64, level l
 * starting at 2^l - 1 + l) are caller-owned host buffers. */
int bf_bisect(const double* pts, int64_t count, int dim, int L, int64_t* perm,
              int64_t* off);

/* ------------------------------------------------------------ operators -- */
/* Dense stored A (m x n, column-major, user order, device memory, lda >= m).
 * The operator keeps a tree-ordered copy in the plan's precision's dtype;
 * the caller's buffer may be freed after the call returns.  Stream-ordered
 * on `stream`. */
int bf_operator_dense(bf_plan plan, const void* A, int64_t lda, int dtype,
                      void* stream, bf_operator* out);

/* A[i,j] = K(t_i, s_j) formed on the fly from the plan's points and kernel
 * (BF_EINVAL if the plan has no kernel or no points). */
int bf_operator_kernel(bf_plan plan, bf_operator* out);

/* The same operator with its entries resident: both orientations (A and
 * A^H) are formed once, on `stream`, as complex64 entry images (the layout
 * bf_set_entry_images describes; 16 bytes per entry of A in all, counted
 * against the plan's mem_cap), and its complex64 products with A and A^H
 * -- bf_operator_apply and the structured sketches of a factorization --
 * stream them instead of re-forming the entries (complex128 products form
 * entries as bf_operator_kernel does).  A factorization of this operator
 * reuses the images instead of forming its own.  Errors: as
 * bf_operator_kernel; BF_ENOMEM when the images do not fit. */
int bf_operator_kernel_cached(bf_plan plan, void* stream, bf_operator* out);

/* A = the factorization F, applied by bf_apply / bf_apply_T (the black box
 * of the exact-recovery and composition workloads).  F must outlive it. */
int bf_operator_factored(bf_fact F, bf_operator* out);

/* A = A1 * A2 (A1: m x k, A2: k x n); both must outlive it. */
int bf_operator_composed(bf_operator A1, bf_operator A2, bf_operator* out);

/* A given by a user callback (m x n). */
int bf_operator_callback(int64_t m, int64_t n, bf_matvec_fn fn, void* ctx,
                         bf_operator* out);

/* Y = op(A) X in user order (device pointers).  Sizes: op N: X n x ncols,
 * Y m x ncols; op T/C: X m x ncols, Y n x ncols. */
int bf_operator_apply(bf_operator A, int op, int64_t ncols, const void* X,
                      int64_t ldx, void* Y, int64_t ldy, int dtype,
                      void* stream);

/* Black-box column counts (products with A, with A^T) since creation. */
int bf_operator_counts(bf_operator A, int64_t* cols_N, int64_t* cols_T);

/* ----------------------------------------------------------- factorize -- */
/* Alg. 2: adaptive leaf bases V^0, U^L (rank doubling from r0), transfer
 * matrices W^1..W^(l_m) and R^(L-1)..R^(l_m) from structured random
 * sketches (Sec. 4.1-4.3) peeled by the factors already recovered, and the
 * centre coupling B^(l_m) by least squares (eq. Bij, Sec. 4.4).
 * A may be NULL (the plan's kernel operator).  Synchronizes `stream` once
 * per level (ranks return to the host to size the next sketch).
 * Errors: BF_ENOTCONVERGED, BF_ECALLBACK, BF_ENOMEM, BF_ECUDA. */
int bf_factor(bf_plan plan, bf_operator A, void* stream, bf_fact* out);

/* Alg. 2 for `count` operators at once, level-synchronously: every phase
 * (leaf passes, each W^l and R^l level, the B solve) runs one launch per
 * kernel covering all blocks of all operators, whatever their size, depth
 * and ranks.  plans[i] (all of one precision) with ops[i] (ops may be NULL
 * or hold NULL entries: the plan's kernel operator).  out: count handles,
 * each identical to what bf_factor would return for that entry; on error all
 * are NULL.  Synchronizes once per phase. */
int bf_factor_batch(int count, const bf_plan* plans, const bf_operator* ops,
                    void* stream, bf_fact* out);

/* y = F x (eq. hybrid_butterfly_mat).  x: n x nrhs, y: m x nrhs, device,
 * user order, dtype BF_C64 or BF_C128 (computed in that precision). */
int bf_apply(bf_fact F, int64_t nrhs, const void* x, int64_t ldx, void* y,
             int64_t ldy, int dtype, void* stream);

/* y = F^T x (op BF_OP_T) or F^H x (op BF_OP_C); x: m x nrhs, y: n x nrhs. */
int bf_apply_T(bf_fact F, int op, int64_t nrhs, const void* x, int64_t ldx,
               void* y, int64_t ldy, int dtype, void* stream);

/* Apply autotuner.  Each stage of an apply of F (op BF_OP_N, BF_OP_T or
 * BF_OP_C; dtype BF_C64 or BF_C128; nrhs right-hand sides) is a batched
 * block product of eq. hybrid_butterfly_mat that the library can run with
 * several kernel shapes; all compute bit-identical results.  This call times
 * every shape on every stage, and the fused apply (bf_set_apply_engine) at
 * every column-slice width that fits, on internal scratch operands (no user
 * data is read or written); it keeps the fastest shape per stage, the
 * fastest slice width, and the faster of the two engines for all later
 * applies of F with a right-hand-side count in the same class (1, 2-4,
 * 5-16, 17-32, 33-64, >64), and writes the tuned device time of one apply
 * in ms to *ms_out (may be NULL).  Synchronises the stream; allocates scratch for
 * its duration.  BF_EINVAL for a bad op/dtype/nrhs, BF_ENOMEM, BF_ECUDA. */
int bf_apply_tune(bf_fact F, int op, int64_t nrhs, int dtype, void* stream, float* ms_out);

/* Graph-captured apply (eq. hybrid_butterfly_mat).  bf_applier_create
 * captures the launches of y = F x (op BF_OP_N), F^T x (BF_OP_T) or
 * F^H x (BF_OP_C) for nrhs right-hand sides of dtype BF_C64/BF_C128, on
 * buffers the applier owns, once into a CUDA graph: the engine bf_apply
 * would use at the time of the call (bf_set_apply_engine, bf_apply_tune;
 * the fused engine, which works on user-order x and y, is replaced by the
 * grouped or the stage launches).  F must outlive the applier; free it
 * with bf_free.  BF_EINVAL, BF_ENOMEM, BF_ECUDA. */
typedef struct bf_applier_s* bf_applier;
int bf_applier_create(bf_fact F, int op, int64_t nrhs, int dtype, bf_applier* out);

/* One apply through the captured graph: x (device, user order, ld ldx,
 * in_rows x nrhs as for bf_apply / bf_apply_T) is gathered into the
 * applier's input, the graph runs, the result is scattered into y (ld ldy).
 * Results equal bf_apply's bit for bit.  Runs of one applier are serialised
 * (a run on another stream waits for the previous one); different appliers
 * of one factorization may run concurrently.  BF_EINVAL for short leading
 * dimensions, BF_ECUDA. */
int bf_applier_run(bf_applier A, const void* x, int64_t ldx, void* y, int64_t ldy, void* stream);

/* Size of the fixed device scratch array used by bf_apply_noalloc (32 MiB).
 * Every GPU on which the library is loaded holds this array until the
 * process exits, whether or not bf_apply_noalloc is ever called. */
#define BF_NOALLOC_SCRATCH_BYTES (32u << 20)

/* Apply without device allocation.  The paper has no counterpart: this is a
 * service for callers that must not allocate device memory while they run --
 * for example an application that handed all device memory to its own pool
 * at start-up (cudaMalloc would fail or fragment that pool), a plug-in
 * running inside a framework that owns the device's memory, or a
 * latency-bound loop whose per-request path may not call cudaMalloc/cudaFree
 * (both can synchronize the whole device).
 * Computes y = F x (op BF_OP_N), F^T x (BF_OP_T) or F^H x (BF_OP_C) exactly
 * as bf_apply / bf_apply_T do, with the same argument meaning and layout;
 * the caller still owns x and y.  All intermediates live in one file-scope
 * device array of BF_NOALLOC_SCRATCH_BYTES:
 *   - the first call on a device looks up that array's device address
 *     (cudaGetSymbolAddress) with the device current and keeps it for the
 *     life of the process; make that first call before capturing the stream
 *     into a CUDA graph.  Resetting the device (cudaDeviceReset) while the
 *     library is loaded is not supported: the kept address would be stale;
 *   - a call that finds no cached task lists for (op, dtype) builds them on
 *     the host and copies them into the array; while the stream is being
 *     captured that copy would outlive its source, so such a call returns
 *     BF_EINVAL (bf_apply with the same op and dtype caches the lists);
 *   - a request that needs more scratch than the array holds (grows with
 *     nrhs and with the factorization's block ranks; nrhs above INT32_MAX
 *     included) returns BF_EINVAL with the byte counts in bf_last_error()
 *     before any GPU work; split the columns into smaller calls;
 *   - every call shares the array and it keeps the last call's contents;
 *     nothing in it needs to start at zero (each call writes every element
 *     it later reads), but calls whose GPU work overlaps -- on different
 *     streams, threads or factorizations -- race on it: serialize them;
 *   - BF_C64 needs the factorization's complex64 copy (a BF_PREC_MIXED
 *     factorization, or one that bf_apply has already run in BF_C64);
 *     otherwise BF_EINVAL.
 * Calls no cudaMalloc, cudaFree or other allocating routine. */
int bf_apply_noalloc(bf_fact F, int op, int64_t nrhs, const void* x,
                     int64_t ldx, void* y, int64_t ldy, int dtype,
                     void* stream);

/* Ranks of one level (2^L int32 to host; block b = tau*2^(L-l) + nu).
 * side 0: row bases V (levels 0..l_m); side 1: column bases U (l_m..L). */
int bf_ranks(bf_fact F, int side, int level, int32_t* out);

/* Statistics (any pointer may be NULL): stored factor entries, black-box
 * columns with A and with A^T used by bf_factor, and its wall time (s). */
int bf_fact_info(bf_fact F, int64_t* stored_entries, int64_t* cols_N,
                 int64_t* cols_T, double* factor_seconds);

/* A-posteriori acceptance record of bf_factor (bf_options.accept_retries;
 * any pointer may be NULL): factorizations run (1 without the check), the
 * r0 of the accepted one, and its sketch error (-1 without the check). */
int bf_fact_accept(bf_fact F, int* attempts, int* r0_used, double* sketch_error);

/* Import a factorization from host blocks (exactly-butterfly operators).
 * rV: (l_m+1) x 2^L ranks of the row bases at levels 0..l_m;
 * rU: (L-l_m+1) x 2^L ranks of the column bases at levels l_m..L.
 * blocks[s], s = 0..L+2, host pointer to the packed column-major blocks of
 * stage s in apply order: V^0, W^1..W^(l_m), B, R^(l_m)..R^(L-1), U^L, each
 * stage's 2^L blocks in block order with ld = block rows.  Block shapes:
 * V^0: |S_nu| x rV0; W^j: (rV[j-1] of the two children) x rV[j];
 * B: rU[l_m] x rV[l_m]; R^j: (rU[j+1] of the two children) x rU[j];
 * U^L: |T_tau| x rU[L].  dtype BF_C128. */
int bf_fact_import(bf_plan plan, const int32_t* rV, const int32_t* rU,
                   const void* const* blocks, int dtype, bf_fact* out);

/* Host copy of stage s's packed blocks (layout of bf_fact_import, complex128);
 * *bytes in: capacity of host_out, out: bytes written (or needed). */
int bf_fact_export(bf_fact F, int stage, void* host_out, size_t* bytes);

/* Checkpoint of a finished factorization (for restarting a server without
 * refactoring; the paper has no counterpart).  bf_fact_save writes F's
 * ranks, every stage's block shapes and entries (complex128, plus the
 * complex64 copy where F has one, so that the reloaded factorization applies
 * bit for bit as F does) and its black-box column counts to `path`;
 * synchronizes the device.  bf_fact_load reads such a file for `plan` (the
 * plan the factorization was built on, or one made with the same geometry
 * and options): BF_EINVAL when the file does not match the plan's n, m, L
 * and l_m, or is truncated or inconsistent; BF_ENOMEM, BF_ECUDA.  The file
 * is native-endian and versioned. */
int bf_fact_save(bf_fact F, const char* path);
int bf_fact_load(bf_plan plan, const char* path, bf_fact* out);

/* Sketch error of Sec. 7 (eq. error): ||A W - F W||_F / ||A W||_F with W a
 * complex Gaussian n x ncols test matrix drawn from the counter-based
 * generator (stream 5<<8, user-order rows); both products are computed in
 * `dtype` (BF_C64 or BF_C128), the norms in FP64.  Synchronizes. */
int bf_error(bf_fact F, bf_operator A, int ncols, uint64_t seed, int dtype,
             void* stream, double* err);

/* Selects the engine of the complex64 sketch products for the whole process:
 * 0 (default) -- tcgen05 tensor cores with the exact three-way bf16 split
 * (operands split into three bf16 parts, 6 products kept: FP32-level);
 * 1 -- SIMT FP32 only; 2 -- tensor cores with split-precision 3xTF32
 * (two TF32 parts, 3 products, ~2^-21 per product); 3 -- the three-way
 * split forced (as 0).  Sketches wider than 48 columns run as column slices.
 * For comparisons and diagnostics; not thread-safe against running
 * factorizations. */
int bf_set_sketch_engine(int engine);

/* Entry images for the whole process (mixed precision, built-in kernel
 * operators): on = 1 (default) -- a factorization first forms every kernel
 * entry once per orientation (A and A^H) in complex64, tiled for the
 * tensor-core sketch kernel (8 bytes per entry and orientation, e.g. 4.3 GB
 * for n = m = 16384), and every structured sketch of Alg. 2 streams that
 * image instead of re-forming the m x n entries (the same bf16 parts and
 * products, summed in another order: results agree to FP32 rounding).  Used while both images fit in half of the free device memory
 * and in half of what mem_cap leaves; freed when the factorization returns.
 * on = 0 -- entries formed on the fly in every sketch.  Errors: BF_EINVAL
 * unless on is 0 or 1.  Not thread-safe against running factorizations. */
int bf_set_entry_images(int on);

/* Failure path of the library's bounded device waits, exercised without a
 * fault.  Every mbarrier wait in the tensor-core kernels and every
 * dependency wait of the persistent apply gives up after 1 s, sets a device
 * flag and returns (freeing its tensor memory); the host then reports
 * BF_ETIMEOUT.  This call runs one wait of each kind with the limit lowered
 * to limit_ns (0 < limit_ns <= 1e9): a one-warp kernel waiting, through the
 * same wait routine, on an mbarrier that nothing completes, then a one-task
 * persistent apply whose task waits on its own flag; it synchronizes
 * `stream` and returns BF_ETIMEOUT when both waits gave up (the designed
 * outcome: the kernels returned and the context stays usable), BF_OK or
 * BF_EINTERNAL when a wait did not give up.  BF_EINVAL for a limit out of
 * range; BF_ETIMEOUT without running if an earlier wait had already given
 * up.  Diagnostic; not thread-safe against running factorizations (they
 * would see the lowered limit). */
int bf_debug_wait_timeout(uint64_t limit_ns, void* stream);

/* Selects the apply engine for the whole process (bf_apply, bf_apply_T,
 * bf_error; eq. hybrid_butterfly_mat).  Two engines compute bit-identical
 * results:
 *   - stages: L + 3 batched block-product launches plus a gather and a
 *     scatter (kernel shapes per stage as tuned by bf_apply_tune);
 *   - fused: two launches, one CTA per (subtree, column slice) each; the
 *     first carries the input side of the factorization (V^0, W^1..W^(l_m),
 *     B, or for F^H / F^T U^H, R^H levels, B^H) for one subtree of the
 *     input-side tree in shared memory, the second the output side for one
 *     subtree of the output-side tree, with one exchange of the centre-level
 *     vectors between them (the split of the paper's hybrid layout, Sec. 6.2,
 *     on the CTAs of one GPU); the tree permutations and the conjugation of
 *     F^T are folded into the loads and stores; used where a subtree's
 *     intermediates fit in shared memory.
 *   - persistent: the grouped engine's runs (below) in one cooperative
 *     launch: a (group, column slice) task starts once the groups it reads
 *     have written their rows (per-task flags, bounded waits), every run
 *     writes its own rows of one stacked buffer, and a task's factor tiles
 *     are staged while it waits; results equal the stage engine's bit for
 *     bit.
 *   - grouped: the stages in runs of 1-4 consecutive stages, one launch
 *     per run; the blocks of a run fall into small connected groups (for
 *     the W levels and depth 3: 4 + 4 + 4 blocks reading 8 blocks of the
 *     level below; complex64 groups of blocks of rank <= 16 with fewer
 *     last-stage blocks merged up to 4), one CTA per (group, column slice)
 *     copies the group's image --
 *     its descriptors and factor blocks, packed once per plan -- while it
 *     waits for the previous launch, then its input rows, and computes the
 *     run's inner stages in shared memory; ceil((L + 3) / depth) launches,
 *     results equal to the stage engine's bit for bit; the tuner picks the
 *     depth, the merging and the slice width.  The plan's images hold a
 *     packed copy of the factor entries of the direction and dtype plus
 *     descriptors; over mem_cap the plan is not built and the stage
 *     launches serve.
 * engine 0 (default): the engine bf_apply_tune measured fastest for the
 * right-hand-side class; untuned, the stage launches for the first two
 * applies of a factorization in each direction and dtype, then grouped
 * where it applies (its plan takes about a millisecond of host time to
 * build once), at a depth set by the largest block rank (<= 16: 3 for
 * complex64, 2 for complex128; <= 32: 2; else 1); 1: stages only; 2: fused
 * wherever it applies; 3: persistent wherever it applies (not when x and y
 * overlap); 4: grouped wherever it applies.  BF_EINVAL otherwise.  Not
 * thread-safe against running applies. */
int bf_set_apply_engine(int engine);

/* Run depth of the grouped apply engine (diagnostic): 0 (default) the depth
 * bf_apply_tune chose (untuned: from the largest block rank, see
 * bf_set_apply_engine); 1-4 that many stages per launch for
 * every later grouped apply.  BF_EINVAL otherwise.  Not thread-safe against
 * running applies. */
int bf_set_grouped_depth(int depth);

/* Group merging of the grouped apply engine (diagnostic): 0 (default) the
 * merging bf_apply_tune chose (untuned: complex64 groups merged until they
 * hold 4 blocks of their run's last stage when every rank is <= 16, else
 * and for complex128 unmerged);
 * 1-16 groups merged until they hold that many (1: unmerged) in every
 * grouped plan built later (a plan is rebuilt when its depth or merging
 * changes).  Results do not depend on it.  BF_EINVAL otherwise.  Not
 * thread-safe against running applies. */
int bf_set_grouped_merge(int merge);

/* Stage-kernel shape for every apply stage launch in this process
 * (diagnostic): v = -1 (default) uses the shapes bf_apply_tune chose, else
 * the untuned default; v = 0..7 forces that shape (0 many-warp, 1 rows,
 * 2 block, 3-5 wide register tiles, 6-7 staged in shared memory).  Every
 * shape computes the same sums in the same order, so results do not change,
 * bit for bit.  Applies captured in an applier keep the shapes of their
 * capture.  BF_EINVAL outside -1..7.  Not thread-safe against running
 * applies. */
int bf_set_stage_variant(int v);

/* Factorization schedule for the whole process: on = 1 (default) -- the
 * two sides of Alg. 2, the row bases (loop "V" and the W levels) and the
 * column bases (loop "U" and the R levels above the centre), which do not
 * depend on each other until the centre level l_m (Secs. 4.2-4.3), run on
 * two host threads and two streams, joined before the centre level (R^(l_m),
 * X = V^H Omega, the B solve); every phase's launches are the same as in
 * the sequential order, so results are identical.  Used for operators bound
 * to the plan (dense and built-in kernel operators) without a memory cap;
 * others run sequentially.  on = 0 -- always sequential.  BF_EINVAL
 * otherwise.  Not thread-safe against running factorizations. */
int bf_set_parallel_sides(int on);

/* ------------------------------------------------------------- common -- */
/* Frees a bf_plan, bf_fact, bf_operator or bf_applier (NULL-safe). */
void bf_free(void* handle);

/* Reason for the last failure on this thread ("" if none). */
const char* bf_last_error(void);

/* Number of kernels this library has launched in this process so far
 * (all threads, all devices; monotone).  Diagnostic: the difference of two
 * readings around a region is the number of library kernels launched in it.
 * Never fails. */
unsigned long long bf_launch_count(void);

/* Number of host synchronisations this library has made in this process so
 * far (all threads; monotone): every stream or device synchronisation and
 * every synchronous copy to or from the device.  A factorization makes one
 * per QR phase of Alg. 2 (the ranks a phase reveals size the next phase's
 * sketch; the phase's tensor-core wait flag comes back with them), one after
 * the centre level's solve and one at the end of each side; building an
 * apply plan or a tuner run adds its own.  Waits for a slot of the
 * library's pinned upload staging ring (a copy enqueued earlier in the same
 * thread) are not counted.  Diagnostic, like bf_launch_count; never fails. */
unsigned long long bf_sync_count(void);

/* Device-side Gaussian test/sketch matrix of the counter-based generator:
 * G[i, c - col0] for rows row0..row0+rows-1, columns col0..col1-1 of
 * (seed, stream) into a device buffer (ld >= rows), dtype C64/C128. */
int bf_gaussian(uint64_t seed, uint32_t stream_id, int64_t row0, int64_t rows,
                int64_t col0, int64_t col1, void* out, int64_t ld, int dtype,
                void* stream);

#ifdef __cplusplus
}
#endif
#endif /* BUTTERFLY_H */
