"""Thin ctypes binding over libbutterfly.so (include/butterfly.h).

Argument marshalling only: every step of the factorization and apply runs in
the library's CUDA kernels.  Tensors are torch CUDA tensors; matrices are
passed column-major (a (rows, cols) tensor with stride(0) == 1), which this
module arranges.  Importing it loads the library and raises if it is missing
-- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbutterfly.so")

BF_C64, BF_C128 = 0, 1
OPS = {"N": 0, "T": 1, "C": 2}
PREC = {"fp64": 0, "mixed": 1}
KERNELS = {"none": 0, "helmholtz2d": 1, "helmholtz3d": 2, "dft": 3}
STATUS = {0: "BF_OK", -1: "BF_EINVAL", -2: "BF_ENOMEM", -3: "BF_ECALLBACK", -4: "BF_ENOTCONVERGED",
          -5: "BF_ECUDA", -6: "BF_ETIMEOUT", -7: "BF_EUNSUPPORTED", -8: "BF_EINTERNAL"}


class BFError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Options(C.Structure):
    _fields_ = [("p", C.c_int), ("r0", C.c_int), ("r_max", C.c_int), ("seed", C.c_uint64),
                ("precision", C.c_int), ("mem_cap", C.c_size_t), ("qr_fp64", C.c_int),
                ("hybrid_level", C.c_int), ("accept_retries", C.c_int), ("leaf_passes", C.c_int)]


class KernelDesc(C.Structure):
    _fields_ = [("type", C.c_int), ("wavenumber", C.c_double)]


MATVEC_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int, C.c_int64, C.c_void_p, C.c_int64,
                        C.c_void_p, C.c_int64, C.c_int, C.c_void_p)

_lib = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run paper_2002_03400_gb300/build.py (no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double
    sig = {
        "bf_options_default": (None, [C.POINTER(Options)]),
        "bf_last_error": (C.c_char_p, []),
        "bf_plan_create": (i32, [vp, i64, vp, i64, i32, C.POINTER(KernelDesc), i32, dbl, C.POINTER(Options), C.POINTER(vp)]),
        "bf_bisect": (i32, [vp, i64, i32, i32, vp, vp]),
        "bf_plan_info": (i32, [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i64), C.POINTER(i64)]),
        "bf_plan_trees": (i32, [vp, vp, vp, vp, vp]),
        "bf_operator_dense": (i32, [vp, vp, i64, i32, vp, C.POINTER(vp)]),
        "bf_operator_kernel": (i32, [vp, C.POINTER(vp)]),
        "bf_operator_kernel_cached": (i32, [vp, vp, C.POINTER(vp)]),
        "bf_operator_factored": (i32, [vp, C.POINTER(vp)]),
        "bf_operator_composed": (i32, [vp, vp, C.POINTER(vp)]),
        "bf_operator_callback": (i32, [i64, i64, MATVEC_FN, vp, C.POINTER(vp)]),
        "bf_operator_apply": (i32, [vp, i32, i64, vp, i64, vp, i64, i32, vp]),
        "bf_operator_counts": (i32, [vp, C.POINTER(i64), C.POINTER(i64)]),
        "bf_factor": (i32, [vp, vp, vp, C.POINTER(vp)]),
        "bf_factor_batch": (i32, [i32, C.POINTER(vp), C.POINTER(vp), vp, C.POINTER(vp)]),
        "bf_apply": (i32, [vp, i64, vp, i64, vp, i64, i32, vp]),
        "bf_apply_T": (i32, [vp, i32, i64, vp, i64, vp, i64, i32, vp]),
        "bf_apply_noalloc": (i32, [vp, i32, i64, vp, i64, vp, i64, i32, vp]),
        "bf_ranks": (i32, [vp, i32, i32, vp]),
        "bf_fact_info": (i32, [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(dbl)]),
        "bf_fact_import": (i32, [vp, vp, vp, C.POINTER(vp), i32, C.POINTER(vp)]),
        "bf_fact_export": (i32, [vp, i32, vp, C.POINTER(C.c_size_t)]),
        "bf_fact_save": (i32, [vp, C.c_char_p]),
        "bf_fact_load": (i32, [vp, C.c_char_p, C.POINTER(vp)]),
        "bf_error": (i32, [vp, vp, i32, C.c_uint64, i32, vp, C.POINTER(dbl)]),
        "bf_free": (None, [vp]),
        "bf_set_sketch_engine": (i32, [i32]),
        "bf_set_entry_images": (i32, [i32]),
        "bf_set_apply_engine": (i32, [i32]),
        "bf_set_stage_variant": (i32, [i32]),
        "bf_set_grouped_depth": (i32, [i32]),
        "bf_set_grouped_merge": (i32, [i32]),
        "bf_set_parallel_sides": (i32, [i32]),
        "bf_launch_count": (C.c_ulonglong, []),
        "bf_sync_count": (C.c_ulonglong, []),
        "bf_apply_tune": (i32, [vp, i32, i64, i32, vp, C.POINTER(C.c_float)]),
        "bf_applier_create": (i32, [vp, i32, i64, i32, C.POINTER(vp)]),
        "bf_applier_run": (i32, [vp, vp, i64, vp, i64, vp]),
        "bf_gaussian": (i32, [C.c_uint64, C.c_uint32, i64, i64, i64, i64, vp, i64, i32, vp]),
        "bf_fact_accept": (i32, [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(dbl)]),
        "bf_debug_wait_timeout": (i32, [C.c_uint64, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def exported_symbols():
    """Names declared in include/butterfly.h that the binding expects."""
    return ["bf_options_default", "bf_last_error", "bf_bisect", "bf_plan_create", "bf_plan_info", "bf_plan_trees",
            "bf_operator_dense", "bf_operator_kernel", "bf_operator_kernel_cached", "bf_operator_factored", "bf_operator_composed",
            "bf_operator_callback", "bf_operator_apply", "bf_operator_counts", "bf_factor",
            "bf_factor_batch", "bf_apply",
            "bf_apply_T", "bf_apply_noalloc", "bf_ranks", "bf_fact_info", "bf_fact_import", "bf_fact_export", "bf_fact_save", "bf_fact_load", "bf_error",
            "bf_free", "bf_gaussian", "bf_set_sketch_engine", "bf_set_entry_images", "bf_launch_count", "bf_apply_tune",
            "bf_applier_create", "bf_applier_run", "bf_fact_accept", "bf_debug_wait_timeout",
            "bf_set_apply_engine", "bf_set_stage_variant", "bf_set_grouped_depth", "bf_set_grouped_merge", "bf_set_parallel_sides", "bf_sync_count"]


def launch_count() -> int:
    """Kernels the library has launched in this process so far."""
    return int(lib().bf_launch_count())


def sync_count() -> int:
    """Host synchronisations the library's factorizations have made so far."""
    return int(lib().bf_sync_count())


def set_sketch_engine(engine: str):
    """'tensor' (default: tcgen05 with the exact three-way bf16 split),
    'simt', 'tensor-3xtf32' (two TF32 parts) or 'tensor-split3' (the
    exact three-way bf16 split, as the default)."""
    check(lib().bf_set_sketch_engine({"tensor": 0, "simt": 1, "tensor-3xtf32": 2, "tensor-split3": 3}[engine]))


def set_entry_images(on: bool):
    """Entry images on (default: a mixed-precision factorization of a built-in
    kernel operator forms its entries once, bf16-split, and every sketch reads
    them) or off (entries formed on the fly in every sketch)."""
    check(lib().bf_set_entry_images(1 if on else 0))


def debug_wait_timeout(limit_ns: int, stream=None) -> int:
    """Status of one bounded wait that nothing completes, run with its limit
    lowered to limit_ns (bf_debug_wait_timeout): -6 (BF_ETIMEOUT) is the
    designed outcome."""
    return int(lib().bf_debug_wait_timeout(int(limit_ns), _stream(stream)))


def set_parallel_sides(on: bool):
    """Run the two sides of Alg. 2 (row bases and column bases) concurrently
    on two host threads and streams (default) or one after the other."""
    check(lib().bf_set_parallel_sides(1 if on else 0))


def set_apply_engine(engine: str):
    """'auto' (default: the engine bf_apply_tune measured fastest for the
    right-hand-side class; untuned: the stage launches for a factorization's
    first two applies, then the grouped engine where it applies), 'stages',
    'fused', 'persistent' or 'grouped' (the last three wherever they
    apply)."""
    check(lib().bf_set_apply_engine({"auto": 0, "stages": 1, "fused": 2, "persistent": 3, "grouped": 4}[engine]))


def set_stage_variant(v: int):
    """Stage-kernel shape for every apply stage: -1 (default) tuned or
    default shapes, 0..7 that shape everywhere (results do not change)."""
    check(lib().bf_set_stage_variant(int(v)))


STAGE_VARIANTS = 8


def set_grouped_depth(depth: int):
    """Stages per launch of the grouped apply engine: 0 (default) the tuned
    depth (untuned: set by the largest block rank), 1..4 that depth for every
    later grouped apply."""
    check(lib().bf_set_grouped_depth(int(depth)))


def set_grouped_merge(merge: int):
    """Group merging of the grouped apply engine: 0 (default) the tuned
    choice (untuned: complex64 groups merged up to 4 last-stage blocks when
    every rank is <= 16),
    1..16 groups merged up to that many blocks (1: unmerged) in every grouped
    plan built later; results do not depend on it."""
    check(lib().bf_set_grouped_merge(int(merge)))


def check(rc: int):
    if rc != 0:
        raise BFError(rc, lib().bf_last_error().decode())


def _dt(t: torch.Tensor) -> int:
    if t.dtype == torch.complex128:
        return BF_C128
    if t.dtype == torch.complex64:
        return BF_C64
    raise TypeError(f"complex64 or complex128 expected, got {t.dtype}")


def _tdtype(d: int):
    return torch.complex128 if d == BF_C128 else torch.complex64


def colmajor(x: torch.Tensor) -> torch.Tensor:
    """View of x (rows, cols) whose memory is column-major (stride(0) == 1)."""
    if x.dim() == 1:
        x = x.reshape(-1, 1)
    if x.stride(0) == 1 and (x.shape[1] <= 1 or x.stride(1) >= x.shape[0]):
        return x
    return x.t().contiguous().t()


def empty_cm(rows: int, cols: int, dtype, device="cuda") -> torch.Tensor:
    return torch.empty((cols, rows), dtype=dtype, device=device).t()


def _ld(x: torch.Tensor) -> int:
    return max(x.stride(1) if x.shape[1] > 1 else x.shape[0], x.shape[0], 1)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class _Handle:
    _h = None

    def free(self):
        if self._h:
            lib().bf_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Plan(_Handle):
    """Trees and parameters (bf_plan_create)."""

    def __init__(self, src=None, tgt=None, n=None, m=None, kernel="none", wavenumber=0.0, leaf=16,
                 tol=1e-6, p=2, r0=4, r_max=1024, seed=0, precision="fp64", mem_cap=0,
                 qr_fp64=False, hybrid_level=-1, accept_retries=0, leaf_passes=0):
        L = lib()
        opt = Options()
        L.bf_options_default(C.byref(opt))
        opt.p, opt.r0, opt.r_max, opt.seed = p, r0, r_max, seed
        opt.precision = PREC[precision] if isinstance(precision, str) else int(precision)
        opt.mem_cap = mem_cap
        opt.qr_fp64 = 1 if qr_fp64 else 0
        opt.hybrid_level, opt.accept_retries, opt.leaf_passes = hybrid_level, accept_retries, leaf_passes
        kd = KernelDesc(KERNELS[kernel] if isinstance(kernel, str) else int(kernel), float(wavenumber))
        self._keep = []
        if src is not None:
            s = np.ascontiguousarray(src, dtype=np.float64)
            t = np.ascontiguousarray(tgt, dtype=np.float64)
            if s.ndim == 1:
                s = s.reshape(-1, 1)
                t = t.reshape(-1, 1)
            n, m, dim = s.shape[0], t.shape[0], s.shape[1]
            self._keep = [s, t]
            sp, tp = s.ctypes.data_as(C.c_void_p), t.ctypes.data_as(C.c_void_p)
        else:
            m = n if m is None else m
            dim, sp, tp = 0, None, None
        h = C.c_void_p()
        check(L.bf_plan_create(sp, n, tp, m, dim, C.byref(kd), leaf, tol, C.byref(opt), C.byref(h)))
        self._h = h
        self.precision = opt.precision
        Lv, lm, nn, mm = C.c_int(), C.c_int(), C.c_int64(), C.c_int64()
        check(L.bf_plan_info(h, C.byref(Lv), C.byref(lm), C.byref(nn), C.byref(mm)))
        self.L, self.lm, self.n, self.m = Lv.value, lm.value, nn.value, mm.value

    def trees(self):
        nlev = sum((1 << l) + 1 for l in range(self.L + 1))
        pS = np.empty(self.n, dtype=np.int64)
        pT = np.empty(self.m, dtype=np.int64)
        oS = np.empty(nlev, dtype=np.int64)
        oT = np.empty(nlev, dtype=np.int64)
        check(lib().bf_plan_trees(self._h, pS.ctypes.data, pT.ctypes.data, oS.ctypes.data, oT.ctypes.data))
        offS, offT, q = [], [], 0
        for l in range(self.L + 1):
            offS.append(oS[q:q + (1 << l) + 1].copy())
            offT.append(oT[q:q + (1 << l) + 1].copy())
            q += (1 << l) + 1
        return pS, offS, pT, offT


class Operator(_Handle):
    """Black-box A (bf_operator_*)."""

    def __init__(self, handle, m, n, keep=()):
        self._h = handle
        self.m, self.n = m, n
        self._keep = list(keep)

    @classmethod
    def dense(cls, plan: Plan, A: torch.Tensor, stream=None):
        A = colmajor(A)
        h = C.c_void_p()
        check(lib().bf_operator_dense(plan._h, C.c_void_p(A.data_ptr()), _ld(A), _dt(A), _stream(stream), C.byref(h)))
        return cls(h, plan.m, plan.n, keep=[plan])

    @classmethod
    def kernel(cls, plan: Plan, cached: bool = False, stream=None):
        """Built-in kernel operator; cached=True keeps its entries resident
        as complex64 entry images (bf_operator_kernel_cached)."""
        h = C.c_void_p()
        if cached:
            check(lib().bf_operator_kernel_cached(plan._h, _stream(stream), C.byref(h)))
        else:
            check(lib().bf_operator_kernel(plan._h, C.byref(h)))
        return cls(h, plan.m, plan.n, keep=[plan])

    @classmethod
    def factored(cls, F: "Factorization"):
        h = C.c_void_p()
        check(lib().bf_operator_factored(F._h, C.byref(h)))
        return cls(h, F.m, F.n, keep=[F])

    @classmethod
    def composed(cls, A1: "Operator", A2: "Operator"):
        h = C.c_void_p()
        check(lib().bf_operator_composed(A1._h, A2._h, C.byref(h)))
        return cls(h, A1.m, A2.n, keep=[A1, A2])

    @classmethod
    def callback(cls, m: int, n: int, fn):
        """fn(op, ncols, X_ptr, ldx, Y_ptr, ldy, dtype, stream_ptr) -> int (0 = ok)."""
        def tramp(ctx, op, ncols, X, ldx, Y, ldy, dtype, stream):
            try:
                return int(fn(op, ncols, X, ldx, Y, ldy, dtype, stream))
            except Exception:
                return 99
        cfn = MATVEC_FN(tramp)
        h = C.c_void_p()
        check(lib().bf_operator_callback(m, n, cfn, None, C.byref(h)))
        return cls(h, m, n, keep=[cfn])

    def apply(self, X: torch.Tensor, op: str = "N", stream=None) -> torch.Tensor:
        X = colmajor(X)
        rows = self.m if op == "N" else self.n
        Y = empty_cm(rows, X.shape[1], X.dtype, X.device)
        check(lib().bf_operator_apply(self._h, OPS[op], X.shape[1], C.c_void_p(X.data_ptr()), _ld(X),
                                      C.c_void_p(Y.data_ptr()), _ld(Y), _dt(X), _stream(stream)))
        return Y

    def counts(self):
        a, b = C.c_int64(), C.c_int64()
        check(lib().bf_operator_counts(self._h, C.byref(a), C.byref(b)))
        return a.value, b.value


class Factorization(_Handle):
    """A resident hybrid butterfly factorization (bf_factor / bf_fact_import)."""

    def __init__(self, handle, plan: Plan):
        self._h = handle
        self.plan = plan
        self.m, self.n, self.L, self.lm = plan.m, plan.n, plan.L, plan.lm

    @classmethod
    def factor(cls, plan: Plan, A: Operator | None = None, stream=None):
        h = C.c_void_p()
        check(lib().bf_factor(plan._h, A._h if A is not None else None, _stream(stream), C.byref(h)))
        F = cls(h, plan)
        F._op = A
        return F

    def save(self, path: str):
        """bf_fact_save: a checkpoint file of this factorization."""
        check(lib().bf_fact_save(self._h, str(path).encode()))

    @classmethod
    def load(cls, plan: Plan, path: str):
        """bf_fact_load: a factorization saved by save(), for `plan`."""
        h = C.c_void_p()
        check(lib().bf_fact_load(plan._h, str(path).encode(), C.byref(h)))
        return cls(h, plan)

    @classmethod
    def factor_batch(cls, plans: list, ops: list | None = None, stream=None) -> list:
        """bf_factor_batch: all operators level-synchronously, one launch per
        kernel per phase."""
        cnt = len(plans)
        ph = (C.c_void_p * cnt)(*[p._h.value for p in plans])
        oh = None
        if ops is not None:
            oh = (C.c_void_p * cnt)(*[(o._h.value if o is not None else None) for o in ops])
        out = (C.c_void_p * cnt)()
        check(lib().bf_factor_batch(cnt, ph, oh, _stream(stream), out))
        res = []
        for i in range(cnt):
            F = cls(C.c_void_p(out[i]), plans[i])
            F._op = ops[i] if ops is not None else None
            res.append(F)
        return res

    @classmethod
    def import_blocks(cls, plan: Plan, rV: np.ndarray, rU: np.ndarray, stages: list):
        rV = np.ascontiguousarray(rV, dtype=np.int32)
        rU = np.ascontiguousarray(rU, dtype=np.int32)
        bufs = [np.ascontiguousarray(s, dtype=np.complex128) for s in stages]
        arr = (C.c_void_p * len(bufs))(*[b.ctypes.data for b in bufs])
        h = C.c_void_p()
        check(lib().bf_fact_import(plan._h, rV.ctypes.data, rU.ctypes.data, arr, BF_C128, C.byref(h)))
        return cls(h, plan)

    def apply(self, x: torch.Tensor, op: str = "N", stream=None) -> torch.Tensor:
        x = colmajor(x)
        rows = self.m if op == "N" else self.n
        y = empty_cm(rows, x.shape[1], x.dtype, x.device)
        args = (x.shape[1], C.c_void_p(x.data_ptr()), _ld(x), C.c_void_p(y.data_ptr()), _ld(y), _dt(x), _stream(stream))
        if op == "N":
            check(lib().bf_apply(self._h, *args))
        else:
            check(lib().bf_apply_T(self._h, OPS[op], *args))
        return y

    def apply_into(self, x: torch.Tensor, y: torch.Tensor, op: str = "N", stream=None):
        """Apply with caller-provided column-major buffers (no allocation here)."""
        args = (x.shape[1], C.c_void_p(x.data_ptr()), _ld(x), C.c_void_p(y.data_ptr()), _ld(y), _dt(x), _stream(stream))
        if op == "N":
            check(lib().bf_apply(self._h, *args))
        else:
            check(lib().bf_apply_T(self._h, OPS[op], *args))

    def tune(self, nrhs: int, dtype=torch.complex64, op: str = "N", stream=None) -> float:
        """Autotunes the apply's stage kernels for this right-hand-side class;
        returns the tuned device time of one apply in ms."""
        ms = C.c_float()
        dt = 0 if dtype == torch.complex64 else 1
        check(lib().bf_apply_tune(self._h, OPS[op], nrhs, dt, _stream(stream), C.byref(ms)))
        return ms.value

    def applier(self, nrhs: int, dtype=torch.complex64, op: str = "N") -> "Applier":
        """A graph-captured apply for nrhs right-hand sides (bf_applier)."""
        return Applier(self, nrhs, dtype, op)

    def ranks(self, side: int, level: int) -> np.ndarray:
        out = np.empty(1 << self.L, dtype=np.int32)
        check(lib().bf_ranks(self._h, side, level, out.ctypes.data))
        return out

    def info(self) -> dict:
        s, a, b, t = C.c_int64(), C.c_int64(), C.c_int64(), C.c_double()
        check(lib().bf_fact_info(self._h, C.byref(s), C.byref(a), C.byref(b), C.byref(t)))
        return {"stored_entries": s.value, "cols_N": a.value, "cols_T": b.value, "seconds": t.value}

    def accept_info(self) -> dict:
        """A-posteriori acceptance record (bf_fact_accept)."""
        a, r, e = C.c_int(), C.c_int(), C.c_double()
        check(lib().bf_fact_accept(self._h, C.byref(a), C.byref(r), C.byref(e)))
        return {"attempts": a.value, "r0": r.value, "sketch_error": e.value}

    def export_stage(self, stage: int) -> np.ndarray:
        nb = C.c_size_t(0)
        check(lib().bf_fact_export(self._h, stage, None, C.byref(nb)))
        out = np.empty(nb.value // 16, dtype=np.complex128)
        check(lib().bf_fact_export(self._h, stage, out.ctypes.data, C.byref(nb)))
        return out

    def error(self, A: Operator, ncols: int = 16, seed: int = 0, dtype=torch.complex128, stream=None) -> float:
        e = C.c_double()
        d = BF_C128 if dtype == torch.complex128 else BF_C64
        check(lib().bf_error(self._h, A._h, ncols, seed, d, _stream(stream), C.byref(e)))
        return e.value


def bisect(points, count: int, L: int):
    """Host-only tree build (bf_bisect): (perm, [off per level])."""
    if points is not None:
        pts = np.ascontiguousarray(points, dtype=np.float64)
        if pts.ndim == 1:
            pts = pts.reshape(-1, 1)
        pp, dim = pts.ctypes.data_as(C.c_void_p), pts.shape[1]
    else:
        pts, pp, dim = None, None, 0
    perm = np.empty(count, dtype=np.int64)
    off = np.empty(sum((1 << l) + 1 for l in range(L + 1)), dtype=np.int64)
    check(lib().bf_bisect(pp, count, dim, L, perm.ctypes.data, off.ctypes.data))
    out, q = [], 0
    for l in range(L + 1):
        out.append(off[q:q + (1 << l) + 1].copy())
        q += (1 << l) + 1
    return perm, out


def gaussian(seed: int, stream_id: int, rows: int, col0: int, col1: int, dtype=torch.complex128,
             row0: int = 0, stream=None) -> torch.Tensor:
    """Device Gaussian matrix of the library's counter-based generator."""
    out = empty_cm(rows, col1 - col0, dtype)
    check(lib().bf_gaussian(seed, stream_id, row0, rows, col0, col1, C.c_void_p(out.data_ptr()), max(rows, 1),
                            _dt(out), _stream(stream)))
    return out


def exact_factorization(plan: Plan, eb) -> Factorization:
    """Imports an exactly-butterfly operator (inputs.ExactButterfly) whose
    block order matches the plan's index-order trees."""
    L, lm, nb, r = eb.L, eb.lm, 1 << eb.L, eb.r
    rV = np.full((lm + 1, nb), r, dtype=np.int32)
    rU = np.full((L - lm + 1, nb), r, dtype=np.int32)
    cm = lambda blocks: np.concatenate([np.asfortranarray(b).ravel(order="F") for b in blocks])
    stages = [cm(eb.V0)]
    stages += [cm(eb.W[j]) for j in range(1, lm + 1)]
    stages += [cm(eb.B)]
    stages += [cm(eb.R[j]) for j in range(lm, L)]
    stages += [cm(eb.U)]
    return Factorization.import_blocks(plan, rV, rU, stages)


class Applier(_Handle):
    """bf_applier: the apply's stage chain captured once into a CUDA graph;
    run() gathers x, launches the graph and scatters into y."""

    def __init__(self, F: Factorization, nrhs: int, dtype=torch.complex64, op: str = "N"):
        h = C.c_void_p()
        dt = BF_C64 if dtype == torch.complex64 else BF_C128
        check(lib().bf_applier_create(F._h, OPS[op], nrhs, dt, C.byref(h)))
        self._h = h
        self._keep = [F]
        self.nrhs, self.dtype, self.op = nrhs, dtype, op
        self.rows_out = F.m if op == "N" else F.n

    def run(self, x: torch.Tensor, y: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        x = colmajor(x)
        if x.shape[1] != self.nrhs or x.dtype != self.dtype:
            raise ValueError("x does not match the applier's column count or dtype")
        if y is None:
            y = empty_cm(self.rows_out, self.nrhs, x.dtype, x.device)
        check(lib().bf_applier_run(self._h, C.c_void_p(x.data_ptr()), _ld(x), C.c_void_p(y.data_ptr()), _ld(y),
                                   _stream(stream)))
        return y
