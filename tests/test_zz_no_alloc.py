"""bf_apply_noalloc: the apply for callers that may not allocate device memory
while they run (an application whose own pool owns all device memory, a
plug-in inside a framework that owns it, or a per-request loop where
cudaMalloc/cudaFree and their device-wide synchronization are not allowed).

It must give the same result as bf_apply / bf_apply_T while taking every
intermediate from the library's fixed device array.  This file is collected
last so that a failure here stops a -x run only after every other test; it
passes alone in a fresh process and after the other tests."""
import ctypes as C
import ctypes.util
import os

import numpy as np
import pytest
import torch

from paper_2002_03400_gb300 import api, inputs

pytestmark = pytest.mark.gpu


def _noalloc(F, op, x, y):
    L = api.lib()
    s = torch.cuda.current_stream().cuda_stream
    return L.bf_apply_noalloc(F._h, api.OPS[op], x.shape[1], C.c_void_p(x.data_ptr()), api._ld(x),
                              C.c_void_p(y.data_ptr()), api._ld(y), api._dt(x), C.c_void_p(s))


def _cudart():
    """The CUDA runtime (for the device's default memory pool, where every
    stream-ordered allocation of the library lands)."""
    for name in ("/usr/local/cuda/lib64/libcudart.so", ctypes.util.find_library("cudart")):
        if name and (os.path.exists(name) or not name.startswith("/")):
            try:
                return C.CDLL(name)
            except OSError:
                pass
    pytest.skip("libcudart not found")


def _pool_high(rt, reset):
    """High-water mark of bytes in use in the current device's default pool
    (cudaMemPoolAttrUsedMemHigh = 8); reset=True lowers it to the current use
    first, so a later rise means something was allocated in between."""
    dev = C.c_int(0)
    assert rt.cudaGetDevice(C.byref(dev)) == 0
    pool = C.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(C.byref(pool), dev) == 0
    v = C.c_uint64(0)
    if reset:
        assert rt.cudaMemPoolSetAttribute(pool, 8, C.byref(v)) == 0
    assert rt.cudaMemPoolGetAttribute(pool, 8, C.byref(v)) == 0
    cur = C.c_uint64(0)
    assert rt.cudaMemPoolGetAttribute(pool, 7, C.byref(cur)) == 0   # UsedMemCurrent
    return v.value, cur.value


def _rel(a, b):
    torch.cuda.synchronize()
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("op", ["N", "T", "C"])
def test_noalloc_matches_bf_apply_on_two_calls(op):
    n, leaf, r, nrhs = 2048, 32, 8, 7
    eb = inputs.exact_butterfly(n, leaf, r, seed=1)
    F = api.exact_factorization(api.Plan(n=n, leaf=leaf), eb)
    x = api.colmajor(torch.from_numpy(inputs.random_rhs(n, nrhs, seed=2)).cuda())
    outs = []
    # first call before bf_apply has built this factorization's task lists,
    # second call after
    y1 = api.empty_cm(n, nrhs, torch.complex128)
    assert _noalloc(F, op, x, y1) == 0, api.lib().bf_last_error()
    ref = F.apply(x, op)
    y2 = api.empty_cm(n, nrhs, torch.complex128)
    y2.fill_(float("nan"))
    assert _noalloc(F, op, x, y2) == 0, api.lib().bf_last_error()
    for y in (y1, y2):
        assert _rel(y, ref) <= 1e-13


def test_noalloc_permuted_plan_complex64_and_limits():
    """Non-identity trees (gather/scatter through the array), complex64 from
    a mixed-precision factorization, and the size limit."""
    g = inputs.cap_pair(700, m=650)
    plan = api.Plan(g.src, g.tgt, kernel=g.kernel, wavenumber=g.wavenumber, leaf=24, tol=1e-6,
                    precision="mixed")
    F = api.Factorization.factor(plan, api.Operator.kernel(plan))
    for dt, tol in ((torch.complex64, 1e-6), (torch.complex128, 1e-13)):
        x = api.colmajor(torch.from_numpy(inputs.random_rhs(700, 5, seed=3)).to(dt).cuda())
        ref = F.apply(x)
        for _ in range(2):
            y = api.empty_cm(650, 5, dt)
            assert _noalloc(F, "N", x, y) == 0, api.lib().bf_last_error()
            assert _rel(y, ref) <= tol
    # a request above BF_NOALLOC_SCRATCH_BYTES is refused before any GPU work
    x = api.empty_cm(700, 1, torch.complex128)
    big = C.c_int64(1 << 22)
    L = api.lib()
    rc = L.bf_apply_noalloc(F._h, 0, big, C.c_void_p(x.data_ptr()), 700, C.c_void_p(x.data_ptr()), 700,
                            api.BF_C128, None)
    assert rc == -1 and b"BF_NOALLOC_SCRATCH_BYTES" in L.bf_last_error()
    # complex64 on a factorization that has no complex64 copy is refused
    eb = inputs.exact_butterfly(512, 16, 4, seed=5)
    F64 = api.exact_factorization(api.Plan(n=512, leaf=16), eb)
    x32 = api.empty_cm(512, 2, torch.complex64)
    assert _noalloc(F64, "N", x32, api.empty_cm(512, 2, torch.complex64)) == -1


def test_noalloc_allocates_nothing_and_refuses_wrapping_sizes():
    """The defining property: neither the uncached first call (task lists
    built on the host and copied into the array) nor a cached call takes
    memory from the device's pool -- its high-water mark does not move.
    And a column count whose byte size would wrap a 64-bit product is
    refused before any GPU work."""
    rt = _cudart()
    n, leaf, r, nrhs = 1024, 16, 6, 9
    eb = inputs.exact_butterfly(n, leaf, r, seed=7)
    F = api.exact_factorization(api.Plan(n=n, leaf=leaf), eb)
    x = api.colmajor(torch.from_numpy(inputs.random_rhs(n, nrhs, seed=8)).cuda())
    y = api.empty_cm(n, nrhs, torch.complex128)
    for op in ("C", "N"):                  # C: uncached task lists, N: cached below
        if op == "N":
            F.apply(x)                         # caches the op-N lists (allocates, outside the window)
        torch.cuda.synchronize()
        _pool_high(rt, reset=True)
        base_high, base_cur = _pool_high(rt, reset=False)
        assert _noalloc(F, op, x, y) == 0, api.lib().bf_last_error()
        torch.cuda.synchronize()
        high, cur = _pool_high(rt, reset=False)
        assert high <= max(base_high, base_cur) and cur == base_cur, (op, base_high, high, base_cur, cur)
    L = api.lib()
    for big in (1 << 60, (1 << 62) + 3, (1 << 31)):
        rc = L.bf_apply_noalloc(F._h, 0, C.c_int64(big), C.c_void_p(x.data_ptr()), n, C.c_void_p(y.data_ptr()), n,
                                api.BF_C128, None)
        assert rc == -1 and b"BF_NOALLOC_SCRATCH_BYTES" in L.bf_last_error(), big
