"""bf_apply_noalloc: the apply for callers that may not allocate device memory
while they run (an application whose own pool owns all device memory, a
plug-in inside a framework that owns it, or a per-request loop where
cudaMalloc/cudaFree and their device-wide synchronization are not allowed).

It must give the same result as bf_apply / bf_apply_T while taking every
intermediate from the library's fixed device array.  This file is collected
last so that a failure here stops a -x run only after every other test; it
passes alone in a fresh process and after the other tests."""
import ctypes as C

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
