"""CPU tests of the C-ABI library: it builds, loads without a GPU, exports
every entry point include/butterfly.h declares, and its host-only logic
(the bisection trees of Sec. 3.1) matches the oracle bit for bit."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2002_03400_gb300 import build
    return build.build()


def _declared():
    src = open(os.path.join(ROOT, "include", "butterfly.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*|unsigned long long)\s+\**(bf_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_planned_entry_points():
    names = _declared()
    for need in ("bf_plan_create", "bf_factor", "bf_apply", "bf_apply_T", "bf_free", "bf_ranks"):
        assert need in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2002_03400_gb300 import api
    assert sorted(api.exported_symbols()) == _declared()


def test_options_defaults_and_error_string(libpath):
    from paper_2002_03400_gb300 import api
    o = api.Options()
    api.lib().bf_options_default(ctypes.byref(o))
    assert (o.p, o.r0, o.r_max, o.seed, o.precision, o.mem_cap, o.qr_fp64) == (2, 4, 1024, 0, 0, 0, 0)
    assert (o.hybrid_level, o.accept_retries, o.leaf_passes) == (-1, 0, 0)
    rc = api.lib().bf_bisect(None, 0, 0, 3, None, None)
    assert rc == -1 and b"bad arguments" in api.lib().bf_last_error()


@pytest.mark.parametrize("kind,count,L", [("line", 1024, 6), ("caps", 777, 5), ("arcs", 1000, 6),
                                          ("index", 999, 4), ("dft", 256, 4), ("hemi_src", 1500, 7),
                                          ("hemi_tgt", 1023, 6)])
def test_host_bisection_matches_oracle(libpath, kind, count, L):
    from oracle.tree import bisect as obisect
    from paper_2002_03400_gb300 import api, inputs
    g = {"line": lambda: inputs.line_pair(count).src, "caps": lambda: inputs.cap_pair(count).tgt,
         "arcs": lambda: inputs.arc_pair(count, 3).tgt, "index": lambda: None,
         "dft": lambda: inputs.dft_points(count).tgt, "hemi_src": lambda: inputs.hemisphere_pair(count).src,
         "hemi_tgt": lambda: inputs.hemisphere_pair(count).tgt}[kind]()
    p, off = api.bisect(g, count, L)
    po, offo = obisect(g, count, L)
    assert np.array_equal(p, po)
    for a, b in zip(off, offo):
        assert np.array_equal(a, b)


def test_plan_rejects_bad_sizes_without_touching_the_gpu(libpath):
    from paper_2002_03400_gb300 import api
    h = ctypes.c_void_p()
    L = api.lib()
    assert L.bf_plan_create(None, 0, None, 4, 0, None, 4, 1e-6, None, ctypes.byref(h)) == -1
    assert L.bf_plan_create(None, 16, None, 16, 0, None, 16, 1e-6, None, ctypes.byref(h)) == -1   # L = 0
    assert L.bf_plan_create(None, 64, None, 64, 0, None, 8, -1.0, None, ctypes.byref(h)) == -1
    assert not h.value
