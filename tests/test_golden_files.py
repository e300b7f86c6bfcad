"""The stored oracle values of the full-size parity tests (written by
tests/golden/make_goldens.py from oracle/ alone) are what they claim: the
files parse, carry every level's ranks, and their sampled rows of A Omega
are the kernel's own products (recomputed here for a few rows) while the
stored F Omega rows lie within the Thm 5.3 bound 2 sqrt(L+2) eps of them."""
import math
import os
import sys

import numpy as np
import pytest

from oracle import butterfly as ob
from oracle import operators as oo
from paper_2002_03400_gb300 import inputs

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, HERE)
import make_goldens as mg   # noqa: E402


@pytest.mark.parametrize("name,L,lm", [("line_pair_n16384.txt", 10, 5), ("caps_n16384.txt", 8, 4),
                                       ("caps_composition_n16384.txt", 8, 4)])
def test_stored_file_is_consistent(name, L, lm):
    d = mg.read(os.path.join(HERE, name))
    assert d["L"] == L and d["lm"] == lm
    assert sorted(d["rV"]) == list(range(lm + 1)) and sorted(d["rU"]) == list(range(lm, L + 1))
    for r in list(d["rV"].values()) + list(d["rU"].values()):
        assert r.shape == (1 << L,) and r.min() >= 1
    assert d["F"].shape == (mg.ROW_SAMPLE, mg.PROBE_COLS) and d["A"].shape == d["F"].shape
    assert np.array_equal(d["rows"], mg.sample_rows(mg.N))
    gap = np.linalg.norm(d["F"] - d["A"]) / np.linalg.norm(d["A"])
    assert gap <= 2 * math.sqrt(L + 2) * 1e-6, gap


@pytest.mark.parametrize("name", ["line_pair_n16384.txt", "caps_n16384.txt"])
def test_stored_exact_rows_are_kernel_products(name):
    d = mg.read(os.path.join(HERE, name))
    Om = ob.error_probe(mg.N, mg.PROBE_SEED, mg.PROBE_COLS)
    rows = d["rows"][:8]
    if name.startswith("line"):
        g = inputs.line_pair(mg.N)
        want = oo.kernel_entries(oo.HELMHOLTZ_2D, g.wavenumber, g.tgt[rows], g.src) @ Om
    else:
        P1, P2, _, k = mg.cap_triple(mg.N)
        want = oo.kernel_entries(oo.HELMHOLTZ_3D, k, P2[rows], P1) @ Om
    assert np.linalg.norm(d["A"][:8] - want) <= 1e-10 * np.linalg.norm(want)
