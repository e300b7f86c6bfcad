"""Pins for oracle.tree (Sec. 3.1): complete bisection trees."""
import numpy as np
import pytest

from oracle.tree import bisect, depth_for_leaf
from paper_2002_03400_gb300 import inputs


def _check_tree(perm, off, count, L):
    assert sorted(perm.tolist()) == list(range(count))          # a permutation
    for lev in range(L + 1):
        o = off[lev]
        assert len(o) == (1 << lev) + 1 and o[0] == 0 and o[-1] == count
        sizes = np.diff(o)
        assert sizes.min() >= 1
        if lev < L:                                             # children split parent: ceil / floor
            ch = np.diff(off[lev + 1])
            assert np.array_equal(ch[0::2] + ch[1::2], sizes)
            assert np.array_equal(ch[0::2], (sizes + 1) // 2)


def test_depth_for_leaf():
    assert depth_for_leaf(1024, 16) == 6
    assert depth_for_leaf(16384, 32) == 9
    assert depth_for_leaf(1000, 16) == 6
    assert depth_for_leaf(16, 16) == 0


@pytest.mark.parametrize("n", [64, 1000, 1024])
def test_index_order(n):
    L = depth_for_leaf(n, 16)
    perm, off = bisect(None, n, L)
    _check_tree(perm, off, n, L)
    assert np.array_equal(perm, np.arange(n))


def test_line_is_identity_and_caps_split_at_median():
    g = inputs.line_pair(256)
    perm, off = bisect(g.src, 256, 4)
    assert np.array_equal(perm, np.arange(256))
    pts = inputs.cap_points(500, (0, 0, 0), 60.0, axis=(1, 0, 0))
    L = 4
    perm, off = bisect(pts, 500, L)
    _check_tree(perm, off, 500, L)
    # brute force at the root: child 0 = the ceil(s/2) smallest along the widest axis
    ext = pts.max(0) - pts.min(0)
    ax = int(np.argmax(ext))
    key = sorted(range(500), key=lambda i: (pts[i, ax], i))
    assert set(perm[:off[1][1]].tolist()) == set(key[:250])
