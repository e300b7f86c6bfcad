"""Bisection trees T_S and T_T (Sec. 3.1, hierarchical partitioning).

A point set is split recursively into two children until depth L; both trees
are complete with 2^l nodes at level l (root = level 0, leaves = level L).
Reading of the paper (it leaves the bisection rule open): a node of s points
splits into ceil(s/2) and floor(s/2) points.  With points given, the node's
points are ordered by the coordinate of largest bounding-box extent (ties
between axes -> lowest axis; ties between points -> lower original index)
and the first ceil(s/2) form child 0.  Without points, index order is used.

Output: ``perm`` (tree position -> original index) and ``off[l]``, the
2^l + 1 boundaries of the level-l nodes in tree order, so node (l, i) owns
tree positions off[l][i] .. off[l][i+1]-1.

Parity: pinned by tests/test_oracle_tree.py (partition invariants, sizes,
brute-force median check).
"""
import numpy as np


def depth_for_leaf(n: int, leaf: int) -> int:
    L = 0
    while -(-n // (1 << L)) > leaf:
        L += 1
    return L


def bisect(points, count: int, L: int):
    idx = np.arange(count)
    pts = None if points is None else np.asarray(points, dtype=np.float64).reshape(count, -1)
    off = [np.array([0, count])]
    nodes = [idx]
    for lev in range(L):
        nxt = []
        for node in nodes:
            s = len(node)
            h = (s + 1) // 2
            if pts is not None and s > 1:
                sub = pts[node]
                ext = sub.max(axis=0) - sub.min(axis=0)
                ax = int(np.argmax(ext))          # first max -> lowest axis
                order = np.lexsort((node, sub[:, ax]))   # key: coordinate, then index
                node = node[order]
            nxt.append(node[:h])
            nxt.append(node[h:])
        nodes = nxt
        sizes = np.array([len(x) for x in nodes])
        off.append(np.concatenate([[0], np.cumsum(sizes)]))
    perm = np.concatenate(nodes) if nodes else idx
    return perm.astype(np.int64), off
