"""Pins for oracle.operators: kernel formulas against numpy.fft and direct
evaluation; black-box column counting; composition."""
import cmath
import math

import numpy as np

from oracle import operators as oo
from paper_2002_03400_gb300 import inputs


def test_dft_kernel_is_numpy_fft():
    n = 64
    g = inputs.dft_points(n)
    A = oo.kernel_entries(oo.DFT, 1.0, g.tgt, g.src)
    x = np.random.default_rng(0).standard_normal(n) + 0j
    assert np.allclose(A @ x, np.fft.fft(x), atol=1e-10)


def test_helmholtz_entries_direct():
    g = inputs.line_pair(32)
    A = oo.kernel_entries(oo.HELMHOLTZ_2D, g.wavenumber, g.tgt, g.src)
    i, j = 5, 17
    r = math.hypot(g.tgt[i, 0] - g.src[j, 0], g.tgt[i, 1] - g.src[j, 1])
    assert abs(A[i, j] - cmath.exp(-1j * g.wavenumber * r) / r) < 1e-13
    assert abs(g.wavenumber - math.pi * 32 / 4) < 1e-12           # 8 points per wavelength
    c = inputs.cap_pair(40)
    B = oo.kernel_entries(oo.HELMHOLTZ_3D, c.wavenumber, c.tgt, c.src)
    r = float(np.linalg.norm(c.tgt[3] - c.src[7]))
    assert abs(B[3, 7] - cmath.exp(1j * c.wavenumber * r) / (4 * math.pi * r)) < 1e-13


def test_kernel_op_chunks_and_counts():
    g = inputs.arc_pair(300, seed=1)
    op = oo.KernelOp(oo.HELMHOLTZ_2D, g.wavenumber, g.tgt, g.src, rows_per_chunk=64)
    A = op.dense()
    X = np.random.default_rng(1).standard_normal((300, 3)) + 0j
    assert np.allclose(op.matvec(X), A @ X)
    assert np.allclose(op.matvec_T(X), A.T @ X)
    assert op.cols_N == 3 and op.cols_T == 3


def test_composition():
    r = np.random.default_rng(2)
    A1 = r.standard_normal((20, 30)) + 1j * r.standard_normal((20, 30))
    A2 = r.standard_normal((30, 25)) + 1j * r.standard_normal((30, 25))
    C = oo.ComposedOp(oo.DenseOp(A1), oo.DenseOp(A2))
    X = r.standard_normal((25, 2)) + 0j
    Y = r.standard_normal((20, 2)) + 0j
    assert np.allclose(C.matvec(X), A1 @ A2 @ X)
    assert np.allclose(C.matvec_T(Y), (A1 @ A2).T @ Y)
