"""Black-box operators for the oracle: products with A and with A^T.

Alg. 2 only assumes a routine that multiplies A = K(T, S) (m x n) and its
transpose by arbitrary matrices (Sec. 4.1).  Every operator here counts the
columns it is applied to, so tests can check the black-box schedule of
Sec. 4.5.  Rows/columns are in the user's original point order.

Kernels (entries A[i, j] = K(t_i, s_j), r = |t_i - s_j|):
  helmholtz2d : exp(-i k r) / r
  helmholtz3d : exp(+i k r) / (4 pi r)          (eq. 3dkernel with kappa = k/2pi)
  dft         : exp(-2 pi i t_i s_j)           (1-D points)

Parity: the kernel formulas are pinned in tests/test_oracle_operators.py by
numpy.fft.fft (DFT) and direct evaluation of single entries.
"""
import numpy as np

HELMHOLTZ_2D = 1
HELMHOLTZ_3D = 2
DFT = 3


def kernel_entries(kind: int, k: float, tgt: np.ndarray, src: np.ndarray) -> np.ndarray:
    tgt = np.asarray(tgt, dtype=np.float64)
    src = np.asarray(src, dtype=np.float64)
    if kind == DFT:
        return np.exp(-2j * np.pi * np.outer(tgt[:, 0], src[:, 0]))
    d = tgt[:, None, :] - src[None, :, :]
    r = np.sqrt(np.sum(d * d, axis=2))
    if kind == HELMHOLTZ_2D:
        return np.exp(-1j * k * r) / r
    if kind == HELMHOLTZ_3D:
        return np.exp(1j * k * r) / (4.0 * np.pi * r)
    raise ValueError(f"unknown kernel {kind}")


class CountingOp:
    """Base: counts black-box columns for products with A and A^T."""

    def __init__(self, m: int, n: int):
        self.m, self.n = m, n
        self.cols_N = 0
        self.cols_T = 0

    def matvec(self, X):
        self.cols_N += X.shape[1]
        return self._matvec(X)

    def matvec_T(self, X):
        self.cols_T += X.shape[1]
        return self._matvec_T(X)


class DenseOp(CountingOp):
    def __init__(self, A: np.ndarray):
        super().__init__(*A.shape)
        self.A = np.asarray(A, dtype=np.complex128)

    def _matvec(self, X):
        return self.A @ X

    def _matvec_T(self, X):
        return self.A.T @ X


class KernelOp(CountingOp):
    """Entries formed on the fly, ``rows_per_chunk`` target rows at a time."""

    def __init__(self, kind, k, tgt, src, rows_per_chunk=512):
        super().__init__(len(tgt), len(src))
        self.kind, self.k = kind, k
        self.tgt = np.asarray(tgt, dtype=np.float64).reshape(self.m, -1)
        self.src = np.asarray(src, dtype=np.float64).reshape(self.n, -1)
        self.chunk = rows_per_chunk

    def _matvec(self, X):
        Y = np.empty((self.m, X.shape[1]), dtype=np.complex128)
        for i0 in range(0, self.m, self.chunk):
            i1 = min(self.m, i0 + self.chunk)
            Y[i0:i1] = kernel_entries(self.kind, self.k, self.tgt[i0:i1], self.src) @ X
        return Y

    def _matvec_T(self, X):
        Y = np.zeros((self.n, X.shape[1]), dtype=np.complex128)
        for i0 in range(0, self.m, self.chunk):
            i1 = min(self.m, i0 + self.chunk)
            Y += kernel_entries(self.kind, self.k, self.tgt[i0:i1], self.src).T @ X[i0:i1]
        return Y

    def dense(self):
        return kernel_entries(self.kind, self.k, self.tgt, self.src)


class FactorOp(CountingOp):
    """A given by a hybrid butterfly factorization (oracle.butterfly.Factorization)."""

    def __init__(self, F):
        super().__init__(F.m, F.n)
        self.F = F

    def _matvec(self, X):
        from .butterfly import apply
        return apply(self.F, X, "N")

    def _matvec_T(self, X):
        from .butterfly import apply
        return apply(self.F, X, "T")


class ComposedOp(CountingOp):
    """A = A1 A2 applied through its factors: A X = A1 (A2 X),
    A^T X = A2^T (A1^T X)."""

    def __init__(self, A1, A2):
        super().__init__(A1.m, A2.n)
        self.A1, self.A2 = A1, A2

    def _matvec(self, X):
        return self.A1.matvec(self.A2.matvec(X))

    def _matvec_T(self, X):
        return self.A2.matvec_T(self.A1.matvec_T(X))
