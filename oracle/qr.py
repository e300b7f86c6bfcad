"""Column-pivoted Householder QR with truncation (Alg. 1 step 3).

W P = Q R with P a column permutation, Q with orthonormal columns, R upper
triangular; U = Q restricted to the revealed rank.  Readings of the paper
(it fixes neither the truncation rule nor the pivot tie-break):

* the rank is #{j : |R_jj| > eps * |R_11|} -- relative to the block, the
  "relative error threshold" the error analysis of Sec. 5 assumes; under
  column pivoting |R_jj| is non-increasing, so the factorization stops at the
  first pivot at or below the threshold.  The rank is at least 1; a zero
  block returns the first unit vector.
* the pivot is the trailing column of largest 2-norm, ties to the lowest
  index (LAPACK convention); norms are recomputed at every step.
* complex Householder reflector H = I - 2 v v^H / (v^H v) with
  v = x - alpha e1, alpha = -exp(i arg x_0) ||x||, so R_jj = alpha.

Parity: pinned by tests/test_oracle_qr.py against scipy.linalg.qr(pivoting=True)
(LAPACK geqp3), orthonormality, and the Halko et al. bound on matrices with
prescribed singular values.
"""
import numpy as np


def pivoted_qr_truncated(W: np.ndarray, eps: float):
    """Return (Q[:, :rank], rank, |R_jj| for the factorized steps, perm)."""
    A = np.array(W, dtype=np.complex128, copy=True)
    s, k = A.shape
    perm = np.arange(k)
    reflectors = []
    diag = []
    nrm0 = None
    for j in range(min(s, k)):
        norms2 = np.sum(np.abs(A[j:, j:]) ** 2, axis=0)
        p = j + int(np.argmax(norms2))            # first maximum -> lowest index
        if p != j:
            A[:, [j, p]] = A[:, [p, j]]
            perm[[j, p]] = perm[[p, j]]
        nrm = float(np.sqrt(norms2[p - j]))
        if nrm0 is None:
            nrm0 = nrm
        if nrm == 0.0 or nrm <= eps * nrm0:
            break
        x = A[j:, j]
        phase = x[0] / abs(x[0]) if x[0] != 0 else 1.0
        alpha = -phase * nrm
        v = x.copy()
        v[0] -= alpha
        beta = np.real(np.vdot(v, v))
        A[j:, j:] -= np.outer(v, (2.0 / beta) * (v.conj() @ A[j:, j:]))
        reflectors.append((j, v, beta))
        diag.append(nrm)
    rank = max(len(reflectors), 1)
    Q = np.zeros((s, rank), dtype=np.complex128)
    Q[np.arange(rank), np.arange(rank)] = 1.0
    for j, v, beta in reversed(reflectors):      # Q = H_0 H_1 ... H_{rank-1} [I; 0]
        Q[j:, :] -= np.outer(v, (2.0 / beta) * (v.conj() @ Q[j:, :]))
    return Q, rank, np.array(diag), perm
