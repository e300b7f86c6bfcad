"""Pins for oracle.qr (Alg. 1 step 3): LAPACK geqp3 via scipy, orthonormality,
the truncation rule, and the randomized range-finder error (Alg. 1 / Halko
et al. Thm 10.7) on matrices with prescribed singular values."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.qr import pivoted_qr_truncated
from oracle import rng


def _cgauss(seed, s, k):
    r = np.random.default_rng(seed)
    return (r.standard_normal((s, k)) + 1j * r.standard_normal((s, k))) / np.sqrt(2)


@pytest.mark.parametrize("shape", [(16, 18), (32, 34), (20, 12), (7, 7), (64, 72)])
def test_matches_lapack_geqp3_untruncated(shape):
    W = _cgauss(shape[0] * 100 + shape[1], *shape)
    Q, rank, diag, perm = pivoted_qr_truncated(W, 0.0)
    q2, r2, p2 = sla.qr(W, mode="economic", pivoting=True)
    assert rank == min(shape)
    assert np.allclose(diag, np.abs(np.diag(r2)), rtol=1e-12)
    # LAPACK downdates norms; with random data no near-ties, same pivots
    assert np.array_equal(perm[:rank], p2[:rank])
    # same column space, column by column up to a phase
    ph = np.sum(Q.conj() * q2[:, :rank], axis=0)
    assert np.allclose(np.abs(ph), 1.0, atol=1e-12)


def test_orthonormal_and_reconstructs():
    W = _cgauss(1, 30, 40)
    Q, rank, diag, perm = pivoted_qr_truncated(W, 0.0)
    assert np.allclose(Q.conj().T @ Q, np.eye(rank), atol=1e-14)
    assert np.linalg.norm(W - Q @ (Q.conj().T @ W)) < 1e-12 * np.linalg.norm(W)
    assert np.all(np.diff(diag) <= 1e-12)           # |R_jj| non-increasing


def test_truncation_rule_relative_to_first_pivot():
    # columns with norms 1, 1e-3, 1e-7 along orthogonal directions
    s = 10
    E = np.eye(s, dtype=np.complex128)
    W = np.stack([E[:, 0], 1e-3 * E[:, 1], 1e-7 * E[:, 2]], axis=1)
    assert pivoted_qr_truncated(W, 1e-6)[1] == 2      # 1e-7 <= 1e-6 * 1 dropped
    assert pivoted_qr_truncated(W, 1e-2)[1] == 1
    assert pivoted_qr_truncated(W, 1e-8)[1] == 3


def test_degenerate_blocks():
    Q, rank, _, _ = pivoted_qr_truncated(np.zeros((5, 4)), 1e-6)
    assert rank == 1 and np.allclose(Q[:, 0], np.eye(5)[:, 0])
    v = _cgauss(2, 6, 1)
    Q, rank, _, _ = pivoted_qr_truncated(np.hstack([v, 2j * v, -v]), 1e-10)
    assert rank == 1
    assert np.allclose(np.abs(Q[:, 0].conj() @ v[:, 0]), np.linalg.norm(v))
    Q, rank, _, _ = pivoted_qr_truncated(_cgauss(3, 1, 5), 1e-6)   # one row
    assert rank == 1 and np.isclose(abs(Q[0, 0]), 1.0)


@pytest.mark.parametrize("q,eps", [(5, 1e-6), (12, 1e-8)])
def test_randomized_range_finder_error(q, eps):
    """Alg. 1 with oversampling p on A with singular values 1 (x q) then
    eps/100: rank = q and ||A - U U^H A|| is at the level of the tail."""
    m, n, p = 80, 60, 4
    r = np.random.default_rng(q)
    Uq, _ = np.linalg.qr(r.standard_normal((m, m)) + 1j * r.standard_normal((m, m)))
    Vq, _ = np.linalg.qr(r.standard_normal((n, n)) + 1j * r.standard_normal((n, n)))
    sv = np.concatenate([np.ones(q), np.full(min(m, n) - q, eps / 100)])
    A = (Uq[:, :n] * sv) @ Vq.conj().T
    Om = rng.gaussian(11, 1, np.arange(n), 0, q + p)
    U, rank, _, _ = pivoted_qr_truncated(A @ Om, eps)
    assert rank == q
    err = np.linalg.norm(A - U @ (U.conj().T @ A), 2)
    assert err < 50 * eps / 100 * np.sqrt(n)          # Halko Thm 10.7 scale: C * sigma_{q+1}
    # an svd-based check of the same subspace
    assert np.linalg.norm(U @ U.conj().T - Uq[:, :q] @ Uq[:, :q].conj().T, 2) < 1e-6
