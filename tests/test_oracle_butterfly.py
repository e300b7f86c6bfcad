"""Pins for oracle.butterfly (Alg. 2, eq. hybrid_butterfly_mat, eq. error).

Nothing here compares the oracle with itself: each check is a closed form,
an invariant, a theorem of the paper, a library routine or brute force."""
import math

import numpy as np
import pytest

from oracle import butterfly as ob
from oracle import operators as oo
from oracle.tree import depth_for_leaf
from paper_2002_03400_gb300 import inputs


def _nested_U(F, j, sigma, mu):
    """Explicit column basis U_{sigma,mu} (eq. nested_basis)."""
    if j == F.L:
        return F.U[sigma]
    top = _nested_U(F, j + 1, 2 * sigma, mu >> 1)
    bot = _nested_U(F, j + 1, 2 * sigma + 1, mu >> 1)
    R = F.R[j][sigma * (1 << (F.L - j)) + mu]
    D = np.zeros((top.shape[0] + bot.shape[0], top.shape[1] + bot.shape[1]), dtype=complex)
    D[:top.shape[0], :top.shape[1]] = top
    D[top.shape[0]:, top.shape[1]:] = bot
    return D @ R


def _nested_V(F, j, sigma, mu):
    """Explicit row basis V_{sigma,mu} (eq. nested_basis_col)."""
    if j == 0:
        return F.V0[mu]
    top = _nested_V(F, j - 1, sigma >> 1, 2 * mu)
    bot = _nested_V(F, j - 1, sigma >> 1, 2 * mu + 1)
    W = F.W[j][sigma * (1 << (F.L - j)) + mu]
    D = np.zeros((top.shape[0] + bot.shape[0], top.shape[1] + bot.shape[1]), dtype=complex)
    D[:top.shape[0], :top.shape[1]] = top
    D[top.shape[0]:, top.shape[1]:] = bot
    return D @ W


def _exact(n, leaf, r, seed):
    eb = inputs.exact_butterfly(n, leaf, r, seed)
    Ft = ob.from_blocks(eb)
    return eb, Ft, oo.FactorOp(Ft)


@pytest.mark.parametrize("n,leaf,r", [(512, 8, 4), (2048, 32, 8), (1024, 16, 6)])
def test_exact_butterfly_recovery(n, leaf, r):
    """Sec. 7.1: an exactly-butterfly matrix of rank r is recovered to machine
    precision with ranks exactly r at every block."""
    eb, Ft, op = _exact(n, leaf, r, seed=1)
    F = ob.factor(op, None, None, eb.L, 1e-12, 2, 4, seed=0)
    A = ob.dense(Ft)
    assert np.linalg.norm(A - ob.dense(F)) <= 1e-12 * np.linalg.norm(A)
    assert ob.sketch_error(op, F, seed=9) <= 1e-12
    for j in F.rV:
        assert np.all(F.rV[j] == r)
    for j in F.rU:
        assert np.all(F.rU[j] == r)
    # all outer and transfer factors are orthonormal, so ||A||_F^2 = sum ||B||_F^2
    sB = sum(np.linalg.norm(b) ** 2 for b in F.B)
    assert abs(sB - np.linalg.norm(A) ** 2) <= 1e-10 * sB
    sBt = sum(np.linalg.norm(b) ** 2 for b in eb.B)
    assert abs(sB - sBt) <= 1e-10 * sBt
    # O(n log n) storage: exact count of stored entries (Sec. 4.5)
    L, lm, nb = eb.L, eb.lm, 1 << eb.L
    want = n * r + n * r + nb * r * r + (lm + (L - lm)) * nb * 2 * r * r
    assert F.stored_entries() == want


def test_blackbox_schedule():
    """Sec. 4.1 / 4.5: level l needs 2^l (r+p) products with A^T and
    2^(L-l) (r+p) with A, r = max(r1 + r2)."""
    n, leaf, r, p = 1024, 8, 4, 2
    eb, Ft, op = _exact(n, leaf, r, seed=2)
    F = ob.factor(op, None, None, eb.L, 1e-12, p, 4, seed=0)
    L, lm = eb.L, eb.lm
    k = 2 * r + p
    for l in range(1, lm + 1):
        assert F.bb_cols[f"W{l}"] == (1 << l) * k
    for l in range(lm, L):
        assert F.bb_cols[f"R{l}"] == (1 << (L - l)) * k
    # leaf loops: r0 = 4 = r is not > r, doubling to 8 gives k = 10 >= leaf 8 (saturated)
    assert F.bb_cols["V0"] == 10 and F.bb_cols["U0"] == 10
    tot_T = F.bb_cols["V0"] + sum((1 << l) * k for l in range(1, lm + 1))
    tot_N = F.bb_cols["U0"] + sum((1 << (L - l)) * k for l in range(lm, L))
    assert op.cols_T == tot_T and op.cols_N == tot_N


@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-8])
def test_dense_brute_force_helmholtz(eps):
    """Thm 5.3: ||A - F||_F <= sqrt(L+2) eps ||A||_F (x2 safety for the
    high-probability assumption on Alg. 1), with F formed by brute force."""
    n = 512
    g = inputs.line_pair(n)
    A = oo.kernel_entries(oo.HELMHOLTZ_2D, g.wavenumber, g.tgt, g.src)
    L = depth_for_leaf(n, 16)
    F = ob.factor(oo.DenseOp(A), g.src, g.tgt, L, eps, 2, 4, seed=0)
    err = np.linalg.norm(A - ob.dense(F)) / np.linalg.norm(A)
    assert err <= 2 * math.sqrt(L + 2) * eps
    assert err >= 1e-3 * eps          # a truncated factorization, not an exact copy


def test_theorems_5_1_and_5_2_per_level():
    """Thm 5.1: sum over level-l blocks of ||K - U U^H K||^2 <= (L-l+1) eps^2 ||A||^2
    (l_m <= l <= L); Thm 5.2: ||K - K V V^H||^2 <= (l+1) eps^2 ||A||^2 (0 <= l <= l_m)."""
    n, eps = 256, 1e-5
    g = inputs.arc_pair(n, seed=4)
    A = oo.kernel_entries(oo.HELMHOLTZ_2D, g.wavenumber, g.tgt, g.src)
    L = depth_for_leaf(n, 16)
    F = ob.factor(oo.DenseOp(A), g.src, g.tgt, L, eps, 2, 4, seed=3)
    At = A[np.ix_(F.permT, F.permS)]
    nA2 = np.linalg.norm(A) ** 2
    for l in range(F.lm, L + 1):
        tot = 0.0
        for tau in range(1 << l):
            for nu in range(1 << (L - l)):
                K = At[F.offT[l][tau]:F.offT[l][tau + 1], F.offS[L - l][nu]:F.offS[L - l][nu + 1]]
                U = _nested_U(F, l, tau, nu)
                assert np.allclose(U.conj().T @ U, np.eye(U.shape[1]), atol=1e-12)
                tot += np.linalg.norm(K - U @ (U.conj().T @ K)) ** 2
        assert tot <= 4 * (L - l + 1) * eps ** 2 * nA2
    for l in range(0, F.lm + 1):
        tot = 0.0
        for tau in range(1 << l):
            for nu in range(1 << (L - l)):
                K = At[F.offT[l][tau]:F.offT[l][tau + 1], F.offS[L - l][nu]:F.offS[L - l][nu + 1]]
                V = _nested_V(F, l, tau, nu)
                assert np.allclose(V.conj().T @ V, np.eye(V.shape[1]), atol=1e-12)
                tot += np.linalg.norm(K - (K @ V) @ V.conj().T) ** 2
        assert tot <= 4 * (l + 1) * eps ** 2 * nA2


def test_dft_matches_numpy_fft_and_ranks_do_not_grow():
    """The DFT is a closed-form butterfly (Sec. 1): the factorization applies
    like numpy.fft.fft, and the block ranks at fixed eps do not grow with n."""
    eps = 1e-8
    maxr = []
    for n in (256, 1024, 4096):
        g = inputs.dft_points(n)
        op = oo.KernelOp(oo.DFT, 1.0, g.tgt, g.src)
        L = depth_for_leaf(n, 16)
        F = ob.factor(op, g.src, g.tgt, L, eps, 2, 4, seed=1)
        x = inputs.random_rhs(n, 2, seed=5)
        y = ob.apply(F, x)
        assert np.linalg.norm(y - np.fft.fft(x, axis=0)) <= 2 * math.sqrt(L + 2) * eps * np.linalg.norm(np.fft.fft(x, axis=0)) * 3
        maxr.append(max(max(F.rV[j].max() for j in F.rV), max(F.rU[j].max() for j in F.rU)))
    assert maxr[-1] <= maxr[0] + 2


def test_global_low_rank():
    """A = X Y^H of rank q: every block has rank <= q and A is recovered."""
    n, q = 512, 3
    r = np.random.default_rng(7)
    X = r.standard_normal((n, q)) + 1j * r.standard_normal((n, q))
    Y = r.standard_normal((n, q)) + 1j * r.standard_normal((n, q))
    A = X @ Y.conj().T
    F = ob.factor(oo.DenseOp(A), None, None, 5, 1e-12, 2, 4, seed=2)
    for d in (F.rV, F.rU):
        for j in d:
            assert d[j].max() <= q
    assert np.linalg.norm(A - ob.dense(F)) <= 1e-11 * np.linalg.norm(A)


def test_apply_adjoint_and_transpose():
    g = inputs.line_pair(256)
    A = oo.kernel_entries(oo.HELMHOLTZ_2D, g.wavenumber, g.tgt, g.src)
    F = ob.factor(oo.DenseOp(A), g.src, g.tgt, 4, 1e-6, 2, 4, seed=0)
    D = ob.dense(F)
    x = inputs.random_rhs(256, 3, seed=1)
    assert np.allclose(ob.apply(F, x, "C"), D.conj().T @ x, atol=1e-12)
    assert np.allclose(ob.apply(F, x, "T"), D.T @ x, atol=1e-12)


def test_error_metric_order_of_magnitude():
    """Tables 1-2 report errors of 0.2..2 eps; same order here."""
    n, eps = 1024, 1e-6
    g = inputs.line_pair(n)
    op = oo.DenseOp(oo.kernel_entries(oo.HELMHOLTZ_2D, g.wavenumber, g.tgt, g.src))
    F = ob.factor(op, g.src, g.tgt, 6, eps, 2, 4, seed=0)
    e = ob.sketch_error(op, F, seed=1)
    assert 0.05 * eps <= e <= 2 * math.sqrt(8) * eps


# --- planted mistakes: each must be caught by one of the pins above ---------

def test_planted_transpose_in_B_is_caught(monkeypatch):
    """Reading eq. Bij literally (transpose instead of pseudo-inverse) breaks
    exact recovery."""
    eb, Ft, op = _exact(512, 8, 4, seed=1)
    monkeypatch.setattr(ob.np.linalg, "pinv", lambda X: X.conj().T)
    F = ob.factor(op, None, None, eb.L, 1e-12, 2, 4, seed=0)
    assert ob.sketch_error(op, F, seed=9) > 1e-3


def test_planted_missing_conjugate_is_caught():
    """Using A^T where A^H is needed (dropping the conjugate of the complex
    extension) breaks the brute-force bound."""
    n, eps = 256, 1e-6
    g = inputs.line_pair(n)
    A = oo.kernel_entries(oo.HELMHOLTZ_2D, g.wavenumber, g.tgt, g.src)

    class Wrong(oo.DenseOp):
        def _matvec_T(self, X):
            return self.A.conj().T @ X
    F = ob.factor(Wrong(A), g.src, g.tgt, 4, eps, 2, 4, seed=0)
    err = np.linalg.norm(A - ob.dense(F)) / np.linalg.norm(A)
    assert err > 100 * eps


def test_planted_swapped_stacking_is_caught(monkeypatch):
    """Stacking the two children of a W block in the wrong order breaks exact
    recovery (wrong index in the nested basis)."""
    eb, Ft, op = _exact(512, 8, 4, seed=3)
    real_VH = ob.VH

    def swapped(F, j, sigma, mu, X):
        if j >= 1:
            top = real_VH(F, j - 1, sigma >> 1, 2 * mu + 1, X)
            bot = real_VH(F, j - 1, sigma >> 1, 2 * mu, X)
            return F.W[j][sigma * (1 << (F.L - j)) + mu].conj().T @ np.vstack([top, bot])
        return real_VH(F, j, sigma, mu, X)
    monkeypatch.setattr(ob, "VH", swapped)
    F = ob.factor(op, None, None, eb.L, 1e-12, 2, 4, seed=0)
    monkeypatch.setattr(ob, "VH", real_VH)
    assert ob.sketch_error(op, F, seed=9) > 1e-3


def test_adjacent_hemispheres_weak_admissibility():
    """The 3D experiment's geometry (Sec. 7.3): two hemispheres that meet
    along the equator.  The generator puts every point on the unit sphere,
    sources above and targets below the equator, equal-area (uniform z, mean
    1/2 in |z|), none on the equator.  The factorization of the touching
    surfaces reaches the Thm 5.3 accuracy against the dense matrix, with
    middle-level ranks above those of two separated caps at the same
    sampling and growing with n (the O(n^{1/4}) growth the paper reports
    for this case), while the separated caps' ranks stay put."""
    g = inputs.hemisphere_pair(2000)
    assert np.allclose(np.linalg.norm(g.src, axis=1), 1.0) and np.allclose(np.linalg.norm(g.tgt, axis=1), 1.0)
    assert g.src[:, 2].min() >= 0.5 / 2000 - 1e-15 and g.tgt[:, 2].max() <= -0.5 / 2000 + 1e-15
    assert abs(g.src[:, 2].mean() - 0.5) < 1e-3 and abs(g.tgt[:, 2].mean() + 0.5) < 1e-3
    assert math.isclose(g.wavenumber, 2 * math.pi / (10.0 * math.sqrt(2 * math.pi / 2000)))
    eps = 1e-6
    mid = {}
    for n in (512, 1024):
        for name, geo in (("hemi", inputs.hemisphere_pair(n)), ("caps", inputs.cap_pair(n, ppw=10.0))):
            op = oo.KernelOp(oo.HELMHOLTZ_3D, geo.wavenumber, geo.tgt, geo.src)
            L = inputs.leaf_levels(n, 16)
            F = ob.factor(op, geo.src, geo.tgt, L, eps, 4, 16, seed=0)
            A = op.dense()
            assert np.linalg.norm(A - ob.dense(F)) <= 2 * math.sqrt(L + 2) * eps * np.linalg.norm(A)
            mid[name, n] = int(np.max(F.rV[F.lm]))
    assert mid["hemi", 512] > mid["caps", 512] and mid["hemi", 1024] > mid["caps", 1024]
    assert mid["hemi", 1024] > mid["hemi", 512]
    assert abs(mid["caps", 1024] - mid["caps", 512]) <= 2


@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_hybrid_level_column_and_row_wise(level):
    """Sec. 3.3: the hybrid factorization at any level l (B at l, W levels
    1..l, R levels L-1..l); l = 0 is the column-wise form of Sec. 3.3.1.  An
    exactly-butterfly matrix (rank 4, L = 4) is recovered to machine
    precision with rank 4 at every block for every l, and the black-box
    column count follows the closed form of Sec. 4.1/4.5: the two leaf
    loops take 10 columns each (r0 = 4 doubled once, p = 2), level j of the
    W loop 2^j (4 + 4 + 2) and level j of the R loop 2^(L-j) (4 + 4 + 2) --
    least at l = L/2 ("much higher cost" toward l = 0 and l = L-1)."""
    eb, Ft, op = _exact(256, 16, 4, seed=1)
    A = ob.dense(Ft)
    F = ob.factor(op, None, None, eb.L, 1e-12, 2, 4, seed=0, hybrid_level=level)
    assert F.lm == level
    assert np.linalg.norm(A - ob.dense(F)) <= 1e-12 * np.linalg.norm(A)
    assert all(np.all(F.rV[j] == 4) for j in F.rV) and all(np.all(F.rU[j] == 4) for j in F.rU)
    L = eb.L
    want = 20 + 10 * (sum(2 ** j for j in range(1, level + 1)) + sum(2 ** (L - j) for j in range(level, L)))
    assert sum(F.bb_cols.values()) == want


def test_column_wise_and_row_wise_kernel():
    """Kernel matrix (line pair, n = 512, L = 5): the column-wise form (l = 0)
    and the row-wise form (the transpose of the column-wise factorization of
    A^T, applied with op T) both reach the Thm 5.3 accuracy; l outside
    [0, L-1] is refused."""
    g = inputs.line_pair(512)
    op = oo.KernelOp(oo.HELMHOLTZ_2D, g.wavenumber, g.tgt, g.src)
    A = op.dense()
    L = inputs.leaf_levels(512, 16)
    bound = 2 * math.sqrt(L + 2) * 1e-6
    Fc = ob.factor(op, g.src, g.tgt, L, 1e-6, 2, 4, seed=0, hybrid_level=0)
    assert np.linalg.norm(A - ob.dense(Fc)) <= bound * np.linalg.norm(A)

    class Transposed:
        def __init__(self, o):
            self.o, self.n, self.m = o, o.m, o.n

        def matvec(self, X):
            return self.o.matvec_T(X)

        def matvec_T(self, X):
            return self.o.matvec(X)

    Fr = ob.factor(Transposed(op), g.tgt, g.src, L, 1e-6, 2, 4, seed=0, hybrid_level=0)
    x = inputs.random_rhs(512, 3, seed=2)
    assert np.linalg.norm(ob.apply(Fr, x, "T") - A @ x) <= bound * np.linalg.norm(A @ x)
    with pytest.raises(ValueError):
        ob.factor(op, g.src, g.tgt, L, 1e-6, 2, 4, seed=0, hybrid_level=L)


def test_a_posteriori_acceptance(monkeypatch):
    """The heuristic stop of the leaf loops ("r > max rank", Sec. 4.2) backed
    by an a-posteriori test: the sketch error (Sec. 7) with fresh columns
    must meet the Thm 5.3 bound, else Alg. 2 reruns with r0 doubled.  A
    converged run is accepted at once; with the stop planted to fire after
    the first pass (leaf bases of rank <= r0 + p), the plain factorization
    misses the bound, the checked one retries until the dense error is
    within it, and without retries it reports non-convergence."""
    g = inputs.line_pair(1024)
    op = oo.KernelOp(oo.HELMHOLTZ_2D, g.wavenumber, g.tgt, g.src)
    A = op.dense()
    L = inputs.leaf_levels(1024, 16)
    bound = 2 * math.sqrt(L + 2) * 1e-6
    F, tried = ob.factor_checked(op, g.src, g.tgt, L, 1e-6, 2, 4, seed=0)
    assert len(tried) == 1 and tried[0][1] <= bound
    F0 = ob.factor(op, g.src, g.tgt, L, 1e-6, 2, 4, seed=0)
    assert all(np.array_equal(F.rV[j], F0.rV[j]) for j in F0.rV)
    monkeypatch.setattr(ob, "leaf_loop_done", lambda r, max_rank, k, leaf_max: True)
    Fp = ob.factor(op, g.src, g.tgt, L, 1e-6, 2, 2, seed=0)
    assert ob.sketch_error(op, Fp, 5) > bound and np.linalg.norm(A - ob.dense(Fp)) > bound * np.linalg.norm(A)
    Fc, tried = ob.factor_checked(op, g.src, g.tgt, L, 1e-6, 2, 2, seed=0)
    assert len(tried) >= 2 and [t[0] for t in tried] == [2 * 2 ** i for i in range(len(tried))]
    assert all(e > bound for _, e in tried[:-1]) and tried[-1][1] <= bound
    assert np.linalg.norm(A - ob.dense(Fc)) <= bound * np.linalg.norm(A)
    with pytest.raises(ob.NotConverged):
        ob.factor_checked(op, g.src, g.tgt, L, 1e-6, 2, 2, seed=0, retries=0)
