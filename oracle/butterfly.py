"""Alg. 2 (adaptive randomized hybrid butterfly factorization), its apply and
the error metric -- plain complex128 numpy, step by step in the paper's order.

Notation (Sec. 3):  A = K(T, S) is m x n; T_T and T_S are bisection trees of
depth L; l_m = floor(L/2).  A level-j block is (tau at level j of T_T,
nu at level L-j of T_S); there are 2^L of them at every level and block
(tau, nu) has index b = tau * 2^(L-j) + nu.  Children of node x are 2x, 2x+1.

Factors (eq. hybrid_butterfly_mat):
    A ~= (U^L R^(L-1) ... R^(l_m)) B^(l_m) (W^(l_m) ... W^1 V^0)
  V0[nu]     = V_{t,nu}      |S_nu| x r      row basis of leaf nu (Sec. 3.3.2)
  W[j][b]    = W_{tau,nu}    (r_{p tau,2nu} + r_{p tau,2nu+1}) x r   (eq. nested_basis_col)
  B[b]       = B_{tau,nu}    r^U x r^V at level l_m                  (Sec. 4.4)
  R[j][b]    = R_{tau,nu}    (r_{2tau,p nu} + r_{2tau+1,p nu}) x r   (eq. nested_basis)
  U[tau]     = U_{tau,s}     |T_tau| x r     column basis of leaf tau (Sec. 3.3.1)
  rV[j][b], rU[j][b]  ranks (columns) of the level-j row / column bases.

Complex extension (the paper states the real case and calls the complex one
trivial): every transpose in a projection becomes a conjugate transpose,
K ~= U U^H K and K ~= K V V^H; the black box provides A and A^T and the
oracle forms A^H X = conj(A^T conj(X)).

Readings where the paper is silent or garbled:
  * Alg. 1 truncation and pivoting: see oracle.qr.
  * adaptive leaf loops: r starts at r0 in both loops; each pass appends r
    new random columns to the previous ones (columns are indexed by the
    counter-based generator, so pass t uses columns 0..r+p-1 of one stream);
    stop when r > max revealed rank, or when r + p >= the largest leaf
    (the sketch then spans every leaf); doubling past r_max is an error.
  * sketch width: one width per level, the maximum over its blocks
    (r = max(r1 + r2) in the lines that form Gamma_tau and Omega_nu), + p;
    at l = l_m the width also covers max r^V + p so that V^H Omega has full
    row rank.
  * in the R loop, tau runs over level l of T_T (the listing's "level L-l"
    for tau is read as a typo for level l).
  * eq. Bij: B = (U^H K Omega)(V^H Omega)^+ (pseudo-inverse), the minimizer
    of ||K Omega - U B V^H Omega||_F; B is r^U x r^V.
  * the loop that builds V^0 is the first loop (the listing's comments);
    the text's line references to it are swapped.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import rng
from .qr import pivoted_qr_truncated
from .tree import bisect


class NotConverged(RuntimeError):
    pass


@dataclass
class Factorization:
    n: int
    m: int
    L: int
    lm: int
    permS: np.ndarray
    offS: list
    permT: np.ndarray
    offT: list
    V0: list = field(default_factory=list)
    W: dict = field(default_factory=dict)
    B: list = field(default_factory=list)
    R: dict = field(default_factory=dict)
    U: list = field(default_factory=list)
    rV: dict = field(default_factory=dict)
    rU: dict = field(default_factory=dict)
    widths: dict = field(default_factory=dict)   # sketch width per stage
    bb_cols: dict = field(default_factory=dict)  # black-box columns per stage

    def stored_entries(self) -> int:
        tot = sum(v.size for v in self.V0) + sum(u.size for u in self.U) + sum(b.size for b in self.B)
        tot += sum(w.size for j in self.W for w in self.W[j])
        tot += sum(x.size for j in self.R for x in self.R[j])
        return int(tot)


def make_trees(src, n, tgt, m, L):
    permS, offS = bisect(src, n, L)
    permT, offT = bisect(tgt, m, L)
    return permS, offS, permT, offT


# ---------------------------------------------------------------------------
# nested bases applied recursively (eqs. nested_basis, nested_basis_col)
# ---------------------------------------------------------------------------

def VH(F: Factorization, j: int, sigma: int, mu: int, X: np.ndarray) -> np.ndarray:
    """V_{sigma,mu}^H X[S_mu]; sigma at level j of T_T, mu at level L-j of T_S.
    V_{sigma,mu} = diag(V_{p sigma, 2mu}, V_{p sigma, 2mu+1}) W_{sigma,mu}."""
    L = F.L
    if j == 0:
        a, b = F.offS[L][mu], F.offS[L][mu + 1]
        return F.V0[mu].conj().T @ X[a:b]
    top = VH(F, j - 1, sigma >> 1, 2 * mu, X)
    bot = VH(F, j - 1, sigma >> 1, 2 * mu + 1, X)
    return F.W[j][sigma * (1 << (L - j)) + mu].conj().T @ np.vstack([top, bot])


def UH(F: Factorization, j: int, sigma: int, mu: int, Z: np.ndarray) -> np.ndarray:
    """U_{sigma,mu}^H Z[T_sigma]; sigma at level j of T_T, mu at level L-j of T_S.
    U_{sigma,mu} = diag(U_{2sigma, p mu}, U_{2sigma+1, p mu}) R_{sigma,mu}."""
    L = F.L
    if j == L:
        a, b = F.offT[L][sigma], F.offT[L][sigma + 1]
        return F.U[sigma].conj().T @ Z[a:b]
    top = UH(F, j + 1, 2 * sigma, mu >> 1, Z)
    bot = UH(F, j + 1, 2 * sigma + 1, mu >> 1, Z)
    return F.R[j][sigma * (1 << (L - j)) + mu].conj().T @ np.vstack([top, bot])


# ---------------------------------------------------------------------------
# Alg. 2
# ---------------------------------------------------------------------------

def leaf_loop_done(r: int, max_rank: int, k: int, leaf_max: int) -> bool:
    """The adaptive stop of the leaf loops (Alg. 2, loops "V" and "U"): the
    guess r exceeds every leaf rank the sketch revealed, or the sketch width
    k = r + p already spans the largest leaf (the heuristic of Sec. 4.2)."""
    return r > max_rank or k >= leaf_max


def factor(op, src, tgt, leaf_levels: int, eps: float, p: int, r0: int, seed: int,
           r_max: int = 4096, hybrid_level: int | None = None) -> Factorization:
    """Adaptive randomized hybrid butterfly factorization (Alg. 2).

    ``op`` is a black box (oracle.operators) in user order; ``src``/``tgt``
    are the point sets (or None for index order) the trees are built on.
    ``hybrid_level`` is the level l of eq. hybrid_butterfly_mat where B sits
    (Alg. 2 uses l_m = floor(L/2), the default); any 0 <= l <= L-1 runs the
    same loops (W levels 1..l, R levels L-1..l, B at l).  l = 0 is the
    column-wise factorization of Sec. 3.3.1 with its outer factor E^0 kept
    as B^0 V^0^H (the "minor modification" of Sec. 4, at the cost of a
    sketch with 2^(L-l) k columns at every R level); the row-wise one
    (Sec. 3.3.2) is the transpose of the column-wise factorization of A^T."""
    n, m, L = op.n, op.m, leaf_levels
    if L < 1:
        raise ValueError("Alg. 2 needs L >= 1 (the B loop runs at l = l_m <= L-1)")
    lm = L // 2 if hybrid_level is None else int(hybrid_level)
    if not 0 <= lm <= L - 1:
        raise ValueError("the hybrid level must satisfy 0 <= l <= L-1")
    permS, offS, permT, offT = make_trees(src, n, tgt, m, L)
    F = Factorization(n, m, L, lm, permS, offS, permT, offT)
    nb = 1 << L

    def A_tree(X):                 # A X, rows/cols in tree order
        Xu = np.zeros((n, X.shape[1]), dtype=np.complex128)
        Xu[permS] = X
        return op.matvec(Xu)[permT]

    def AH_tree(X):                # A^H X = conj(A^T conj X), tree order
        Xu = np.zeros((m, X.shape[1]), dtype=np.complex128)
        Xu[permT] = X.conj()
        return op.matvec_T(Xu)[permS].conj()

    leafS = np.diff(offS[L])
    leafT = np.diff(offT[L])

    # --- V^0: leaf row bases from Y = A^H Gamma_t (loop "V") -------------
    r = r0
    Y = np.zeros((n, 0), dtype=np.complex128)
    passes = 0
    while True:
        k = r + p
        if Y.shape[1] < k:
            G = rng.gaussian(seed, rng.stream_id(rng.STAGE_V0), np.arange(m), Y.shape[1], k)
            Y = np.hstack([Y, AH_tree(G)])
        passes += 1
        F.V0, ranks = [], np.zeros(nb, dtype=np.int64)
        for nu in range(nb):
            Q, rk, _, _ = pivoted_qr_truncated(Y[offS[L][nu]:offS[L][nu + 1], :k], eps)
            F.V0.append(Q)
            ranks[nu] = rk
        if leaf_loop_done(r, int(ranks.max()), k, int(leafS.max())):
            break
        r *= 2
        if r > r_max:
            raise NotConverged("V^0 rank exceeds r_max")
    F.rV[0] = ranks
    F.widths["V0"] = k
    F.bb_cols["V0"] = Y.shape[1]

    # --- U^L: leaf column bases from Z = A Omega_s (loop "U") -------------
    r = r0
    Z = np.zeros((m, 0), dtype=np.complex128)
    while True:
        k = r + p
        if Z.shape[1] < k:
            O = rng.gaussian(seed, rng.stream_id(rng.STAGE_U0), np.arange(n), Z.shape[1], k)
            Z = np.hstack([Z, A_tree(O)])
        F.U, ranks = [], np.zeros(nb, dtype=np.int64)
        for tau in range(nb):
            Q, rk, _, _ = pivoted_qr_truncated(Z[offT[L][tau]:offT[L][tau + 1], :k], eps)
            F.U.append(Q)
            ranks[tau] = rk
        if leaf_loop_done(r, int(ranks.max()), k, int(leafT.max())):
            break
        r *= 2
        if r > r_max:
            raise NotConverged("U^L rank exceeds r_max")
    F.rU[L] = ranks
    F.widths["U0"] = k
    F.bb_cols["U0"] = Z.shape[1]

    # --- W^l, l = 1..l_m (Sec. 4.3) ---------------------------------------
    for l in range(1, lm + 1):
        prev = F.rV[l - 1]
        nt, nn = 1 << l, 1 << (L - l)
        k = 0
        for tau in range(nt):
            for nu in range(nn):
                base = (tau >> 1) * (2 * nn)
                k = max(k, prev[base + 2 * nu] + prev[base + 2 * nu + 1])
        k += p
        Gc = rng.gaussian(seed, rng.stream_id(rng.STAGE_W, l), np.arange(m), 0, k)
        Gbar = np.zeros((m, nt * k), dtype=np.complex128)       # structured Gamma-bar
        for tau in range(nt):
            a, b = offT[l][tau], offT[l][tau + 1]
            Gbar[a:b, tau * k:(tau + 1) * k] = Gc[a:b]
        Y = AH_tree(Gbar)                                        # K(T_tau, S)^H Gamma_tau
        F.W[l] = [None] * nb
        F.rV[l] = np.zeros(nb, dtype=np.int64)
        for tau in range(nt):
            Yt = Y[:, tau * k:(tau + 1) * k]
            for nu in range(nn):
                P = np.vstack([VH(F, l - 1, tau >> 1, 2 * nu, Yt),
                               VH(F, l - 1, tau >> 1, 2 * nu + 1, Yt)])
                Q, rk, _, _ = pivoted_qr_truncated(P, eps)
                F.W[l][tau * nn + nu] = Q
                F.rV[l][tau * nn + nu] = rk
        F.widths[f"W{l}"] = k
        F.bb_cols[f"W{l}"] = nt * k

    # --- R^l, l = L-1 .. l_m, and B at l_m (Secs. 4.2, 4.4) ---------------
    F.B = [None] * nb
    for l in range(L - 1, lm - 1, -1):
        nxt = F.rU[l + 1]
        nt, nn = 1 << l, 1 << (L - l)
        nn1 = nn >> 1                        # nodes of T_S at level L-l-1
        k = 0
        for tau in range(nt):
            for nu in range(nn):
                k = max(k, nxt[(2 * tau) * nn1 + (nu >> 1)] + nxt[(2 * tau + 1) * nn1 + (nu >> 1)])
        if l == lm:
            k = max(k, int(F.rV[lm].max()))
        k += p
        Oc = rng.gaussian(seed, rng.stream_id(rng.STAGE_R, l), np.arange(n), 0, k)
        Obar = np.zeros((n, nn * k), dtype=np.complex128)       # structured Omega-bar
        for nu in range(nn):
            a, b = offS[L - l][nu], offS[L - l][nu + 1]
            Obar[a:b, nu * k:(nu + 1) * k] = Oc[a:b]
        Z = A_tree(Obar)                                         # K(T, S_nu) Omega_nu
        F.R[l] = [None] * nb
        F.rU[l] = np.zeros(nb, dtype=np.int64)
        for nu in range(nn):
            Zn = Z[:, nu * k:(nu + 1) * k]
            On = Obar[:, nu * k:(nu + 1) * k]
            for tau in range(nt):
                P = np.vstack([UH(F, l + 1, 2 * tau, nu >> 1, Zn),
                               UH(F, l + 1, 2 * tau + 1, nu >> 1, Zn)])
                Q, rk, _, _ = pivoted_qr_truncated(P, eps)
                b = tau * nn + nu
                F.R[l][b] = Q
                F.rU[l][b] = rk
                if l == lm:
                    X = VH(F, lm, tau, nu, On)                   # V_{tau,nu}^H Omega_nu
                    C = Q.conj().T @ P                           # U_{tau,nu}^H K Omega_nu
                    F.B[b] = C @ np.linalg.pinv(X)               # eq. Bij
        F.widths[f"R{l}"] = k
        F.bb_cols[f"R{l}"] = nn * k
    return F


# ---------------------------------------------------------------------------
# apply (eq. hybrid_butterfly_mat) and adjoint
# ---------------------------------------------------------------------------

def _apply_N(F: Factorization, x: np.ndarray) -> np.ndarray:
    L, lm, nb = F.L, F.lm, 1 << F.L
    xt = x[F.permS]
    v = [F.V0[nu].conj().T @ xt[F.offS[L][nu]:F.offS[L][nu + 1]] for nu in range(nb)]
    for j in range(1, lm + 1):                       # W^j
        nn = 1 << (L - j)
        w = [None] * nb
        for s in range(1 << j):
            for mu in range(nn):
                base = (s >> 1) * (2 * nn)
                w[s * nn + mu] = F.W[j][s * nn + mu].conj().T @ np.vstack([v[base + 2 * mu], v[base + 2 * mu + 1]])
        v = w
    u = [F.B[b] @ v[b] for b in range(nb)]           # B^(l_m)
    for j in range(lm, L):                           # R^j: level j -> level j+1
        nn = 1 << (L - j)
        nn1 = nn >> 1
        w = [None] * nb
        for s in range(1 << (j + 1)):
            tau, a = s >> 1, s & 1
            for mu in range(nn1):
                acc = 0
                for c in (0, 1):
                    b = tau * nn + 2 * mu + c
                    r_first = F.rU[j + 1][(2 * tau) * nn1 + mu]
                    rows = slice(0, r_first) if a == 0 else slice(r_first, F.R[j][b].shape[0])
                    acc = acc + F.R[j][b][rows] @ u[b]
                w[s * nn1 + mu] = acc
        u = w
    yt = np.zeros((F.m, x.shape[1]), dtype=np.complex128)
    for tau in range(nb):
        yt[F.offT[L][tau]:F.offT[L][tau + 1]] = F.U[tau] @ u[tau]
    y = np.zeros_like(yt)
    y[F.permT] = yt
    return y


def _apply_H(F: Factorization, x: np.ndarray) -> np.ndarray:
    L, lm, nb = F.L, F.lm, 1 << F.L
    xt = x[F.permT]
    u = [F.U[tau].conj().T @ xt[F.offT[L][tau]:F.offT[L][tau + 1]] for tau in range(nb)]
    for j in range(L - 1, lm - 1, -1):               # R^j^H: level j+1 -> level j
        nn = 1 << (L - j)
        nn1 = nn >> 1
        w = [None] * nb
        for tau in range(1 << j):
            for nu in range(nn):
                top = u[(2 * tau) * nn1 + (nu >> 1)]
                bot = u[(2 * tau + 1) * nn1 + (nu >> 1)]
                w[tau * nn + nu] = F.R[j][tau * nn + nu].conj().T @ np.vstack([top, bot])
        u = w
    v = [F.B[b].conj().T @ u[b] for b in range(nb)]  # B^H
    for j in range(lm, 0, -1):                       # W^j^H: level j -> level j-1
        nn = 1 << (L - j)
        w = [None] * nb
        for rho in range(1 << (j - 1)):
            for kap in range(2 * nn):
                mu, c = kap >> 1, kap & 1
                acc = 0
                for a in (0, 1):
                    b = (2 * rho + a) * nn + mu
                    r_first = F.rV[j - 1][rho * (2 * nn) + 2 * mu]
                    rows = slice(0, r_first) if c == 0 else slice(r_first, F.W[j][b].shape[0])
                    acc = acc + F.W[j][b][rows] @ v[b]
                w[rho * (2 * nn) + kap] = acc
        v = w
    yt = np.zeros((F.n, x.shape[1]), dtype=np.complex128)
    for nu in range(nb):
        yt[F.offS[L][nu]:F.offS[L][nu + 1]] = F.V0[nu] @ v[nu]
    y = np.zeros_like(yt)
    y[F.permS] = yt
    return y


def apply(F: Factorization, x: np.ndarray, op: str = "N") -> np.ndarray:
    """y = F x (op 'N'), F^H x ('C') or F^T x = conj(F^H conj x) ('T');
    x and y in user point order."""
    x = np.asarray(x, dtype=np.complex128)
    vec = x.ndim == 1
    if vec:
        x = x[:, None]
    if op == "N":
        y = _apply_N(F, x)
    elif op == "C":
        y = _apply_H(F, x)
    elif op == "T":
        y = _apply_H(F, x.conj()).conj()
    else:
        raise ValueError(op)
    return y[:, 0] if vec else y


def dense(F: Factorization) -> np.ndarray:
    """The m x n matrix the factors represent (F applied to the identity)."""
    return apply(F, np.eye(F.n, dtype=np.complex128), "N")


def error_probe(n: int, seed: int, cols: int = 16) -> np.ndarray:
    """Test matrix of the error metric (Sec. 7, eq. error): complex Gaussian,
    ``cols`` columns, rows in user order, its own stream."""
    return rng.gaussian(seed, rng.stream_id(rng.STAGE_ERR), np.arange(n), 0, cols)


def factor_checked(op, src, tgt, leaf_levels: int, eps: float, p: int, r0: int, seed: int,
                   check_seed: int = 1009, retries: int = 4, **kw) -> tuple:
    """Alg. 2 with an a-posteriori acceptance test: the sketch error of
    Sec. 7 (eq. error) with fresh test columns must be within the Thm 5.3
    bound 2 sqrt(L+2) eps; otherwise the factorization is redone with the
    initial rank guess r0 doubled (at most `retries` times).  Returns the
    factorization and the list of (r0, error) of every attempt."""
    bound = 2.0 * np.sqrt(leaf_levels + 2) * eps
    tried = []
    for t in range(retries + 1):
        F = factor(op, src, tgt, leaf_levels, eps, p, r0, seed, **kw)
        e = sketch_error(op, F, check_seed + t)
        tried.append((r0, e))
        if e <= bound:
            return F, tried
        r0 *= 2
    raise NotConverged(f"sketch error above {bound:.2e} after {retries} retries: {tried}")


def sketch_error(op, F: Factorization, seed: int, cols: int = 16) -> float:
    """||A Omega - F Omega||_F / ||A Omega||_F (Sec. 7, eq. error)."""
    Om = error_probe(F.n, seed, cols)
    AO = op.matvec(Om)
    FO = apply(F, Om, "N")
    return float(np.linalg.norm(AO - FO) / np.linalg.norm(AO))


# ---------------------------------------------------------------------------
# exactly-butterfly operators given as blocks of constant rank (Sec. 7.1)
# ---------------------------------------------------------------------------

def from_blocks(eb, src=None, tgt=None) -> Factorization:
    """Wrap blocks laid out like paper_2002_03400_gb300.inputs.ExactButterfly
    (index-order trees) as a Factorization."""
    L, lm, r, nb = eb.L, eb.lm, eb.r, 1 << eb.L
    permS, offS, permT, offT = make_trees(src, eb.n, tgt, eb.m, L)
    F = Factorization(eb.n, eb.m, L, lm, permS, offS, permT, offT)
    F.V0 = [eb.V0[i] for i in range(nb)]
    F.U = [eb.U[i] for i in range(nb)]
    F.B = [eb.B[i] for i in range(nb)]
    F.W = {j: [eb.W[j][i] for i in range(nb)] for j in eb.W}
    F.R = {j: [eb.R[j][i] for i in range(nb)] for j in eb.R}
    for j in range(0, lm + 1):
        F.rV[j] = np.full(nb, r)
    for j in range(lm, L + 1):
        F.rU[j] = np.full(nb, r)
    return F
