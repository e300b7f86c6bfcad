"""Fits the sin/cos polynomials of the mixed-precision kernel entries
(kentry.cuh) on |t| <= pi/4 by a Remez exchange on the absolute error:
    sin t ~ t + t^3 (s3 + t^2 (s5 + t^2 s7))
    cos t ~ 1 + t^2 (c2 + t^2 (c4 + t^2 (c6 + t^2 c8)))
in float64, then reports the error of the float32-rounded coefficients
evaluated in float32 with FMA-free rounding at every step (an upper bound
for the device's FMA evaluation).  Run: python fit_sincos.py"""
import numpy as np

A = np.pi / 4


def remez(f, basis, n_iter=30):
    """Minimax fit sum_j a_j basis_j(t) to f on [0, A] (absolute error)."""
    m = len(basis)
    # initial reference: Chebyshev extrema
    x = (A / 2) * (1 - np.cos(np.pi * np.arange(m + 1) / m))
    grid = np.linspace(0, A, 200001)
    for _ in range(n_iter):
        M = np.column_stack([b(x) for b in basis] + [(-1.0) ** np.arange(m + 1)])
        sol = np.linalg.solve(M, f(x))
        a, E = sol[:m], sol[m]
        err = f(grid) - sum(aj * b(grid) for aj, b in zip(a, basis))
        # new reference: alternating extrema of the error
        idx = [0]
        for i in range(1, len(grid) - 1):
            if (err[i] - err[i - 1]) * (err[i + 1] - err[i]) <= 0:
                idx.append(i)
        idx.append(len(grid) - 1)
        idx = np.array(idx)
        # keep m+1 points of largest error with alternating sign
        sel = [idx[0]]
        for i in idx[1:]:
            if np.sign(err[i]) == np.sign(err[sel[-1]]):
                if abs(err[i]) > abs(err[sel[-1]]):
                    sel[-1] = i
            else:
                sel.append(i)
        while len(sel) > m + 1:
            sel.pop(0 if abs(err[sel[0]]) < abs(err[sel[-1]]) else -1)
        if len(sel) < m + 1:
            break
        x = grid[sel]
    return a, np.max(np.abs(err))


def main():
    # sin: residual (sin t - t) fitted by t^3, t^5, t^7
    s, es = remez(lambda t: np.sin(t) - t, [lambda t: t ** 3, lambda t: t ** 5, lambda t: t ** 7])
    c, ec = remez(lambda t: np.cos(t) - 1, [lambda t: t ** 2, lambda t: t ** 4, lambda t: t ** 6, lambda t: t ** 8])
    sf, cf = s.astype(np.float32), c.astype(np.float32)
    t = np.linspace(-A, A, 400001).astype(np.float32)
    t2 = t * t
    ps = (t2 * sf[2] + sf[1]).astype(np.float32)
    ps = (t2 * ps + sf[0]).astype(np.float32)
    sv = ((t * t2) * ps + t).astype(np.float32)
    pc = (t2 * cf[3] + cf[2]).astype(np.float32)
    pc = (t2 * pc + cf[1]).astype(np.float32)
    pc = (t2 * pc + cf[0]).astype(np.float32)
    cv = (t2 * pc + np.float32(1)).astype(np.float32)
    td = t.astype(np.float64)
    print("minimax abs error (float64 coefficients): sin %.3g cos %.3g" % (es, ec))
    print("float32 evaluation max abs error: sin %.3g cos %.3g" % (np.max(np.abs(sv - np.sin(td))),
                                                                    np.max(np.abs(cv - np.cos(td)))))
    for name, v in (("S3", sf[0]), ("S5", sf[1]), ("S7", sf[2]), ("C2", cf[0]), ("C4", cf[1]), ("C6", cf[2]),
                    ("C8", cf[3])):
        print("#define BF_%s %.9ef" % (name, v))


if __name__ == "__main__":
    main()
