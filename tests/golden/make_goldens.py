"""Writes the stored expected values of the full-size parity tests.

Every number in the files this script writes comes from the FP64 oracle
(``oracle/``) on the seeded inputs of ``paper_2002_03400_gb300.inputs``; no
value comes from the CUDA path.  Each file holds, for one configuration:

* the oracle's block ranks at every level (row bases V at levels 0..l_m,
  column bases U at levels l_m..L; block b = tau * 2^(L-l) + nu), for the
  "ranks within +-1 per block" comparison;
* the oracle factorization applied to the error metric's test matrix
  (Sec. 7, eq. error: 16 complex Gaussian columns, ``oracle.butterfly.
  error_probe`` with seed 11), on a seeded sample of output rows, for the
  ||F_gpu Omega - F_oracle Omega|| <= 1e-6 ||A Omega|| comparison;
* the exact product A Omega on the same rows (the operator's own entries,
  or for a composition the product of the two kernel operators).

Configurations (sizes of the benchmark's full-size cases):

* ``line``: the 2-D Helmholtz kernel exp(-i k r)/r between two parallel
  unit segments at distance 1 (the geometry of Sec. 7.2), n = m = 16384,
  8 points per wavelength, leaf 16 (L = 10), tol 1e-6, p = 2, r0 = 16,
  seed 0.
* ``caps``: exp(i k r)/(4 pi r) between two 60-degree caps of unit spheres
  centred at x = -3 and x = 0 (P1 -> P2), n = m = 16384, 8 points per
  wavelength, leaf 64 (L = 8), tol 1e-6, p = 4, r0 = 64 (the 3-D parameters
  of Sec. 7.3), seed 0.
* ``composition``: A = K(P3 <- P2) K(P2 <- P1) (P3 a cap at x = 3 facing
  -x) known only through the oracle factorizations of its two factors
  (each as in ``caps``), recompressed by Alg. 2 with the same parameters.

Usage: python tests/golden/make_goldens.py {line|caps|composition}
(minutes of host time each at n = 16384).
"""
from __future__ import annotations

import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import butterfly as ob            # noqa: E402
from oracle import operators as oo            # noqa: E402
from paper_2002_03400_gb300 import inputs     # noqa: E402

N = 16384
PROBE_SEED = 11
PROBE_COLS = 16
ROW_SAMPLE = 256
ROW_SEED = 2027


def cap_triple(n: int):
    """P1, P2, P3 and the wavenumber of the cap configuration."""
    P1 = inputs.cap_points(n, (-3.0, 0.0, 0.0), 60.0, axis=(1.0, 0.0, 0.0))
    P2 = inputs.cap_points(n, (0.0, 0.0, 0.0), 60.0, axis=(-1.0, 0.0, 0.0))
    P3 = inputs.cap_points(n, (3.0, 0.0, 0.0), 60.0, axis=(-1.0, 0.0, 0.0))
    k = 2.0 * math.pi / (8.0 * math.sqrt(math.pi / n))
    return P1, P2, P3, k


def sample_rows(m: int) -> np.ndarray:
    return np.sort(np.random.default_rng(ROW_SEED).choice(m, ROW_SAMPLE, replace=False))


def write(path: str, header: dict, F, Om: np.ndarray, rows: np.ndarray, exact_rows: np.ndarray) -> None:
    FO = ob.apply(F, Om, "N")[rows]
    with open(path, "w") as f:
        f.write("# Stored oracle values (FP64 oracle, oracle/ only) written by tests/golden/make_goldens.py\n")
        f.write("# Alg. 2 factorization ranks; F Omega and A Omega on sampled rows (Sec. 7, eq. error)\n")
        for k, v in header.items():
            f.write(f"# {k} = {v}\n")
        f.write(f"L {F.L}\nlm {F.lm}\n")
        for j in range(F.lm + 1):
            f.write(f"rV {j} " + " ".join(str(int(r)) for r in F.rV[j]) + "\n")
        for j in range(F.lm, F.L + 1):
            f.write(f"rU {j} " + " ".join(str(int(r)) for r in F.rU[j]) + "\n")
        for i, row in enumerate(rows):
            for name, val in (("F", FO[i]), ("A", exact_rows[i])):
                f.write(f"{name} {int(row)} " + " ".join(f"{z.real:.12e} {z.imag:.12e}" for z in val) + "\n")


def case_line(n: int = N) -> None:
    g = inputs.line_pair(n)
    op = oo.KernelOp(oo.HELMHOLTZ_2D, g.wavenumber, g.tgt, g.src)
    L = inputs.leaf_levels(n, 16)
    t0 = time.perf_counter()
    F = ob.factor(op, g.src, g.tgt, L, 1e-6, 2, 16, seed=0)
    dt = time.perf_counter() - t0
    Om = ob.error_probe(n, PROBE_SEED, PROBE_COLS)
    rows = sample_rows(n)
    exact = oo.kernel_entries(oo.HELMHOLTZ_2D, g.wavenumber, g.tgt[rows], g.src) @ Om
    write(os.path.join(HERE, f"line_pair_n{n}.txt"),
          {"config": f"line pair n=m={n}, helmholtz2d exp(-ikr)/r, 8 ppw, leaf 16, tol 1e-6, p 2, r0 16, seed 0",
           "probe": f"error_probe(n, seed={PROBE_SEED}, cols={PROBE_COLS}); rows: {ROW_SAMPLE} sampled, seed {ROW_SEED}",
           "oracle_seconds": f"{dt:.1f}", "oracle_sketch_error": f"{ob.sketch_error(op, F, 5):.6e}"},
          F, Om, rows, exact)


def _cap_factor(src, tgt, k):
    op = oo.KernelOp(oo.HELMHOLTZ_3D, k, tgt, src)
    L = inputs.leaf_levels(len(src), 64)
    return op, ob.factor(op, src, tgt, L, 1e-6, 4, 64, seed=0)


def case_caps(n: int = N) -> None:
    P1, P2, _, k = cap_triple(n)
    t0 = time.perf_counter()
    op, F = _cap_factor(P1, P2, k)
    dt = time.perf_counter() - t0
    Om = ob.error_probe(n, PROBE_SEED, PROBE_COLS)
    rows = sample_rows(n)
    exact = oo.kernel_entries(oo.HELMHOLTZ_3D, k, P2[rows], P1) @ Om
    write(os.path.join(HERE, f"caps_n{n}.txt"),
          {"config": f"caps P1 -> P2, n=m={n}, helmholtz3d exp(ikr)/(4 pi r), 8 ppw, leaf 64, tol 1e-6, p 4, "
                     "r0 64, seed 0",
           "probe": f"error_probe(n, seed={PROBE_SEED}, cols={PROBE_COLS}); rows: {ROW_SAMPLE} sampled, seed {ROW_SEED}",
           "oracle_seconds": f"{dt:.1f}", "oracle_sketch_error": f"{ob.sketch_error(op, F, 5):.6e}"},
          F, Om, rows, exact)


def case_composition(n: int = N) -> None:
    P1, P2, P3, k = cap_triple(n)
    t0 = time.perf_counter()
    op1, F1 = _cap_factor(P1, P2, k)
    op2, F2 = _cap_factor(P2, P3, k)
    comp = oo.ComposedOp(oo.FactorOp(F2), oo.FactorOp(F1))
    L = inputs.leaf_levels(n, 64)
    F = ob.factor(comp, P1, P3, L, 1e-6, 4, 64, seed=0)
    dt = time.perf_counter() - t0
    Om = ob.error_probe(n, PROBE_SEED, PROBE_COLS)
    rows = sample_rows(n)
    exact = oo.kernel_entries(oo.HELMHOLTZ_3D, k, P3[rows], P2) @ op1.matvec(Om)
    write(os.path.join(HERE, f"caps_composition_n{n}.txt"),
          {"config": f"A = K(P3<-P2) K(P2<-P1), caps n={n}, each factor and the recompression: leaf 64, tol 1e-6, "
                     "p 4, r0 64, seed 0; black box = the oracle factorizations of the two factors",
           "probe": f"error_probe(n, seed={PROBE_SEED}, cols={PROBE_COLS}); rows: {ROW_SAMPLE} sampled, seed {ROW_SEED}",
           "oracle_seconds": f"{dt:.1f}", "oracle_sketch_error": f"{ob.sketch_error(comp, F, 5):.6e}"},
          F, Om, rows, exact)


def read(path: str) -> dict:
    """Parses a file written above: L, lm, rV[j], rU[j], rows, F rows, A rows."""
    out = {"rV": {}, "rU": {}, "rows": [], "F": [], "A": [], "meta": {}}
    with open(path) as f:
        for line in f:
            if line.startswith("#"):
                if " = " in line:
                    k, v = line[2:].split(" = ", 1)
                    out["meta"][k.strip()] = v.strip()
                continue
            t = line.split()
            if t[0] in ("L", "lm"):
                out[t[0]] = int(t[1])
            elif t[0] in ("rV", "rU"):
                out[t[0]][int(t[1])] = np.array([int(v) for v in t[2:]])
            else:
                v = np.array([float(x) for x in t[2:]])
                z = v[0::2] + 1j * v[1::2]
                if t[0] == "F":
                    out["rows"].append(int(t[1]))
                out[t[0]].append(z)
    out["rows"] = np.array(out["rows"])
    out["F"] = np.array(out["F"])
    out["A"] = np.array(out["A"])
    return out


if __name__ == "__main__":
    {"line": case_line, "caps": case_caps, "composition": case_composition}[sys.argv[1]]()
