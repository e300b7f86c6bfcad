"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds only input construction: point geometries, wavenumbers,
random factor blocks for an exactly-butterfly operator, operator-size draws
and request traces.  It contains none of the factorization's arithmetic
(no sketching, peeling, QR truncation, least squares or butterfly apply).

Geometries stand in for the paper's integral-equation workloads:

* ``line_pair``: two parallel segments of length 1 at distance 1, the
  geometry of the 2D scattering experiment (Sec. 7.2), with the kernel
  exp(-i k r)/r evaluated directly instead of the H-matrix inverse.
* ``arc_pair``: two separated circular arcs (batched workload).
* ``cap_points``: Fibonacci-sampled spherical caps (3D kernels, Sec. 7.3
  style surfaces); ``cap_pair`` two separated caps, ``hemisphere_pair``
  the two adjacent hemispheres of the 3D experiment (Sec. 7.3).
* ``exact_butterfly``: random orthonormal U, V, R, W blocks and Gaussian B
  blocks of constant rank r, as in the exact-recovery experiment (Sec. 7.1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# kernel ids shared with include/butterfly.h (bf_kernel_type)
KERNEL_HELMHOLTZ_2D = 1   # exp(-i k r) / r
KERNEL_HELMHOLTZ_3D = 2   # exp(+i k r) / (4 pi r)
KERNEL_DFT = 3            # exp(-2 pi i x y), 1-D points


@dataclass
class Geometry:
    """Source and target point sets (rows = points) plus the kernel to use."""
    src: np.ndarray
    tgt: np.ndarray
    kernel: int
    wavenumber: float
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.src.shape[0]

    @property
    def m(self) -> int:
        return self.tgt.shape[0]

    @property
    def dim(self) -> int:
        return self.src.shape[1]


def line_pair(n: int, m: int | None = None, ppw: float = 8.0) -> Geometry:
    """Sources uniformly spaced on [0,1]x{0}, targets on [0,1]x{1}.

    Point j sits at the midpoint ((j+1/2)/n, y).  The wavenumber gives
    ``ppw`` points per wavelength on the source line: k = 2*pi/(ppw*h),
    h = 1/n (k = pi*n/4 at 8 points per wavelength)."""
    m = n if m is None else m
    src = np.stack([(np.arange(n) + 0.5) / n, np.zeros(n)], axis=1)
    tgt = np.stack([(np.arange(m) + 0.5) / m, np.ones(m)], axis=1)
    k = 2.0 * math.pi / (ppw / n)
    return Geometry(src, tgt, KERNEL_HELMHOLTZ_2D, k, f"line_pair_n{n}",
                    {"ppw": ppw})


def arc_pair(n: int, seed: int, m: int | None = None) -> Geometry:
    """Two separated circular arcs of radius 1, centres (0,0) and (3,0).

    Each arc's opening angle is drawn from U[30, 90] degrees and the arc is
    centred on the line joining the two centres (arc 1 faces +x, arc 2 faces
    -x).  Points are midpoint-uniform in angle.  The points-per-wavelength
    figure is drawn from U[4, 16]; k = 2*pi/(ppw*h) with h the source arc's
    point spacing."""
    m = n if m is None else m
    rng = np.random.default_rng(np.random.SeedSequence([0xA5C, seed]))
    a1 = math.radians(rng.uniform(30.0, 90.0))
    a2 = math.radians(rng.uniform(30.0, 90.0))
    ppw = float(rng.uniform(4.0, 16.0))
    t1 = -a1 / 2 + (np.arange(n) + 0.5) * (a1 / n)
    t2 = math.pi - a2 / 2 + (np.arange(m) + 0.5) * (a2 / m)
    src = np.stack([np.cos(t1), np.sin(t1)], axis=1)
    tgt = np.stack([3.0 + np.cos(t2), np.sin(t2)], axis=1)
    h = a1 / n
    k = 2.0 * math.pi / (ppw * h)
    return Geometry(src, tgt, KERNEL_HELMHOLTZ_2D, k, f"arc_pair_n{n}_s{seed}",
                    {"ppw": ppw, "angle1": a1, "angle2": a2})


def cap_points(n: int, centre, half_angle_deg: float = 60.0,
               axis=(1.0, 0.0, 0.0)) -> np.ndarray:
    """Fibonacci sampling of a spherical cap of the unit sphere.

    The cap is the set of unit vectors within ``half_angle_deg`` of ``axis``,
    translated to ``centre``.  Point j uses the equal-area height
    1 - (j+1/2)/n * (1 - cos(half_angle)) and golden-angle azimuth."""
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    c = 1.0 - math.cos(math.radians(half_angle_deg))
    j = np.arange(n) + 0.5
    z = 1.0 - j / n * c
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    golden = math.pi * (3.0 - math.sqrt(5.0))
    phi = golden * np.arange(n)
    local = np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)
    # rotate local +z onto axis
    ez = np.array([0.0, 0.0, 1.0])
    v = np.cross(ez, axis)
    s = np.linalg.norm(v)
    cth = float(ez @ axis)
    if s < 1e-15:
        rot = np.eye(3) if cth > 0 else np.diag([1.0, -1.0, -1.0])
    else:
        vx = np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])
        rot = np.eye(3) + vx + vx @ vx * ((1 - cth) / (s * s))
    return local @ rot.T + np.asarray(centre, dtype=np.float64)


def cap_pair(n: int, m: int | None = None, ppw: float = 8.0,
             src_centre=(-3.0, 0.0, 0.0), tgt_centre=(0.0, 0.0, 0.0)) -> Geometry:
    """Sources on a 60-degree cap of the unit sphere at ``src_centre`` facing
    +x, targets on a cap of the sphere at ``tgt_centre`` facing -x.  The caps
    have area pi; h = sqrt(pi/n) and k = 2*pi/(ppw*h).  Kernel
    exp(i k r)/(4 pi r)."""
    m = n if m is None else m
    src = cap_points(n, src_centre, 60.0, axis=(1.0, 0.0, 0.0))
    tgt = cap_points(m, tgt_centre, 60.0, axis=(-1.0, 0.0, 0.0))
    h = math.sqrt(math.pi / n)
    k = 2.0 * math.pi / (ppw * h)
    return Geometry(src, tgt, KERNEL_HELMHOLTZ_3D, k, f"cap_pair_n{n}",
                    {"ppw": ppw})


def hemisphere_pair(n: int, m: int | None = None, ppw: float = 10.0) -> Geometry:
    """Two adjacent unit hemispheres (the 3D experiment, Sec. 7.3): sources
    on the upper half of the unit sphere (z > 0), targets on the lower half
    (z < 0), each Fibonacci-sampled with equal-area heights, so the two
    surfaces meet along the equator (weak admissibility: every level has
    blocks that touch).  No point lies on the equator (|z| >= 1/(2n)).  Each
    half has area 2 pi; h = sqrt(2 pi / n) and k = 2 pi / (ppw h), ppw = 10
    as the paper intends.  Kernel exp(i k r)/(4 pi r)."""
    m = n if m is None else m
    src = cap_points(n, (0.0, 0.0, 0.0), 90.0, axis=(0.0, 0.0, 1.0))
    tgt = cap_points(m, (0.0, 0.0, 0.0), 90.0, axis=(0.0, 0.0, -1.0))
    h = math.sqrt(2.0 * math.pi / n)
    k = 2.0 * math.pi / (ppw * h)
    return Geometry(src, tgt, KERNEL_HELMHOLTZ_3D, k, f"hemisphere_pair_n{n}", {"ppw": ppw})


def dft_points(n: int) -> Geometry:
    """1-D points for the DFT matrix A[j, q] = exp(-2 pi i x_j y_q) with
    x_j = j/n (targets) and y_q = q (sources), i.e. A = numpy.fft.fft's
    matrix."""
    tgt = (np.arange(n) / n).reshape(n, 1)
    src = np.arange(n, dtype=np.float64).reshape(n, 1)
    return Geometry(src, tgt, KERNEL_DFT, 1.0, f"dft_n{n}")


# --------------------------------------------------------------------------
# Exactly-butterfly operator (exact-recovery experiment, Sec. 7.1)
# --------------------------------------------------------------------------

def _haar_unitary(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    """rows x cols matrix with orthonormal columns, Haar-distributed:
    QR of a complex Gaussian matrix with the phases of diag(R) moved into Q
    (Mezzadri, Notices AMS 2007)."""
    g = (rng.standard_normal((rows, cols)) + 1j * rng.standard_normal((rows, cols))) / math.sqrt(2)
    q, r = np.linalg.qr(g)
    d = np.diag(r)
    ph = d / np.where(np.abs(d) == 0, 1.0, np.abs(d))
    return q * ph[None, :]


@dataclass
class ExactButterfly:
    """Blocks of a hybrid butterfly with constant rank r at every block.

    Block index at level j (tau at level j of the target tree, nu at level
    L-j of the source tree) is b = tau * 2**(L-j) + nu.  Shapes:
      V0[nu]      : (leaf rows of S_nu) x r     (level 0, tau = root)
      W[j][b]     : 2r x r                       j = 1..lm
      B[b]        : r x r                        level lm
      R[j][b]     : 2r x r                       j = lm..L-1
      U[tau]      : (leaf rows of T_tau) x r    (level L, nu = root)
    Rows of W[j][b] stack (pt, 2nu) then (pt, 2nu+1); rows of R[j][b] stack
    (2tau, pnu) then (2tau+1, pnu).  All of V0, W, R, U have orthonormal
    columns; B is complex Gaussian."""
    n: int
    m: int
    L: int
    lm: int
    r: int
    V0: np.ndarray
    W: dict
    B: np.ndarray
    R: dict
    U: np.ndarray


def exact_butterfly(n: int, leaf: int, r: int, seed: int, m: int | None = None) -> ExactButterfly:
    m = n if m is None else m
    L = int(round(math.log2(n // leaf)))
    assert leaf << L == n and (m % (1 << L)) == 0, "n must be leaf * 2^L"
    lm = L // 2
    nb = 1 << L
    rng = np.random.default_rng(np.random.SeedSequence([0xB0F, seed]))
    V0 = np.stack([_haar_unitary(rng, n >> L, r) for _ in range(nb)])
    W = {j: np.stack([_haar_unitary(rng, 2 * r, r) for _ in range(nb)]) for j in range(1, lm + 1)}
    B = (rng.standard_normal((nb, r, r)) + 1j * rng.standard_normal((nb, r, r))) / math.sqrt(2)
    R = {j: np.stack([_haar_unitary(rng, 2 * r, r) for _ in range(nb)]) for j in range(lm, L)}
    U = np.stack([_haar_unitary(rng, m >> L, r) for _ in range(nb)])
    return ExactButterfly(n, m, L, lm, r, V0, W, B, R, U)


# --------------------------------------------------------------------------
# Batched and serving workloads
# --------------------------------------------------------------------------

def batched_sizes(count: int = 64, seed: int = 3) -> list[int]:
    """Operator sizes drawn uniformly from {1024, 2048, 4096, 8192}."""
    rng = np.random.default_rng(np.random.SeedSequence([0xBA7, seed]))
    return [int(x) for x in rng.choice([1024, 2048, 4096, 8192], size=count)]


def random_rhs(rows: int, cols: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """Complex Gaussian right-hand sides (user point order)."""
    rng = np.random.default_rng(np.random.SeedSequence([0x2E5, seed]))
    x = (rng.standard_normal((rows, cols)) + 1j * rng.standard_normal((rows, cols))) / math.sqrt(2)
    return x.astype(dtype)


@dataclass
class Request:
    t: float          # arrival time (s)
    kind: str         # "apply" or "factor"
    target: int       # index of the resident factorization (apply) or size (factor)
    nrhs: int = 0
    dtype: str = "c128"
    geometry: str = ""


def serving_trace(duration_s: float, rate_hz: float, seed: int,
                  resident: int, factor_sizes=(4096, 16384, 65536),
                  apply_fraction: float = 0.8) -> list[Request]:
    """Poisson arrivals: ``apply_fraction`` applies with 1..64 right-hand
    sides (complex64 or complex128 with equal odds) against one of
    ``resident`` factorizations, the rest factor requests with n drawn from
    ``factor_sizes`` on arcs or caps."""
    rng = np.random.default_rng(np.random.SeedSequence([0x5E7, seed]))
    t = 0.0
    out = []
    while True:
        t += float(rng.exponential(1.0 / rate_hz))
        if t >= duration_s:
            break
        if rng.random() < apply_fraction:
            out.append(Request(t, "apply", int(rng.integers(resident)),
                               int(rng.integers(1, 65)),
                               "c64" if rng.random() < 0.5 else "c128"))
        else:
            out.append(Request(t, "factor", int(rng.choice(factor_sizes)), 0, "c64",
                               "arc" if rng.random() < 0.5 else "cap"))
    return out


def leaf_levels(n: int, leaf: int) -> int:
    """Tree depth L: the smallest L with ceil(n / 2^L) <= leaf."""
    L = 0
    while -(-n // (1 << L)) > leaf:
        L += 1
    return L
