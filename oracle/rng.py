"""Counter-based Gaussian random matrices for the sketches (oracle side).

The paper only asks for i.i.d. normal entries (Alg. 1 step 1; Sec. 4.1).  Both
the oracle and the CUDA path draw them from one published counter-based
generator, Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11), each side implementing it on its own,
so that entry (row g, column c) of a sketch stream is a pure function of
(seed, stream, g, c):

  counter = (g >> 1, c, stream, 0),  key = (seed mod 2^32, seed >> 32)
  (w0, w1, w2, w3) = Philox4x32_10(counter, key)
  (a, b) = (w0, w1) if g is even else (w2, w3)
  u1 = (a + 1/2) / 2^32,  u2 = (b + 1/2) / 2^32
  z = sqrt(-ln u1) * exp(2 pi i u2)          (Box-Muller; E|z|^2 = 1)

so Re z and Im z are independent N(0, 1/2).  Pinned by the Random123
known-answer vectors (tests/golden/philox4x32_10_kat.txt) and by moment tests.
"""
import numpy as np

_M0, _M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
_W0, _W1 = np.uint64(0x9E3779B9), np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)

# stream ids: (stage << 8) | level
STAGE_V0 = 1      # Gamma_t for the leaf row bases V^0   (Alg. 2, loop "V")
STAGE_U0 = 2      # Omega_s for the leaf column bases U^L (Alg. 2, loop "U")
STAGE_W = 3       # Gamma_tau at level l (W^l)
STAGE_R = 4       # Omega_nu at level l (R^l, B)
STAGE_ERR = 5     # 16 test columns of the error metric (Sec. 7, eq. error)


def stream_id(stage: int, level: int = 0) -> int:
    return (stage << 8) | level


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox-4x32 with 10 rounds on arrays of 32-bit counters (held in uint64)."""
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & _MASK for x in (c0, c1, c2, c3))
    k0 = np.uint64(k0) & _MASK
    k1 = np.uint64(k1) & _MASK
    for _ in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> _S32, p0 & _MASK
        hi1, lo1 = p1 >> _S32, p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & _MASK, lo1, (hi0 ^ c3 ^ k1) & _MASK, lo0
        k0 = (k0 + _W0) & _MASK
        k1 = (k1 + _W1) & _MASK
    return c0, c1, c2, c3


def gaussian(seed: int, stream: int, rows, col0: int, col1: int) -> np.ndarray:
    """Complex normal matrix G[i, c - col0] for global rows ``rows`` (tree
    order) and columns col0 <= c < col1 of the given stream."""
    rows = np.asarray(rows, dtype=np.uint64)
    cols = np.arange(col0, col1, dtype=np.uint64)
    g = rows[:, None] + np.zeros_like(cols)[None, :]
    c = np.zeros_like(rows)[:, None] + cols[None, :]
    w0, w1, w2, w3 = philox4x32_10(g >> np.uint64(1), c, np.uint64(stream), 0,
                                   seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    odd = (g & np.uint64(1)).astype(bool)
    a = np.where(odd, w2, w0).astype(np.float64)
    b = np.where(odd, w3, w1).astype(np.float64)
    u1 = (a + 0.5) / 4294967296.0
    u2 = (b + 0.5) / 4294967296.0
    return np.sqrt(-np.log(u1)) * np.exp(2j * np.pi * u2)
