"""Algorithm 1's initialisation, "initialise W_i to a random orthogonal
matrix", as a seeded draw from the Haar distribution: the Q factor (with a
positive-diagonal R) of a v_i x k matrix of independent standard normals.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): it gives the oracle the
W^0 the library draws when srm_init receives no W0, from the same published
definition and shares no code with the CUDA path.

The normals come from the counter-based generator Philox4x64-10 (Salmon,
Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC 2011): key (seed, 0) and counter (b, i, 0, 0) for block b of subject i.
Each 64-bit output word w gives the uniform u = ((w >> 12) + 1/2) 2^-52 in
(0, 1).  The word pairs (w0, w1) and (w2, w3) of block b give entries
4b .. 4b + 3 of G_i, in row-major order, by the Box-Muller transform:
sqrt(-2 ln u_a) cos(2 pi u_b) and sqrt(-2 ln u_a) sin(2 pi u_b).
"""
from __future__ import annotations

import numpy as np

_MASK32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)
# round multipliers and key increments of Philox4x64 (the published constants)
_M0 = np.uint64(0xD2E7470EE14C6C93)
_M1 = np.uint64(0xCA5A826395121157)
_W0 = np.uint64(0x9E3779B97F4A7C15)
_W1 = np.uint64(0xBB67AE8584CAA73B)


def _mulhilo(a: np.uint64, b: np.ndarray):
    """(high, low) 64-bit halves of the 128-bit product a * b, elementwise."""
    a0, a1 = a & _MASK32, a >> _S32
    b0, b1 = b & _MASK32, b >> _S32
    t = a0 * b0
    m1 = a1 * b0 + (t >> _S32)
    m2 = a0 * b1 + (m1 & _MASK32)
    hi = a1 * b1 + (m1 >> _S32) + (m2 >> _S32)
    lo = a * b  # wraps modulo 2^64
    return hi, lo


def philox4x64_10(counter, key):
    """Philox4x64 with ten rounds.  counter: 4 arrays (or ints) of uint64,
    key: 2 uint64.  Returns the 4 output words (uint64 arrays)."""
    with np.errstate(over="ignore"):
        c = [np.asarray(x, dtype=np.uint64) for x in counter]
        k0, k1 = np.uint64(key[0]), np.uint64(key[1])
        for _ in range(10):
            hi0, lo0 = _mulhilo(_M0, c[0])
            hi1, lo1 = _mulhilo(_M1, c[2])
            c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
            k0 = k0 + _W0
            k1 = k1 + _W1
    return c


def unit_open(w: np.ndarray) -> np.ndarray:
    """((w >> 12) + 1/2) 2^-52: a uniform in (0, 1) from a 64-bit word (exact
    in FP64: at least 2^-53, at most 1 - 2^-53)."""
    return ((w >> np.uint64(12)).astype(np.float64) + 0.5) * 2.0 ** -52


def standard_normals(seed: int, subject: int, n: int) -> np.ndarray:
    """The first n normals of subject `subject` (entries of G_i, row-major)."""
    nb = (n + 3) // 4
    b = np.arange(nb, dtype=np.uint64)
    zero = np.zeros(nb, dtype=np.uint64)
    w = philox4x64_10([b, np.full(nb, subject, dtype=np.uint64), zero, zero], (seed, 0))
    z = np.empty((nb, 4))
    for p in range(2):
        r = np.sqrt(-2.0 * np.log(unit_open(w[2 * p])))
        th = 2.0 * np.pi * unit_open(w[2 * p + 1])
        z[:, 2 * p] = r * np.cos(th)
        z[:, 2 * p + 1] = r * np.sin(th)
    return z.reshape(-1)[:n]


def haar_w0(seed: int, subject: int, v: int, k: int) -> np.ndarray:
    """W^0_i (v x k, FP64): Q of the QR factorisation of G_i with the column
    signs that make diag(R) positive."""
    G = standard_normals(seed, subject, v * k).reshape(v, k)
    q, r = np.linalg.qr(G)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s[None, :]
