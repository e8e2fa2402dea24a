"""Philox4x32-10 counter-based generator and Box-Muller normals.

ORACLE -- test infrastructure only (tests, smoke check, benchmark CPU leg).

Philox4x32 with 10 rounds as published by Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC'11): each round multiplies
counter words 0 and 2 by the constants 0xD2511F53 and 0xCD9E8D57, forms
(hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0), and the key is bumped by the Weyl
constants (0x9E3779B9, 0xBB67AE85) between rounds.

Normals: each 32-bit word u gives a uniform U = (u + 1/2) 2^-32 in (0, 1);
the pairs (U0, U1) and (U2, U3) give two normals each by the Box-Muller
transform sqrt(-2 ln Ua) (cos, sin)(2 pi Ub).

The random test matrices W of the peeling algorithm (Sec. 3.1, i.i.d. N(0,1)
entries) are drawn entry by entry from the counter (row, col // 4, level,
stream) under a 64-bit seed key, taking normal number col % 4, so the draw
does not depend on launch geometry.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint32(0x9E3779B9)
W1 = np.uint32(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10; all arguments uint32 arrays (broadcast)."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint32) for v in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint32)
    k1 = np.asarray(k1, dtype=np.uint32)
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    c0, c1, c2, c3 = (v.copy() for v in (c0, c1, c2, c3))
    with np.errstate(over="ignore"):
        for r in range(10):
            if r > 0:
                k0 = (k0 + W0).astype(np.uint32)
                k1 = (k1 + W1).astype(np.uint32)
            p0 = c0.astype(np.uint64) * M0
            p1 = c2.astype(np.uint64) * M1
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & MASK).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & MASK).astype(np.uint32)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def normals(rows, cols, level, stream, seed):
    """Matrix of N(0,1) draws, entry (i, j) from counter (rows[i], cols[j]//4,
    level, stream), normal number cols[j] % 4."""
    rows = np.asarray(rows, dtype=np.int64)[:, None]
    cols = np.asarray(cols, dtype=np.int64)[None, :]
    k0 = np.uint32(seed & 0xFFFFFFFF)
    k1 = np.uint32((seed >> 32) & 0xFFFFFFFF)
    u = philox4x32_10(rows.astype(np.uint32), (cols >> 2).astype(np.uint32),
                      np.uint32(level), np.uint32(stream), k0, k1)
    U = [(w.astype(np.float64) + 0.5) * 2.0 ** -32 for w in u]
    ra = np.sqrt(-2.0 * np.log(U[0]))
    rb = np.sqrt(-2.0 * np.log(U[2]))
    z = [ra * np.cos(2.0 * np.pi * U[1]), ra * np.sin(2.0 * np.pi * U[1]),
         rb * np.cos(2.0 * np.pi * U[3]), rb * np.sin(2.0 * np.pi * U[3])]
    sel = np.broadcast_to(cols & 3, z[0].shape)
    return np.choose(sel, z)
