"""Initial populations (oracle side; test infrastructure).

* Uniform: x_a = lo_a + u (hi_a - lo_a), u from the TAG_SEED stream (c0 = sample,
  c1 = coordinate block, word a % 4).
* Carry Tiger (Sec. 5.1 describes it only as placing the initial samples along rays
  toward the box's corners, edge midpoints and face centres; that one description is
  all the paper gives, so the construction below is a reading): sample i lies on the ray from the box centre c
  to a boundary anchor, x = c + t (e * half), half = (hi - lo) / 2, t uniform in
  (0, 1).  The anchor class cycles with i: i % 3 = 0 face centres (round-robin over
  the 2d faces: axis q // 2, side q % 2 with q = (i // 3) mod 2d), 1 edge midpoints
  (free axis (i // 3) mod d at the centre, every other coordinate at a bound with a
  random sign), 2 vertices (every coordinate at a bound with a random sign).  t is
  word 0 of the TAG_SEED stream with c1 = 0; the signs are the bits of the four
  words with c1 = 1 (bit a % 32 of word a // 32).
"""
from __future__ import annotations

import numpy as np

from . import philox as PX

TAG_SEED = 8


def uniform(lo, hi, n, seed, prob_index=0):
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    d = lo.shape[0]
    i = np.arange(n)
    U = np.empty((n, d))
    for blk in range((d + 3) // 4):
        w = PX.words(seed, i, blk, TAG_SEED, 0, 1, prob_index, 0)
        for v in range(4):
            a = 4 * blk + v
            if a < d:
                U[:, a] = PX.u01(w[:, v])
    return lo + U * (hi - lo)


def carry_tiger_directions(d, n, seed, prob_index=0):
    """Anchor directions e (n, d) with entries in {-1, 0, 1} and the ray positions t (n,)."""
    i = np.arange(n)
    cls, j = i % 3, i // 3
    t = PX.u01(PX.words(seed, i, 0, TAG_SEED, 0, 0, prob_index, 0)[:, 0])
    W = PX.words(seed, i, 1, TAG_SEED, 0, 0, prob_index, 0).astype(np.uint64)
    a = np.arange(d)
    bits = (W[:, a // 32] >> (a % 32).astype(np.uint64)) & np.uint64(1)
    sgn = 2.0 * bits.astype(np.float64) - 1.0
    E = np.zeros((n, d))
    face = cls == 0
    q = j[face] % (2 * d)
    E[np.flatnonzero(face), q // 2] = np.where(q % 2 == 1, 1.0, -1.0)
    edge = np.flatnonzero(cls == 1)
    E[edge] = sgn[edge]
    E[edge, j[edge] % d] = 0.0
    vert = np.flatnonzero(cls == 2)
    E[vert] = sgn[vert]
    return E, t


def carry_tiger(lo, hi, n, seed, prob_index=0):
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    E, t = carry_tiger_directions(lo.shape[0], n, seed, prob_index)
    c, half = 0.5 * (lo + hi), 0.5 * (hi - lo)
    return c + t[:, None] * E * half
