"""Philox4x32-10 and the random-stream layout of the method (oracle side).

Philox4x32-10 is written from its published definition (Salmon, Moraes, Dror,
Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3", SC'11, Section 3): ten
rounds of the 4x32 multiply-hi/lo S-box with the two round multipliers, the
key bumped by the two Weyl constants between rounds.  Pinned by the published
known-answer vectors in tests/golden/philox_kat.txt.

Stream layout (identical on the CUDA side, implemented there separately):

    key = (seed mod 2^32, seed div 2^32)
    ctr = (c0, c1, (tag << 24) | ((cycle & 0xffff) << 8) | (step & 0xff),
           (prob << 16) | (k & 0xffff))

``c0`` is a sample / slot / row index, ``c1`` a sub-index (coordinate block of
four), ``k`` a perturbation index.  Uniforms are u(w) = (2*(w >> 9) + 1) 2^-24
(exact in binary32), normals come from Box-Muller on pairs of words.
"""
from __future__ import annotations

import numpy as np

MUL0, MUL1 = 0xD2511F53, 0xCD9E8D57
WEYL0, WEYL1 = 0x9E3779B9, 0xBB67AE85
MASK32 = np.uint64(0xFFFFFFFF)

# stream tags
TAG_RM = 1          # Repulse Monkey: parent choice (word 0) and ray position (word 1)
TAG_RM_DIR = 2      # Repulse Monkey: ray direction normals
TAG_GR_MAT = 3      # Golden Rooster: Gaussian matrix entries
TAG_GR_T = 4        # Golden Rooster: ray position
TAG_UNIFORM = 5     # uniform redraw in the box
TAG_HLC = 6         # Hands Like Clouds perturbations z_k
TAG_NOISE = 7       # additive evaluation noise


def philox4x32_10(ctr, key):
    """ctr: (..., 4) integers; key: (..., 2) integers.  Returns (..., 4) uint32."""
    c = np.asarray(ctr, dtype=np.uint64) & MASK32
    k = np.asarray(key, dtype=np.uint64) & MASK32
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0 = np.broadcast_to(k[..., 0], c0.shape).copy()
    k1 = np.broadcast_to(k[..., 1], c0.shape).copy()
    for _ in range(10):
        p0 = np.uint64(MUL0) * c0
        p1 = np.uint64(MUL1) * c2
        n0 = (p1 >> np.uint64(32)) ^ c1 ^ k0
        n1 = p1 & MASK32
        n2 = (p0 >> np.uint64(32)) ^ c3 ^ k1
        n3 = p0 & MASK32
        c0, c1, c2, c3 = n0, n1, n2, n3
        k0 = (k0 + np.uint64(WEYL0)) & MASK32
        k1 = (k1 + np.uint64(WEYL1)) & MASK32
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def make_key(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint64)


def make_ctr(c0, c1, tag, cycle, step, prob, k):
    c0 = np.asarray(c0, dtype=np.uint64)
    c1 = np.asarray(c1, dtype=np.uint64)
    c0, c1 = np.broadcast_arrays(c0, c1)
    c2 = np.full(c0.shape, (int(tag) << 24) | ((int(cycle) & 0xFFFF) << 8) | (int(step) & 0xFF), np.uint64)
    c3 = np.full(c0.shape, ((int(prob) & 0xFFFF) << 16) | (int(k) & 0xFFFF), np.uint64)
    return np.stack([c0, c1, c2, c3], axis=-1)


def words(seed, c0, c1, tag, cycle, step, prob, k):
    return philox4x32_10(make_ctr(c0, c1, tag, cycle, step, prob, k), make_key(seed))


def u01(w):
    """Uniform in (0, 1): (2*(w >> 9) + 1) * 2^-24, exact in binary32."""
    w = np.asarray(w, dtype=np.uint64)
    return ((w >> np.uint64(9)) * np.uint64(2) + np.uint64(1)).astype(np.float64) * 2.0 ** -24


def box_muller(w):
    """(..., 4) words -> (..., 4) standard normals, pairs (w0, w1) and (w2, w3)."""
    u = u01(w)
    r01 = np.sqrt(-2.0 * np.log(u[..., 0]))
    r23 = np.sqrt(-2.0 * np.log(u[..., 2]))
    a01 = 2.0 * np.pi * u[..., 1]
    a23 = 2.0 * np.pi * u[..., 3]
    return np.stack([r01 * np.cos(a01), r01 * np.sin(a01), r23 * np.cos(a23), r23 * np.sin(a23)], axis=-1)


def normal_rows(seed, rows, d, tag, cycle, step, prob, k):
    """Standard normals z[r, j] for row ids ``rows`` and coordinates j < d.

    Coordinate j uses normal (j mod 4) of the Philox block with c1 = j // 4.
    """
    rows = np.asarray(rows, dtype=np.uint64)
    nb = (d + 3) // 4
    r2, b2 = np.meshgrid(rows, np.arange(nb, dtype=np.uint64), indexing="ij")
    z = box_muller(words(seed, r2, b2, tag, cycle, step, prob, k))   # (R, nb, 4)
    return z.reshape(rows.shape[0], nb * 4)[:, :d]


def _lowbias32(v):
    """Wellons' 'lowbias32' integer finalizer (xorshift-multiply, 3 rounds)."""
    v = v & MASK32
    v ^= v >> np.uint64(16)
    v = (v * np.uint64(0x7FEB352D)) & MASK32
    v ^= v >> np.uint64(15)
    v = (v * np.uint64(0x846CA68B)) & MASK32
    v ^= v >> np.uint64(16)
    return v


def point_key(X):
    """Two 32-bit words identifying an evaluation point: coordinate j's binary32
    bit pattern b_j is mixed as v_j = lowbias32(b_j xor (j * 0x9E3779B9)); the
    words are sum_j v_j and xor_j v_j (2j + 1) (mod 2^32)."""
    X32 = np.ascontiguousarray(np.asarray(X, dtype=np.float64).astype(np.float32))
    b = X32.view(np.uint32).astype(np.uint64)
    j = np.arange(X32.shape[1], dtype=np.uint64)
    v = _lowbias32(b ^ ((j * np.uint64(0x9E3779B9)) & MASK32)[None, :])
    h1 = v.sum(axis=1) & MASK32
    h2 = np.bitwise_xor.reduce((v * (np.uint64(2) * j + np.uint64(1))[None, :]) & MASK32, axis=1)
    return h1, h2


def point_noise(seed, prob, X):
    """One standard normal per evaluation point (Sec. 5.6 noise, keyed by the point)."""
    h1, h2 = point_key(X)
    ctr = np.stack([h1, h2, np.full_like(h1, TAG_NOISE << 24), np.full_like(h1, (int(prob) & 0xFFFF) << 16)],
                   axis=-1)
    w = philox4x32_10(ctr, make_key(seed))
    u = u01(w)
    return np.sqrt(-2.0 * np.log(u[:, 0])) * np.cos(2.0 * np.pi * u[:, 1])


def uniform_rows(seed, rows, d, tag, cycle, step, prob, k):
    rows = np.asarray(rows, dtype=np.uint64)
    nb = (d + 3) // 4
    r2, b2 = np.meshgrid(rows, np.arange(nb, dtype=np.uint64), indexing="ij")
    u = u01(words(seed, r2, b2, tag, cycle, step, prob, k))
    return u.reshape(rows.shape[0], nb * 4)[:, :d]
