"""Philox4x32-7 and Box-Muller normals for the oracle (numpy, vectorised).

Philox4x32 is defined in Salmon, Moraes, Dror & Shaw, "Parallel random
numbers: as easy as 1, 2, 3" (SC'11), Section 3: a 4x32-bit counter is mixed
by R rounds of two 32x32->64 multiplications whose high halves are xor-ed
with the other two words and a round key; the key is bumped by the Weyl
constants between rounds.  This file is written from that description and
shares nothing with the CUDA implementation.  The filter uses R = 7 rounds:
Salmon et al. report Philox4x32 free of TestU01 BigCrush failures from seven
rounds on (ten being their choice with a safety margin).

The paper being implemented is silent on random numbers.  The filter's
counter layout (a reading of this library, used identically by the CUDA
path) is:

    key  = (seed mod 2^32, seed div 2^32)
    init normals        ctr = (nu // 4, 0, 0, 0)   nu = i*d + t
    propagation normals ctr = (nu // 4, n, 1, 0)   nu = pi*d + t, at time step n
    resampling uniforms ctr = (pi // 4, n, 2, 0)   word pi % 4   (32-bit draws)
    wide uniforms       ctr = (pi // 2, n, 3, 0)   words 2(pi%2), 2(pi%2)+1 (64-bit draws)

where pi is particle i's *group-major* number at step n: with digit k = n mod m,
pi = g*a_k + r, g = (i // (a_k s_k)) * s_k + i % s_k the index of i's group and
r = (i // s_k) % a_k its digit k (see ``butterfly.group_major``).  Numbering the
draws group by group lets one GPU thread that owns a group read its draws
from consecutive counter blocks.

Normals come in Box-Muller pairs: words (w0, w1) give normals 4c, 4c+1 and
(w2, w3) give 4c+2, 4c+3 of counter block c, with

    u = (2*(w0 >> 9) + 1) * 2^-24   in (0, 1), exactly representable in FP32
    v = (w1 >> 8) * 2^-24           in [0, 1), exactly representable in FP32
    z0 = sqrt(-2 ln u) cos(2 pi v),  z1 = sqrt(-2 ln u) sin(2 pi v).

Both u and v are exact binary fractions so that the FP32 device path and this
FP64 path start the transform from identical numbers.
"""
from __future__ import annotations

import numpy as np

MASK32 = np.uint64(0xFFFFFFFF)
# Round multipliers and Weyl key increments published for Philox4x32.
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85

ROUNDS = 7          # rounds of Philox4x32 in the filter's random stream

PURPOSE_INIT = 0
PURPOSE_PROPAGATE = 1
PURPOSE_RESAMPLE = 2
PURPOSE_RESAMPLE_WIDE = 3
PURPOSE_ISLAND = 4


def philox4x32(c0, c1, c2, c3, key, rounds: int = ROUNDS):
    """Philox4x32-R on arrays of counters.  Returns four uint32 arrays.

    c0..c3: array-likes broadcastable to a common shape (values < 2^32).
    key: (k0, k1) python ints < 2^32.
    """
    x0, x1, x2, x3 = (np.asarray(c, dtype=np.uint64) & MASK32 for c in (c0, c1, c2, c3))
    x0, x1, x2, x3 = np.broadcast_arrays(x0, x1, x2, x3)
    k0, k1 = int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF
    for r in range(rounds):
        if r > 0:
            k0 = (k0 + PHILOX_W0) & 0xFFFFFFFF
            k1 = (k1 + PHILOX_W1) & 0xFFFFFFFF
        p0 = PHILOX_M0 * x0          # < 2^64, exact in uint64
        p1 = PHILOX_M1 * x2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        x0, x1, x2, x3 = (hi1 ^ x1 ^ np.uint64(k0), lo1,
                          hi0 ^ x3 ^ np.uint64(k1), lo0)
    return tuple(v.astype(np.uint32) for v in (x0, x1, x2, x3))


def seed_key(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return (seed & 0xFFFFFFFF, seed >> 32)


def box_muller(wa, wb):
    """Two normals (float64) from two uint32 words, by the exact-fraction rule above."""
    wa = np.asarray(wa, dtype=np.uint64)
    wb = np.asarray(wb, dtype=np.uint64)
    u = (2.0 * (wa >> np.uint64(9)).astype(np.float64) + 1.0) * 2.0 ** -24
    v = (wb >> np.uint64(8)).astype(np.float64) * 2.0 ** -24
    rad = np.sqrt(-2.0 * np.log(u))
    ang = 2.0 * np.pi * v
    return rad * np.cos(ang), rad * np.sin(ang)


def normals(seed: int, n: int, purpose: int, count: int, dtype_index=np.int64):
    """Normals number 0..count-1 of stream (n, purpose): float64 array of length count.

    Normal nu sits in counter block nu // 4 at position nu % 4.
    """
    nblocks = (count + 3) // 4
    c = np.arange(nblocks, dtype=np.uint64)
    w0, w1, w2, w3 = philox4x32(c, n, purpose, 0, seed_key(seed))
    z0, z1 = box_muller(w0, w1)
    z2, z3 = box_muller(w2, w3)
    out = np.stack([z0, z1, z2, z3], axis=1).reshape(-1)
    return out[:count]


def resample_words(seed: int, n: int, N: int) -> np.ndarray:
    """32-bit resampling uniforms r_i (uint64 array, values < 2^32) for particles 0..N-1."""
    nblocks = (N + 3) // 4
    c = np.arange(nblocks, dtype=np.uint64)
    w = philox4x32(c, n, PURPOSE_RESAMPLE, 0, seed_key(seed))
    return np.stack(w, axis=1).reshape(-1)[:N].astype(np.uint64)


def resample_words_wide(seed: int, n: int, N: int):
    """64-bit resampling uniforms as (lo, hi) uint64 arrays of 32-bit halves."""
    nblocks = (N + 1) // 2
    c = np.arange(nblocks, dtype=np.uint64)
    w0, w1, w2, w3 = philox4x32(c, n, PURPOSE_RESAMPLE_WIDE, 0, seed_key(seed))
    lo = np.stack([w0, w2], axis=1).reshape(-1)[:N].astype(np.uint64)
    hi = np.stack([w1, w3], axis=1).reshape(-1)[:N].astype(np.uint64)
    return lo, hi


def normals_at(seed: int, n: int, purpose: int, nu) -> np.ndarray:
    """Normals number ``nu`` (any integer array) of stream (n, purpose), float64."""
    nu = np.asarray(nu, dtype=np.uint64)
    w0, w1, w2, w3 = philox4x32(nu >> np.uint64(2), n, purpose, 0, seed_key(seed))
    z0, z1 = box_muller(w0, w1)
    z2, z3 = box_muller(w2, w3)
    pos = (nu & np.uint64(3)).astype(np.int64)
    return np.choose(pos, [z0, z1, z2, z3])


def resample_words_at(seed: int, n: int, idx) -> np.ndarray:
    """32-bit resampling uniforms of particles ``idx`` (uint64 values < 2^32)."""
    idx = np.asarray(idx, dtype=np.uint64)
    w = philox4x32(idx >> np.uint64(2), n, PURPOSE_RESAMPLE, 0, seed_key(seed))
    return np.choose((idx & np.uint64(3)).astype(np.int64), w).astype(np.uint64)


def resample_words_wide_at(seed: int, n: int, idx):
    """64-bit resampling uniforms of particles ``idx`` as (lo, hi) uint64 arrays."""
    idx = np.asarray(idx, dtype=np.uint64)
    w0, w1, w2, w3 = philox4x32(idx >> np.uint64(1), n, PURPOSE_RESAMPLE_WIDE, 0, seed_key(seed))
    odd = (idx & np.uint64(1)).astype(bool)
    lo = np.where(odd, w2, w0).astype(np.uint64)
    hi = np.where(odd, w3, w1).astype(np.uint64)
    return lo, hi


def island_words_at(seed: int, n: int, stage: int, idx) -> np.ndarray:
    """32-bit uniforms of islands ``idx`` at island-resampling stage ``stage`` of time n:
    counter (i / 4, n, PURPOSE_ISLAND, stage), word i mod 4."""
    idx = np.asarray(idx, dtype=np.uint64)
    w = philox4x32(idx >> np.uint64(2), n, PURPOSE_ISLAND, stage, seed_key(seed))
    return np.choose((idx & np.uint64(3)).astype(np.int64), w).astype(np.uint64)
