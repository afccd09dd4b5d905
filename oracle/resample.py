"""Integer multinomial draw inside one interaction group (oracle side).

Algorithm 2 (multinomial resampling) and the sampling line of Algorithm 3
(augmented resampling) draw each new particle i from the weighted empirical
law of the particles j it may interact with,

    P(anc_i = j) = A^{ij} V^j / sum_l A^{il} V^l,

where for the butterfly matrices of Section 1.2 (generalised to mixed radix)
A^{ij} = 1/a for the a members j of i's group.  The paper fixes no number
format for this draw.  This library's reading fixes one integer rule that the
oracle and the CUDA path both implement, so that given equal inputs the
ancestor indices are equal bit for bit:

  1. delta_j = fp32(lw_j - M_G), M_G = max of the group's log-weights
     (so the largest member has delta = 0 exactly);
  2. e_j = fp32(exp(delta_j))  (decision taken in FP32, the kernel's precision);
  3. q_j = floor(e_j * 2^B), B = 24 for groups of a <= 256 members, else 32;
  4. P_j = q_0 + ... + q_j (exact integers), Q = P_{a-1} (>= 2^B > 0);
  5. u_i = floor(r_i * Q / 2^32) with a 32-bit uniform r_i when a <= 256,
     u_i = floor(r_i * Q / 2^64) with a 64-bit uniform when a > 256;
  6. anc_i = min { j : P_j > u_i }  =  #{ j : P_j <= u_i }.

The law of step 6 is exactly  #{r : P_{j-1} <= floor(rQ/2^W) < P_j} / 2^W,
which differs from q_j / Q by less than 2^-W per member; members with
e_j < 2^-B are never drawn (bias at most a * 2^-B of the group weight).
"""
from __future__ import annotations

import numpy as np

NARROW_MAX_RADIX = 256


def qbits(a: int) -> int:
    """Fractional bits of the quantised weights for a group of a members."""
    return 24 if a <= NARROW_MAX_RADIX else 32


def quantise(lw: np.ndarray, axis: int) -> np.ndarray:
    """Steps 1-3 along ``axis`` (the group axis).  Returns uint64 q of lw's shape.

    Non-finite log-weights are treated as -inf (weight zero).  A group whose
    members are all -inf gets q = 0 everywhere; ``draw`` then keeps every
    particle in place.
    """
    lw = np.where(np.isfinite(lw), lw, -np.inf)
    a = lw.shape[axis]
    M = np.max(lw, axis=axis, keepdims=True)
    with np.errstate(invalid="ignore"):
        delta = (lw - M).astype(np.float32)
    delta = np.where(np.isfinite(M), delta, np.float32(-np.inf))
    e = np.exp(delta.astype(np.float64)).astype(np.float32)
    q = np.floor(e.astype(np.float64) * 2.0 ** qbits(a))
    return q.astype(np.uint64)


def mulhi64(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """floor(x * y / 2^64) for uint64 arrays, by 32-bit limbs (exact)."""
    m = np.uint64(0xFFFFFFFF)
    s = np.uint64(32)
    x = np.asarray(x, dtype=np.uint64)
    y = np.asarray(y, dtype=np.uint64)
    xl, xh = x & m, x >> s
    yl, yh = y & m, y >> s
    p00, p01, p10, p11 = xl * yl, xl * yh, xh * yl, xh * yh
    mid = (p00 >> s) + (p01 & m) + (p10 & m)
    return p11 + (p01 >> s) + (p10 >> s) + (mid >> s)


def scaled_uniform(r, Q, a: int, r_hi=None) -> np.ndarray:
    """Step 5: the integer uniform u in [0, Q)."""
    r = np.asarray(r, dtype=np.uint64)
    Q = np.asarray(Q, dtype=np.uint64)
    if a <= NARROW_MAX_RADIX:
        return (r * Q) >> np.uint64(32)       # r < 2^32 and Q <= 2^32: no overflow
    r64 = (np.asarray(r_hi, dtype=np.uint64) << np.uint64(32)) | r
    return mulhi64(r64, Q)


def draw(q: np.ndarray, u: np.ndarray, axis: int) -> np.ndarray:
    """Steps 4 and 6 along ``axis``: member index (within the group) of each draw.

    q: quantised weights with the group on ``axis``; u: integer uniforms of the
    same shape (one per new particle, u < Q of its group).  Returns int64.
    A group with Q = 0 (all weights zero) maps every member to itself.
    """
    P = np.cumsum(q, axis=axis, dtype=np.uint64)
    a = q.shape[axis]
    Pm = np.moveaxis(P, axis, -1)            # (..., a) prefix sums per group
    um = np.moveaxis(np.asarray(u, dtype=np.uint64), axis, -1)   # (..., a) draws per group
    if a <= 64:
        count = (Pm[..., None, :] <= um[..., :, None]).sum(axis=-1)   # #{j : P_j <= u_i}
    else:
        flatP = Pm.reshape(-1, a)
        flatu = um.reshape(-1, a)
        count = np.empty(flatu.shape, dtype=np.int64)
        for g in range(flatP.shape[0]):
            count[g] = np.searchsorted(flatP[g], flatu[g], side="right")
        count = count.reshape(um.shape)
    Q = Pm[..., -1:]
    self_idx = np.broadcast_to(np.arange(a), count.shape)
    count = np.where(Q == 0, self_idx, count)
    return np.moveaxis(count, -1, axis).astype(np.int64)


def exact_law(q: np.ndarray, a_bits_wide: bool = False) -> np.ndarray:
    """Exact law of the member index drawn from quantised weights q (1-D), as
    probabilities: P(j) = #{r in [0, 2^W): P_{j-1} <= floor(r Q / 2^W) < P_j} / 2^W.

    #{r : floor(r Q / 2^W) < P} = ceil(P 2^W / Q), computed with Python integers.
    """
    W = 64 if a_bits_wide else 32
    P = np.cumsum(np.asarray(q, dtype=np.uint64)).tolist()
    Q = int(P[-1])
    bound = [0] + [-(-(int(p) << W) // Q) for p in P]   # ceil(P*2^W/Q)
    counts = [bound[j + 1] - bound[j] for j in range(len(P))]
    return np.array([c / float(1 << W) for c in counts])
