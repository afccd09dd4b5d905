"""Butterfly interaction matrices (oracle side, dense, for small N).

Section 1.2 defines the radix-2 matrices of augmented resampling as Kronecker
products,  A_s = I_{2^{S-s}} (x) 1_{1/2} (x) I_{2^{s-1}} (x) 1_{1/M}.
Following the Remark after Lemma 3 (any doubly stochastic A_s whose product
is 1_{1/N} will do), this library reads particle indices in mixed radix,
N = a_0 a_1 ... a_{m-1}, digit 0 least significant, and lets step k mix digit
k only:

    A_k = I_{N/(a_k s_k)} (x) 1_{1/a_k} (x) I_{s_k},    s_k = a_0 ... a_{k-1}.

Index i = h*(a_k s_k) + r*s_k + l  (h, r, l the digits above, at, below k).
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np


def strides(radices: Sequence[int]) -> List[int]:
    """s_k = a_0 * ... * a_{k-1}."""
    out, s = [], 1
    for a in radices:
        out.append(s)
        s *= int(a)
    return out


def ones_over(k: int) -> np.ndarray:
    """The paper's 1_{1/k}: a k x k matrix of ones times 1/k."""
    return np.full((k, k), 1.0 / k)


def mixed_radix_A(radices: Sequence[int], k: int) -> np.ndarray:
    """Dense A_k = I_{N/(a_k s_k)} (x) 1_{1/a_k} (x) I_{s_k}."""
    N = int(np.prod(radices))
    a = int(radices[k])
    s = strides(radices)[k]
    return np.kron(np.kron(np.eye(N // (a * s)), ones_over(a)), np.eye(s))


def paper_A(S: int, M: int, s: int) -> np.ndarray:
    """Eq. (A matrices), Section 1.2: A_s = I_{2^{S-s}} (x) 1_{1/2} (x) I_{2^{s-1}} (x) 1_{1/M}, s = 1..S."""
    return np.kron(np.kron(np.kron(np.eye(2 ** (S - s)), ones_over(2)), np.eye(2 ** (s - 1))),
                   ones_over(M))


def group_members(i: int, radices: Sequence[int], k: int) -> List[int]:
    """Indices j that share every mixed-radix digit with i except digit k."""
    a = int(radices[k])
    s = strides(radices)[k]
    h, rem = divmod(i, a * s)
    l = rem % s
    return [h * a * s + r * s + l for r in range(a)]


def lemma1_partners(i: int, s: int) -> List[int]:
    """Lemma 1, eq. (explicit nonzero elements): 1-based PE indices j with
    (I_{2^{S-s}} (x) 1_{1/2} (x) I_{2^{s-1}})^{ij} != 0, for 1-based i."""
    return [((i - 1) % 2 ** (s - 1)) + (q - 1) * 2 ** (s - 1) + 2 ** s * ((i - 1) // 2 ** s) + 1
            for q in (1, 2)]


def section4_pairs(S: int, s: int):
    """Section 4.3: the pairs P_{i,s} = (l_s^i, r_s^i), 1-based, in the paper's order."""
    left, right = [], []
    for i in range(1, 2 ** (S - s) + 1):
        for j in range(1, 2 ** (s - 1) + 1):
            left.append(2 ** s * (i - 1) + (j - 1) + 1)
            right.append(2 ** s * (i - 1) + (j - 1) + 1 + 2 ** (s - 1))
    return list(zip(left, right))


def group_index(i, radices: Sequence[int], k: int):
    """Index of i's group among the N / a_k groups of digit k: (i // (a_k s_k)) * s_k + i % s_k."""
    a = int(radices[k])
    s = strides(radices)[k]
    i = np.asarray(i, dtype=np.int64)
    return (i // (a * s)) * s + i % s


def group_major(N: int, radices: Sequence[int], k: int) -> np.ndarray:
    """pi(i) = g*a_k + r for i = 0..N-1: particles numbered group by group at a step on
    digit k (g = group_index(i), r = digit k of i).  A permutation of 0..N-1."""
    a = int(radices[k])
    s = strides(radices)[k]
    i = np.arange(N, dtype=np.int64)
    return group_index(i, radices, k) * a + (i // s) % a


def set_A(radices: Sequence[int], k: int) -> np.ndarray:
    """Stage matrix of the digit set {0, k} (k >= 1): the groups are the indices that
    share every digit except digits 0 and k, each of size a_0 a_k, so A = A_k A_0
    (the two digit stages commute).  With radices (M, 2, ..., 2) this is the paper's
    A_s of eq. (A matrices) for s = k."""
    return mixed_radix_A(radices, k) @ mixed_radix_A(radices, 0)


def set_group_index(i, radices: Sequence[int], k: int):
    """Group of i for the digit set {0, k}: g = h (s_k / a_0) + l' with h the digits
    above k and l' the digits 1..k-1 of i."""
    a0, a = int(radices[0]), int(radices[k])
    s = strides(radices)[k]
    i = np.asarray(i, dtype=np.int64)
    return (i // (a * s)) * (s // a0) + (i % s) // a0


def set_group_major(N: int, radices: Sequence[int], k: int) -> np.ndarray:
    """pi(i) = g a_0 a_k + rho for the digit set {0, k}, rho = r_k a_0 + r_0 (digit k
    major, digit 0 minor: the first PE's particles, then its partner's)."""
    a0, a = int(radices[0]), int(radices[k])
    s = strides(radices)[k]
    i = np.arange(N, dtype=np.int64)
    rho = ((i // s) % a) * a0 + i % a0
    return set_group_index(i, radices, k) * (a0 * a) + rho
