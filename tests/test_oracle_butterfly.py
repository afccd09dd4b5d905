"""Pins for the butterfly interaction structure (Section 1.2, Lemmas 1-2, Figures 1-2)."""
import itertools
import os

import numpy as np
import pytest

from oracle import butterfly as bf


def _read_fig1(path):
    blocks, cur = {}, None
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("A"):
            cur = line
            blocks[cur] = []
        else:
            blocks[cur].append([int(v) for v in line.split()])
    return {k: np.array(v) for k, v in blocks.items()}


def test_fig1_matrices(golden_dir):
    """Figure 1: A_1, A_2 for m = 4 PEs, M = 3, from eq. (A matrices)."""
    pat = _read_fig1(os.path.join(golden_dir, "fig1_A_m4_M3.txt"))
    for s in (1, 2):
        want = 0.5 * np.kron(pat[f"A{s}"], np.full((3, 3), 1.0 / 3))
        np.testing.assert_array_equal(bf.paper_A(S=2, M=3, s=s), want)
    # Lemma 2: the product over all stages is 1_{1/N}
    prod = bf.paper_A(2, 3, 2) @ bf.paper_A(2, 3, 1)
    np.testing.assert_allclose(prod, np.full((12, 12), 1 / 12), atol=1e-15)


def test_fig2_pairs(golden_dir):
    """Figure 2 / Section 4.3: pairs P_{i,s} for m = 8 PEs."""
    for line in open(os.path.join(golden_dir, "fig2_pairs_m8.txt")):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        s = int(parts[0])
        want = [tuple(int(v) for v in p.split(",")) for p in parts[1:]]
        assert bf.section4_pairs(3, s) == want
        # each pair is exactly the nonzero set of Lemma 1 for its members
        for l, r in want:
            assert sorted(bf.lemma1_partners(l, s)) == [l, r]
            assert sorted(bf.lemma1_partners(r, s)) == [l, r]


RADIX_SETS = [(2, 2), (2, 3), (3, 2, 2), (4, 2), (2, 2, 2), (5,), (3, 4), (2, 3, 4)]


@pytest.mark.parametrize("radices", RADIX_SETS)
def test_lemma1_lemma2_mixed_radix(radices):
    """Lemma 1 (symmetric, idempotent, doubly stochastic) and Lemma 2 (product = 1_{1/N})
    for the mixed-radix generalisation that the Remark after Lemma 3 allows."""
    N = int(np.prod(radices))
    prod = np.eye(N)
    for k in range(len(radices)):
        A = bf.mixed_radix_A(radices, k)
        np.testing.assert_allclose(A, A.T)
        np.testing.assert_allclose(A @ A, A, atol=1e-15)
        np.testing.assert_allclose(A.sum(0), 1)
        np.testing.assert_allclose(A.sum(1), 1)
        # nonzero columns of row i are exactly i's group (all digits but k shared)
        for i in range(N):
            nz = sorted(np.nonzero(A[i])[0].tolist())
            assert nz == sorted(bf.group_members(i, radices, k))
            assert np.isclose(A[i, i], 1.0 / radices[k])
        prod = A @ prod
    np.testing.assert_allclose(prod, np.full((N, N), 1.0 / N), atol=1e-14)


@pytest.mark.parametrize("S", [1, 2, 3, 4, 5])
def test_lemma1_explicit_partner_formula(S):
    """Eq. (explicit nonzero elements) equals the nonzero columns of I (x) 1_{1/2} (x) I."""
    m = 2 ** S
    for s in range(1, S + 1):
        B = np.kron(np.kron(np.eye(2 ** (S - s)), bf.ones_over(2)), np.eye(2 ** (s - 1)))
        for i in range(1, m + 1):
            want = sorted((np.nonzero(B[i - 1])[0] + 1).tolist())
            assert sorted(bf.lemma1_partners(i, s)) == want
            assert B[i - 1, i - 1] == 0.5


@pytest.mark.parametrize("S,M", [(2, 3), (3, 2), (2, 1)])
def test_paper_stage_is_product_of_two_digit_stages(S, M):
    """The paper's A_s mixes one PE bit and the within-PE digit at once: with radices
    (M, 2, ..., 2) (within-PE digit least significant) it is A_{digit s} A_{digit 0}."""
    radices = (M,) + (2,) * S
    for s in range(1, S + 1):
        want = bf.paper_A(S, M, s)
        # the paper's Kronecker order puts the within-PE factor innermost (least significant)
        got = bf.mixed_radix_A(radices, s) @ bf.mixed_radix_A(radices, 0)
        np.testing.assert_allclose(got, want, atol=1e-15)


@pytest.mark.parametrize("radices", [(2, 2), (3, 4, 2), (4, 8, 2), (5,)])
def test_group_major_numbering_is_a_permutation(radices):
    """Draw numbering at each digit: a permutation in which each group's members are
    consecutive, in digit order."""
    N = int(np.prod(radices))
    for k in range(len(radices)):
        pi = bf.group_major(N, radices, k)
        assert np.array_equal(np.sort(pi), np.arange(N))
        for i in range(N):
            mem = bf.group_members(i, radices, k)
            assert [int(pi[j]) for j in mem] == list(range(int(pi[mem[0]]), int(pi[mem[0]]) + radices[k]))
