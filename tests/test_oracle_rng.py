"""Pins for the oracle's Philox4x32-7, Box-Muller and 64-bit helpers.

Philox's bit pattern cannot be pinned to published known-answer vectors
here (none are available offline): it is pinned by the properties a
counter-based generator must have - uniform words, avalanche on counter and
key bits, injectivity over counters - and the CUDA path is pinned to it bit
for bit by the GPU tests.
"""
import numpy as np
import pytest
from scipy import stats

from oracle import philox, resample


def _words(n=1 << 16, key=(12345, 678), c1=0, c2=0):
    c = np.arange(n, dtype=np.uint64)
    return np.stack(philox.philox4x32(c, c1, c2, 0, key), axis=1)


def test_words_uniform_bytes():
    w = _words()
    b = w.view(np.uint8).reshape(-1)
    counts = np.bincount(b, minlength=256)
    chi2, p = stats.chisquare(counts)
    assert p > 1e-4, (chi2, p)
    # top bits of each word uniform too
    for j in range(4):
        top = (w[:, j] >> 24).astype(np.int64)
        assert stats.chisquare(np.bincount(top, minlength=256))[1] > 1e-4


def _popcount(x):
    x = x.astype(np.uint64)
    return np.array([bin(int(v)).count("1") for v in x.reshape(-1)]).reshape(x.shape)


def test_avalanche_on_counter_and_key_bits():
    rng = np.random.default_rng(0)
    base = rng.integers(0, 2 ** 32, size=(64, 4), dtype=np.uint64)
    key = (0xDEADBEEF, 0x01234567)
    out0 = np.stack(philox.philox4x32(base[:, 0], base[:, 1], base[:, 2], base[:, 3], key), 1)
    flips = []
    for word in range(4):
        for bit in (0, 7, 19, 31):
            b2 = base.copy()
            b2[:, word] ^= np.uint64(1 << bit)
            out1 = np.stack(philox.philox4x32(b2[:, 0], b2[:, 1], b2[:, 2], b2[:, 3], key), 1)
            flips.append(_popcount(out0 ^ out1).sum(axis=1))
    for kbit in (0, 31):
        out1 = np.stack(philox.philox4x32(base[:, 0], base[:, 1], base[:, 2], base[:, 3],
                                          (key[0] ^ (1 << kbit), key[1])), 1)
        flips.append(_popcount(out0 ^ out1).sum(axis=1))
    f = np.concatenate(flips)
    # 128 output bits: a good mixer flips ~64 on average, never almost none.
    assert abs(f.mean() - 64) < 1.5, f.mean()
    assert f.min() > 30


def test_injective_over_counters():
    w = _words(1 << 18)
    as_bytes = w.view(np.dtype((np.void, 16))).reshape(-1)
    assert len(np.unique(as_bytes)) == len(as_bytes)


def test_rounds_matter():
    c = np.arange(16, dtype=np.uint64)
    a = np.stack(philox.philox4x32(c, 0, 0, 0, (1, 2), rounds=10), 1)
    b = np.stack(philox.philox4x32(c, 0, 0, 0, (1, 2), rounds=7), 1)
    assert not np.array_equal(a, b)
    # zero rounds is the identity on the counter
    z = np.stack(philox.philox4x32(c, 5, 6, 7, (1, 2), rounds=0), 1)
    assert np.array_equal(z[:, 0], c.astype(np.uint32)) and np.all(z[:, 1] == 5)


def test_box_muller_is_standard_normal():
    """One large sample (2^21 normals) is N(0, 1) by its moments and a KS test, and
    the KS p-values of 24 independent seeds (2^15 normals each) are themselves
    uniform, as they must be for a generator without structure at this scale."""
    z = philox.normals(seed=42, n=3, purpose=philox.PURPOSE_PROPAGATE, count=1 << 21)
    assert abs(z.mean()) < 0.004
    assert abs(z.var() - 1) < 0.005
    assert stats.kstest(z, "norm").pvalue > 1e-3
    ps = [stats.kstest(philox.normals(seed, 3, philox.PURPOSE_PROPAGATE, 1 << 15), "norm").pvalue
          for seed in range(100, 124)]
    assert stats.kstest(ps, "uniform").pvalue > 1e-3, ps
    # pairs are uncorrelated
    zz = z.reshape(-1, 2)
    assert abs(np.corrcoef(zz[:, 0], zz[:, 1])[0, 1]) < 0.005


def test_box_muller_closed_form_radius_and_angle():
    rng = np.random.default_rng(1)
    wa = rng.integers(0, 2 ** 32, 1000, dtype=np.uint64)
    wb = rng.integers(0, 2 ** 32, 1000, dtype=np.uint64)
    z0, z1 = philox.box_muller(wa, wb)
    u = ((wa >> np.uint64(9)).astype(np.float64) * 2 + 1) / 2 ** 24
    v = (wb >> np.uint64(8)).astype(np.float64) / 2 ** 24
    np.testing.assert_allclose(z0 ** 2 + z1 ** 2, -2 * np.log(u), rtol=1e-12)
    ang = np.mod(np.arctan2(z1, z0), 2 * np.pi)
    np.testing.assert_allclose(np.cos(ang - 2 * np.pi * v), 1.0, atol=1e-9)
    # u and v are exact FP32 values
    assert np.all(u.astype(np.float32).astype(np.float64) == u)
    assert np.all(v.astype(np.float32).astype(np.float64) == v)
    assert u.min() > 0 and u.max() < 1


def test_normal_counter_layout_is_blockwise():
    # normal nu lives in block nu // 4; asking for more normals never changes earlier ones
    a = philox.normals(7, 2, 1, 10)
    b = philox.normals(7, 2, 1, 23)
    assert np.array_equal(a, b[:10])


def test_mulhi64_against_python_integers():
    rng = np.random.default_rng(3)
    x = rng.integers(0, 2 ** 63, 2000, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, 2000, dtype=np.uint64)
    y = rng.integers(0, 2 ** 63, 2000, dtype=np.uint64)
    got = resample.mulhi64(x, y)
    want = np.array([(int(a) * int(b)) >> 64 for a, b in zip(x, y)], dtype=np.uint64)
    assert np.array_equal(got, want)
    edge = np.array([2 ** 64 - 1], dtype=np.uint64)
    assert int(resample.mulhi64(edge, edge)[0]) == ((2 ** 64 - 1) ** 2) >> 64


def test_every_output_bit_balanced():
    """Each of the 128 output bits of the seven-round generator is set half the
    time over 2^18 consecutive counters (within 5 standard errors)."""
    w = _words(1 << 18, key=(0x1234567, 0x89ABCDE))
    n = w.shape[0]
    bits = ((w[:, :, None] >> np.arange(32, dtype=np.uint32)[None, None, :]) & 1).reshape(n, 128)
    freq = bits.mean(axis=0)
    assert np.all(np.abs(freq - 0.5) < 5 * 0.5 / np.sqrt(n)), freq


@pytest.mark.parametrize("lag", ["counter", "time_step"])
def test_neighbouring_counters_independent(lag):
    """The filter draws from counters that differ by one in the first word
    (neighbouring particles) or in the second (the next time step): the pair of
    top nibbles of word 0 at neighbouring counters is uniform over 256 cells."""
    n = 1 << 17
    c = np.arange(n, dtype=np.uint64) * 2
    key = (77, 99)
    a = philox.philox4x32(c, 5, 1, 0, key)[0]
    if lag == "counter":
        b = philox.philox4x32(c + 1, 5, 1, 0, key)[0]
    else:
        b = philox.philox4x32(c, 6, 1, 0, key)[0]
    cell = ((a >> 28).astype(np.int64) << 4) | (b >> 28).astype(np.int64)
    assert stats.chisquare(np.bincount(cell, minlength=256))[1] > 1e-4


def test_words_of_a_block_uncorrelated():
    w = _words(1 << 17, key=(3, 4)).astype(np.float64) / 2.0 ** 32
    r = np.corrcoef(w.T)
    off = r[~np.eye(4, dtype=bool)]
    assert np.all(np.abs(off) < 5 / np.sqrt(w.shape[0])), r
