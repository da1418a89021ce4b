"""Pins of the oracle's random numbers: Philox4x32-10 against the known-answer vectors
of its published definition, and the Box-Muller normals against the normal law."""
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(v, 16) for v in line.split()]
        yield w[0:4], w[4:6], w[6:10]


@pytest.mark.parametrize("ctr,key,expect", list(_kat()))
def test_philox_known_answers(ctr, key, expect):
    out = oracle.philox4x32_10(ctr, key)
    assert [int(v) for v in out] == expect


def test_normals_are_unit_gaussian():
    from scipy import stats
    g = oracle.normals(np.arange(200000, dtype=np.uint32), seed=42, step=7, tag=0)
    flat = g.ravel()
    assert abs(flat.mean()) < 5 / np.sqrt(flat.size)
    assert abs(flat.var() - 1) < 5 * np.sqrt(2 / flat.size)
    assert stats.kstest(flat, "norm").pvalue > 1e-4
    # fourth moment of the normal law (3), each of the eight normals of a draw on its own
    for q in range(8):
        assert abs(np.mean(g[:, q] ** 4) - 3) < 5 * np.sqrt(96 / g.shape[0])
    # the eight normals of one draw (four Box-Muller pairs) are mutually uncorrelated
    c = np.corrcoef(g.T)
    off = c[~np.eye(8, dtype=bool)]
    assert np.abs(off).max() < 5 / np.sqrt(g.shape[0])
    # tails: |n| is bounded by sqrt(-2 ln 2^-21) since u1 >= 2^-21
    assert np.abs(flat).max() <= np.sqrt(-2 * np.log(2.0 ** -21)) + 1e-12


def test_angles_are_uniform_and_radii_rayleigh():
    # a pair (n0, n1) = r (cos theta, sin theta): theta uniform on 4096 equally spaced
    # angles, r^2 / 2 exponential (the law of -ln u1)
    g = oracle.normals(np.arange(100000, dtype=np.uint32), seed=5, step=1, tag=2)
    n0, n1 = g[:, 0::2].ravel(), g[:, 1::2].ravel()
    th = np.mod(np.arctan2(n1, n0), 2 * np.pi)
    slot = th / (2 * np.pi / 4096) - 0.5
    np.testing.assert_allclose(slot, np.round(slot), atol=1e-6)       # on the 4096 angles
    counts = np.bincount(np.round(slot).astype(int) % 4096, minlength=4096)
    from scipy import stats
    assert stats.chisquare(counts).pvalue > 1e-4
    r2h = (n0 * n0 + n1 * n1) / 2
    assert stats.kstest(r2h, "expon").pvalue > 1e-4


def test_counter_fields_select_independent_streams():
    idx = np.arange(50000, dtype=np.uint32)
    base = oracle.normals(idx, seed=42, step=5, tag=0)
    for kw in [dict(seed=43, step=5, tag=0), dict(seed=42, step=6, tag=0), dict(seed=42, step=5, tag=2),
               dict(seed=42 + (1 << 32), step=5, tag=0), dict(seed=42, step=5 + (1 << 32), tag=0)]:
        other = oracle.normals(idx, **kw)
        c = np.corrcoef(base.ravel(), other.ravel())[0, 1]
        assert abs(c) < 5 / np.sqrt(base.size)
    # same counter, same numbers
    np.testing.assert_array_equal(base, oracle.normals(idx, seed=42, step=5, tag=0))


def test_normals_follow_counter_layout():
    # counter = (index, step lo, step hi, tag), key = (seed lo, seed hi); each output word w
    # feeds one Box-Muller pair with u1 = ((w >> 12) + 1/2) 2^-20, u2 = ((w & 4095) + 1/2) 2^-12
    seed, step, tag, index = 0x0123456789ABCDEF, (5 << 32) + 17, 2, 99
    w = oracle.philox4x32_10([index, step & 0xFFFFFFFF, step >> 32, tag], [seed & 0xFFFFFFFF, seed >> 32])
    w = w.astype(np.int64)
    u1 = ((w >> 12) + 0.5) / 2.0 ** 20
    u2 = ((w & 4095) + 0.5) / 2.0 ** 12
    r = np.sqrt(-2 * np.log(u1))
    expect = np.stack([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)], axis=1).ravel()
    got = oracle.normals([index], seed, step, tag)[0]
    np.testing.assert_allclose(got, expect, rtol=1e-14, atol=1e-15)
