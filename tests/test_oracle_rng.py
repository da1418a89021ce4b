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
    g = oracle.normals(np.arange(200000, dtype=np.uint32), seed=42, step=7, tag=0).ravel()
    assert abs(g.mean()) < 5 / np.sqrt(g.size)
    assert abs(g.var() - 1) < 5 * np.sqrt(2 / g.size)
    assert stats.kstest(g, "norm").pvalue > 1e-4
    # the two normals of a Box-Muller pair are uncorrelated
    p = oracle.normals(np.arange(100000, dtype=np.uint32), seed=3, step=0, tag=1)
    assert abs(np.mean(p[:, 0] * p[:, 1])) < 5 / np.sqrt(p.shape[0])
    # tails: |n| is bounded by sqrt(-2 ln 2^-24) since u1 >= 2^-24
    assert np.abs(g).max() <= np.sqrt(-2 * np.log(2.0 ** -24)) + 1e-12


def test_counter_fields_select_independent_streams():
    idx = np.arange(50000, dtype=np.uint32)
    base = oracle.normals(idx, seed=42, step=5, tag=0)
    for kw in [dict(seed=43, step=5, tag=0), dict(seed=42, step=6, tag=0), dict(seed=42, step=5, tag=1),
               dict(seed=42 + (1 << 32), step=5, tag=0), dict(seed=42, step=5 + (1 << 32), tag=0)]:
        other = oracle.normals(idx, **kw)
        c = np.corrcoef(base.ravel(), other.ravel())[0, 1]
        assert abs(c) < 5 / np.sqrt(base.size)
    # same counter, same numbers
    np.testing.assert_array_equal(base, oracle.normals(idx, seed=42, step=5, tag=0))


def test_normals_follow_counter_layout():
    # counter = (index, step lo, step hi, tag), key = (seed lo, seed hi); words (0,1) and
    # (2,3) feed Box-Muller with u = (x >> 9 + 1/2) 2^-23
    seed, step, tag, index = 0x0123456789ABCDEF, (5 << 32) + 17, 2, 99
    w = oracle.philox4x32_10([index, step & 0xFFFFFFFF, step >> 32, tag], [seed & 0xFFFFFFFF, seed >> 32])
    u = ((w.astype(np.float64) // 512) + 0.5) / 2.0 ** 23
    r1 = np.sqrt(-2 * np.log(u[0]))
    r2 = np.sqrt(-2 * np.log(u[2]))
    expect = [r1 * np.cos(2 * np.pi * u[1]), r1 * np.sin(2 * np.pi * u[1]),
              r2 * np.cos(2 * np.pi * u[3]), r2 * np.sin(2 * np.pi * u[3])]
    got = oracle.normals([index], seed, step, tag)[0]
    np.testing.assert_allclose(got, expect, rtol=1e-14, atol=1e-15)
