"""Pins of the Cannon ring-exchange oracle (section 5, matrix
multiplication) against what the algorithm and arithmetic fix: a
brute-force triple loop on tiny inputs, the library product, exact
identities (identity and permutation factors), the ring schedule covering
every block once, and the FP32 error bound on known sums."""

import itertools

import numpy as np
import pytest

from oracle import cannon as oc
from workloads import matmul as mm


def brute(a, b):
    n = len(a)
    c = [[0.0] * n for _ in range(n)]
    for i, j, k in itertools.product(range(n), range(n), range(n)):
        c[i][j] += a[i][k] * b[k][j]
    return np.array(c)


@pytest.mark.parametrize("n,p", [(6, 1), (6, 2), (6, 3), (12, 4), (12, 6)])
def test_matches_brute_force_triple_loop(n, p):
    rng = np.random.default_rng(n * 10 + p)
    a = rng.integers(-5, 6, size=(n, n)).astype(np.float64)
    b = rng.integers(-5, 6, size=(n, n)).astype(np.float64)
    c, _ = oc.cannon(a, b, p)
    assert np.array_equal(c, brute(a.tolist(), b.tolist()))


@pytest.mark.parametrize("p", [1, 2, 3, 4, 8])
def test_matches_library_product(p):
    n = 96
    _, _, a, b = mm.pair(n, 40 + p, "uniform")
    c, _ = oc.cannon(a, b, p)
    assert np.allclose(c, a @ b, rtol=0, atol=1e-12)


def test_schedule_covers_every_block_once():
    for p in (1, 2, 3, 5, 8):
        sch = oc.schedule(p)
        assert len(sch) == p
        seen = [(r, j) for step in sch for (r, j) in step]
        assert sorted(seen) == [(r, j) for r in range(p) for j in range(p)]
        for step in sch:       # each stripe is held by exactly one rank
            assert sorted(j for _, j in step) == list(range(p))
    _, blocks = oc.cannon(np.eye(8), np.eye(8), 4)
    assert [(s, r, j) for s, r, j in blocks] == \
        [(s, r, j) for s, step in enumerate(oc.schedule(4)) for r, j in step]


def test_identity_and_permutation_are_exact():
    n, p = 24, 4
    _, _, _, b = mm.pair(n, 7, "uniform")
    c, _ = oc.cannon(np.eye(n), b, p)
    assert np.array_equal(c, b)
    perm = np.random.default_rng(3).permutation(n)
    pm = np.eye(n)[perm]
    c, _ = oc.cannon(pm, b, p)
    assert np.array_equal(c, b[perm])
    c, _ = oc.cannon(b, pm.T, p)                # column permutation
    assert np.array_equal(c, b[:, perm])


def test_rejects_ragged_stripes():
    with pytest.raises(ValueError):
        oc.cannon(np.eye(10), np.eye(10), 3)


def test_entry_and_bound():
    _, _, a, b = mm.pair(32, 5, "dyadic")
    full = a @ b
    for i, j in [(0, 0), (5, 31), (31, 7)]:
        assert oc.entry(a, b, i, j) == full[i, j]
        assert oc.entry_abs(a, b, i, j) >= abs(full[i, j])
    # the bound holds for a sum rounded in FP32 left to right
    rng = np.random.default_rng(9)
    t = rng.uniform(-1, 1, 4096).astype(np.float32)
    s = np.float32(0.0)
    for v in t:
        s = np.float32(s + v)
    exact = float(np.sum(t.astype(np.float64)))
    assert abs(float(s) - exact) <= oc.fp32_sum_bound(4096, np.abs(t).sum())


def test_dyadic_inputs_are_exact_bf16_and_sum_exactly():
    a_bits, bt_bits, a, b = mm.pair(64, 11, "dyadic")
    assert np.array_equal(mm.bf16_values(a_bits), a)
    assert np.array_equal(mm.bf16_values(bt_bits).T, b)
    # all values are multiples of 1/16 in [-1, 1]
    assert np.all(np.abs(a) <= 1) and np.all((a * 16) == np.round(a * 16))


def test_bf16_rounding_is_nearest_even():
    x = np.array([1.0, 1.00390625, 1.01171875, -1.00390625, 65504.0],
                 dtype=np.float32)
    assert mm.round_bf16_bits(x).tolist() == [0x3F80, 0x3F80, 0x3F82, 0xBF80,
                                              0x4780]
