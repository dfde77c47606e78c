"""Pins for the oracle's norm quadtree (Sec. 2, Eqs. 1-3).

The leaf values are checked against exact rational arithmetic (fractions),
which is independent of the oracle's double-double accumulation; a plain
floating-point sum is shown to differ on the same data, so a dropped
low-order term would fail here."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_counts.json")


def _wide_matrix(n, seed):
    rng = np.random.default_rng(seed)
    mag = 10.0 ** rng.uniform(-9, 3, size=(n, n))
    sign = np.where(rng.random((n, n)) < 0.5, -1.0, 1.0)
    return mag * sign


def _exact_sq_sum(vals):
    return sum((Fraction(float(v)) ** 2 for v in vals), Fraction(0))


@pytest.mark.parametrize("n,b", [(12, 4), (10, 4), (7, 3), (9, 16)])
def test_leaf_norms_are_correctly_rounded_exact_sums(n, b):
    a = _wide_matrix(n, n * 7 + b)
    got = oracle.leaf_norms2(a, b)
    nb = -(-n // b)
    P = got.shape[0]
    assert P == 1 << oracle.depth(nb)
    plain_differs = 0
    for I in range(P):
        for K in range(P):
            blk = a[I * b:(I + 1) * b, K * b:(K + 1) * b]
            if I >= nb or K >= nb:
                assert got[I, K] == 0.0
                continue
            exact = float(_exact_sq_sum(blk.ravel()))
            assert got[I, K] == exact, (I, K)
            s = 0.0
            for v in blk.ravel():
                s += v * v
            plain_differs += s != exact
    if n >= 10 and b >= 4:
        assert plain_differs > 0, "data too benign to tell exact from plain sums"


def test_pyramid_parents_are_rounded_sums_of_children():
    a = _wide_matrix(40, 3)
    tiers = oracle.norm_pyramid(a, 4)   # nb = 10 -> depth 4, P = 16
    assert len(tiers) == 5
    assert tiers[-1].shape == (16, 16)
    for t in range(len(tiers) - 1):
        child = tiers[t + 1]
        par = tiers[t]
        for I in range(par.shape[0]):
            for J in range(par.shape[1]):
                ex = sum((Fraction(float(child[2 * I + i, 2 * J + j]))
                          for i in range(2) for j in range(2)), Fraction(0))
                assert par[I, J] == float(ex)
    # the root is ||A||_F^2 (Eq. 2 applied to the whole matrix)
    exact = float(_exact_sq_sum(a.ravel()))
    assert tiers[0][0, 0] == pytest.approx(exact, rel=4e-16)


def test_parent_norm_bounds_children():
    """Monotone rounding keeps every parent >= each child, which makes the
    recursive culling set equal the flat one."""
    a = _wide_matrix(64, 11)
    tiers = oracle.norm_pyramid(a, 4)
    for t in range(len(tiers) - 1):
        c = tiers[t + 1]
        p = np.repeat(np.repeat(tiers[t], 2, axis=0), 2, axis=1)
        assert np.all(p >= c)


def test_zero_and_ragged_leaves():
    a = np.zeros((5, 5))
    a[4, 4] = 3.0
    n2 = oracle.leaf_norms2(a, 2)        # nb = 3 -> P = 4
    assert n2.shape == (4, 4)
    expect = np.zeros((4, 4))
    expect[2, 2] = 9.0
    assert np.array_equal(n2, expect)


def test_padding_matches_paper():
    gold = json.load(open(GOLD))
    for case in gold["padding"]:
        for b in (16, 32, 64):
            nb = -(-case["n"] // b)
            assert b * (1 << oracle.depth(nb)) == case["padded"], case["cite"]
