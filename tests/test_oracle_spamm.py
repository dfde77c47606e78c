"""Pins for the oracle's SpAMM (Eq. 4, Algorithm 1).

- the recursive walk's surviving triples equal a brute-force enumeration of
  the leaf predicate, and come out with k increasing per output leaf;
- tau = 0 keeps exactly the structurally nonzero products ("exact in
  structure"); tau = infinity keeps none;
- tau = 0 values equal numpy's dense product within Higham's gamma_n bound;
- tau > 0 values stay within the sub-multiplicative error bound;
- a hand-worked example with leaf size 1, and the paper's printed
  potential-task counts (Sec. 4.2).
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1403_7458_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_counts.json")
U = 2.0 ** -53


def _gamma(m):
    return m * U / (1 - m * U)


def _sorted(t):
    t = np.asarray(t).reshape(-1, 3)
    order = np.lexsort((t[:, 1], t[:, 2], t[:, 0]))   # by i, then j, then k
    return t[order]


def _block_sparse(n, b, seed, fill=0.4):
    rng = np.random.default_rng(seed)
    nb = -(-n // b)
    mask = rng.random((nb, nb)) < fill
    a = rng.standard_normal((n, n))
    for I in range(nb):
        for K in range(nb):
            if not mask[I, K]:
                a[I * b:(I + 1) * b, K * b:(K + 1) * b] = 0.0
    return a, mask


@pytest.mark.parametrize("n,b,tau", [(256, 32, 1e-6), (250, 16, 1e-3), (300, 32, 1e-1),
                                     (192, 16, 0.0), (128, 8, 1e-8)])
def test_recursive_set_equals_flat_set(n, b, tau):
    a = synth.decaying_matrix(n, n + b, decay=1.3)
    c, tasks = oracle.spamm(a, a, b, tau, want_tasks=True)
    nb = -(-n // b)
    n2 = oracle.leaf_norms2(a, b)
    flat = oracle.flat_tasks(n2, n2, nb, tau)
    assert len(tasks) == len(flat)
    assert np.array_equal(_sorted(tasks), flat)
    # visit order: for each output leaf (i, j), k increases
    seen = {}
    for i, k, j in tasks:
        assert seen.get((i, j), -1) < k
        seen[(i, j)] = k


def test_tau_zero_is_exact_in_structure():
    a, ma = _block_sparse(96, 8, 1)
    b, mb = _block_sparse(96, 8, 2)
    c, tasks = oracle.spamm(a, b, 8, 0.0, want_tasks=True)
    expect = [(i, k, j) for i in range(12) for j in range(12) for k in range(12)
              if ma[i, k] and mb[k, j]]
    assert np.array_equal(_sorted(tasks), np.array(expect, dtype=np.int32).reshape(-1, 3))


def test_tau_infinite_culls_everything():
    a = synth.decaying_matrix(128, 5)
    c, tasks = oracle.spamm(a, a, 16, 1e300, want_tasks=True)
    assert len(tasks) == 0
    assert not np.any(c)


def test_task_set_shrinks_with_tau():
    a = synth.decaying_matrix(256, 9)
    sets = []
    for tau in (0.0, 1e-10, 1e-6, 1e-3, 1e-1):
        _, t = oracle.spamm(a, a, 16, tau, want_tasks=True)
        sets.append({tuple(x) for x in t})
    for s0, s1 in zip(sets, sets[1:]):
        assert s1 <= s0
    assert len(sets[0]) > len(sets[-1])


@pytest.mark.parametrize("n,b", [(256, 32), (200, 16), (64, 64)])
def test_tau_zero_matches_dense_product(n, b):
    rng = np.random.default_rng(n)
    a = rng.standard_normal((n, n))
    bm = rng.standard_normal((n, n))
    c = oracle.spamm(a, bm, b, 0.0)
    ref = a @ bm
    bound = _gamma(n) * (np.abs(a) @ np.abs(bm))
    assert np.all(np.abs(c - ref) <= 2 * bound)
    # and the oracle's own dense triple loop agrees to the same bound
    assert np.all(np.abs(oracle.gemm(a, bm) - ref) <= 2 * bound)


@pytest.mark.parametrize("tau", [1e-6, 1e-4, 1e-2])
def test_tau_error_bound(tau):
    n, b = 320, 16
    a = synth.decaying_matrix(n, 3, decay=1.0)
    c, tasks = oracle.spamm(a, a, b, tau, want_tasks=True)
    nb = n // b
    n2 = oracle.leaf_norms2(a, b)[:nb, :nb]
    nrm = np.sqrt(n2)
    keep = np.zeros((nb, nb, nb), dtype=bool)
    keep[tasks[:, 0], tasks[:, 1], tasks[:, 2]] = True
    # sum over culled k of ||A_ik|| ||B_kj|| bounds each culled leaf's error
    prod = nrm[:, :, None] * nrm[None, :, :]           # [i, k, j]
    culled = np.where(keep, 0.0, prod).sum(axis=1)       # [i, j]
    bound = np.sqrt((culled ** 2).sum())
    err = np.linalg.norm(a @ a - c)
    slack = 1e-12 * np.linalg.norm(np.abs(a) @ np.abs(a))
    assert err <= bound + slack
    assert err > 0.0 or bound == 0.0


def test_values_equal_sum_of_kept_leaf_products():
    n, b, tau = 192, 32, 1e-4
    a = synth.decaying_matrix(n, 21, decay=1.0)
    bm = synth.decaying_matrix(n, 22, decay=1.2)
    c, tasks = oracle.spamm(a, bm, b, tau, want_tasks=True)
    ref = np.zeros((n, n))
    for i, k, j in tasks:
        ref[i * b:(i + 1) * b, j * b:(j + 1) * b] += (
            a[i * b:(i + 1) * b, k * b:(k + 1) * b] @ bm[k * b:(k + 1) * b, j * b:(j + 1) * b])
    bound = _gamma(n) * (np.abs(a) @ np.abs(bm))
    assert np.all(np.abs(c - ref) <= 2 * bound)


def test_worked_example_leaf_size_one():
    """Leaf size 1: every node of the leaf tier is one element and its norm is
    |a_ij|, so Eq. 4 keeps the term a_ik b_kj iff |a_ik| |b_kj| > tau."""
    A = np.array([[1.0, 0.5, 0.0, 0.01],
                  [0.5, 1.0, 0.1, 0.0],
                  [0.0, 0.1, 1.0, 0.5],
                  [0.01, 0.0, 0.5, 1.0]])
    tau = 0.02
    # |products| that survive: 1*1, 1*.5, .5*.5, 1*.1, .5*.1 ; culled: .1*.1 = .01,
    # anything with .01 (at most .01), anything with 0.
    C = oracle.spamm(A, A, 1, tau)
    expect = np.array([
        [1 * 1 + .5 * .5, 1 * .5 + .5 * 1, .5 * .1, 0.0],
        [.5 * 1 + 1 * .5, .5 * .5 + 1 * 1, 1 * .1 + .1 * 1, .1 * .5],
        [.1 * .5, .1 * 1 + 1 * .1, 1 * 1 + .5 * .5, 1 * .5 + .5 * 1],
        [0.0, .5 * .1, .5 * 1 + 1 * .5, .5 * .5 + 1 * 1],
    ])
    assert np.allclose(C, expect, rtol=0, atol=1e-15)
    # the dropped terms: C_00 loses .01*.01, C_11 loses .1*.1, C_03 loses
    # 1*.01 + .01*1, C_02 and C_13 lose .01*.5
    assert np.allclose(A @ A - C, [[1e-4, 0, .005, .02], [0, .01, 0, .005],
                                   [.005, 0, .01, 0], [.02, .005, 0, 1e-4]], atol=1e-15)


def test_paper_potential_task_counts():
    gold = json.load(open(GOLD))
    for case in gold["potential_tasks"]:
        m = case["nc_over_nb"]
        a = np.ones((m, m))
        _, tasks = oracle.spamm(a, a, 1, 0.0, want_tasks=True)
        assert len(tasks) == case["tasks"], case["cite"]


def test_openmp_walk_equals_serial_walk():
    a = synth.decaying_matrix(384, 4)
    c1 = oracle.spamm(a, a, 16, 1e-6, nthreads=1)
    c4 = oracle.spamm(a, a, 16, 1e-6, nthreads=4)
    assert np.array_equal(c1, c4)
