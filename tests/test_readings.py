"""CPU checks of two readings the CUDA path relies on, against the oracle and
plain arithmetic (no GPU):

- a leaf takes part in a kept triple of Eq. 4 only if its squared norm times
  the largest squared norm among its partners passes the test, so slicing
  only such leaves loses no product (the slicing kernel's skip rule);
- the idempotency error summed from squares of FP64 differences cut to FP32
  (23 fraction bits, FP32 sums of at most 32 terms, FP64 across them) stays
  within 2^-17 of the FP64 sum, far below what the stopping rule compares.
"""
import numpy as np

import oracle
from paper_1403_7458_gb300 import synth


def _leaf_tier(a, leaf):
    return oracle.norm_pyramid(a, leaf)[-1]


def test_leaves_failing_against_their_largest_partner_are_in_no_kept_triple():
    n, leaf = 512, 16
    for seed, tau in ((3, 1e-4), (4, 1e-6), (5, 1e-2)):
        a = synth.decaying_matrix(n, seed)
        b = synth.decaying_matrix(n, seed + 20, decay=1.2)
        na, nbn = _leaf_tier(a, leaf), _leaf_tier(b, leaf)
        nb = -(-n // leaf)
        na, nbn = na[:nb, :nb], nbn[:nb, :nb]
        tasks = oracle.flat_tasks(na, nbn, nb, tau)
        assert len(tasks) > 0
        tau2 = tau * tau
        # A leaf (i, k): its partners are B's row k; B leaf (k, j): A's column k
        keep_a = na * nbn.max(axis=1)[None, :] > tau2
        keep_b = nbn * na.max(axis=0)[:, None] > tau2
        used_a = np.zeros((nb, nb), dtype=bool)
        used_b = np.zeros((nb, nb), dtype=bool)
        used_a[tasks[:, 0], tasks[:, 1]] = True
        used_b[tasks[:, 1], tasks[:, 2]] = True
        # every leaf a kept triple uses passes its test, and every leaf that
        # passes has a partner with which it is kept (the rule is exact)
        assert np.array_equal(used_a, keep_a)
        assert np.array_equal(used_b, keep_b)
        if tau >= 1e-2:
            assert keep_a.sum() < (na > 0).sum()  # the rule skips leaves here


def _trunc32(d):
    """FP64 values cut to FP32 by dropping fraction bits (as the update does)."""
    bits = d.view(np.uint64)
    sign = (bits >> np.uint64(63)).astype(np.uint32) << np.uint32(31)
    e = ((bits >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64) - 896
    m = ((bits >> np.uint64(29)) & np.uint64(0x7FFFFF)).astype(np.uint32)
    out = np.where(e > 0, sign | (np.clip(e, 0, 254).astype(np.uint32) << np.uint32(23)) | m, np.uint32(0))
    return out.view(np.float32)


def test_idempotency_squares_in_fp32_stay_within_bound():
    rng = np.random.default_rng(11)
    for scale in (1e-2, 1e-6, 1e-10):
        # one leaf of 32 x 32 differences, lane l holding elements l + 32 u
        d = scale * rng.standard_normal(1024) * np.exp(rng.uniform(-8, 0, 1024))
        ref = float(np.sum(d * d))
        f = _trunc32(d).reshape(32, 32)  # [u][lane]
        lane = np.zeros(32, dtype=np.float32)
        for u in range(32):  # FP32 multiply-add per lane, in element order
            lane = (lane + f[u] * f[u]).astype(np.float32)
        got = float(np.sum(lane.astype(np.float64)))
        assert abs(got - ref) <= 2.0 ** -17 * ref
