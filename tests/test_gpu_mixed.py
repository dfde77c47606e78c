"""Mixed-precision (exact BF16 slices on tcgen05) SpAMM and SP2 vs references.

1. Bit-exact against a test-side integer model of the same arithmetic: each
   element scaled by the matrix's power of two 2^-sigma (max|x| < 2^sigma),
   rounded half-up to X = round(|x| 2^(7s - sigma)), cut into base-128 digits;
   slice pairs p + q < s summed exactly per diagonal d = p + q;
   C = RN(2^(sigmaA + sigmaB - 7s - 7) sum_d S_d 128^(s-1-d)).  The model
   also confirms that the sum of the absolute values of every diagonal's
   terms stays below 2^24, so that every partial FP32 sum is exact whatever
   the order of accumulation.  Beyond that the diagonals round in FP32
   (tested separately on a dense matrix near 0.99).
2. Against the FP64 oracle (the definition of SpAMM) within the rigorous
   elementwise bound of the slicing:
     |dC_ij| <= sum_l over kept leaves of (|a_il| eb + ea |b_lj| + ea eb
                + (s-1) 2^(sigmaA+sigmaB-7s)) + 2^-52 |C_ij|,
   ea = 2^(sigmaA-7s-1), eb = 2^(sigmaB-7s-1) (rounding of each element),
   the (s-1) term bounding the dropped pairs p + q >= s.
3. SP2: ||P_mixed - P_FP64||_F <= 1e-6 (the target accuracy), with the
   same stopping rule.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1403_7458_gb300 import synth

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _sigma(a):
    mx = np.abs(a).max()
    return 0 if mx == 0 else math.frexp(mx)[1]


def _digits(a, s):
    sig = _sigma(a)
    X = np.floor(np.abs(a) * 2.0 ** (7 * s - sig) + 0.5).astype(np.int64)
    sign = np.where(a < 0, -1, 1).astype(np.int64)
    d = []
    for p in range(s):
        v = X >> (7 * (s - 1 - p))
        if p > 0:
            v = v & 127
        d.append(sign * v)
    return d, sig


def _model(a, b, leaf, tau, s):
    """Exact integer model of the sliced leaf products over the oracle's
    task list (same predicate, same norms)."""
    n = a.shape[0]
    _, tasks = oracle.spamm(a, b, leaf, tau, want_tasks=True)
    da, sa = _digits(a, s)
    db, sb = _digits(b, s)
    nb = -(-n // leaf)
    npad = nb * leaf
    pad = lambda m: np.pad(m, ((0, npad - n), (0, npad - n)))
    da = [pad(x) for x in da]
    db = [pad(x) for x in db]
    S = np.zeros((s, npad, npad), dtype=np.int64)
    T = np.zeros((s, npad, npad), dtype=np.int64)   # sums of |terms| per diagonal
    aa = [np.abs(x) for x in da]
    ab = [np.abs(x) for x in db]
    for i, k, j in tasks:
        ri, rk, rj = slice(i * leaf, (i + 1) * leaf), slice(k * leaf, (k + 1) * leaf), slice(j * leaf, (j + 1) * leaf)
        for p in range(s):
            for q in range(s - p):
                S[p + q, ri, rj] += da[p][ri, rk] @ db[q][rk, rj]
                T[p + q, ri, rj] += aa[p][ri, rk] @ ab[q][rk, rj]
    # every partial FP32 sum of a diagonal is exact when the sum of the
    # absolute values of its terms stays below 2^24 (in whatever order the
    # tensor core adds them): the condition under which the bits must match
    assert T.max() < 2 ** 24, "model: FP32 sums would not be provably exact"
    cint = np.zeros((npad, npad), dtype=object)
    for d in range(s):
        cint = cint + S[d].astype(object) * (128 ** (s - 1 - d))
    e = sa + sb - 7 * s - 7
    c = np.vectorize(lambda v: math.ldexp(float(v), e))(cint).astype(np.float64)
    return c[:n, :n], tasks, sa, sb


@pytest.mark.parametrize("n,tau,s,seed,leaf", [(256, 1e-6, 5, 0, 32), (200, 1e-4, 4, 1, 32), (320, 1e-8, 6, 2, 32),
                                               (130, 0.0, 3, 3, 32), (256, 1e-6, 7, 4, 32),
                                               (200, 1e-6, 7, 5, 16), (136, 1e-4, 3, 6, 16),
                                               (300, 1e-6, 4, 7, 64), (192, 0.0, 3, 8, 64)])
def test_mixed_spamm_bit_exact_vs_integer_model(cuda_lib, n, tau, s, seed, leaf):
    a = synth.decaying_matrix(n, seed)
    b = synth.decaying_matrix(n, seed + 50, decay=1.3)
    A = cuda_lib.tree_build(_dev(a), leaf=leaf)
    B = cuda_lib.tree_build(_dev(b), leaf=leaf)
    C, st = cuda_lib.multiply(A, B, tau, prec=cuda_lib.OZAKI_BF16, slices=s, stats=True)
    got = cuda_lib.to_dense(C).cpu().numpy()
    want, tasks, _, _ = _model(a, b, leaf, tau, s)
    assert st["tasks"] == len(tasks)
    assert np.array_equal(got, want), np.abs(got - want).max()
    assert st["sums_rounded"] == 0  # every diagonal sum stayed below 2^24


def test_exact_slices_dense_near_constant_within_fp32_accumulation_bound(cuda_lib):
    """A dense matrix of entries near 0.99 at N = 4096 (leaf 32, 7 slices,
    tau = 0: 128 products per output leaf, all slices nonzero): the diagonal
    sums reach about 2^26, beyond the 2^24 below which FP32 sums of integers
    are exact.  The result is then the sliced product with each diagonal
    rounded in FP32: on sampled output leaves it lies within that rounding
    bound of the exact integer model (each accumulation step rounds to at
    most 2 units of 2^-23 of the running magnitude, which the sum of |terms|
    bounds), and within FP32-level relative accuracy of the FP64 product.
    The combination of the diagonals must not overflow (it did in int64
    before: S_0 2^42 > 2^63)."""
    n, leaf, s = 4096, 32, 7
    rng = np.random.default_rng(21)
    a = 0.99 + 0.005 * rng.uniform(-1.0, 1.0, size=(n, n))
    A = cuda_lib.tree_build(_dev(a), leaf=leaf)
    C, st = cuda_lib.multiply(A, A, 0.0, prec=cuda_lib.OZAKI_BF16, slices=s, stats=True)
    assert st["tasks"] == (n // leaf) ** 3
    # the leading diagonal sums (about 2^26) are reported as rounded: every
    # output element has one, and the product reports each at most once
    assert 0 < st["sums_rounded"] <= n * n
    got = cuda_lib.to_dense(C).cpu().numpy()
    da, sg = _digits(a, s)
    e = 2 * sg - 7 * s - 7
    worst = 0.0
    for i, j in [(0, 0), (5, 77), (127, 3), (64, 64), (31, 100), (90, 127)]:
        ri, rj = slice(i * leaf, (i + 1) * leaf), slice(j * leaf, (j + 1) * leaf)
        Sd = [np.zeros((leaf, leaf), dtype=np.int64) for _ in range(s)]
        Td = [np.zeros((leaf, leaf), dtype=np.int64) for _ in range(s)]
        for p in range(s):
            for q in range(s - p):
                Sd[p + q] += da[p][ri, :] @ da[q][:, rj]
                Td[p + q] += np.abs(da[p][ri, :]) @ np.abs(da[q][:, rj])
        assert max(t.max() for t in Td) > 2 ** 24          # the case the test is about
        exact = sum(Sd[d].astype(object) * (128 ** (s - 1 - d)) for d in range(s))
        model = np.vectorize(lambda v: math.ldexp(float(v), e))(exact).astype(np.float64)
        # accumulation steps into diagonal d of one element: (d + 1) slice
        # pairs x 2 instructions (K = 16 each) for every one of the 128 k
        bound = sum(math.ldexp(1.0, e + 7 * (s - 1 - d)) * (2 * (d + 1) * (n // leaf)) * 2.0 ** -22
                    * Td[d].astype(np.float64) for d in range(s))
        g = got[ri, rj]
        assert np.all(np.abs(g - model) <= bound + 2.0 ** -52 * np.abs(model))
        ref = a[ri, :] @ a[:, rj]
        worst = max(worst, float(np.max(np.abs(g - ref) / np.abs(ref))))
    assert worst < 1e-4, worst                         # FP32-level over 256 accumulation steps


def test_sp2_slicing_overflow_is_reported(cuda_lib):
    """SP2 slices its iterates with the fixed scale |x| < 2.  F = diag(2, ...,
    2, -2) starts from X0 = diag(0, ..., 0, 1); at tau = 2.5 its only product
    (squared norms 1 x 1 < tau^2) is culled, so the first iteration takes
    X <- 2X (tr X < Ne) and the iterate's 2 is out of range.  Its leaf then
    passes Eq. 4 (4 x 4 > tau^2), so the second product uses its slices: the
    solve must fail with E_INVAL and say so, not compute with saturated
    digits."""
    n = 64
    f = np.diag(np.r_[np.full(n - 1, 2.0), -2.0])
    F = cuda_lib.tree_build(_dev(f), leaf=32)
    with pytest.raises(cuda_lib.SpammError) as ei:
        cuda_lib.sp2_solve(F, n / 2, 2.5, prec=cuda_lib.OZAKI_BF16, slices=7, fixed_iters=4)
    assert ei.value.status == cuda_lib.E_INVAL
    assert "slicing range" in str(ei.value)
    # the same solve with FP64 leaf products runs (no slicing)
    P, r = cuda_lib.sp2_solve(F, n / 2, 2.5, fixed_iters=4)
    assert r["iters"] == 4


def test_sp2_unused_out_of_range_leaves_are_not_sliced(cuda_lib):
    """Slicing skips leaves that no product uses (their norm fails Eq. 4
    against every partner), so an out-of-range iterate that takes part in no
    product is no error: with every product culled (tau huge) the mixed solve
    runs X <- 2X like the FP64 one and gives the same iterate."""
    n = 64
    f = np.diag(np.r_[np.full(n - 1, 2.0), -2.0])
    F = cuda_lib.tree_build(_dev(f), leaf=32)
    Pm, rm = cuda_lib.sp2_solve(F, n / 2, 1e10, prec=cuda_lib.OZAKI_BF16, slices=7, fixed_iters=4)
    Pf, rf = cuda_lib.sp2_solve(F, n / 2, 1e10, fixed_iters=4)
    assert rm["iters"] == rf["iters"] == 4
    pm = cuda_lib.to_dense(Pm).cpu().numpy()
    assert np.array_equal(pm, cuda_lib.to_dense(Pf).cpu().numpy())
    assert pm[-1, -1] >= 2.0  # left the slicing range without being sliced


@pytest.mark.parametrize("n,tau,s", [(512, 1e-6, 5), (384, 1e-8, 6), (256, 1e-3, 4)])
def test_mixed_spamm_within_slicing_bound_of_fp64(cuda_lib, n, tau, s):
    a = synth.decaying_matrix(n, 9)
    A = cuda_lib.tree_build(_dev(a), leaf=32)
    C, _ = cuda_lib.multiply(A, A, tau, prec=cuda_lib.OZAKI_BF16, slices=s)
    got = cuda_lib.to_dense(C).cpu().numpy()
    ref, tasks = oracle.spamm(a, a, 32, tau, want_tasks=True)
    sg = _sigma(a)
    ea = eb = 2.0 ** (sg - 7 * s - 1)
    # per output element: sum over kept leaves of the per-term bound
    nb = -(-n // 32)
    keep = np.zeros((nb, nb, nb), dtype=bool)
    keep[tasks[:, 0], tasks[:, 1], tasks[:, 2]] = True
    absA = np.abs(np.pad(a, ((0, nb * 32 - n),) * 2))
    bound = np.zeros((nb * 32, nb * 32))
    for i in range(nb):
        for j in range(nb):
            ks = np.nonzero(keep[i, :, j])[0]
            if len(ks) == 0:
                continue
            cols = np.concatenate([np.arange(k * 32, k * 32 + 32) for k in ks])
            Ai = absA[i * 32:(i + 1) * 32][:, cols]
            Bj = absA[cols][:, j * 32:(j + 1) * 32]
            bound[i * 32:(i + 1) * 32, j * 32:(j + 1) * 32] = (
                Ai.sum(axis=1)[:, None] * eb + ea * Bj.sum(axis=0)[None, :]
                + len(cols) * (ea * eb + (s - 1) * 2.0 ** (2 * sg - 7 * s)))
    bound = bound[:n, :n] + 2.0 ** -52 * np.abs(ref)
    assert np.all(np.abs(got - ref) <= bound)


def test_mixed_rejects_unsupported(cuda_lib):
    a = synth.decaying_matrix(128, 0)
    A64 = cuda_lib.tree_build(_dev(a), leaf=64)
    # 7 slices x leaf 64 = 448 accumulator columns > 256
    with pytest.raises(cuda_lib.SpammError) as ei:
        cuda_lib.multiply(A64, A64, 1e-6, prec=cuda_lib.OZAKI_BF16)
    assert ei.value.status == cuda_lib.E_NOTSUP
    A = cuda_lib.tree_build(_dev(a), leaf=32)
    for bad in (9, 2):
        with pytest.raises(cuda_lib.SpammError) as ei:
            cuda_lib.multiply(A, A, 1e-6, prec=cuda_lib.OZAKI_BF16, slices=bad)
        assert ei.value.status == cuda_lib.E_NOTSUP
    with pytest.raises(cuda_lib.SpammError) as ei:
        cuda_lib.multiply(A, A, 1e-6, prec=17)
    assert ei.value.status == cuda_lib.E_NOTSUP
    # SP2 on the tensor path needs the diagonal traces: leaf 16 or 32
    F64 = cuda_lib.tree_build(_dev(synth.tb_hamiltonian(128, 0)), leaf=64)
    with pytest.raises(cuda_lib.SpammError) as ei:
        cuda_lib.sp2_solve(F64, 64, 1e-8, prec=cuda_lib.TF32)
    assert ei.value.status == cuda_lib.E_NOTSUP


@pytest.mark.parametrize("n,s", [(1024, 6), (1024, 7), (4096, 7)])
def test_mixed_sp2_matches_fp64_sp2(cuda_lib, n, s):
    h = synth.tb_hamiltonian(n, 1)
    F = cuda_lib.tree_build(_dev(h), leaf=32)
    P64, r64 = cuda_lib.sp2_solve(F, n / 2, 1e-8)
    Pm, rm = cuda_lib.sp2_solve(F, n / 2, 1e-8, prec=cuda_lib.OZAKI_BF16, slices=s,
                                fixed_iters=r64["iters"])
    p64 = cuda_lib.to_dense(P64).cpu().numpy()
    pm = cuda_lib.to_dense(Pm).cpu().numpy()
    assert np.linalg.norm(pm - p64) <= 1e-6
    assert abs(np.trace(pm) - n / 2) < 1e-6
    assert np.linalg.norm(pm @ pm - pm) < 1e-5


@pytest.mark.parametrize("n,s,leaf", [(1000, 7, 32), (1050, 4, 32), (1050, 3, 32), (500, 7, 16)])
def test_mixed_sp2_symmetric_mode_is_bit_identical(cuda_lib, n, s, leaf):
    """Forming only the upper block triangle of X^2 and mirroring it gives
    the same bits as forming every leaf (exact slice arithmetic on an exactly
    symmetric iterate).  The symmetric product reads its B leaves from the
    tile-major slices by tensor copies, the full product from the per-leaf
    transposed array; s <= 4 at leaf 32 runs two-column tiles (odd leaf
    counts: the last tile has one column)."""
    h = synth.tb_hamiltonian(n, 4)
    F = cuda_lib.tree_build(_dev(h), leaf=leaf)
    Ps, rs = cuda_lib.sp2_solve(F, n / 2, 1e-8, prec=cuda_lib.OZAKI_BF16, slices=s, fixed_iters=12)
    Pf, rf = cuda_lib.sp2_solve(F, n / 2, 1e-8, prec=cuda_lib.OZAKI_BF16, slices=s, fixed_iters=12,
                                symmetric=False)
    assert rs["symmetric"] == 1 and rf["symmetric"] == 0
    ps = cuda_lib.to_dense(Ps).cpu().numpy()
    assert np.array_equal(ps, cuda_lib.to_dense(Pf).cpu().numpy())
    assert np.array_equal(ps, ps.T)
    # traces, branches and task counts agree exactly; ||X^2 - X||_F is the same
    # sum in another order (the fused update walks leaf rows, not columns)
    hs, hf = rs["history"], rf["history"]
    cols = [c for c in range(hs.shape[1]) if c != 2]
    assert np.array_equal(hs[:, cols], hf[:, cols])
    assert np.allclose(hs[:, 2], hf[:, 2], rtol=1e-12, atol=0)


def test_mixed_sp2_asymmetric_input_uses_full_product(cuda_lib):
    n = 256
    h = synth.tb_hamiltonian(n, 5)
    h[3, 7] += 1e-13                      # no longer exactly symmetric
    F = cuda_lib.tree_build(_dev(h), leaf=32)
    P, r = cuda_lib.sp2_solve(F, n / 2, 1e-8, prec=cuda_lib.OZAKI_BF16, fixed_iters=4)
    assert r["symmetric"] == 0


def _kept_abs_product(a, b, leaf, tasks):
    """sum over kept leaf products of |A_ik| |B_kj| (elementwise) and the
    number of terms K per output element."""
    n = a.shape[0]
    nb = -(-n // leaf)
    npad = nb * leaf
    pa = np.pad(np.abs(a), ((0, npad - n),) * 2)
    pb = np.pad(np.abs(b), ((0, npad - n),) * 2)
    acc = np.zeros((npad, npad))
    kcnt = np.zeros((nb, nb))
    for i, k, j in tasks:
        acc[i * leaf:(i + 1) * leaf, j * leaf:(j + 1) * leaf] += (
            pa[i * leaf:(i + 1) * leaf, k * leaf:(k + 1) * leaf] @ pb[k * leaf:(k + 1) * leaf, j * leaf:(j + 1) * leaf])
        kcnt[i, j] += leaf
    K = np.kron(kcnt, np.ones((leaf, leaf)))
    return acc[:n, :n], K[:n, :n]


@pytest.mark.parametrize("prec_name,n,tau,leaf", [("BF16", 384, 1e-6, 32), ("BF16X3", 384, 1e-6, 32),
                                                  ("BF16X3", 256, 0.0, 32), ("TF32", 384, 1e-6, 32),
                                                  ("TF32X3", 384, 1e-6, 32), ("TF32", 200, 1e-6, 16),
                                                  ("TF32X3", 320, 1e-6, 64), ("BF16X3", 300, 1e-6, 64),
                                                  ("BF16", 200, 1e-4, 16), ("TF32X3", 136, 0.0, 16)])
def test_float_split_modes_within_rounding_bounds(cuda_lib, prec_name, n, tau, leaf):
    """Operands rounded to nearest in BF16 (u = 2^-8) or TF32 (u = 2^-11, plus
    2^-24 for the FP32 step on the way), exact products, FP32 accumulation of
    K terms (u_f = 2^-24; the bound takes 2K u_f for the accumulator):
      one term : |dC| <= (2 u + u^2 + 2 K u_f (1 + u)^2) sum |a||b|
      3 terms  : |dC| <= (5 u^2 + 3 K u_f) sum |a||b|   (dropped lo*lo and
                 residuals below u^2 |x|)."""
    prec = getattr(cuda_lib, prec_name)
    a = synth.decaying_matrix(n, 13)
    b = synth.decaying_matrix(n, 14, decay=1.3)
    A = cuda_lib.tree_build(_dev(a), leaf=leaf)
    B = cuda_lib.tree_build(_dev(b), leaf=leaf)
    C, st = cuda_lib.multiply(A, B, tau, prec=prec, stats=True)
    got = cuda_lib.to_dense(C).cpu().numpy()
    ref, tasks = oracle.spamm(a, b, leaf, tau, want_tasks=True)
    assert st["tasks"] == len(tasks)
    absab, K = _kept_abs_product(a, b, leaf, tasks)
    u = 2.0 ** -8 if prec_name.startswith("BF16") else 2.0 ** -11 + 2.0 ** -24
    uf = 2.0 ** -24
    if not prec_name.endswith("X3"):
        coef = 2 * u + u * u + 2 * K * uf * (1 + u) ** 2
    else:
        coef = 5 * u * u + 3 * K * uf
    bound = coef * absab + 2.0 ** -52 * np.abs(ref)
    err = np.abs(got - ref)
    assert np.all(err <= bound), (err / np.maximum(absab, 1e-300)).max()
    # and not far below the one-term rounding of its own type (the operands
    # really were rounded: a wrong element type would show up here)
    if not prec_name.endswith("X3"):
        assert err.max() > 0.01 * u * absab.max()
    else:
        assert err.max() < (2 * u) * absab.max()


def test_float_split_sp2_misses_target_that_exact_slices_meet(cuda_lib):
    n = 1024
    h = synth.tb_hamiltonian(n, 1)
    F = cuda_lib.tree_build(_dev(h), leaf=32)
    P64, r64 = cuda_lib.sp2_solve(F, n / 2, 1e-8)
    p64 = cuda_lib.to_dense(P64).cpu().numpy()
    errs = {}
    for name in ("BF16X3", "OZAKI_BF16"):
        P, r = cuda_lib.sp2_solve(F, n / 2, 1e-8, prec=getattr(cuda_lib, name), fixed_iters=r64["iters"])
        errs[name] = np.linalg.norm(cuda_lib.to_dense(P).cpu().numpy() - p64)
    assert errs["OZAKI_BF16"] <= 1e-6 < errs["BF16X3"] < 1e-1


@pytest.mark.parametrize("prec_name,leaf,slices", [("OZAKI_BF16", 32, 7), ("TF32", 16, 0), ("BF16X3", 64, 0),
                                                   ("OZAKI_BF16", 64, 4)])
def test_tile_cull_counts_match_oracle_with_early_skip(cuda_lib, prec_name, leaf, slices):
    """Surviving triples of the tile cull (deep quadtree, sparse matrix: the
    32-leaf early skip fires) equal the oracle's flat enumeration."""
    n, tau = 4096, 1e-8
    h = synth.tb_hamiltonian(n, 5, decay=1.0)
    g = synth.decaying_matrix(n, 6, decay=1.1)
    A = cuda_lib.tree_build(_dev(h), leaf=leaf)
    B = cuda_lib.tree_build(_dev(g), leaf=leaf)
    nb = A.nb
    want_ab = len(oracle.flat_tasks(oracle.leaf_norms2(h, leaf), oracle.leaf_norms2(g, leaf), nb, tau))
    want_aa = len(oracle.flat_tasks(oracle.leaf_norms2(h, leaf), oracle.leaf_norms2(h, leaf), nb, tau))
    prec = getattr(cuda_lib, prec_name)
    _, st = cuda_lib.multiply(A, B, tau, prec=prec, slices=slices, stats=True)
    assert st["tasks"] == want_ab
    _, st = cuda_lib.multiply(A, A, tau, prec=prec, slices=slices, stats=True)
    assert st["tasks"] == want_aa


@pytest.mark.parametrize("prec_name,leaf,n", [("OZAKI_BF16", 32, 1000), ("TF32", 64, 1000), ("BF16X3", 16, 1000),
                                              ("TF32", 32, 1050), ("BF16X3", 32, 1000)])
def test_tiles_without_work_are_zero_in_a_reused_output(cuda_lib, prec_name, leaf, n):
    """Tiles without work are never handed out; their output leaves are
    zeroed by a separate pass.  Reuse an output that held a dense product
    and check that a sparse product overwrites every leaf (two-column tiles
    at leaf 32 for the float splits; n = 1050: an odd number of leaf
    columns)."""
    h = synth.tb_hamiltonian(n, 8, decay=1.0)
    A = cuda_lib.tree_build(_dev(h), leaf=leaf)
    prec = getattr(cuda_lib, prec_name)
    C, _ = cuda_lib.multiply(A, A, 0.0, prec=prec)               # every tile has work
    assert np.count_nonzero(cuda_lib.to_dense(C).cpu().numpy()) > 0.5 * n * n
    C, st = cuda_lib.multiply(A, A, 1e-3, C=C, prec=prec, stats=True)  # most tiles empty
    got = cuda_lib.to_dense(C).cpu().numpy()
    ref, tasks = oracle.spamm(h, h, leaf, 1e-3, want_tasks=True)
    assert st["tasks"] == len(tasks)
    nb = -(-n // leaf)
    has = np.zeros((nb, nb), dtype=bool)
    has[tasks[:, 0], tasks[:, 2]] = True
    mask = np.kron(has, np.ones((leaf, leaf), dtype=bool))[:n, :n]
    assert not np.any(got[~mask])                                 # leaves without tasks: exactly 0
    absab, K = _kept_abs_product(h, h, leaf, tasks)
    # the rest: the product (loose: each mode's own bound is tested elsewhere;
    # exact slices err in absolute terms, float splits in relative terms)
    assert np.all(np.abs(got - ref) <= 0.02 * absab + 1e-9 * absab.max())


@pytest.mark.parametrize("prec_name", ["FP64", "OZAKI_BF16", "TF32X3"])
def test_sp2_graph_replay_matches_direct_launches(cuda_lib, prec_name):
    """After the first four iterations SP2 replays a captured CUDA graph of
    four iterations; the result must equal enqueuing every launch directly."""
    n = 1024
    h = synth.tb_hamiltonian(n, 2)
    F = cuda_lib.tree_build(_dev(h), leaf=32)
    prec = getattr(cuda_lib, prec_name)
    Pg, rg = cuda_lib.sp2_solve(F, n / 2, 1e-8, prec=prec, timing=True)
    Pd, rd = cuda_lib.sp2_solve(F, n / 2, 1e-8, prec=prec, timing=True, flags=cuda_lib.F_NOGRAPH)
    assert rd["graphed"] == 0
    assert rg["iters"] > 8 and rg["graphed"] >= 4
    assert rg["iters"] == rd["iters"] and rg["stop_reason"] == rd["stop_reason"]
    assert np.array_equal(rg["history"], rd["history"])
    assert np.array_equal(cuda_lib.to_dense(Pg).cpu().numpy(), cuda_lib.to_dense(Pd).cpu().numpy())
    # launches of replayed iterations are still counted
    assert abs(rg["launches"] - rd["launches"]) <= 4
    assert rg["ms_gemm"] > 0


def test_mixed_sp2_leaf16_matches_fp64(cuda_lib):
    """Leaf 16 on the tensor path (tiles of 8 leaf rows; diagonal traces
    reduced over 16-lane halves of a warp)."""
    n = 1024
    h = synth.tb_hamiltonian(n, 4)
    F = cuda_lib.tree_build(_dev(h), leaf=16)
    P64, r64 = cuda_lib.sp2_solve(F, n / 2, 1e-8)
    P, r = cuda_lib.sp2_solve(F, n / 2, 1e-8, prec=cuda_lib.OZAKI_BF16, slices=7, fixed_iters=r64["iters"])
    assert r["symmetric"] == 1
    assert np.array_equal(r["history"][:, 4], r64["history"][:, 4])      # task counts
    d = cuda_lib.to_dense(P).cpu().numpy() - cuda_lib.to_dense(P64).cpu().numpy()
    assert np.linalg.norm(d) <= 1e-6


def test_release_scratch_then_reuse(cuda_lib):
    n = 512
    a = synth.decaying_matrix(n, 3)
    A = cuda_lib.tree_build(_dev(a), leaf=32)
    C1, _ = cuda_lib.multiply(A, A, 1e-6, prec=cuda_lib.OZAKI_BF16)
    want = cuda_lib.to_dense(C1).cpu().numpy()
    cuda_lib.release_scratch(A)
    cuda_lib.release_scratch(C1)
    C2, _ = cuda_lib.multiply(A, A, 1e-6, C=C1, prec=cuda_lib.OZAKI_BF16)
    assert np.array_equal(cuda_lib.to_dense(C2).cpu().numpy(), want)


@pytest.mark.parametrize("n", [1, 17, 33, 129])
@pytest.mark.parametrize("prec_name,leaf", [("OZAKI_BF16", 32), ("TF32", 16), ("BF16X3", 64), ("FP64", 16)])
def test_tiny_and_ragged_sizes(cuda_lib, n, prec_name, leaf):
    """Sizes below one leaf, one tile and ragged edges: the task set equals
    the oracle's, padding leaves stay zero, values match the FP64 product."""
    a = synth.decaying_matrix(n, 11) if n > 1 else np.array([[0.75]])
    A = cuda_lib.tree_build(_dev(a), leaf=leaf)
    prec = getattr(cuda_lib, prec_name)
    for tau in (0.0, 1e-6, 1e300):
        C, st = cuda_lib.multiply(A, A, tau, prec=prec, stats=True)
        ref, tasks = oracle.spamm(a, a, leaf, tau, want_tasks=True)
        assert st["tasks"] == len(tasks)
        got = cuda_lib.to_dense(C).cpu().numpy()
        absab = np.abs(a) @ np.abs(a)
        if prec_name == "FP64":
            bound = 1e-12 * absab
        elif prec_name == "OZAKI_BF16":  # absolute: slices resolve 2^(sigma - 49)
            bound = 1e-12 * absab.max() * np.ones_like(absab)
        else:                            # float splits: relative to |a||a|
            bound = 1e-2 * absab
        assert np.all(np.abs(got - ref) <= bound + 1e-300)
        if tau == 1e300:
            assert not np.any(got)


def test_mixed_sp2_trace_above_rule_matches_fp64(cuda_lib):
    """Branch rule 1 (X^2 iff tr X > Ne) on the tensor path: same task counts
    and branches as the FP64 solve with the same rule, P within 1e-6."""
    n = 1024
    h = synth.tb_hamiltonian(n, 6)
    F = cuda_lib.tree_build(_dev(h), leaf=32)
    P64, r64 = cuda_lib.sp2_solve(F, n / 2, 1e-8, rule=cuda_lib.RULE_TRACE_ABOVE)
    P, r = cuda_lib.sp2_solve(F, n / 2, 1e-8, rule=cuda_lib.RULE_TRACE_ABOVE, prec=cuda_lib.OZAKI_BF16,
                              slices=7, fixed_iters=r64["iters"])
    assert np.array_equal(r["history"][:, 3], r64["history"][:, 3])
    assert np.array_equal(r["history"][:, 4], r64["history"][:, 4])
    d = cuda_lib.to_dense(P).cpu().numpy() - cuda_lib.to_dense(P64).cpu().numpy()
    assert np.linalg.norm(d) <= 1e-6


def test_sp2_max_iter_returns_the_last_iterate(cuda_lib):
    n = 512
    h = synth.tb_hamiltonian(n, 7)
    F = cuda_lib.tree_build(_dev(h), leaf=32)
    for prec in (cuda_lib.FP64, cuda_lib.OZAKI_BF16):
        P, r = cuda_lib.sp2_solve(F, n / 2, 1e-8, prec=prec, max_iter=3)
        assert r["iters"] == 3 and r["stop_reason"] == cuda_lib.STOP_MAXITER and not r["converged"]
        P3, r3 = cuda_lib.sp2_solve(F, n / 2, 1e-8, prec=prec, fixed_iters=3)
        assert np.array_equal(cuda_lib.to_dense(P).cpu().numpy(), cuda_lib.to_dense(P3).cpu().numpy())


def test_split_tf32_sp2_close_to_fp64(cuda_lib):
    n = 1024
    h = synth.tb_hamiltonian(n, 8)
    F = cuda_lib.tree_build(_dev(h), leaf=32)
    P64, r64 = cuda_lib.sp2_solve(F, n / 2, 1e-8)
    P, r = cuda_lib.sp2_solve(F, n / 2, 1e-8, prec=cuda_lib.TF32X3, fixed_iters=r64["iters"])
    d = np.linalg.norm(cuda_lib.to_dense(P).cpu().numpy() - cuda_lib.to_dense(P64).cpu().numpy())
    assert d < 1e-3
