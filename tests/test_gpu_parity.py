"""CUDA path vs the CPU oracle, through the C ABI, on identical seeded inputs.

Bars:
- squared norms of every quadtree tier: bit-exact (both sides round the exact
  sum once);
- culled task lists: bit-exact (same predicate, same norms);
- FP64 leaf products: |C_gpu - C_oracle| <= 2 n u (|A||B|)_ij elementwise
  (both sum the same kept terms, k increasing, in FP64; the CUDA kernel uses
  fused multiply-adds, the oracle separate roundings, so each entry can differ
  by at most the gamma_n bound of either evaluation);
- SP2: same Gershgorin bounds (same sums, same order), same task counts and
  branches until X is idempotent to 1e-6 (beyond that the two branch values
  differ by O(e^2) and rounding may pick either), and
  ||P_gpu - P_oracle||_F <= 1e-10 + 10 e, with e the oracle's final
  idempotency error: once X stalls at the SpAMM error floor, each further
  iteration moves X by O(e) and either side may take the other branch.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1403_7458_gb300 import synth

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def _torch():
    import torch
    return torch


def _dev(a):
    torch = _torch()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _wide(n, seed):
    rng = np.random.default_rng(seed)
    return 10.0 ** rng.uniform(-9, 3, size=(n, n)) * np.where(rng.random((n, n)) < .5, -1., 1.)


def _sorted_gpu_tasks(off, k, nb):
    g = np.repeat(np.arange(nb * nb), np.diff(off))
    i, j = g // nb, g % nb
    t = np.stack([i, k.astype(np.int64), j], axis=1)
    order = np.lexsort((t[:, 1], t[:, 2], t[:, 0]))
    return t[order]


@pytest.mark.parametrize("n,b", [(200, 16), (200, 32), (130, 64), (1024, 32), (33, 32)])
def test_norm_pyramid_bit_exact(cuda_lib, n, b):
    a = _wide(n, n + b)
    A = cuda_lib.tree_build(_dev(a), leaf=b)
    ref = oracle.norm_pyramid(a, b)
    assert A.depth == len(ref) - 1
    for t, r in enumerate(ref):
        got = cuda_lib.norms(A, t)
        assert np.array_equal(got, r), (t, np.abs(got - r).max())


def test_tree_build_from_host_memory(cuda_lib):
    a = synth.decaying_matrix(100, 1)
    A = cuda_lib.tree_build(a, leaf=16)          # numpy = host pointer
    back = np.zeros((100, 100))
    cuda_lib.to_dense(A, out=back)
    assert np.array_equal(back, a)
    assert np.array_equal(cuda_lib.norms(A, A.depth), oracle.leaf_norms2(a, 16))


def test_host_transfers_in_row_blocks_with_row_pitch(cuda_lib):
    """Host input and output go through the device in row blocks (here four
    blocks of 256 rows at n = 1000, b = 16): a host matrix with a row pitch
    larger than n builds the same handle as its device copy, and the dense
    output lands in a pitched host buffer without touching the padding."""
    import torch
    n, b = 1000, 16
    a = synth.decaying_matrix(n, 4)
    big = torch.zeros((n, n + 40), dtype=torch.float64)  # host memory, row pitch n + 40
    big[:, :n] = torch.from_numpy(a)
    A = cuda_lib.tree_build(big[:, :n], leaf=b)
    assert np.array_equal(cuda_lib.norms(A, A.depth), oracle.leaf_norms2(a, b))
    out = torch.full((n, n + 24), -1.0, dtype=torch.float64)
    cuda_lib.to_dense(A, out=out[:, :n])
    assert np.array_equal(out[:, :n].numpy(), a)
    assert bool((out[:, n:] == -1.0).all())
    # with a drop threshold: the host build equals the device build
    Ah = cuda_lib.tree_build(big[:, :n], leaf=b, drop=1e-3)
    Ad = cuda_lib.tree_build(_dev(a), leaf=b, drop=1e-3)
    assert Ah.stored == Ad.stored < Ad.nb * Ad.nb
    assert np.array_equal(cuda_lib.to_dense(Ah).cpu().numpy(), cuda_lib.to_dense(Ad).cpu().numpy())


@pytest.mark.parametrize("n,b,tau,kind", [(1024, 32, 1e-6, "dec"), (1000, 16, 1e-6, "dec"), (512, 64, 1e-8, "dec"),
                                          (384, 32, 0.0, "dec"), (384, 32, 1e-2, "dec"), (256, 32, 1e300, "dec"),
                                          (3000, 16, 1e-6, "dec"), (4096, 32, 1e-8, "tb"), (4100, 64, 1e-6, "tb")])
def test_task_list_bit_exact(cuda_lib, n, b, tau, kind):
    """Flat enumeration of Eq. 4 by the oracle vs the GPU's list; the larger
    cases have quadtrees deep enough for the early skip of whole 32-leaf
    steps of k (and sparse enough, "tb": decay 1.0, for it to fire)."""
    a = synth.decaying_matrix(n, 7) if kind == "dec" else synth.tb_hamiltonian(n, 7, decay=1.0)
    A = cuda_lib.tree_build(_dev(a), leaf=b)
    off, k = cuda_lib.task_list(A, A, tau)
    nb = A.nb
    n2 = oracle.leaf_norms2(a, b)
    flat = oracle.flat_tasks(n2, n2, nb, tau)
    got = _sorted_gpu_tasks(off, k, nb)
    assert got.shape == flat.shape
    assert np.array_equal(got, flat.astype(np.int64))
    # k increasing inside every group
    for g in range(0, nb * nb, max(1, nb * nb // 97)):
        ks = k[off[g]:off[g + 1]]
        assert np.all(np.diff(ks.astype(np.int64)) > 0)


def test_task_list_matches_recursive_walk_distinct_operands(cuda_lib):
    n, b, tau = 320, 32, 1e-5
    a = synth.decaying_matrix(n, 3, decay=1.0)
    bm = synth.decaying_matrix(n, 4, decay=2.0)
    A = cuda_lib.tree_build(_dev(a), leaf=b)
    B = cuda_lib.tree_build(_dev(bm), leaf=b)
    off, k = cuda_lib.task_list(A, B, tau)
    _, rec = oracle.spamm(a, bm, b, tau, want_tasks=True)
    order = np.lexsort((rec[:, 1], rec[:, 2], rec[:, 0]))
    assert np.array_equal(_sorted_gpu_tasks(off, k, A.nb), rec[order].astype(np.int64))


@pytest.mark.parametrize("n,b,tau,seed", [(1024, 32, 1e-6, 0), (1000, 16, 1e-6, 1),
                                          (640, 64, 1e-8, 2), (300, 32, 0.0, 3),
                                          (96, 32, 1e-3, 4)])
def test_spamm_fp64_values(cuda_lib, n, b, tau, seed):
    a = synth.decaying_matrix(n, seed)
    bm = synth.decaying_matrix(n, seed + 100, decay=1.2)
    A = cuda_lib.tree_build(_dev(a), leaf=b)
    B = cuda_lib.tree_build(_dev(bm), leaf=b)
    C, st = cuda_lib.multiply(A, B, tau, stats=True)
    c = cuda_lib.to_dense(C).cpu().numpy()
    ref, tasks = oracle.spamm(a, bm, b, tau, want_tasks=True)
    assert st["tasks"] == len(tasks)
    assert st["flops_useful"] == 2.0 * b ** 3 * len(tasks)
    bound = 2 * n * U * (np.abs(a) @ np.abs(bm))
    assert np.all(np.abs(c - ref) <= bound + 1e-300)
    # C's quadtree is built from the stored leaves
    for t, r in enumerate(oracle.norm_pyramid(c, b)):
        assert np.array_equal(cuda_lib.norms(C, t), r)


def test_spamm_reuses_output_handle(cuda_lib):
    a = synth.decaying_matrix(256, 5)
    A = cuda_lib.tree_build(_dev(a), leaf=32)
    C, _ = cuda_lib.multiply(A, A, 1e-6)
    first = cuda_lib.to_dense(C).cpu().numpy()
    C2, _ = cuda_lib.multiply(A, A, 1e-1, C=C)
    assert C2 is C
    ref = oracle.spamm(a, a, 32, 1e-1)
    assert np.allclose(cuda_lib.to_dense(C).cpu().numpy(), ref, atol=1e-12, rtol=0)
    assert not np.array_equal(first, cuda_lib.to_dense(C).cpu().numpy())


def test_spamm_deterministic(cuda_lib):
    a = synth.decaying_matrix(768, 6)
    A = cuda_lib.tree_build(_dev(a), leaf=32)
    C1, _ = cuda_lib.multiply(A, A, 1e-8)
    C2, _ = cuda_lib.multiply(A, A, 1e-8)
    assert np.array_equal(cuda_lib.to_dense(C1).cpu().numpy(), cuda_lib.to_dense(C2).cpu().numpy())


@pytest.mark.parametrize("n,b,tau", [(512, 32, 1e-8), (300, 16, 1e-6), (256, 64, 0.0)])
def test_sp2_fp64_matches_oracle(cuda_lib, n, b, tau):
    h = synth.tb_hamiltonian(n, n)
    F = cuda_lib.tree_build(_dev(h), leaf=b)
    P, rep = cuda_lib.sp2_solve(F, n / 2, tau)
    p = cuda_lib.to_dense(P).cpu().numpy()
    p_ref, hist, stop = oracle.sp2(h, b, n / 2, tau)
    lo, hi = oracle.gershgorin(h)
    assert rep["emin"] == lo and rep["emax"] == hi       # same sums in the same order
    assert rep["stop_reason"] == stop
    assert rep["iters"] == len(hist)
    gh = rep["history"]
    # task counts and branches agree until X is idempotent to ~1e-6
    for r_gpu, r_ref in zip(gh, hist):
        if r_ref[oracle.H_IDEM] < 1e-6:
            break
        assert r_gpu[oracle.H_BRANCH] == r_ref[oracle.H_BRANCH]
        assert r_gpu[oracle.H_TASKS] == r_ref[oracle.H_TASKS]
        assert r_gpu[oracle.H_TR] == pytest.approx(r_ref[oracle.H_TR], abs=1e-9)
    assert np.linalg.norm(p - p_ref) <= 1e-10 + 10 * hist[-1, oracle.H_IDEM]


@pytest.mark.parametrize("n,b", [(1000, 32), (777, 16), (900, 64)])
def test_sp2_fp64_symmetric_mode_is_bit_identical(cuda_lib, n, b):
    """FP64 leaf products of an exactly symmetric iterate: forming only the
    upper block triangle of X^2 and storing each C_ij also as C_ji^T gives
    the same bits as forming every leaf (the mirror sums the same products
    in the same order, factors swapped)."""
    h = synth.tb_hamiltonian(n, 7)
    F = cuda_lib.tree_build(_dev(h), leaf=b)
    Ps, rs = cuda_lib.sp2_solve(F, n / 2, 1e-8, fixed_iters=10)
    Pf, rf = cuda_lib.sp2_solve(F, n / 2, 1e-8, fixed_iters=10, symmetric=False)
    assert rs["symmetric"] == 1 and rf["symmetric"] == 0
    ps = cuda_lib.to_dense(Ps).cpu().numpy()
    assert np.array_equal(ps, cuda_lib.to_dense(Pf).cpu().numpy())
    assert np.array_equal(ps, ps.T)
    assert np.array_equal(rs["history"], rf["history"])
    # leaf products formed: all of them in the full product, the upper block
    # triangle (diagonal leaves once, the others for both) when symmetric
    assert rf["flops_tensor"] == rf["flops_useful"]
    assert rs["flops_useful"] / 2 <= rs["flops_tensor"] < rs["flops_useful"]


def test_sp2_first_iterations_config1_size(cuda_lib):
    """N = 4096 tight-binding Hamiltonian, tau = 1e-8: the oracle runs three
    SP2 iterations (fixed-iteration mode) and the GPU must agree on every
    task count and branch, with P within 1e-9."""
    n, b, tau = 4096, 32, 1e-8
    h = synth.tb_hamiltonian(n, 0)
    F = cuda_lib.tree_build(_dev(h), leaf=b)
    P, rep = cuda_lib.sp2_solve(F, n / 2, tau, fixed_iters=3)
    p_ref, hist, stop = oracle.sp2(h, b, n / 2, tau, fixed_iters=3)
    gh = rep["history"]
    assert np.array_equal(gh[:, oracle.H_TASKS], hist[:, oracle.H_TASKS])
    assert np.array_equal(gh[:, oracle.H_BRANCH], hist[:, oracle.H_BRANCH])
    p = cuda_lib.to_dense(P).cpu().numpy()
    assert np.linalg.norm(p - p_ref) <= 1e-9


def test_sp2_full_config1_properties(cuda_lib):
    """Full N = 4096 solve at tau = 1e-8: trace, idempotency and commutation
    hold at the SpAMM error level (the oracle needs minutes for this size)."""
    torch = _torch()
    n, b, tau = 4096, 32, 1e-8
    h = synth.tb_hamiltonian(n, 0)
    hd = _dev(h)
    F = cuda_lib.tree_build(hd, leaf=b)
    P, rep = cuda_lib.sp2_solve(F, n / 2, tau)
    assert rep["stop_reason"] in (cuda_lib.STOP_CONVERGED, cuda_lib.STOP_STAGNATED)
    p = cuda_lib.to_dense(P)
    assert abs(torch.trace(p).item() - n / 2) < 1e-6
    assert torch.linalg.norm(p @ p - p).item() < 1e-5
    assert torch.linalg.norm(hd @ p - p @ hd).item() < 1e-4


def test_bad_arguments_raise(cuda_lib):
    a = synth.decaying_matrix(64, 0)
    A = cuda_lib.tree_build(_dev(a), leaf=32)
    B = cuda_lib.tree_build(_dev(synth.decaying_matrix(96, 0)), leaf=32)
    with pytest.raises(cuda_lib.SpammError) as ei:
        cuda_lib.multiply(A, B, 1e-6)
    assert ei.value.status == cuda_lib.E_INVAL
    with pytest.raises(cuda_lib.SpammError):
        cuda_lib.multiply(A, A, -1.0)
    with pytest.raises(cuda_lib.SpammError):
        cuda_lib.multiply(A, A, float("nan"))
    with pytest.raises(cuda_lib.SpammError):
        cuda_lib.tree_build(_dev(a), leaf=24)
    with pytest.raises(cuda_lib.SpammError):
        cuda_lib.sp2_solve(A, 64.0, 1e-8)     # Ne must be < n


def test_spamm_sampled_leaves_at_n16384(cuda_lib):
    """A product at the precision-study size (N = 16384, tight-binding
    Hamiltonian, tau = 1e-8): 24 output leaves recomputed one by one from the
    definition (Eq. 4 on the oracle's leaf norms, k increasing) and compared
    with the FP64 path (within 2 gamma_K) and the 7-slice path (within the
    slicing bound)."""
    n, b, tau = 16384, 32, 1e-8
    h = synth.tb_hamiltonian(n, 3)
    F = cuda_lib.tree_build(_dev(h), leaf=b)
    n2 = oracle.leaf_norms2(h, b)
    nb = n // b
    C64, st = cuda_lib.multiply(F, F, tau, stats=True)
    Cx, stx = cuda_lib.multiply(F, F, tau, prec=cuda_lib.OZAKI_BF16, slices=7, stats=True)
    assert st["tasks"] == stx["tasks"]
    torch = _torch()
    rng = np.random.default_rng(5)
    picks = [(i, min(nb - 1, max(0, i + d))) for i, d in zip(rng.integers(0, nb, 24), rng.integers(-6, 7, 24))]
    d64 = cuda_lib.to_dense(C64)
    dx = cuda_lib.to_dense(Cx)
    sig = math.frexp(np.abs(h).max())[1]
    for i, j in picks:
        ks = [k for k in range(nb) if n2[i, k] * n2[k, j] > tau * tau]
        ref = np.zeros((b, b))
        absref = np.zeros((b, b))
        rowsum = np.zeros(b)
        colsum = np.zeros(b)
        for k in ks:
            a_ik = h[i * b:(i + 1) * b, k * b:(k + 1) * b]
            b_kj = h[k * b:(k + 1) * b, j * b:(j + 1) * b]
            ref += a_ik @ b_kj
            absref += np.abs(a_ik) @ np.abs(b_kj)
            rowsum += np.abs(a_ik).sum(axis=1)
            colsum += np.abs(b_kj).sum(axis=0)
        got64 = d64[i * b:(i + 1) * b, j * b:(j + 1) * b].cpu().numpy()
        gotx = dx[i * b:(i + 1) * b, j * b:(j + 1) * b].cpu().numpy()
        K = max(1, len(ks) * b)
        g = K * 2.0 ** -53 / (1 - K * 2.0 ** -53)
        assert np.all(np.abs(got64 - ref) <= 2 * g * absref + 1e-300), (i, j)
        # rounding of every element to 7 slices (e each) and the dropped
        # slice pairs p + q >= 7, as in the mixed-precision tests
        e = 2.0 ** (sig - 7 * 7 - 1)
        slack = rowsum[:, None] * e + e * colsum[None, :] + K * (e * e + 6 * 2.0 ** (2 * sig - 49))
        assert np.all(np.abs(gotx - ref) <= slack + 2 * g * absref + 1e-300), (i, j)
    del d64, dx
    torch.cuda.empty_cache()


@pytest.mark.parametrize("drop", [0.0, 1e-6, 1e-3])
def test_sparse_leaf_storage_equals_dense_with_dropped_leaves_zeroed(cuda_lib, drop):
    """spamm_tree_build with a drop threshold stores only the leaves with
    ||leaf||_F > drop; everything after behaves as the dense matrix with the
    other leaves set to zero: norms, task lists, FP64 and exact-slice
    products, and SP2 (F stored sparsely), bit for bit."""
    n, b = 2048, 32
    h = synth.tb_hamiltonian(n, 1, decay=1.0)
    nb = n // b
    n2 = oracle.leaf_norms2(h, b)[:nb, :nb]
    keep = n2 > drop * drop
    hz = h * np.kron(keep, np.ones((b, b)))
    S = cuda_lib.tree_build(_dev(h), leaf=b, drop=drop)
    D = cuda_lib.tree_build(_dev(hz), leaf=b, drop=-1.0)
    assert S.stored == int(keep.sum()) < nb * nb and D.stored == nb * nb
    assert np.array_equal(cuda_lib.to_dense(S).cpu().numpy(), hz)
    for t in range(S.depth + 1):
        assert np.array_equal(cuda_lib.norms(S, t), cuda_lib.norms(D, t))
    for prec, sl in ((cuda_lib.FP64, 0), (cuda_lib.OZAKI_BF16, 7), (cuda_lib.TF32, 0)):
        Cs, ss = cuda_lib.multiply(S, S, 1e-8, prec=prec, slices=sl, stats=True)
        Cd, sd = cuda_lib.multiply(D, D, 1e-8, prec=prec, slices=sl, stats=True)
        assert ss["tasks"] == sd["tasks"]
        assert np.array_equal(cuda_lib.to_dense(Cs).cpu().numpy(), cuda_lib.to_dense(Cd).cpu().numpy())
    for prec, sl in ((cuda_lib.FP64, 0), (cuda_lib.OZAKI_BF16, 7)):
        Ps, rs = cuda_lib.sp2_solve(S, n / 2, 1e-8, prec=prec, slices=sl)
        Pd, rd = cuda_lib.sp2_solve(D, n / 2, 1e-8, prec=prec, slices=sl)
        assert np.array_equal(rs["history"], rd["history"])
        assert np.array_equal(cuda_lib.to_dense(Ps).cpu().numpy(), cuda_lib.to_dense(Pd).cpu().numpy())
    # a handle with absent leaves is an input only
    with pytest.raises(cuda_lib.SpammError) as ei:
        cuda_lib.multiply(D, D, 1e-8, C=S)
    assert ei.value.status == cuda_lib.E_INVAL
    with pytest.raises(cuda_lib.SpammError) as ei:
        cuda_lib.sp2_solve(D, n / 2, 1e-8, P=S)
    assert ei.value.status == cuda_lib.E_INVAL


def test_sp2_rejects_an_asymmetric_hamiltonian(cuda_lib):
    n = 256
    h = synth.tb_hamiltonian(n, 5)
    h[3, 40] += 1e-3                      # mirror leaves' norms now differ
    F = cuda_lib.tree_build(_dev(h), leaf=32)
    with pytest.raises(cuda_lib.SpammError) as ei:
        cuda_lib.sp2_solve(F, n / 2, 1e-8)
    assert ei.value.status == cuda_lib.E_INVAL


def test_device_watchdog_gives_up_and_the_context_survives(cuda_lib):
    """Every wait in the library's kernels is bounded; a wait on a barrier that
    nothing completes gives up and is reported as E_TIMEOUT, after which the
    device still computes."""
    import time
    t0 = time.perf_counter()
    assert cuda_lib.watchdog_selftest(200) == cuda_lib.E_TIMEOUT
    assert 0.1 < time.perf_counter() - t0 < 5.0
    a = synth.decaying_matrix(128, 0)
    A = cuda_lib.tree_build(_dev(a), leaf=32)
    C, st = cuda_lib.multiply(A, A, 1e-6, stats=True)
    ref, tasks = oracle.spamm(a, a, 32, 1e-6, want_tasks=True)
    assert st["tasks"] == len(tasks)


def test_sp2_history_records_leaf_fill(cuda_lib):
    n, b = 2048, 32
    h = synth.tb_hamiltonian(n, 2, decay=1.0)
    F = cuda_lib.tree_build(_dev(h), leaf=b)
    for prec in (cuda_lib.FP64, cuda_lib.OZAKI_BF16):
        P, rep = cuda_lib.sp2_solve(F, n / 2, 1e-8, prec=prec)
        nb = n // b
        fill = float((cuda_lib.norms(P, P.depth)[:nb, :nb] > 0).mean())
        hist = rep["history"]
        assert hist.shape[1] == cuda_lib.H_COLS
        assert hist[-1, cuda_lib.H_FILL] == pytest.approx(fill, abs=0.5 / (nb * nb))
        assert np.all((hist[:, cuda_lib.H_FILL] > 0) & (hist[:, cuda_lib.H_FILL] <= 1))
