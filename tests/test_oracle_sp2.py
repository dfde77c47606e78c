"""Pins for the oracle's SP2 (cited in Sec. 4) and its Gershgorin start.

At tau = 0 SP2 must produce the spectral projector onto the Ne lowest
eigenvectors, which numpy's dense eigensolver gives independently; at
tau > 0 the trace, idempotency and commutation with F must hold to the
SpAMM error level."""
import math

import numpy as np
import pytest

import oracle
from paper_1403_7458_gb300 import synth


def _projector(h, ne):
    w, v = np.linalg.eigh(h)
    return v[:, :ne] @ v[:, :ne].T, w


def test_gershgorin_contains_spectrum():
    for seed in range(3):
        h = synth.tb_hamiltonian(150, seed)
        lo, hi = oracle.gershgorin(h)
        w = np.linalg.eigvalsh(h)
        assert lo <= w[0] and w[-1] <= hi


def test_gershgorin_closed_forms():
    d = np.diag([3.0, -1.5, 0.25])
    assert oracle.gershgorin(d) == (-1.5, 3.0)
    m = np.array([[1.0, -2.0], [-2.0, 5.0]])
    assert oracle.gershgorin(m) == (-1.0, 7.0)


@pytest.mark.parametrize("n,b,rule", [(128, 16, 0), (192, 32, 0), (160, 32, 1)])
def test_sp2_tau_zero_equals_eigenprojector(n, b, rule):
    h = synth.tb_hamiltonian(n, n)
    ne = n // 2
    p, hist, stop = oracle.sp2(h, b, ne, 0.0, rule=rule)
    assert stop == oracle.STOP_CONVERGED
    pe, w = _projector(h, ne)
    assert w[ne] - w[ne - 1] > 1.0                  # the model is gapped
    assert np.linalg.norm(p - pe) < 1e-10 * np.sqrt(n)
    assert abs(np.trace(p) - ne) < 1e-10
    assert np.linalg.norm(p @ p - p) < 1e-10
    assert np.linalg.norm(h @ p - p @ h) < 1e-9


def test_sp2_branch_and_trace_history():
    n = 128
    h = synth.tb_hamiltonian(n, 1)
    ne = n // 2
    p, hist, stop = oracle.sp2(h, 16, ne, 0.0)
    for t1, t2, e, br, nt, tn in hist:
        take = abs(t2 - ne) < abs(2 * t1 - t2 - ne)
        assert br == (1.0 if take else 0.0)
        assert tn == pytest.approx(t2 if take else 2 * t1 - t2, abs=1e-9)
        assert 0 < nt <= (n // 16) ** 3
    # first iterate: X0 = (emax I - F)/(emax - emin) has trace (n emax - tr F)/(emax - emin)
    lo, hi = oracle.gershgorin(h)
    assert hist[0, 0] == pytest.approx((n * hi - np.trace(h)) / (hi - lo), rel=1e-13)


def test_sp2_with_culling_holds_to_spamm_error_level():
    n = 384
    h = synth.tb_hamiltonian(n, 2)
    ne = n // 2
    p, hist, stop = oracle.sp2(h, 32, ne, 1e-8)
    assert stop in (oracle.STOP_CONVERGED, oracle.STOP_STAGNATED)
    pe, _ = _projector(h, ne)
    assert abs(np.trace(p) - ne) < 1e-7
    assert np.linalg.norm(p @ p - p) < 1e-6
    assert np.linalg.norm(h @ p - p @ h) < 1e-5
    assert np.linalg.norm(p - pe) < 1e-5
    # the paper's error metric Tr[F (P - P~)] against the tau = 0 projector
    p0, _, _ = oracle.sp2(h, 32, ne, 0.0)
    assert abs(np.trace(h @ (p0 - p))) < 1e-6


def test_sp2_fixed_iterations():
    h = synth.tb_hamiltonian(96, 3)
    p, hist, stop = oracle.sp2(h, 16, 48, 1e-8, fixed_iters=7)
    assert stop == oracle.STOP_FIXED
    assert hist.shape[0] == 7


def _spamm_leaf1(x, tau):
    """SpAMM with leaf size 1, straight from its definition (Eq. 4): C_ij =
    sum over k of x_ik x_kj for the k whose squared norms pass,
    x_ik^2 x_kj^2 > tau^2, in increasing k."""
    n = len(x)
    c = [[0.0] * n for _ in range(n)]
    for i in range(n):
        for j in range(n):
            s = 0.0
            for k in range(n):
                a, b = x[i][k], x[k][j]
                if (a * a) * (b * b) > tau * tau:
                    s = s + a * b
            c[i][j] = s
    return c


def _sp2_leaf1(f, ne, tau, trace_tol=1e-10, idem_tol=1e-8, max_iter=100):
    """The SP2 loop written out on plain Python lists (Gershgorin start,
    trace-distance branch, the stopping rule: converged, stagnated when
    e < 1e-3 and e > e_(n-2) / 2, or max_iter).  Returns (iterations, stop
    reason, [(e, took X^2)])."""
    n = len(f)
    lo, hi = math.inf, -math.inf
    for i in range(n):
        s = 0.0
        for j in range(n):
            if j != i:
                s += abs(f[i][j])
        lo = min(lo, f[i][i] - s)
        hi = max(hi, f[i][i] + s)
    x = [[((hi if i == j else 0.0) - f[i][j]) / (hi - lo) for j in range(n)] for i in range(n)]
    eh = [math.inf] * 3
    hist = []
    for it in range(1, max_iter + 1):
        x2 = _spamm_leaf1(x, tau)
        t1 = sum(x[i][i] for i in range(n))
        t2 = sum(x2[i][i] for i in range(n))
        e = math.sqrt(sum((x2[i][j] - x[i][j]) ** 2 for i in range(n) for j in range(n)))
        take = abs(t2 - ne) < abs(2.0 * t1 - t2 - ne)
        x = x2 if take else [[2.0 * x[i][j] - x2[i][j] for j in range(n)] for i in range(n)]
        tn = sum(x[i][i] for i in range(n))
        hist.append((e, take))
        eh = [eh[1], eh[2], e]
        if abs(tn - ne) < trace_tol and e < idem_tol:
            return it, oracle.STOP_CONVERGED, hist
        if it >= 3 and e < 1e-3 and e > 0.5 * eh[0]:
            return it, oracle.STOP_STAGNATED, hist
    return max_iter, oracle.STOP_MAXITER, hist


def test_sp2_stagnation_stop_matches_brute_force_leaf1():
    """Pin of the stopping rule's stagnation branch: tiny symmetric matrices
    with leaf size 1, where culling leaves an error floor that ||X^2 - X||_F
    cannot get below.  The oracle must stop at the same iteration, for the
    same reason, with the same branches and e history as the loop written
    out above on plain lists (seeded cases; the first three that stagnate
    after at least four iterations)."""
    rng = np.random.default_rng(1)
    cases = 0
    for _ in range(4000):
        n = int(rng.integers(2, 5))
        a = rng.uniform(-1, 1, size=(n, n))
        a = np.round((a + a.T) / 2, 4)
        for i in range(n):
            a[i, i] = np.round(rng.uniform(-2, 2), 3)
        ne = int(rng.integers(1, n))
        tau = float(10.0 ** rng.uniform(-6, -1))
        it, reason, hist = _sp2_leaf1(a.tolist(), ne, tau)
        if reason != oracle.STOP_STAGNATED or it < 4:
            continue
        _, h, stop = oracle.sp2(a, 1, ne, tau)
        assert stop == oracle.STOP_STAGNATED
        assert len(h) == it
        assert np.array_equal(h[:, oracle.H_BRANCH], [1.0 if t else 0.0 for _, t in hist])
        assert np.allclose(h[:, oracle.H_IDEM], [e for e, _ in hist], rtol=1e-9, atol=1e-15)
        cases += 1
        if cases == 3:
            break
    assert cases == 3
