"""Pins for the oracle's SP2 (cited in Sec. 4) and its Gershgorin start.

At tau = 0 SP2 must produce the spectral projector onto the Ne lowest
eigenvectors, which numpy's dense eigensolver gives independently; at
tau > 0 the trace, idempotency and commutation with F must hold to the
SpAMM error level."""
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
