"""Structure of the synthetic inputs (the stand-ins for the paper's water
Fockians): site counts, Morton order, symmetry, decay and the gapped
on-site pattern."""
import numpy as np
import pytest

from paper_1403_7458_gb300 import synth


def test_sites_layout_and_order():
    rng = np.random.default_rng(0)
    pos, gen = synth.water_sites(1024, rng)
    assert pos.shape == (1024, 3)
    assert sorted(gen.tolist()) == list(range(1024))
    # 341 three-site clusters + 1 extra site; cube of 30 A^3 per cluster
    side = (30.0 * 342) ** (1 / 3)
    assert pos.min() >= -1.0 - 1e-9 and pos.max() <= side + 1.0 + 1e-9
    keys = synth.morton3(pos)
    assert np.all(np.diff(keys.astype(np.float64)) >= 0)
    # cluster members sit 1 A from their centre
    inv = np.empty(1024, dtype=np.int64)
    inv[gen] = np.arange(1024)
    for c in range(341):
        p0 = pos[inv[3 * c]]
        for m in (1, 2):
            assert abs(np.linalg.norm(pos[inv[3 * c + m]] - p0) - 1.0) < 1e-12


def test_decaying_matrix_properties():
    a = synth.decaying_matrix(300, 4)
    assert np.array_equal(a, a.T)
    assert np.all(np.diag(a) == 1.0)
    pos, _ = synth.water_sites(300, np.random.default_rng(4))
    r = synth.distances(pos)
    off = ~np.eye(300, dtype=bool)
    env = np.exp(-r / 1.5)
    assert np.all(np.abs(a[off]) <= env[off] * (1 + 1e-15))
    assert np.all(np.abs(a[off]) >= 0.5 * env[off] * (1 - 1e-15))
    assert np.array_equal(a, synth.decaying_matrix(300, 4))


def test_hamiltonian_properties():
    h = synth.tb_hamiltonian(200, 7)
    assert np.array_equal(h, h.T)
    pos, gen = synth.water_sites(200, np.random.default_rng(7))
    assert np.array_equal(np.diag(h), np.where(gen % 2 == 0, -2.0, 2.0))
    off = h[~np.eye(200, dtype=bool)]
    assert np.all(off <= 0.0)
    assert np.all((off == 0.0) | (np.abs(off) >= 1e-12))


def test_batch_sizes():
    n, lam = synth.batch_sizes(64, 0)
    assert len(n) == 64 and all(512 <= x <= 8192 and x % 32 == 0 for x in n)
    assert all(1.0 <= x <= 2.0 for x in lam)


def test_hamiltonian_torch_matches_numpy_generator():
    torch = pytest.importorskip("torch")
    for n, decay in ((300, 1.2), (1100, 1.0)):
        h = synth.tb_hamiltonian(n, 3, decay=decay)
        ht = synth.tb_hamiltonian_torch(n, 3, decay=decay, device="cpu", rows_per_block=256).numpy()
        # same sites, same cut pattern; values equal up to the rounding of
        # r / decay (an ulp of an argument up to ~28 moves exp by ~28 ulp)
        assert np.array_equal(h == 0, ht == 0)
        assert np.array_equal(np.diag(h), np.diag(ht))
        assert np.allclose(h, ht, rtol=1e-14, atol=0)


def test_hamiltonian_block_is_the_leading_principal_block():
    from paper_1403_7458_gb300 import synth
    full = synth.tb_hamiltonian(1500, seed=3, decay=1.0)
    blk = synth.tb_hamiltonian_block(1500, 700, seed=3, decay=1.0)
    assert np.array_equal(blk, full[:700, :700])
