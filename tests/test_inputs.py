"""The seeded synthetic inputs follow their stated recipe: exact spectral
edges, Haar rotations, reproducible seeds, the lattice's structure and its
closed-form gap bound, and the batch / serving distributions."""
import math

import numpy as np
import pytest

from paper_1101_0265_gb300 import inputs as I


@pytest.mark.parametrize("n,nocc,gap", [(64, 32, 0.1), (100, 25, 1e-3), (7, 3, 0.5)])
def test_dense_spectrum_edges_and_rotation(n, nocc, gap):
    h = I.dense_hamiltonian(n, nocc, gap, config=81, instance=2)
    lam = h.lam
    # the four edges are present exactly, nocc eigenvalues below the gap
    assert lam[0] == -1.0 and lam[-1] == 1.0
    assert lam[nocc - 1] == -gap / 2 and lam[nocc] == gap / 2
    assert np.all(np.diff(lam) >= 0) and np.count_nonzero(lam < 0) == nocc
    assert (h.lmin, h.lmax, h.homo, h.lumo) == (-1.0, 1.0, -gap / 2, gap / 2)
    # Q orthogonal, F = Q diag(lam) Q^T exactly symmetric with that spectrum
    assert np.max(np.abs(h.Q.T @ h.Q - np.eye(n))) < 1e-12
    assert np.array_equal(h.F, h.F.T)
    assert np.max(np.abs(np.linalg.eigvalsh(h.F) - lam)) < 1e-12


def test_seeds_are_reproducible_and_distinct():
    a = I.dense_hamiltonian(40, 20, 0.1, config=5, instance=1)
    b = I.dense_hamiltonian(40, 20, 0.1, config=5, instance=1)
    c = I.dense_hamiltonian(40, 20, 0.1, config=5, instance=2)
    d = I.dense_hamiltonian(40, 20, 0.1, config=6, instance=1)
    assert np.array_equal(a.F, b.F)
    assert not np.array_equal(a.F, c.F) and not np.array_equal(a.F, d.F)
    assert I.seed_for(5, 1) != I.seed_for(5, 2) != I.seed_for(6, 1)


def test_haar_columns_are_unbiased():
    # the sign folding makes the first column's entries symmetric about 0:
    # over many draws their mean is near zero (an unfolded QR biases signs)
    rng = np.random.default_rng(3)
    means = np.mean([I.haar_orthogonal(6, rng)[:, 0] for _ in range(4000)], axis=0)
    assert np.max(np.abs(means)) < 0.03


def test_lattice_structure_and_gap_bound():
    L = 8
    lat = I.lattice_hamiltonian(L, config=3, instance=1)
    n = L ** 3
    assert lat.n == n and lat.nocc == n // 2
    idx = I.lattice_site_index(L)
    # the ordering is a permutation; each 32-site block is a 4 x 4 x 2 sub-cube
    assert np.array_equal(np.sort(idx.ravel()), np.arange(n))
    x, y, z = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    for blk in range(n // 32):
        sel = (idx // 32) == blk
        assert np.ptp(x[sel]) == 3 and np.ptp(y[sel]) == 3 and np.ptp(z[sel]) == 1
    F = lat.dense()
    assert np.array_equal(F, F.T)
    # nearest-neighbour hopping only (periodic): six neighbours per site,
    # each bond -1 +- 0.1; onsite +-0.5 by sublattice, plus small noise
    off = F - np.diag(np.diag(F))
    assert np.all(np.count_nonzero(off, axis=1) == 6)
    nz = off[off != 0]
    assert np.all((nz >= -1.1) & (nz <= -0.9))
    pos = np.empty(n, dtype=int)
    pos[idx.ravel()] = ((x + y + z) % 2).ravel()
    d = np.diag(F)
    assert np.all(np.where(pos == 0, d > 0.2, d < -0.2))
    # hopping joins opposite sublattices only (bipartite)
    r, c = np.nonzero(off)
    assert np.all(pos[r] != pos[c])
    # every eigenvalue clears the closed-form bound, nocc of them negative
    ev = np.linalg.eigvalsh(F)
    assert np.min(np.abs(ev)) >= lat.gap_bound > 0.3
    assert np.count_nonzero(ev < 0) == lat.nocc


def test_lattice_rejects_sizes_that_break_blocks():
    with pytest.raises(ValueError):
        I.lattice_hamiltonian(6)


def test_batch_and_serve_distributions():
    b = I.batch_specs(512)
    ns = np.array([s.n for s in b])
    gaps = np.array([s.gap for s in b])
    assert ns.min() >= 64 and ns.max() <= 2048
    assert 1e-3 <= gaps.min() and gaps.max() <= 1e-1
    # log-uniform: the median of log n sits near the middle of the range
    assert abs(np.median(np.log(ns)) - 0.5 * (math.log(64) + math.log(2048))) < 0.3
    assert all(0.3 * s.n - 1 <= s.nocc <= 0.7 * s.n + 1 for s in b)
    assert [s.n for s in I.batch_specs(512)] == list(ns)            # reproducible
    sv = I.serve_specs(100.0, 400)
    t = np.array([s.arrival for s in sv])
    assert np.all(np.diff(t) > 0)
    # Poisson arrivals: mean inter-arrival time near 1 / rate
    assert abs(np.mean(np.diff(t)) - 0.01) < 0.002
    schemes = [s.scheme for s in sv]
    assert 0.4 < schemes.count("TC_SF") / len(schemes) < 0.6
    ns = np.array([s.n for s in sv])
    assert ns.min() >= 128 and ns.max() <= 8192


def test_reflected_recipe_keeps_the_spectrum():
    # the serving stream's O(n^2) recipe: dense, symmetric, exactly the dense
    # recipe's spectrum, reproducible per instance
    torch = pytest.importorskip("torch")
    sp = I.serve_specs(100.0, 3)[1]
    sp = I.InstanceSpec(n=96, nocc=40, gap=sp.gap, scheme=sp.scheme, arrival=0.0, instance=sp.instance,
                        config=sp.config)
    F, h = I.reflected_hamiltonian_device(sp, "cpu")
    F2, _ = I.reflected_hamiltonian_device(sp, "cpu")
    A = F.numpy()
    assert np.array_equal(A, F2.numpy())
    assert np.array_equal(A, A.T)
    ev = np.linalg.eigvalsh(A)
    assert np.max(np.abs(ev - np.sort(h.lam))) <= 1e-12
    assert h.homo == h.lam[h.nocc - 1] and h.lumo == h.lam[h.nocc]
    assert np.count_nonzero(np.abs(A - np.diag(np.diag(A))) > 1e-14) > 0.9 * 96 * 95
