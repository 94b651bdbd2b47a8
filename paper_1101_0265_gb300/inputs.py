"""Seeded synthetic inputs for density-matrix purification.

This module builds Hamiltonians and request streams only.  It holds none of
the purification arithmetic: no spectral map, no density matrix, no bound
estimate.  Both the CPU oracle (through the tests) and the GPU library consume
what it returns, so a mistake here cannot hide a disagreement between them.

Workloads (all synthetic; the paper's own tests are diagonal test
Hamiltonians with prescribed chemical potential and band gap, and it notes
that a result for given mu and gap carries over to every Hamiltonian with the
same mu and gap, so a rotated diagonal matrix is an equally valid test case):

* ``dense_hamiltonian``: F = Q diag(lambda) Q^T with Q Haar-orthogonal.  The
  occupied eigenvalues fill [-1, -gap/2], the unoccupied ones [gap/2, 1], and
  the four edges -1, -gap/2, gap/2, 1 are present exactly, so lambda_min,
  lambda_homo, lambda_lumo, lambda_max and mu = 0 are known in closed form.
* ``diagonal_hamiltonian``: the paper's diagonal test matrices.
* ``lattice_hamiltonian``: a cubic tight-binding model with a gap around 0,
  sites ordered by 4x4x2 sub-cubes so that 32-site blocks are spatially
  compact.
* ``batch_specs`` / ``serve_specs``: many instances of uneven size;
  ``dense_hamiltonian_device`` builds one on a CUDA device with torch (same
  recipe, torch's generator) when thousands of large inputs are needed.

Seeds: every instance draws from ``numpy.random.Generator(PCG64(s))`` with
``s = splitmix64(BASE_SEED ^ splitmix64(config) ^ splitmix64(instance + 1))``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 11010265
_MASK = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def splitmix64(x: int) -> int:
    """The SplitMix64 output function of Steele, Lea and Flood (2014),
    applied to ``x + golden gamma`` (one step of the published generator)."""
    z = (x + _GOLDEN) & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def seed_for(config: int, instance: int = 0) -> int:
    return splitmix64(BASE_SEED ^ splitmix64(config) ^ splitmix64(instance + 1))


def rng_for(config: int, instance: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed_for(config, instance)))


@dataclass
class Hamiltonian:
    """A symmetric test Hamiltonian with its known spectral landmarks.

    ``F`` is row-major float64 (n x n).  ``lam`` is the prescribed spectrum
    (ascending) and ``Q`` the eigenvectors used to build F (None for diagonal
    and lattice inputs).  ``homo``/``lumo`` are the eigenvalues just below
    and just above the gap; ``nocc`` counts eigenvalues below ``mu``."""

    F: np.ndarray
    n: int
    nocc: int
    mu: float
    lmin: float
    lmax: float
    homo: float
    lumo: float
    lam: np.ndarray | None = None
    Q: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def gap(self) -> float:
        return self.lumo - self.homo


def haar_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal matrix: QR of a standard normal matrix
    with the signs of R's diagonal folded into Q (Mezzadri 2007)."""
    Z = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(Z)
    Q *= np.sign(np.diag(R))[None, :]
    return Q


def gapped_spectrum(n: int, nocc: int, gap: float, rng: np.random.Generator,
                    lo: float = -1.0, hi: float = 1.0, mu: float = 0.0) -> np.ndarray:
    """nocc eigenvalues in [lo, mu - gap/2] and n - nocc in [mu + gap/2, hi],
    with both ends of each band present exactly; returned ascending."""
    if not (0 < nocc < n):
        raise ValueError("need 0 < nocc < n")
    homo, lumo = mu - gap / 2.0, mu + gap / 2.0
    occ = _band(nocc, lo, homo, rng, homo)
    vir = _band(n - nocc, lumo, hi, rng, lumo)
    return np.sort(np.concatenate([occ, vir]))


def _band(m: int, a: float, b: float, rng: np.random.Generator, single: float) -> np.ndarray:
    """m values in [a, b] containing both ends (only ``single`` when m == 1)."""
    if m == 1:
        return np.array([single], dtype=np.float64)
    ends = np.array([a, b], dtype=np.float64)
    if m == 2:
        return ends
    return np.concatenate([ends, rng.uniform(a, b, m - 2)])


def _symmetric(F: np.ndarray) -> np.ndarray:
    F = 0.5 * (F + F.T)
    return np.ascontiguousarray(F)


def dense_hamiltonian(n: int, nocc: int, gap: float, config: int = 1, instance: int = 0,
                      lo: float = -1.0, hi: float = 1.0) -> Hamiltonian:
    """F = Q diag(lambda) Q^T, Q Haar from the instance's seed."""
    rng = rng_for(config, instance)
    lam = gapped_spectrum(n, nocc, gap, rng, lo, hi)
    Q = haar_orthogonal(n, rng)
    F = _symmetric((Q * lam[None, :]) @ Q.T)
    return Hamiltonian(F=F, n=n, nocc=nocc, mu=0.0, lmin=float(lam[0]), lmax=float(lam[-1]),
                       homo=float(lam[nocc - 1]), lumo=float(lam[nocc]), lam=lam, Q=Q,
                       meta={"kind": "dense", "gap": gap, "config": config, "instance": instance})


def diagonal_hamiltonian(lam, mu: float) -> Hamiltonian:
    """The paper's diagonal test matrices: F = diag(lam)."""
    lam = np.sort(np.asarray(lam, dtype=np.float64))
    nocc = int(np.count_nonzero(lam < mu))
    if not (0 < nocc < lam.size):
        raise ValueError("mu must split the spectrum")
    return Hamiltonian(F=np.diag(lam), n=lam.size, nocc=nocc, mu=mu, lmin=float(lam[0]),
                       lmax=float(lam[-1]), homo=float(lam[nocc - 1]), lumo=float(lam[nocc]),
                       lam=lam, Q=np.eye(lam.size), meta={"kind": "diagonal"})


def unit_interval_spectrum(n: int, mu: float, gap: float, config: int = 7,
                           instance: int = 0) -> np.ndarray:
    """Spectrum of width 1 on [0, 1] with a gap of width ``gap`` centred on mu
    and all four edges present; the setting of the paper's multiplication
    count experiments (spectral width 1)."""
    rng = rng_for(config, instance)
    nocc = max(2, min(n - 2, int(round(n * mu))))
    homo, lumo = mu - gap / 2.0, mu + gap / 2.0
    return np.sort(np.concatenate([_band(nocc, 0.0, homo, rng, homo),
                                   _band(n - nocc, lumo, 1.0, rng, lumo)]))


# ----------------------------------------------------------------------------
# Cubic tight-binding lattice (block-sparse workload)
# ----------------------------------------------------------------------------

def lattice_site_index(L: int):
    """Site ordering by 4x4x2 sub-cubes (32 sites), blocks and sites within a
    block both in lexicographic (x, y, z) order.  Returns idx[x, y, z]."""
    if L % 4:
        raise ValueError("L must be a multiple of 4")
    x, y, z = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    nbx, nby, nbz = L // 4, L // 4, L // 2
    blk = ((x // 4) * nby + (y // 4)) * nbz + (z // 2)
    off = ((x % 4) * 4 + (y % 4)) * 2 + (z % 2)
    del nbx
    return blk * 32 + off


@dataclass
class Lattice:
    n: int
    L: int
    rows: np.ndarray   # COO, both triangles, diagonal included
    cols: np.ndarray
    vals: np.ndarray
    onsite: np.ndarray
    gap_bound: float   # |lambda| >= gap_bound for every eigenvalue (Weyl)
    nocc: int

    def dense(self) -> np.ndarray:
        F = np.zeros((self.n, self.n))
        np.add.at(F, (self.rows, self.cols), self.vals)
        return F


def lattice_hamiltonian(L: int, config: int = 3, instance: int = 0,
                        onsite: float = 0.5, onsite_sigma: float = 0.05,
                        hop: float = -1.0, hop_spread: float = 0.1) -> Lattice:
    """Periodic L^3 cubic lattice: onsite 0.5*s + N(0, sigma) with sublattice
    sign s = (-1)^(x+y+z), nearest-neighbour hopping -1 + U(-0.1, 0.1) drawn
    once per bond.  Without the onsite noise, H^2 = 0.25 I + K^2 for the
    bipartite hopping K, so every |lambda| >= 0.5; with the noise, Weyl's
    inequality gives |lambda| >= 0.5 - max|noise|."""
    if L % 4:
        raise ValueError("L must be a multiple of 4 (bipartite under periodic wrap, whole blocks)")
    rng = rng_for(config, instance)
    idx = lattice_site_index(L)
    n = L ** 3
    x, y, z = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    s = np.where((x + y + z) % 2 == 0, 1.0, -1.0)
    noise = rng.normal(0.0, onsite_sigma, size=(L, L, L))
    eps = onsite * s + noise
    rows = [idx.ravel()]
    cols = [idx.ravel()]
    vals = [eps.ravel()]
    for axis in range(3):
        nb = np.roll(idx, -1, axis=axis)
        t = hop + rng.uniform(-hop_spread, hop_spread, size=(L, L, L))
        a, b, tv = idx.ravel(), nb.ravel(), t.ravel()
        rows += [a, b]
        cols += [b, a]
        vals += [tv, tv]
    rows = np.concatenate(rows).astype(np.int64)
    cols = np.concatenate(cols).astype(np.int64)
    vals = np.concatenate(vals)
    on = np.empty(n)
    on[idx.ravel()] = eps.ravel()
    return Lattice(n=n, L=L, rows=rows, cols=cols, vals=vals, onsite=on,
                   gap_bound=float(onsite - np.max(np.abs(noise))), nocc=n // 2)


# ----------------------------------------------------------------------------
# Many instances: batch and serving stream
# ----------------------------------------------------------------------------

@dataclass
class InstanceSpec:
    n: int
    nocc: int
    gap: float
    scheme: str
    arrival: float = 0.0
    instance: int = 0
    config: int = 4


def batch_specs(count: int = 256, n_lo: int = 64, n_hi: int = 2048, gap_lo: float = 1e-3,
                gap_hi: float = 1e-1, config: int = 4) -> list[InstanceSpec]:
    """n log-uniform in [n_lo, n_hi], gap log-uniform, nocc = round(U(0.3, 0.7) n)."""
    rng = rng_for(config, 0)
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        gap = float(math.exp(rng.uniform(math.log(gap_lo), math.log(gap_hi))))
        nocc = int(round(rng.uniform(0.3, 0.7) * n))
        nocc = min(max(nocc, 2), n - 2)
        out.append(InstanceSpec(n=n, nocc=nocc, gap=gap, scheme="TC_SF", instance=i + 1,
                                config=config))
    return out


def serve_specs(rate: float, count: int, n_lo: int = 128, n_hi: int = 8192,
                gap_lo: float = 1e-4, gap_hi: float = 1e-1, config: int = 5) -> list[InstanceSpec]:
    """Poisson arrivals at ``rate`` per second; half fixed-mu, half
    trace-correcting; sizes and gaps log-uniform."""
    rng = rng_for(config, int(rate))
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        gap = float(math.exp(rng.uniform(math.log(gap_lo), math.log(gap_hi))))
        nocc = int(round(rng.uniform(0.3, 0.7) * n))
        nocc = min(max(nocc, 2), n - 2)
        scheme = "FIXED_MU_SF" if rng.uniform() < 0.5 else "TC_SF"
        out.append(InstanceSpec(n=n, nocc=nocc, gap=gap, scheme=scheme, arrival=t,
                                instance=i + 1, config=config))
    return out


def instance_hamiltonian(spec: InstanceSpec) -> Hamiltonian:
    return dense_hamiltonian(spec.n, spec.nocc, spec.gap, config=spec.config,
                             instance=spec.instance)


def reflected_hamiltonian_device(spec: InstanceSpec, device="cuda", reflections: int = 3):
    """A cheaper dense recipe for long request streams: F = H_k .. H_1
    diag(lambda) H_1 .. H_k with k random Householder reflections H = I - 2 v
    v^T (|v| = 1, v from a seeded torch generator), each applied to both
    sides in O(n^2).  The spectrum is exactly that of the dense recipe (the
    same numpy generator), F is dense and symmetric; the eigenvectors are not
    Haar-distributed, which purification does not depend on.  Returns (F as a
    float64 CUDA tensor, Hamiltonian metadata without F or Q)."""
    import torch
    rng = rng_for(spec.config, spec.instance)
    lam = gapped_spectrum(spec.n, spec.nocc, spec.gap, rng)
    g = torch.Generator(device=device)
    g.manual_seed(seed_for(spec.config, spec.instance) & ((1 << 63) - 1))
    F = torch.diag(torch.from_numpy(lam).to(device))
    for _ in range(reflections):
        v = torch.randn(spec.n, generator=g, dtype=torch.float64, device=device)
        v = v / torch.linalg.vector_norm(v)
        w = F @ v                       # H F H = F - 2 v w^T - 2 w v^T + 4 (v^T w) v v^T
        c = torch.dot(v, w)
        F = F - 2.0 * torch.outer(v, w) - 2.0 * torch.outer(w, v) + 4.0 * c * torch.outer(v, v)
    F = 0.5 * (F + F.T)
    meta = Hamiltonian(F=None, n=spec.n, nocc=spec.nocc, mu=0.0, lmin=float(lam[0]),
                       lmax=float(lam[-1]), homo=float(lam[spec.nocc - 1]),
                       lumo=float(lam[spec.nocc]), lam=lam, Q=None,
                       meta={"kind": "reflected-device", "gap": spec.gap, "scheme": spec.scheme,
                             "reflections": reflections})
    return F.contiguous(), meta


def dense_hamiltonian_device(spec: InstanceSpec, device="cuda", keep_q: bool = False):
    """The dense recipe built on a GPU with torch (Haar Q from a seeded torch
    generator, spectrum from the numpy generator as above).  Returns
    (F as a float64 CUDA tensor, Hamiltonian metadata without F; its Q is the
    CUDA tensor of eigenvectors when keep_q, else None)."""
    import torch
    rng = rng_for(spec.config, spec.instance)
    lam = gapped_spectrum(spec.n, spec.nocc, spec.gap, rng)
    g = torch.Generator(device=device)
    g.manual_seed(seed_for(spec.config, spec.instance) & ((1 << 63) - 1))
    Z = torch.randn(spec.n, spec.n, generator=g, dtype=torch.float64, device=device)
    Q, R = torch.linalg.qr(Z)
    Q = Q * torch.sign(torch.diagonal(R))[None, :]
    lt = torch.from_numpy(lam).to(device)
    F = (Q * lt[None, :]) @ Q.T
    F = 0.5 * (F + F.T)
    meta = Hamiltonian(F=None, n=spec.n, nocc=spec.nocc, mu=0.0, lmin=float(lam[0]),
                       lmax=float(lam[-1]), homo=float(lam[spec.nocc - 1]),
                       lumo=float(lam[spec.nocc]), lam=lam, Q=Q if keep_q else None,
                       meta={"kind": "dense-device", "gap": spec.gap, "scheme": spec.scheme})
    return F.contiguous(), meta
