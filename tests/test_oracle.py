"""Pins for the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with a retyped copy of its own formulas:
each pin comes from a definition (fixed points and vanishing derivatives of
P_{i,j}, Eq. 3's fold condition, D = theta(mu I - F)), from a library routine
(eigh, a scalar root finder), from functional calculus on the eigenbasis, or
from a claim the paper states (half the multiplications, speedup growing as
the gap closes, independent of mu).
"""
import math
import os

import numpy as np
import pytest
import sympy
from scipy.optimize import brentq

from oracle import purify_oracle as O
from paper_1101_0265_gb300 import inputs as I

SCHEMES = O.SCHEMES


# --- P_{i,j}: degree 1+i+j, fixed points 0 and 1, i vanishing derivatives at
# 0 and j at 1 (the paper's definition of the notation) ---------------------

@pytest.mark.parametrize("fn,i,j", [(O.P10, 1, 0), (O.P01, 0, 1), (O.P11, 1, 1)])
def test_polynomial_family_definition(fn, i, j):
    x = sympy.Symbol("x")
    p = sympy.nsimplify(sympy.expand(fn(x)), rational=True)
    assert sympy.degree(p, x) == 1 + i + j
    assert p.subs(x, 0) == 0 and p.subs(x, 1) == 1
    for d in range(1, i + 1):
        assert sympy.diff(p, x, d).subs(x, 0) == 0
    for d in range(1, j + 1):
        assert sympy.diff(p, x, d).subs(x, 1) == 0
    # and the next derivative does not vanish (exactly i and j)
    assert sympy.diff(p, x, i + 1).subs(x, 0) != 0
    assert sympy.diff(p, x, j + 1).subs(x, 1) != 0


# --- Algorithm 1's alpha solves Eq. 3 (independently, by root finding) ---------

@pytest.mark.parametrize("beta", [1e-9, 1e-4, 0.01, 0.1, 0.25, 0.4, 0.49, 0.4999])
def test_fixed_mu_alpha_solves_eq3(beta):
    def g(a):
        return O.P11(a * (beta - 0.5) + 0.5) - O.P11(0.5 * (1.0 - a))
    a_root = brentq(g, 1.0 + 1e-12, math.sqrt(3.0) + 1e-9, xtol=1e-15, rtol=1e-15)
    a = O.fixed_mu_alpha(beta)
    assert a >= 1.0
    assert abs(a - a_root) <= 1e-12 * a
    # the fold is complete: the stretched interval [0.5(1-a), a(b-0.5)+0.5]
    # straddles 0, so the unoccupied part folds over itself
    assert 0.5 * (1 - a) <= 0.0 <= a * (beta - 0.5) + 0.5


def test_fixed_mu_alpha_limits():
    # alpha -> 1 (plain McWeeny) as beta -> 0; alpha = sqrt(3) at beta = 1/2
    assert abs(O.fixed_mu_alpha(0.0) - 1.0) < 1e-15
    assert abs(O.fixed_mu_alpha(0.5) - math.sqrt(3.0)) < 1e-15


# --- Algorithm 2's alpha makes the folded ends meet --------------------------

@pytest.mark.parametrize("beta,betabar", [(0.45, 0.6), (0.3, 0.9), (0.1, 0.95), (0.49, 0.51),
                                          (0.2, 0.55), (0.02, 0.3)])
def test_tc_alpha_fold_condition(beta, betabar):
    # P10 branch: the images of 0 and beta under x -> (1+a)x - a have equal
    # squares, i.e. the stretched unoccupied interval is folded onto itself.
    a10 = O.tc_alpha("P10", beta, betabar)
    root10 = brentq(lambda a: O.P10(-a) - O.P10((1 + a) * beta - a), 1e-14, 1.0, xtol=1e-16)
    assert abs(a10 - root10) < 1e-12
    # P01 branch: the images of 1 and beta-bar under x -> (1+a)x meet under 2y - y^2.
    a01 = O.tc_alpha("P01", beta, betabar)
    root01 = brentq(lambda a: O.P01(1 + a) - O.P01((1 + a) * betabar), 1e-14, 1.0, xtol=1e-16)
    assert abs(a01 - root01) < 1e-12
    assert a10 >= 0 and a01 >= 0


# --- the scalar bound tracks the gap edges exactly (diagonal test matrices,
# the paper's own test setting) ---------------------------------------------

@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("mu,gap", [(0.5, 0.1), (0.25, 0.01), (0.8, 0.02)])
def test_scalar_bound_tracks_edges_on_diagonal(scheme, mu, gap):
    lam = I.unit_interval_spectrum(40, mu, gap)
    h = I.diagonal_hamiltonian(lam, mu)
    X, r = O.purify(h.F, scheme, 0.0, 1.0, mu=mu, homo=h.homo, lumo=h.lumo, tol=1e-12)
    assert r.converged
    # rerun step by step, checking every iterate's spectrum against the bound
    x_unocc = np.diag(X)[h.nocc:]
    x_occ = np.diag(X)[:h.nocc]
    b, bb = r.betas[-1], r.betabars[-1]
    assert x_unocc.max() <= b + 1e-15 and x_unocc.min() >= -1e-15
    assert x_occ.min() >= bb - 1e-15 and x_occ.max() <= 1 + 1e-15
    for k in range(1, r.iterations + 1):
        Xk, rk = O.purify(h.F, scheme, 0.0, 1.0, mu=mu, homo=h.homo, lumo=h.lumo, tol=0.0,
                          max_iter=k)
        d = np.diag(Xk)
        # the lumo / homo images are the bound itself (the edge is attained)
        assert abs(d[h.nocc] - rk.betas[-1]) <= 1e-13
        assert abs(d[h.nocc - 1] - rk.betabars[-1]) <= 1e-13
        assert d[h.nocc:].max() <= rk.betas[-1] + 1e-13
        assert d[:h.nocc].min() >= rk.betabars[-1] - 1e-13


# --- functional calculus: on F = Q diag(lam) Q^T the matrix recursion equals
# Q diag(f(lam)) Q^T with f the composed scalar maps ------------------------

def _scalar_compose(scheme, r, x):
    x = np.array(x, dtype=np.float64)
    if scheme.startswith("FIXED_MU"):
        for a in r.alphas:
            xs = a * (x - 0.5) + 0.5
            x = O.P11(xs)
    else:
        for br, a in zip(r.branches, r.alphas):
            x = O.P10((1 + a) * x - a) if br == "P10" else O.P01((1 + a) * x)
    return x


@pytest.mark.parametrize("scheme", SCHEMES)
def test_matrix_recursion_is_functional_calculus(scheme):
    h = I.dense_hamiltonian(48, 20, 0.2, config=90)
    for k in (1, 2, 5):
        X, r = O.purify(h.F, scheme, h.lmin, h.lmax, mu=0.0, homo=h.homo, lumo=h.lumo,
                        tol=0.0, max_iter=k)
        c0, c1 = r.f0
        x0 = c0 + c1 * h.lam
        fx = _scalar_compose(scheme, r, x0)
        ref = (h.Q * fx[None, :]) @ h.Q.T
        assert np.max(np.abs(X - ref)) < 1e-12
        # f0 maps the spectrum into [0, 1] with occupied states above
        assert x0.min() >= -1e-15 and x0.max() <= 1 + 1e-15
        assert x0[: h.nocc].min() > x0[h.nocc:].max()


# --- brute force: D = theta(mu I - F) by eigendecomposition ------------------

@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("n,nocc,gap", [(64, 32, 0.1), (96, 30, 0.01), (33, 17, 0.3)])
def test_density_matches_eigendecomposition(scheme, n, nocc, gap):
    h = I.dense_hamiltonian(n, nocc, gap, config=91)
    tol = 1e-12
    D, r = O.purify(h.F, scheme, h.lmin, h.lmax, mu=0.0, homo=h.homo, lumo=h.lumo, tol=tol)
    assert r.converged and r.err_bound <= tol
    D_ref = O.density_by_eigh(h.F, 0.0)
    assert np.max(np.abs(D - D_ref)) <= tol + 1e-11
    D_cf = O.density_closed_form(h.Q, h.lam, 0.0)
    assert np.max(np.abs(D - D_cf)) <= tol + 1e-11
    # invariants: trace = nocc, idempotent, commutes with F
    assert abs(np.trace(D) - nocc) < 1e-10
    assert O.idempotency_error(D) < 1e-10
    assert O.commutator_norm(D, h.F) < 1e-10


def test_density_on_diagonal_is_step_function():
    lam = I.unit_interval_spectrum(50, 0.3, 0.05)
    h = I.diagonal_hamiltonian(lam, 0.3)
    for scheme in SCHEMES:
        D, r = O.purify(h.F, scheme, 0.0, 1.0, mu=0.3, homo=h.homo, lumo=h.lumo, tol=1e-13)
        expect = np.diag((lam < 0.3).astype(float))
        assert np.max(np.abs(D - expect)) <= 1e-13


def test_trace_rule_niklasson():
    # alpha = 0 with the trace rule: Niklasson's TC2.  It needs only nocc;
    # without gap bounds it stops on idempotency.
    h = I.dense_hamiltonian(64, 21, 0.1, config=92)
    D, r = O.purify_tc(h.F, h.lmin, h.lmax, tol=1e-10, scaled=False, branch_rule="trace",
                       nocc=h.nocc, max_iter=100)
    assert r.converged
    D_ref = O.density_by_eigh(h.F, 0.0)
    assert np.max(np.abs(D - D_ref)) < 1e-9
    # with bounds given, the trace rule and the beta rule reach the same D
    D2, r2 = O.purify_tc(h.F, h.lmin, h.lmax, h.homo, h.lumo, tol=1e-12, scaled=False,
                         branch_rule="trace", nocc=h.nocc)
    assert np.max(np.abs(D2 - D_ref)) < 1e-11


def test_tie_takes_p01_branch():
    # symmetric gap: beta + beta-bar == 1 exactly -> the strict test is false
    b, bb = O.tc_beta0(-1.0, 1.0, -0.05, 0.05)
    assert b + bb == 1.0
    assert O.tc_branch_by_beta(b, bb) == "P01"


# --- the paper's claims about multiplication counts (Fig. 3 protocol:
# spectral width 1, accuracy 1e-9) -------------------------------------------

def _counts(mu, xi, tol=1e-9):
    g = O.fixed_mu_gamma(0.0, 1.0, mu)
    b = O.fixed_mu_beta0(g, mu, mu - xi / 2, mu + xi / 2)
    mcw_sf = 2 * len(O.fixed_mu_schedule(b, tol, 10_000, True)[0])
    mcw_mono = 2 * len(O.fixed_mu_schedule(b, tol, 10_000, False)[0])
    tb, tbb = O.tc_beta0(0.0, 1.0, mu - xi / 2, mu + xi / 2)
    tc_sf = len(O.tc_schedule(tb, tbb, tol, 10_000, True))
    tc_mono = len(O.tc_schedule(tb, tbb, tol, 10_000, False))
    return mcw_mono, mcw_sf, tc_mono, tc_sf


def golden_counts():
    """Rows (mu, xi, mcweeny_mono, mcweeny_scaled, tc_mono, tc_scaled) of
    tests/golden/scalar_counts.txt (written from the oracle by
    tests/golden/make_scalar_counts.py)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "scalar_counts.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    return [(float(r[0]), float(r[1])) + tuple(int(v) for v in r[2:]) for r in rows]


def test_scalar_counts_golden():
    # the stored counts are reproduced exactly; they show the paper's claims
    # (about half the multiplications; cost growing with 1/xi) and the mirror
    # symmetry of both schemes in mu about the middle of the spectrum
    rows = golden_counts()
    assert len(rows) == 12
    by = {}
    for mu, xi, mm, ms, tm, ts in rows:
        assert _counts(mu, xi) == (mm, ms, tm, ts), (mu, xi)
        assert 0.4 <= ms / mm <= 0.65 and 0.4 <= ts / tm <= 0.65
        by[(round(mu, 2), xi)] = (mm, ms, tm, ts)
    for mu in (0.1, 0.25, 0.4):
        assert by[(mu, 0.01)] == by[(round(1 - mu, 2), 0.01)]
    gap_sweep = [by[(0.5, 10.0 ** -k)] for k in range(1, 7)]
    for col in range(4):
        assert all(a[col] <= b[col] for a, b in zip(gap_sweep, gap_sweep[1:]))


def test_config_counts_golden():
    # the dense configurations' counts (spectrum [-1, 1], mu = 0) stored in
    # tests/golden/config_counts.txt are reproduced exactly; scaling never
    # costs more, a tighter tolerance never costs less
    from tests.golden.make_scalar_counts import config_counts
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config_counts.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 12
    by = {}
    for r in rows:
        gap, tol = float(r[0]), float(r[1])
        c = tuple(int(v) for v in r[2:])
        assert config_counts(gap, tol) == c, (gap, tol)
        assert c[1] <= c[0] and c[3] <= c[2]
        by[(gap, tol)] = c
    for gap in (1e-1, 1e-2, 1e-3, 1e-4):
        for col in range(4):
            assert by[(gap, 1e-6)][col] <= by[(gap, 1e-9)][col] <= by[(gap, 1e-12)][col]


def test_half_the_multiplications():
    # Abstract and Fig. 3b: about half the multiplications, "around twice as fast"
    for xi in (1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6):
        mm, ms, tm, ts = _counts(0.5, xi)
        assert 0.4 <= ms / mm <= 0.65, (xi, mm, ms)
        assert 0.4 <= ts / tm <= 0.65, (xi, tm, ts)


def test_speedup_grows_as_gap_closes_and_cost_is_logarithmic():
    xis = [10.0 ** -k for k in range(1, 9)]
    c = np.array([_counts(0.5, xi) for xi in xis], dtype=float)
    saved_mcw = c[:, 0] - c[:, 1]
    saved_tc = c[:, 2] - c[:, 3]
    assert np.all(np.diff(saved_mcw) >= 0) and saved_mcw[-1] > saved_mcw[0]
    assert np.all(np.diff(saved_tc) >= 0) and saved_tc[-1] > saved_tc[0]
    # counts grow linearly in ln(1/xi) (cost O(ln(width/gap)))
    x = np.log(1.0 / np.array(xis))
    for col in range(4):
        slope, icept = np.polyfit(x, c[:, col], 1)
        resid = c[:, col] - (slope * x + icept)
        assert slope > 0 and np.max(np.abs(resid)) <= 2.5


def test_speedup_independent_of_mu():
    # Fig. 3a: xi = 0.01, mu varied; the ratio stays near one half everywhere
    ratios = []
    for mu in (0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9):
        mm, ms, tm, ts = _counts(mu, 0.01)
        ratios += [ms / mm, ts / tm]
    assert min(ratios) >= 0.45 and max(ratios) <= 0.65


def test_mirror_symmetry_in_mu():
    # theta(mu I - F) for mu -> 1 - mu is the complement problem: equal counts
    for mu in (0.1, 0.25, 0.4):
        assert _counts(mu, 0.01) == _counts(1.0 - mu, 0.01)


def test_gap_zero_alpha1_fixed_point():
    # beta = 1/2 (no gap) is a fixed point of Algorithm 1's scalar map: the
    # method cannot converge, which is why a zero gap is rejected
    a = O.fixed_mu_alpha(0.5)
    bs = a * (0.5 - 0.5) + 0.5
    assert O.P11(bs) == 0.5


# --- spectral bounds ---------------------------------------------------------

def test_gershgorin_contains_spectrum():
    h = I.dense_hamiltonian(80, 40, 0.1, config=93)
    lo, hi = O.gershgorin(h.F)
    assert lo <= h.lam[0] and hi >= h.lam[-1]
    d = np.array([3.0, -2.0, 0.5])
    assert O.gershgorin(np.diag(d)) == (-2.0, 3.0)
    # 2x2 with known discs
    F = np.array([[1.0, -2.0], [-2.0, 4.0]])
    assert O.gershgorin(F) == (-1.0, 6.0)


def test_splitmix64_published_vector():
    # SplitMix64 seeded with 1234567: first outputs of the reference generator
    seq = [O._splitmix64((1234567 + i * O._GOLDEN) & O._MASK) for i in range(5)]
    assert seq == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                   4593380528125082431, 16408922859458223821]


def test_lanczos_full_recovers_spectrum():
    h = I.dense_hamiltonian(24, 12, 0.3, config=94)
    q = O.lanczos_start(24)
    a, b = O.lanczos(h.F, 24, q)
    T = np.diag(a) + np.diag(b[:-1], 1) + np.diag(b[:-1], -1)
    assert np.max(np.abs(np.linalg.eigvalsh(T) - h.lam)) < 1e-8
    # tridiagonal of the Lanczos basis: V^T F V = T for a few steps
    k = 6
    a, b = O.lanczos(h.F, k, q)
    V = [q / np.linalg.norm(q)]
    vp = np.zeros(24)
    for j in range(k - 1):
        w = h.F @ V[-1] - (b[j - 1] * vp if j else 0.0) - a[j] * V[-1]
        vp = V[-1]
        V.append(w / b[j])
    V = np.array(V).T
    Tk = np.diag(a) + np.diag(b[:k - 1], 1) + np.diag(b[:k - 1], -1)
    assert np.max(np.abs(V.T @ h.F @ V - Tk)) < 1e-12
    assert np.max(np.abs(V.T @ V - np.eye(k))) < 1e-12


def test_lanczos_bounds_bracket_extremes():
    h = I.dense_hamiltonian(300, 150, 0.1, config=95)
    lo, hi = O.lanczos_bounds(h.F, 30)
    g_lo, g_hi = O.gershgorin(h.F)
    assert g_lo <= lo and hi <= g_hi
    # the estimates bracket the extreme eigenvalues -1, 1 and are far tighter
    # than Gershgorin on a dense matrix
    assert lo <= -1.0 + 1e-12 and hi >= 1.0 - 1e-12
    assert lo > -1.05 and hi < 1.05
    assert g_hi - g_lo > 4.0


# --- block truncation (the sparsity discussion: drop small elements while
# controlling the error each step adds) ---------------------------------------

def _random_blocky(nb, seed, bs=32):
    rng = np.random.default_rng(seed)
    scales = 10.0 ** rng.uniform(-9, 0, size=(nb, nb))
    scales = np.triu(scales) + np.triu(scales, 1).T
    X = rng.standard_normal((nb * bs, nb * bs)) * np.repeat(np.repeat(scales, bs, 0), bs, 1)
    return 0.5 * (X + X.T)


@pytest.mark.parametrize("tau", [0.0, 1e-8, 1e-6, 1e-4])
def test_truncation_error_bound_and_greed(tau):
    X = _random_blocky(6, 3)
    Xt, keep = O.truncate_blocks(X, tau)
    assert np.array_equal(keep, keep.T)
    dropped = X - Xt
    # the step moves X by at most tau in the Frobenius (hence 2-) norm
    assert np.linalg.norm(dropped) <= tau * (1 + 1e-12)
    assert np.linalg.norm(dropped, 2) <= tau * (1 + 1e-12)
    # greedy and maximal: the smallest kept block would overflow the budget
    N = O.block_norms(X)
    kept = [(N[i, j], i, j) for i in range(6) for j in range(i, 6) if keep[i, j]]
    if kept and tau > 0:
        m, i, j = min(kept)
        w = 1.0 if i == j else 2.0
        assert np.linalg.norm(dropped) ** 2 + w * m * m > tau * tau
    # every dropped block is no larger than every kept block
    if kept:
        drop_norms = [N[i, j] for i in range(6) for j in range(i, 6) if not keep[i, j]]
        if drop_norms:
            assert max(drop_norms) <= min(k[0] for k in kept)


def test_block_norms_definition():
    X = _random_blocky(3, 4)
    N = O.block_norms(X)
    for i in range(3):
        for j in range(3):
            assert abs(N[i, j] - np.sqrt(np.sum(X[32 * i:32 * i + 32, 32 * j:32 * j + 32] ** 2))) < 1e-12


def test_truncated_purification_reduces_to_plain_at_tau_zero():
    h = I.dense_hamiltonian(96, 40, 0.05, config=96)
    X, r, nnzb = O.purify_tc_truncated(h.F, h.lmin, h.lmax, h.homo, h.lumo, 0.0, tol=1e-12)
    Xp, rp = O.purify_tc(h.F, h.lmin, h.lmax, h.homo, h.lumo, tol=1e-12)
    assert r.iterations == rp.iterations
    assert np.max(np.abs(X - Xp)) < 1e-14
    assert all(k == 6 for k in nnzb)  # 3 x 3 blocks, none exactly zero: 6 with I <= J


def test_lattice_gap_and_truncated_density():
    # the cubic lattice's spectrum keeps |lambda| >= 0.5 - max|onsite noise|
    lat = I.lattice_hamiltonian(8)
    F = lat.dense()
    lam = np.linalg.eigvalsh(F)
    assert np.min(np.abs(lam)) >= lat.gap_bound
    assert np.count_nonzero(lam < 0) == lat.nocc
    lo, hi = O.gershgorin(F)
    g = lat.gap_bound
    tau = 1e-6
    X, r, nnzb = O.purify_tc_truncated(F, lo, hi, -g, g, tau, tol=1e-10)
    D = O.density_by_eigh(F, 0.0)
    # each step adds at most tau; errors in the block coupling occupied and
    # unoccupied states are amplified by at most 1 / (mapped gap)
    mapped_gap = 2 * g / (hi - lo)
    assert np.linalg.norm(X - D, 2) <= 1e-10 + (r.iterations + 1) * tau / mapped_gap
    assert abs(np.trace(X) - lat.nocc) < 1e-3


def test_truncation_budget_spreads_over_the_schedule():
    # a total budget eps: tau = eps / (m + 1) for the m scheduled iterations
    # and X_0; the scaled schedule (fewer iterations) truncates harder, and
    # the result stays within eps / (mapped gap) of the exact density
    lat = I.lattice_hamiltonian(8)
    F = lat.dense()
    lo, hi = O.gershgorin(F)
    g = lat.gap_bound
    eps = 1e-4
    D = O.density_by_eigh(F, 0.0)
    mapped_gap = 2 * g / (hi - lo)
    runs = {}
    for scaled in (True, False):
        X, r, nnzb = O.purify_tc_truncated(F, lo, hi, -g, g, None, tol=1e-10, scaled=scaled,
                                           tau_budget=eps)
        assert r.tau == pytest.approx(eps / (r.iterations + 1), rel=1e-15)
        assert np.linalg.norm(X - D, 2) <= 1e-10 + eps / mapped_gap
        runs[scaled] = (r, nnzb)
    assert runs[True][0].iterations < runs[False][0].iterations
    assert runs[True][0].tau > runs[False][0].tau
    # a zero budget truncates only exact zeros: the untruncated recursion
    X0, r0, _ = O.purify_tc_truncated(F, lo, hi, -g, g, None, tol=1e-10, tau_budget=0.0)
    Xp, rp = O.purify_tc(F, lo, hi, -g, g, tol=1e-10)
    assert np.max(np.abs(X0 - Xp)) < 1e-13


# --- gap edges from the purification (interior eigenvalues) -----------------

@pytest.mark.parametrize("n,nocc,gap,cfg", [(300, 120, 0.05, 1), (500, 250, 0.01, 2), (400, 100, 2e-3, 3),
                                            (256, 128, 0.1, 4), (200, 60, 1e-4, 5)])
def test_gap_estimate_is_inner_and_tight(n, nocc, gap, cfg):
    h = I.dense_hamiltonian(n, nocc, gap, config=cfg)
    he, le, steps = O.estimate_gap(h.F, h.lmin, h.lmax, h.nocc)
    w = h.lmax - h.lmin
    assert h.homo <= he < le <= h.lumo
    assert he - h.homo <= 1e-12 * w and h.lumo - le <= 1e-12 * w
    assert steps > 0


def test_gap_estimate_diagonal_and_lattice():
    # diagonal F: the recursion acts entry by entry
    lam = np.sort(np.concatenate([np.linspace(-1, -0.03, 70), np.linspace(0.02, 1, 50)]))
    h = I.diagonal_hamiltonian(lam, 0.0)
    he, le, _ = O.estimate_gap(h.F, -1.0, 1.0, 70)
    assert -0.03 <= he < le <= 0.02 and he + 0.03 < 1e-12 and 0.02 - le < 1e-12
    # the 8^3 lattice against its eigendecomposition
    lat = I.lattice_hamiltonian(8)
    F = lat.dense()
    ev = np.linalg.eigvalsh(F)
    lo, hi = O.gershgorin(F)
    he, le, _ = O.estimate_gap(F, lo, hi, lat.nocc)
    assert ev[lat.nocc - 1] <= he < le <= ev[lat.nocc]
    assert he - ev[lat.nocc - 1] < 1e-8 and ev[lat.nocc] - le < 1e-8


def test_gap_filters_pick_their_side():
    # the occupied filter x^4 (1 - x) peaks for the occupied eigenvalue
    # nearest 1/2 and the unoccupied one x (1 - x)^4 for the unoccupied one,
    # on spectra where every eigenvalue has x (1 - x) < 1/16
    rng = np.random.default_rng(0)
    occ = 1.0 - rng.uniform(1e-6, 0.06, 40)
    unocc = rng.uniform(1e-6, 0.06, 30)
    x = np.concatenate([occ, unocc])
    p = O.GAP_FILTER_POWER
    assert np.argmax(x ** p * (1 - x)) == np.argmin(occ)
    assert np.argmax(x * (1 - x) ** p) - 40 == np.argmax(unocc)


# --- higher-order fixed-mu polynomials P_{m,m} ---------------------------------

@pytest.mark.parametrize("i,j", [(1, 0), (0, 1), (1, 1), (3, 3), (1, 3), (3, 1), (2, 2), (5, 5)])
def test_P_ij_closed_form_matches_definition(i, j):
    # degree 1 + i + j, P(0) = 0, P(1) = 1, i vanishing derivatives at 0 and j
    # at 1: 2 + i + j conditions fix the polynomial
    sympy = pytest.importorskip("sympy")
    x = sympy.symbols("x")
    P = sympy.nsimplify(sympy.expand(O.P_ij(i, j, x)), rational=True)
    assert sympy.degree(P, x) == 1 + i + j
    assert P.subs(x, 0) == 0 and P.subs(x, 1) == 1
    for d in range(1, i + 1):
        assert sympy.diff(P, x, d).subs(x, 0) == 0
    for d in range(1, j + 1):
        assert sympy.diff(P, x, d).subs(x, 1) == 0
    assert O.P_ij(1, 1, 0.3) == pytest.approx(O.P11(0.3), rel=1e-15)


def test_pmm_alpha_solves_the_scaling_equation():
    for beta in np.linspace(0.01, 0.499, 40):
        # m = 1 is Algorithm 1's closed form
        assert O.pmm_alpha(1, beta) == pytest.approx(O.fixed_mu_alpha(beta), rel=4e-16, abs=0)
        a = O.pmm_alpha(3, beta)
        assert 1.0 <= a <= 1.0 / (1.0 - 2.0 * beta)
        lhs = O.P_ij(3, 3, a * (beta - 0.5) + 0.5)
        rhs = O.P_ij(3, 3, 0.5 * (1.0 - a))
        assert abs(lhs - rhs) <= 1e-14


def test_pmm_scheme():
    h = I.dense_hamiltonian(160, 60, 1e-3, config=10)
    Dx = O.density_closed_form(h.Q, h.lam, 0.0)
    # m = 1 is Algorithm 1
    X1, r1 = O.purify_fixed_mu_pmm(h.F, h.lmin, h.lmax, 0.0, h.homo, h.lumo, m=1, tol=1e-12)
    Xa, ra = O.purify_fixed_mu(h.F, h.lmin, h.lmax, 0.0, h.homo, h.lumo, tol=1e-12)
    assert r1.iterations == ra.iterations and r1.multiplications == ra.multiplications
    assert np.max(np.abs(X1 - Xa)) < 1e-12
    # m = 3: converges to D; scaling saves iterations; per multiplication it
    # is no better than m = 1 (the finding the bench reports)
    X3, r3 = O.purify_fixed_mu_pmm(h.F, h.lmin, h.lmax, 0.0, h.homo, h.lumo, m=3, tol=1e-12)
    _, r3m = O.purify_fixed_mu_pmm(h.F, h.lmin, h.lmax, 0.0, h.homo, h.lumo, m=3, tol=1e-12, scaled=False)
    assert r3.converged and np.max(np.abs(X3 - Dx)) < 1e-11
    assert r3.iterations < r3m.iterations and r3.iterations < r1.iterations
    assert r3.multiplications > r1.multiplications
    # functional calculus: on a diagonal F the recursion acts entry by entry
    lam = np.concatenate([np.linspace(-1, -0.05, 20), np.linspace(0.05, 1, 20)])
    hd = I.diagonal_hamiltonian(lam, 0.0)
    Xd, rd = O.purify_fixed_mu_pmm(hd.F, -1.0, 1.0, 0.0, -0.05, 0.05, m=3, tol=1e-12)
    x = (0.0 - lam) / O.fixed_mu_gamma(-1.0, 1.0, 0.0) + 0.5
    for a in rd.alphas:
        x = O.P_ij(3, 3, a * (x - 0.5) + 0.5)
    assert np.max(np.abs(np.diag(Xd) - x)) < 1e-13


# --- asymmetric P_{i,j}: scaling about the unstable fixed point ----------------

def test_pij_fixed_points():
    for i, j in ((1, 3), (3, 1), (1, 5), (3, 5)):
        c = O.pij_fixed_point(i, j)
        assert 0.0 < c < 1.0 and abs(O.P_ij(i, j, c) - c) < 1e-15
        assert O.pij_fixed_point(j, i) == pytest.approx(1.0 - c, abs=1e-15)  # P_ij(x) = 1 - P_ji(1 - x)
    assert O.pij_fixed_point(3, 3) == pytest.approx(0.5, abs=1e-15)


def test_pij_alpha_reduces_and_folds():
    for beta in np.linspace(0.02, 0.49, 25):
        assert O.pij_alpha(1, 1, 0.5, beta, 1.0 - beta) == pytest.approx(O.fixed_mu_alpha(beta), rel=1e-15)
        assert O.pij_alpha(3, 3, 0.5, beta, 1.0 - beta) == pytest.approx(O.pmm_alpha(3, beta), rel=1e-14)
    # asymmetric: the binding side folds exactly, the other not past its edge
    c = O.pij_fixed_point(3, 1)
    for beta, betabar in ((0.2, 0.9), (0.7, 0.95), (0.5, 0.99)):
        a = O.pij_alpha(3, 1, c, beta, betabar)
        gu = O.P_ij(3, 1, a * (beta - c) + c) - O.P_ij(3, 1, c * (1 - a))
        go = O.P_ij(3, 1, c + a * (1 - c)) - O.P_ij(3, 1, a * (betabar - c) + c)
        assert a >= 1.0 and gu >= -1e-15 and go >= -1e-15 and min(gu, go) < 1e-12


@pytest.mark.parametrize("i,j", [(1, 3), (3, 1), (3, 3)])
def test_pij_scheme_bounds_track_the_eigenvalues(i, j):
    # on a diagonal F the recursion acts entry by entry: after every iteration
    # the unoccupied images lie in [0, beta] and the occupied in [betabar, 1]
    lam = np.concatenate([np.linspace(-1, -0.02, 30), np.linspace(0.03, 1, 25)])
    h = I.diagonal_hamiltonian(lam, 0.0)
    c = O.pij_fixed_point(i, j)
    gamma = max((0.0 + 1.0) / (1.0 - c), (1.0 - 0.0) / c)
    x = c + (0.0 - lam) / gamma
    beta, betabar = c - 0.03 / gamma, c + 0.02 / gamma
    _, steps = O.pij_schedule(i, j, beta, betabar, 1e-12, 200)
    occ = lam < 0
    for a, b, bb in steps:
        x = O.P_ij(i, j, a * (x - c) + c)
        assert np.all(x[~occ] <= b + 1e-15) and np.all(x[~occ] >= -1e-15)
        assert np.all(x[occ] >= bb - 1e-15) and np.all(x[occ] <= 1 + 1e-15)
    X, r = O.purify_fixed_mu_pij(h.F, -1.0, 1.0, 0.0, -0.02, 0.03, i, j, tol=1e-12)
    assert r.converged and np.max(np.abs(np.diag(X) - occ)) < 1e-12
    assert np.max(np.abs(np.diag(X) - x)) < 1e-13


def test_pij_scheme_dense():
    h = I.dense_hamiltonian(150, 50, 1e-3, config=11)
    Dx = O.density_closed_form(h.Q, h.lam, 0.0)
    for i, j in ((1, 3), (3, 1)):
        X, r = O.purify_fixed_mu_pij(h.F, h.lmin, h.lmax, 0.0, h.homo, h.lumo, i, j, tol=1e-12)
        _, rm = O.purify_fixed_mu_pij(h.F, h.lmin, h.lmax, 0.0, h.homo, h.lumo, i, j, tol=1e-12,
                                      scaled=False)
        assert r.converged and np.max(np.abs(X - Dx)) < 1e-11
        assert r.iterations < rm.iterations
        assert r.multiplications == O.PIJ_PRODUCTS[(i, j)] * r.iterations
    # i = j = 3 through the general route is the P_{m,m} scheme
    X3, r3 = O.purify_fixed_mu_pij(h.F, h.lmin, h.lmax, 0.0, h.homo, h.lumo, 3, 3, tol=1e-12)
    Xm, rm3 = O.purify_fixed_mu_pmm(h.F, h.lmin, h.lmax, 0.0, h.homo, h.lumo, m=3, tol=1e-12)
    assert r3.iterations == rm3.iterations and np.max(np.abs(X3 - Xm)) < 1e-11
