"""GPU parity of the float64 path against the CPU oracle (through the C ABI)."""
import math

import numpy as np
import pytest

from oracle import purify_oracle as O
from paper_1101_0265_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    from paper_1101_0265_gb300 import build
    build.build()
    import paper_1101_0265_gb300 as P
    return P


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# --- kernel units -------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 31, 63, 64, 65, 127, 130, 257, 600])
def test_symm_product_f64(P, n):
    h = I.dense_hamiltonian(max(n, 2), max(n // 2, 1), 0.1, config=80, instance=n)
    X = h.F[:n, :n].copy() if n > 1 else np.array([[0.7]])
    X = 0.5 * (X + X.T)
    X2 = X @ X
    out = torch.empty((n, n), dtype=torch.float64, device="cuda")
    P.k_symm_product_f64(_cuda(X), _cuda(X), out)          # X X
    got = out.cpu().numpy()
    assert np.array_equal(got, got.T)
    assert np.max(np.abs(got - X2)) <= 1e-14 * n * max(1.0, np.max(np.abs(X)) ** 2) + 1e-15
    P.k_symm_product_f64(_cuda(X2), _cuda(X), out)         # X^2 X (commuting)
    ref = X2 @ X
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-13 * n + 1e-15


@pytest.mark.parametrize("n", [5, 64, 129, 300])
def test_step_f64_epilogue_and_reductions(P, n):
    h = I.dense_hamiltonian(n, n // 3 + 1, 0.2, config=81, instance=n)
    X = (h.lmax * np.eye(n) - h.F) / (h.lmax - h.lmin)
    cP, cE, cI, dY, dI = -1.3, 2.2, 0.25, 0.8, 0.1
    out = torch.empty((n, n), dtype=torch.float64, device="cuda")
    red = torch.zeros(3, dtype=torch.float64, device="cuda")
    Xd = _cuda(X)
    P.k_step_f64(Xd, Xd, Xd, out, cP, cE, cI, dY, dI, red)
    torch.cuda.synchronize()
    S = X @ X
    Y = cP * S + cE * X + cI * np.eye(n)
    C = dY * Y + dI * np.eye(n)
    got = out.cpu().numpy()
    assert np.max(np.abs(got - C)) < 1e-13
    r = red.cpu().numpy()
    assert abs(r[0] - np.trace(Y)) < 1e-11
    assert abs(r[1] - np.sum((X - S) ** 2)) < 1e-11 * max(1.0, np.sum((X - S) ** 2))
    assert abs(r[2] - np.sum(Y ** 2)) < 1e-11 * np.sum(Y ** 2)


@pytest.mark.parametrize("n", [1, 7, 33, 512, 1000])
def test_gershgorin_f64(P, n):
    h = I.dense_hamiltonian(max(n, 2), max(n // 2, 1), 0.05, config=82, instance=n)
    F = h.F[:n, :n].copy()
    lohi = torch.zeros(2, dtype=torch.float64, device="cuda")
    P.k_gershgorin_f64(_cuda(F), lohi)
    lo, hi = O.gershgorin(F)
    got = lohi.cpu().numpy()
    scale = np.abs(F).sum(axis=1).max()
    assert abs(got[0] - lo) <= 1e-13 * scale and abs(got[1] - hi) <= 1e-13 * scale


@pytest.mark.parametrize("n,k", [(50, 10), (300, 24), (1024, 32)])
def test_lanczos_f64(P, n, k):
    h = I.dense_hamiltonian(n, n // 2, 0.1, config=83, instance=n)
    a, b = P.k_lanczos_f64(_cuda(h.F), k)
    ao, bo = O.lanczos(h.F, k, O.lanczos_start(n))
    assert np.max(np.abs(a - ao)) < 1e-9 and np.max(np.abs(b - bo)) < 1e-9
    # the extremal Ritz values agree closely
    T = lambda a_, b_: np.diag(a_) + np.diag(b_[:-1], 1) + np.diag(b_[:-1], -1)
    assert np.max(np.abs(np.linalg.eigvalsh(T(a, b))[[0, -1]]
                         - np.linalg.eigvalsh(T(ao, bo))[[0, -1]])) < 1e-11
    # reductions in a fixed order: the same coefficients on every call
    a2, b2 = P.k_lanczos_f64(_cuda(h.F), k)
    assert np.array_equal(a, a2) and np.array_equal(b, b2)


# --- whole purification parity --------------------------------------------------

def _run(P, h, scheme, tol=1e-12, max_iter=200, precision="fp64", bounds=True, **opts):
    pur = P.Purifier(precision=precision, **opts)
    kw = dict(lmin=h.lmin, lmax=h.lmax, homo=h.homo, lumo=h.lumo) if bounds else {}
    pur.set_hamiltonian(h.F, nocc=h.nocc, mu=0.0, **kw)
    code = pur.run(scheme, tol, max_iter)
    D = pur.density()
    st = pur.stats()
    pur.close()
    return code, D, st


@pytest.mark.parametrize("scheme", O.SCHEMES)
def test_purify_parity_n256(P, scheme):
    # dense F n = 256, nocc = 128, gap 0.1 on [-1, 1], tol 1e-12
    h = I.dense_hamiltonian(256, 128, 0.1, config=1)
    code, D, st = _run(P, h, scheme)
    Do, r = O.purify(h.F, scheme, h.lmin, h.lmax, mu=0.0, homo=h.homo, lumo=h.lumo, tol=1e-12)
    assert code == P.OK
    assert st["iterations"] == r.iterations and st["multiplications"] == r.multiplications
    assert np.max(np.abs(D - Do)) <= 1e-10
    assert abs(st["trace"] - r.traces[-1]) < 1e-9
    assert st["trace_err"] < 1e-9
    if scheme.startswith("TC"):
        assert abs(st["idem_err_fro"] - r.idem[-1]) < 1e-9
    assert np.max(np.abs(D - O.density_closed_form(h.Q, h.lam, 0.0))) < 1e-10


@pytest.mark.parametrize("n,nocc,gap", [(100, 3, 0.3), (333, 200, 0.02), (129, 64, 0.001),
                                        (2, 1, 0.5), (65, 64, 0.1)])
@pytest.mark.parametrize("scheme", ["FIXED_MU_SF", "TC_SF", "TC_MONO"])
def test_purify_parity_ragged(P, n, nocc, gap, scheme):
    h = I.dense_hamiltonian(n, nocc, gap, config=84, instance=n)
    code, D, st = _run(P, h, scheme)
    Do, r = O.purify(h.F, scheme, h.lmin, h.lmax, mu=0.0, homo=h.homo, lumo=h.lumo, tol=1e-12)
    assert code == P.OK and st["iterations"] == r.iterations
    # early rounding is amplified by 1 / (mapped gap); the bound scales with it
    tol = 1e-10 if gap >= 0.01 else 1e-9
    assert np.max(np.abs(D - Do)) <= tol


def test_purify_diagonal_paper_setting(P):
    # the paper's diagonal test Hamiltonians: spectral width 1, mu = 0.5
    lam = I.unit_interval_spectrum(200, 0.5, 0.01)
    h = I.diagonal_hamiltonian(lam, 0.5)
    for scheme in O.SCHEMES:
        pur = P.Purifier()
        pur.set_hamiltonian(h.F, nocc=h.nocc, mu=0.5, lmin=0.0, lmax=1.0, homo=h.homo, lumo=h.lumo)
        pur.run(scheme, 1e-9, 500)
        D = pur.density()
        st = pur.stats()
        Do, r = O.purify(h.F, scheme, 0.0, 1.0, mu=0.5, homo=h.homo, lumo=h.lumo, tol=1e-9)
        assert st["multiplications"] == r.multiplications
        assert np.max(np.abs(D - Do)) < 1e-12
        assert np.max(np.abs(D - np.diag((lam < 0.5).astype(float)))) <= 1e-9


def test_estimated_bounds(P):
    h = I.dense_hamiltonian(400, 150, 0.05, config=85)
    pur = P.Purifier(lanczos_steps=32)
    pur.set_hamiltonian(h.F, nocc=h.nocc, mu=0.0, homo=h.homo, lumo=h.lumo)
    st = pur.stats()
    lo, hi = O.lanczos_bounds(h.F, 32)
    assert abs(st["lmin"] - min(lo, h.homo)) < 1e-9 and abs(st["lmax"] - max(hi, h.lumo)) < 1e-9
    assert st["lmin"] <= h.lmin + 1e-12 and st["lmax"] >= h.lmax - 1e-12
    pur.run("TC_SF", 1e-12)
    D = pur.density()
    Do, _ = O.purify(h.F, "TC_SF", st["lmin"], st["lmax"], homo=h.homo, lumo=h.lumo, tol=1e-12)
    assert np.max(np.abs(D - Do)) < 1e-10
    # Gershgorin only
    pur2 = P.Purifier(lanczos_steps=0)
    pur2.set_hamiltonian(h.F, nocc=h.nocc, mu=0.0, homo=h.homo, lumo=h.lumo)
    g = O.gershgorin(h.F)
    st2 = pur2.stats()
    assert abs(st2["lmin"] - g[0]) < 1e-10 and abs(st2["lmax"] - g[1]) < 1e-10


def test_trace_rule_parity(P):
    h = I.dense_hamiltonian(200, 70, 0.1, config=86)
    pur = P.Purifier(branch_rule="trace")
    pur.set_hamiltonian(h.F, nocc=h.nocc, lmin=h.lmin, lmax=h.lmax)
    pur.run("TC_MONO", 1e-10, 100)
    D = pur.density()
    st = pur.stats()
    Do, r = O.purify_tc(h.F, h.lmin, h.lmax, tol=1e-10, scaled=False, branch_rule="trace",
                        nocc=h.nocc, max_iter=100)
    assert st["iterations"] == r.iterations
    assert np.max(np.abs(D - Do)) < 1e-10


def test_device_pointers_and_strided_host(P):
    h = I.dense_hamiltonian(150, 60, 0.1, config=87)
    pur = P.Purifier()
    Fd = _cuda(h.F)
    pur.set_hamiltonian(Fd, nocc=h.nocc, mu=0.0, lmin=h.lmin, lmax=h.lmax, homo=h.homo, lumo=h.lumo)
    pur.run("TC_SF", 1e-12)
    Dd = torch.empty((150, 150), dtype=torch.float64, device="cuda")
    pur.density(Dd)
    # padded host input (leading dimension > n)
    big = np.zeros((150, 170))
    big[:, :150] = h.F
    pur2 = P.Purifier()
    pur2.set_hamiltonian(big[:, :150], nocc=h.nocc, mu=0.0, lmin=h.lmin, lmax=h.lmax,
                         homo=h.homo, lumo=h.lumo)
    pur2.run("TC_SF", 1e-12)
    Dh = np.zeros((150, 160))
    pur2.density(Dh[:, :150])
    assert np.array_equal(Dd.cpu().numpy(), Dh[:, :150])
    # only the upper triangle is read
    Fu = np.triu(h.F)
    pur2.set_hamiltonian(Fu, nocc=h.nocc, mu=0.0, lmin=h.lmin, lmax=h.lmax, homo=h.homo,
                         lumo=h.lumo)
    pur2.run("TC_SF", 1e-12)
    assert np.array_equal(pur2.density(), Dh[:, :150])


def test_errors(P):
    h = I.dense_hamiltonian(64, 32, 0.1, config=88)
    pur = P.Purifier()
    with pytest.raises(P.PurifyError) as e:
        pur.run("TC_SF")
    assert e.value.code == P.ERR_STATE
    with pytest.raises(P.PurifyError) as e:
        pur.set_hamiltonian(h.F, nocc=32, lmin=-1, lmax=1, homo=0.05, lumo=-0.05)
    assert e.value.code == P.ERR_BOUNDS
    pur.set_hamiltonian(h.F, nocc=32, mu=0.0, lmin=-1, lmax=1, homo=-0.05, lumo=0.05)
    code = pur.run("TC_SF", 1e-12, max_iter=3)
    assert code == P.ERR_NOT_CONVERGED
    st = pur.stats()
    assert st["iterations"] == 3 and st["status"] == P.ERR_NOT_CONVERGED
    assert pur.density().shape == (64, 64)
    # wrong gap bounds: occupied and unoccupied states mixed up -> trace != nocc
    pur.set_hamiltonian(h.F, nocc=32, lmin=-1, lmax=1, homo=0.3, lumo=0.35)
    assert pur.run("TC_SF", 1e-12, check=False) == P.ERR_BOUNDS
    # zero gap is rejected for fixed mu
    pur.set_hamiltonian(h.F, nocc=32, mu=0.05, lmin=-1, lmax=1, homo=-0.05, lumo=0.05)
    assert pur.run("FIXED_MU_SF", 1e-12, check=False) == P.ERR_BOUNDS
    with pytest.raises(P.PurifyError) as e:
        pur.set_hamiltonian(h.F[:0, :0], nocc=0, lmin=-1, lmax=1)
    assert e.value.code == P.ERR_INVALID_ARG


@pytest.mark.parametrize("nocc", [2048, 1024])
def test_purify_fp64_full_size_closed_form(P, nocc):
    # dense F n = 4096, gap 1e-2: compare with D = Q_occ Q_occ^T and check the
    # invariants (the oracle's recursion would take tens of seconds here)
    h = I.dense_hamiltonian(4096, nocc, 1e-2, config=2, instance=nocc)
    code, D, st = _run(P, h, "TC_SF", tol=1e-12)
    assert code == P.OK
    Dc = O.density_closed_form(h.Q, h.lam, 0.0)
    # rounding of F itself (~1e-16 |F| sqrt(n)) is amplified by 1 / gap
    assert np.max(np.abs(D - Dc)) < 1e-10
    assert st["trace_err"] < 1e-8


@pytest.mark.parametrize("scheme,gap", [("FIXED_MU_P33_SF", 1e-2), ("FIXED_MU_P33_MONO", 1e-2),
                                        ("FIXED_MU_P33_SF", 1e-4)])
def test_p33_fixed_mu_parity(P, scheme, gap):
    # the fixed-mu scheme with P_{3,3}: five float64 products per iteration
    h = I.dense_hamiltonian(260, 100, gap, config=88)
    pur = P.Purifier(precision="fp64")
    pur.set_hamiltonian(h.F, nocc=h.nocc, mu=0.0, lmin=h.lmin, lmax=h.lmax, homo=h.homo, lumo=h.lumo)
    pur.run(scheme, 1e-12, 200)
    D, st = pur.density(), pur.stats()
    pur.close()
    Do, r = O.purify_fixed_mu_pmm(h.F, h.lmin, h.lmax, 0.0, h.homo, h.lumo, m=3, tol=1e-12,
                                  scaled=scheme.endswith("_SF"))
    assert st["iterations"] == r.iterations
    assert st["multiplications"] == r.multiplications == 5 * r.iterations
    assert np.max(np.abs(D - Do)) < 1e-10
    assert abs(st["trace"] - h.nocc) < 1e-9


@pytest.mark.parametrize("scheme,ij", [("FIXED_MU_P13_SF", (1, 3)), ("FIXED_MU_P31_SF", (3, 1)),
                                       ("FIXED_MU_P31_MONO", (3, 1))])
def test_asymmetric_pij_parity(P, scheme, ij):
    # scaled about the unstable fixed point c != 1/2; mu placed off-centre
    h = I.dense_hamiltonian(240, 90, 5e-3, config=90)
    pur = P.Purifier(precision="fp64")
    pur.set_hamiltonian(h.F, nocc=h.nocc, mu=0.0, lmin=h.lmin, lmax=h.lmax, homo=h.homo, lumo=h.lumo)
    pur.run(scheme, 1e-12, 200)
    D, st = pur.density(), pur.stats()
    pur.close()
    Do, r = O.purify_fixed_mu_pij(h.F, h.lmin, h.lmax, 0.0, h.homo, h.lumo, *ij, tol=1e-12,
                                  scaled=scheme.endswith("_SF"))
    assert st["iterations"] == r.iterations and st["multiplications"] == r.multiplications
    assert np.max(np.abs(D - Do)) < 1e-10
    assert abs(st["trace"] - h.nocc) < 1e-9
