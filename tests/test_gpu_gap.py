"""GPU tests of the gap-edge estimate (trace-rule steps, filtered Lanczos on
each side, inverse maps): against the oracle's same procedure, against the
exact spectrum (the estimates must lie inside the gap), and as the gap
bounds of a following purification."""
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


CASES = [(300, 120, 0.05, 1), (500, 250, 0.01, 2), (400, 100, 2e-3, 3), (1000, 400, 1e-3, 6)]


@pytest.mark.parametrize("n,nocc,gap,cfg", CASES)
def test_fp64_estimate_matches_oracle_and_is_inner(P, n, nocc, gap, cfg):
    h = I.dense_hamiltonian(n, nocc, gap, config=cfg)
    w = h.lmax - h.lmin
    ho, lo, _ = O.estimate_gap(h.F, h.lmin, h.lmax, h.nocc)
    pur = P.Purifier(precision="fp64")
    pur.set_hamiltonian(h.F, nocc=h.nocc, lmin=h.lmin, lmax=h.lmax)
    he, le = pur.estimate_gap(40)
    assert h.homo <= he < le <= h.lumo
    assert abs(he - ho) <= 1e-11 * w and abs(le - lo) <= 1e-11 * w
    st = pur.stats()
    assert st["homo"] == he and st["lumo"] == le
    pur.close()


@pytest.mark.parametrize("n,nocc,gap,cfg", CASES + [(2048, 1024, 1e-2, 7)])
def test_mixed_estimate_then_purify(P, n, nocc, gap, cfg):
    # the estimate is inside the gap and tight; the purification that uses it
    # takes the iterations of the exact gap and reaches the exact density
    h = I.dense_hamiltonian(n, nocc, gap, config=cfg)
    w = h.lmax - h.lmin
    pur = P.Purifier(precision="mixed")
    pur.set_hamiltonian(h.F, nocc=h.nocc, lmin=h.lmin, lmax=h.lmax)
    he, le = pur.estimate_gap(40)
    assert h.homo <= he < le <= h.lumo
    assert he - h.homo <= 1e-6 * w and h.lumo - le <= 1e-6 * w
    pur.run("TC_SF", 1e-9, 200)
    D, st = pur.density(), pur.stats()
    pur.close()
    _, r = O.purify(h.F, "TC_SF", h.lmin, h.lmax, homo=h.homo, lumo=h.lumo, tol=1e-9)
    assert st["iterations"] == r.iterations
    assert np.max(np.abs(D - O.density_closed_form(h.Q, h.lam, 0.0))) <= 3e-7


@pytest.mark.parametrize("precision,tight", [("fp64", 1e-9), ("mixed", 1e-4)])
def test_lattice_estimate(P, precision, tight):
    lat = I.lattice_hamiltonian(8)
    F = lat.dense()
    ev = np.linalg.eigvalsh(F)
    glo, ghi = O.gershgorin(F)
    pur = P.Purifier(precision=precision)
    pur.set_hamiltonian_coo(lat.n, lat.rows, lat.cols, lat.vals, nocc=lat.nocc, lmin=glo, lmax=ghi)
    he, le = pur.estimate_gap(40)
    pur.close()
    assert ev[lat.nocc - 1] <= he < le <= ev[lat.nocc]
    assert he - ev[lat.nocc - 1] <= tight and ev[lat.nocc] - le <= tight


def test_estimate_errors(P):
    h = I.dense_hamiltonian(100, 40, 0.1, config=8)
    pur = P.Purifier(precision="mixed")
    with pytest.raises(P.PurifyError):
        pur.estimate_gap(40)                      # no Hamiltonian yet
    pur.set_hamiltonian(h.F, lmin=h.lmin, lmax=h.lmax)
    with pytest.raises(P.PurifyError):
        pur.estimate_gap(40)                      # nocc unknown
    pur.set_hamiltonian(h.F, nocc=h.nocc, lmin=h.lmin, lmax=h.lmax)
    with pytest.raises(P.PurifyError):
        pur.estimate_gap(2)                       # too few Lanczos steps
    he, le = pur.estimate_gap(40)
    with pytest.raises(P.PurifyError):
        pur.density()                             # no density after an estimate
    pur.close()
