"""The fused epilogue's per-step reductions (trace and idempotency norm of
Algorithm 1 / Algorithm 2 steps) against the oracle's, step by step, on both
precisions, read back through purify_step_history."""
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


# Per-element tolerance of the iterates against the oracle's: 1e-12 for the
# float64 path, 5e-8 for the mixed path (its final-density bound at n = 256).
# A trace sums n diagonal elements; a Frobenius norm of an n x n difference
# moves by at most n times the elementwise error.
@pytest.mark.parametrize("precision,elt", [("fp64", 1e-12), ("mixed", 5e-8)])
@pytest.mark.parametrize("scheme", ["TC_SF", "TC_MONO", "FIXED_MU_SF", "FIXED_MU_MONO"])
def test_step_reductions_match_oracle(P, precision, elt, scheme):
    n = 256
    h = I.dense_hamiltonian(n, 100, 0.05, config=80)
    pur = P.Purifier(precision=precision)
    pur.set_hamiltonian(h.F, nocc=h.nocc, mu=0.0, lmin=h.lmin, lmax=h.lmax, homo=h.homo, lumo=h.lumo)
    assert pur.run(scheme, 1e-12, 200) == P.OK
    tr, idem = pur.step_history()
    pur.close()
    _, r = O.purify(h.F, scheme, h.lmin, h.lmax, mu=0.0, homo=h.homo, lumo=h.lumo, tol=1e-12)
    assert len(tr) == r.iterations == len(r.traces)
    np.testing.assert_allclose(tr, r.traces, rtol=0, atol=n * elt)
    if scheme.startswith("TC"):
        assert len(r.idem) == len(idem)
        # early steps: ||X - X^2||_F is O(1) and must agree to the relative
        # level of the iterates; late steps sit at the rounding floor
        np.testing.assert_allclose(idem, r.idem, rtol=1e-6, atol=2 * n * elt)
        assert idem[0] > 1.0          # X_0 is far from idempotent
    else:
        assert np.all(np.isnan(idem))
    # the last trace equals the run's statistic
    assert abs(tr[-1] - h.nocc) < 1e-3


def test_step_reductions_trace_rule(P):
    # Niklasson's branch rule on the mixed path: the per-step traces that
    # chose the branches match the oracle's run with the same rule
    n = 300
    h = I.dense_hamiltonian(n, 140, 0.1, config=81)
    pur = P.Purifier(precision="mixed", branch_rule="trace")
    pur.set_hamiltonian(h.F, nocc=h.nocc, mu=0.0, lmin=h.lmin, lmax=h.lmax, homo=h.homo, lumo=h.lumo)
    assert pur.run("TC_SF", 1e-12, 200) == P.OK
    tr, idem = pur.step_history()
    pur.close()
    _, r = O.purify_tc(h.F, h.lmin, h.lmax, h.homo, h.lumo, tol=1e-12, branch_rule="trace", nocc=h.nocc)
    assert len(tr) == r.iterations
    np.testing.assert_allclose(tr, r.traces, rtol=0, atol=n * 5e-8)
    np.testing.assert_allclose(idem, r.idem, rtol=1e-6, atol=2 * n * 5e-8)


def test_step_history_before_a_run(P):
    pur = P.Purifier(precision="mixed")
    with pytest.raises(P.PurifyError):
        pur.step_history()
    pur.close()
