"""Failure detection on the device without a fault: the product kernel's work
waits are bounded, and a wait that runs out stops the kernel cleanly (it
records the role that gave up, waits for its own copies and MMAs, frees
tensor memory and exits); the call returns PURIFY_ERR_DEVICE_TIMEOUT and the
context stays usable.

The test shortens the work waits (purify_options.wait_kcycles) to a thousand
cycles, far below one tile's MMAs (~300 k cycles at n = 256), so the epilogue's
wait for the first tile's accumulators must give up; nothing else is changed.
The waits for copies and MMAs in flight at teardown keep their full bound, so
every launch still ends by itself.
"""
import numpy as np
import pytest

from oracle import purify_oracle as O
from paper_1101_0265_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EPI_WAIT = 4      # device flag bit: an epilogue warp's wait gave up
PLAN = 8          # device flag bit: internal k-chunk plan check (must stay clear)


@pytest.fixture(scope="module")
def P():
    from paper_1101_0265_gb300 import build
    build.build()
    import paper_1101_0265_gb300 as P
    return P


@pytest.mark.parametrize("scheme", ["TC_SF", "FIXED_MU_SF"])
def test_short_device_waits_time_out_then_recover(P, scheme):
    h = I.dense_hamiltonian(256, 120, 0.05, config=82)
    ref, _ = O.purify(h.F, scheme, h.lmin, h.lmax, mu=0.0, homo=h.homo, lumo=h.lumo, tol=1e-12)
    pur = P.Purifier(precision="mixed", wait_kcycles=1)
    pur.set_hamiltonian(h.F, nocc=h.nocc, mu=0.0, lmin=h.lmin, lmax=h.lmax, homo=h.homo, lumo=h.lumo)
    code = pur.run(scheme, 1e-12, 200, check=False)
    assert code == P.ERR_DEVICE_TIMEOUT, P.strerror(code)
    flag = pur.stats()["device_flag"]
    assert flag & EPI_WAIT and not flag & PLAN, flag
    torch.cuda.synchronize()            # the context is intact
    # the same handle with the default bound: a correct purification
    pur.set_options(wait_kcycles=0)
    assert pur.run(scheme, 1e-12, 200) == P.OK
    assert pur.stats()["device_flag"] == 0
    err = float(np.max(np.abs(pur.density() - ref)))
    pur.close()
    assert err <= 5e-8, err


@pytest.mark.parametrize("rounds", [False, True])
def test_timeout_in_a_batch(P, rounds):
    # the batch engine's launches (one queue launch, whose items also wait on
    # the device for their instance's previous product, or one grouped launch
    # per round) honour the same bound
    hs = [I.dense_hamiltonian(n, n // 2, 0.1, config=83, instance=n) for n in (130, 260)]
    B = P.Batch(wait_kcycles=1)
    ids = [B.add(h.F, h.nocc, h.lmin, h.lmax, h.homo, h.lumo, scheme="TC_SF", tol=1e-10, mu=0.0) for h in hs]
    with pytest.raises(P.PurifyError) as e:
        B.run(use_graph=False, rounds=rounds)
    assert e.value.code == P.ERR_DEVICE_TIMEOUT
    B.close()
    torch.cuda.synchronize()            # the context is intact
    # a fresh batch with the default bound is correct
    B = P.Batch()
    ids = [B.add(h.F, h.nocc, h.lmin, h.lmax, h.homo, h.lumo, scheme="TC_SF", tol=1e-10, mu=0.0) for h in hs]
    B.run(use_graph=False, rounds=rounds)
    for i, h in zip(ids, hs):
        ref, _ = O.purify(h.F, "TC_SF", h.lmin, h.lmax, mu=0.0, homo=h.homo, lumo=h.lumo, tol=1e-10)
        assert np.max(np.abs(B.density(i) - ref)) <= 5e-8
    B.close()


@pytest.mark.parametrize("scheme", ["TC_SF", "FIXED_MU_SF"])
def test_short_waits_in_a_queue_launch_run(P, scheme):
    # n = 3200 runs as queue launches (consecutive products overlapping, items
    # waiting on the device for the row panels they read): with 1000-cycle
    # waits the dependency and hand-off waits give up, the call returns
    # PURIFY_ERR_DEVICE_TIMEOUT, the context stays usable, and the same
    # handle with the default bound matches the closed form
    h = I.dense_hamiltonian(3200, 1500, 0.05, config=84)
    pur = P.Purifier(precision="mixed", wait_kcycles=1)
    pur.set_hamiltonian(h.F, nocc=h.nocc, mu=0.0, lmin=h.lmin, lmax=h.lmax, homo=h.homo, lumo=h.lumo)
    code = pur.run(scheme, 1e-10, 200, check=False)
    assert code == P.ERR_DEVICE_TIMEOUT, P.strerror(code)
    flag = pur.stats()["device_flag"]
    assert flag and not flag & PLAN, flag
    torch.cuda.synchronize()
    pur.set_options(wait_kcycles=0)
    assert pur.run(scheme, 1e-10, 200) == P.OK
    assert pur.stats()["device_flag"] == 0
    err = float(np.max(np.abs(pur.density() - O.density_closed_form(h.Q, h.lam, 0.0))))
    pur.close()
    assert err <= 1e-6, err
