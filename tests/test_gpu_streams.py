"""Stream ordering at the C ABI: a handle works on its own stream but is
joined to the caller's stream, so device inputs still being produced on the
caller's stream are read only once complete, and the caller's stream waits
for the results."""
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


def _late_input(F_host):
    """A device copy of F that only completes after a long device-side delay
    queued on torch's current stream."""
    Fd = torch.zeros(F_host.shape, dtype=torch.float64, device="cuda")
    src = torch.from_numpy(F_host).pin_memory()
    torch.cuda._sleep(200_000_000)          # ~0.1 s of device time first
    Fd.copy_(src, non_blocking=True)
    return Fd


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_handle_waits_for_callers_stream(P, precision):
    h = I.dense_hamiltonian(300, 120, 0.05, config=62)
    Do, _ = O.purify(h.F, "TC_SF", h.lmin, h.lmax, homo=h.homo, lumo=h.lumo, tol=1e-12)
    pur = P.Purifier(precision=precision)                 # joined to torch's current stream
    pur.set_hamiltonian(_late_input(h.F), nocc=h.nocc, lmin=h.lmin, lmax=h.lmax, homo=h.homo,
                        lumo=h.lumo)
    pur.run("TC_SF", 1e-12)
    Dd = torch.empty((300, 300), dtype=torch.float64, device="cuda")
    pur.density(Dd)
    Dd.mul_(1.0)                                          # a torch op after the library's write
    assert np.max(np.abs(Dd.cpu().numpy() - Do)) <= (1e-10 if precision == "fp64" else 1e-7)


def test_batch_waits_for_callers_stream(P):
    h = I.dense_hamiltonian(257, 100, 0.05, config=63)
    Do, _ = O.purify(h.F, "TC_SF", h.lmin, h.lmax, homo=h.homo, lumo=h.lumo, tol=1e-10)
    B = P.Batch()
    i = B.add(_late_input(h.F), h.nocc, h.lmin, h.lmax, h.homo, h.lumo, scheme="TC_SF", tol=1e-10)
    B.run(use_graph=True)
    assert np.max(np.abs(B.density(i) - Do)) <= 1e-7
    B.close()


def test_host_input_is_read_before_the_call_returns(P):
    # a pinned host F may be overwritten as soon as set_hamiltonian / batch
    # add return
    from paper_1101_0265_gb300 import inputs as I
    from oracle import purify_oracle as O
    h = I.dense_hamiltonian(2048, 1000, 0.05, config=76)
    Dx = O.density_closed_form(h.Q, h.lam, 0.0)
    F = torch.from_numpy(h.F.copy()).pin_memory()
    pur = P.Purifier(precision="mixed")
    pur.set_hamiltonian(F, nocc=h.nocc, mu=0.0, lmin=h.lmin, lmax=h.lmax, homo=h.homo, lumo=h.lumo)
    F.fill_(float("nan"))
    pur.run("TC_SF", 1e-9, 200)
    assert np.max(np.abs(pur.density() - Dx)) < 3e-7
    pur.close()
    F.copy_(torch.from_numpy(h.F))
    B = P.Batch()
    i = B.add(F, h.nocc, h.lmin, h.lmax, h.homo, h.lumo, scheme="TC_SF", tol=1e-9, mu=0.0)
    F.fill_(float("nan"))
    B.run()
    assert np.max(np.abs(B.density(i) - Dx)) < 3e-7
    B.close()


@pytest.mark.parametrize("n,scheme", [(1000, "TC_SF"), (2200, "FIXED_MU_SF"), (4096, "TC_SF")])
def test_concurrent_handles_equal_solo_runs(P, n, scheme):
    # Two handles on their own streams, driven from two host threads, run
    # split products at the same time, so a launch's CTAs need not all be
    # resident and the split parts go to whichever CTAs claim them: the
    # densities must still equal solo runs bit for bit (split parts are added
    # in part order, whoever computes them).
    import threading
    hs = [I.dense_hamiltonian(n, n // 2, 0.01, config=72, instance=k) for k in range(2)]

    def run(h, stream=None):
        pur = P.Purifier(precision="mixed", stream=stream)
        pur.set_hamiltonian(h.F, nocc=h.nocc, mu=0.0, lmin=h.lmin, lmax=h.lmax, homo=h.homo, lumo=h.lumo)
        assert pur.run(scheme, 1e-10, 200) == P.OK
        D = pur.density()
        pur.close()
        return D

    solo = [run(h) for h in hs]
    streams = [torch.cuda.Stream() for _ in hs]
    got = [None, None]
    errs = []

    def worker(k):
        try:
            for _ in range(3):
                got[k] = run(hs[k], streams[k].cuda_stream)
                assert np.array_equal(got[k], solo[k])
        except Exception as e:  # reported after the join
            errs.append(e)
    ths = [threading.Thread(target=worker, args=(k,)) for k in range(2)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    assert not errs, errs
