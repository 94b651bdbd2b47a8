"""GPU tests of the batch engine: many purifications of uneven size in one
queue launch or in grouped tensor-core launches per round (with and without
a CUDA graph), and continuous batching.  Every
result must equal the same purification run alone, bit for bit, and the
CPU oracle to the mixed path's tolerance."""
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


SPECS = [  # n, nocc, gap, scheme
    (64, 20, 0.05, "TC_SF"), (100, 61, 0.002, "FIXED_MU_SF"), (129, 64, 0.01, "TC_SF"),
    (200, 77, 0.1, "TC_MONO"), (256, 128, 1e-3, "TC_SF"), (300, 150, 0.02, "FIXED_MU_SF"),
    (383, 200, 0.05, "FIXED_MU_MONO"), (511, 300, 0.004, "TC_SF"), (640, 320, 0.03, "TC_SF"),
    (77, 30, 0.2, "FIXED_MU_SF"),
]


def _hams():
    return [I.dense_hamiltonian(n, nocc, gap, config=60, instance=i) for i, (n, nocc, gap, _) in
            enumerate(SPECS)]


def _alone(P, h, scheme, tol):
    # whole tiles, as in the batch's grouped launches (a split of the last
    # wave changes the order of the inexact level's additions)
    pur = P.Purifier(precision="mixed", split_k=False)
    pur.set_hamiltonian(h.F, nocc=h.nocc, mu=0.0, lmin=h.lmin, lmax=h.lmax, homo=h.homo, lumo=h.lumo)
    pur.run(scheme, tol, 300)
    D = pur.density()
    st = pur.stats()
    pur.close()
    return D, st


@pytest.mark.parametrize("use_graph,rounds", [(True, False), (False, False), (True, True), (False, True)])
def test_batch_equals_alone_and_oracle(P, use_graph, rounds):
    # rounds=False: one queue launch, each instance advancing on its own;
    # rounds=True: one grouped launch per round
    hs = _hams()
    tol = 1e-10
    B = P.Batch()
    ids = [B.add(h.F, h.nocc, h.lmin, h.lmax, h.homo, h.lumo, scheme=sp[3], tol=tol, mu=0.0)
           for h, sp in zip(hs, SPECS)]
    for rep in range(2):  # the second run replays the captured graph
        B.run(use_graph=use_graph, rounds=rounds)
        for i, h, sp in zip(ids, hs, SPECS):
            assert B.done(i)
            D = B.density(i)
            Da, sta = _alone(P, h, sp[3], tol)
            assert np.array_equal(D, Da), (sp, np.max(np.abs(D - Da)))
            st = B.stats(i)
            assert st["iterations"] == sta["iterations"]
            assert st["multiplications"] == sta["multiplications"]
            assert abs(st["trace"] - h.nocc) < 1e-6
            if rep == 0:
                Do, r = O.purify(h.F, sp[3], h.lmin, h.lmax, mu=0.0, homo=h.homo, lumo=h.lumo,
                                 tol=tol)
                assert st["iterations"] == r.iterations
                assert np.max(np.abs(D - Do)) <= 3e-7
    B.close()


def test_continuous_batching_equals_alone(P):
    # requests arrive while others are running: admit two, step, admit three
    # more, step ... ; results are those of each request alone
    hs = _hams()
    tol = 1e-9
    B = P.Batch()
    pending = list(range(len(hs)))
    live = {}
    rounds = 0
    while pending or live:
        for _ in range(min(2 + rounds % 2, len(pending))):
            k = pending.pop(0)
            h = hs[k]
            live[k] = B.add(h.F, h.nocc, h.lmin, h.lmax, h.homo, h.lumo, scheme=SPECS[k][3], tol=tol,
                            mu=0.0)
        active, finished = B.step()
        rounds += 1
        for k, i in list(live.items()):
            if B.done(i):
                D = B.density(i)
                Da, _ = _alone(P, hs[k], SPECS[k][3], tol)
                assert np.array_equal(D, Da), SPECS[k]
                before = B.bytes_in_use()
                B.release(i)
                assert B.bytes_in_use() < before
                del live[k]
        assert rounds < 500
    assert B.bytes_in_use() == 0
    B.close()


@pytest.mark.parametrize("k", [1, 3])
def test_continuous_batching_with_queue_advance_equals_alone(P, k):
    # requests arrive while others run; every call advances each active one
    # by up to k products in one queue launch; results are those alone
    hs = _hams()
    tol = 1e-9
    B = P.Batch()
    pending = list(range(len(hs)))
    live = {}
    calls = 0
    while pending or live:
        for _ in range(min(3, len(pending))):
            j = pending.pop(0)
            h = hs[j]
            live[j] = B.add(h.F, h.nocc, h.lmin, h.lmax, h.homo, h.lumo, scheme=SPECS[j][3], tol=tol, mu=0.0)
        active, finished = B.advance(k)
        calls += 1
        for j, i in list(live.items()):
            if B.done(i):
                Da, _ = _alone(P, hs[j], SPECS[j][3], tol)
                assert np.array_equal(B.density(i), Da), SPECS[j]
                B.release(i)
                del live[j]
        assert calls < 500
    assert B.bytes_in_use() == 0
    B.close()


def test_batch_device_inputs_and_footprint(P):
    h = I.dense_hamiltonian(300, 100, 0.05, config=61)
    B = P.Batch()
    Fd = torch.from_numpy(h.F).cuda()
    i = B.add(Fd, h.nocc, h.lmin, h.lmax, h.homo, h.lumo, scheme="TC_SF", tol=1e-9)
    assert 0 < B.bytes_in_use() <= P.batch_footprint(300)
    B.run()
    Dd = torch.empty((300, 300), dtype=torch.float64, device="cuda")
    B.density(i, Dd)
    Da, _ = _alone(P, h, "TC_SF", 1e-9)
    assert np.array_equal(Dd.cpu().numpy(), Da)
    with pytest.raises(P.PurifyError):
        B.add(h.F, h.nocc, h.lmin, h.lmax, h.lumo, h.homo)       # homo > lumo
    B.close()


def test_queue_many_products_per_cta(P):
    # more instances and products than CTAs can hold claims for at once: the
    # claim ring wraps many times; mixed digit counts in one launch (the
    # small-gap instances need more digit planes than the wide-gap ones)
    specs = [(96 + 32 * (k % 7), 40 + k, 10 ** (-1 - (k % 3)), "TC_SF" if k % 2 else "FIXED_MU_SF")
             for k in range(24)]
    hs = [I.dense_hamiltonian(n, nocc, gap, config=64, instance=k) for k, (n, nocc, gap, _) in enumerate(specs)]
    B = P.Batch()
    ids = [B.add(h.F, h.nocc, h.lmin, h.lmax, h.homo, h.lumo, scheme=sp[3], tol=1e-10, mu=0.0)
           for h, sp in zip(hs, specs)]
    B.run(use_graph=True)
    digits = set()
    alone = {}
    for k, (i, h, sp) in enumerate(zip(ids, hs, specs)):
        D = B.density(i)
        alone[k] = _alone(P, h, sp[3], 1e-10)[0]
        assert np.array_equal(D, alone[k]), sp
        digits.add(B.stats(i)["digit_max"])
    assert len(digits) > 1, digits
    # a changed set of instances is staged again into the same device buffer
    # (the tensor maps change under the same addresses): still exact
    for i in ids[::2]:
        B.release(i)
    keep = {k: i for k, i in enumerate(ids) if k % 2}
    for use_graph in (False, True):
        B.run(use_graph=use_graph)
        for k, i in keep.items():
            assert np.array_equal(B.density(i), alone[k]), (use_graph, specs[k])
    B.close()


def test_queue_equals_rounds_on_a_mixed_batch(P):
    # 96 instances of the batch workload (n log-uniform in [64, 2048], gaps
    # log-uniform in [1e-3, 1e-1]): products of 5 and 6 digits share the
    # queue launch and its CTAs, so an epilogue warp can be on an item of one
    # digit count while another warp of the CTA is on the other; every
    # density must still equal the per-round engine's, bit for bit
    dev = torch.device("cuda:0")
    specs = I.batch_specs(96)
    B = P.Batch()
    ids = []
    for sp in specs:
        F, h = I.dense_hamiltonian_device(sp, dev)
        ids.append(B.add(F, h.nocc, h.lmin, h.lmax, h.homo, h.lumo, scheme="TC_SF", tol=1e-9, mu=0.0))
        del F
    B.run(use_graph=False, rounds=True)
    ref = [B.density(i) for i in ids]
    digits = {B.stats(i)["digit_max"] for i in ids}
    assert len(digits) > 1, digits
    for use_graph in (False, True, True):
        B.run(use_graph=use_graph, rounds=False)
        bad = [k for k, i in enumerate(ids) if not np.array_equal(B.density(i), ref[k])]
        assert not bad, (use_graph, bad[:8])
    B.close()
