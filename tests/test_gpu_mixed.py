"""GPU tests of the mixed path: digit-plane products on the tcgen05 tensor
cores, and whole purifications against the CPU oracle."""
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


def _sym_int(n, lim, rng):
    A = rng.integers(-lim, lim + 1, size=(n, n)).astype(np.float64)
    return np.triu(A) + np.triu(A, 1).T


@pytest.mark.parametrize("n", [128, 200, 256, 383])
def test_one_digit_products_are_exact(P, n):
    # X = 2^(e-8) d with integer d: one digit, level 0 only; the tensor-core
    # sum of integer products must be exact
    rng = np.random.default_rng(n)
    for e in (0, 1):
        dA = _sym_int(n, 48, rng)
        dB = _sym_int(n, 48, rng)
        A = dA * 2.0 ** (e - 8)
        B = dB * 2.0 ** (e - 8)
        out = torch.empty((n, n), dtype=torch.float64, device="cuda")
        P.k_digit_product_f64(_cuda(A), _cuda(B), out, 1, e, e)
        got = out.cpu().numpy()
        ref = A @ B.T           # upper triangle of A B^T, mirrored
        iu = np.triu_indices(n)
        assert np.array_equal(got[iu], ref[iu])
        assert np.array_equal(got, got.T)


@pytest.mark.parametrize("n", [130, 256])
def test_two_digit_inputs_three_digit_product_exact(P, n):
    # inputs with exactly two digits; with three product digits every nonzero
    # digit pair is kept and every level is exact
    # (leading digit 8 bits, remainder digits 7 bits up to n = 4096)
    rng = np.random.default_rng(7 + n)
    d0 = _sym_int(n, 40, rng)
    d1 = _sym_int(n, 60, rng)
    A = d0 * 2.0 ** -8 + d1 * 2.0 ** -15
    out = torch.empty((n, n), dtype=torch.float64, device="cuda")
    P.k_digit_product_f64(_cuda(A), _cuda(A), out, 3, 0, 0)
    ref = A @ A
    assert np.array_equal(out.cpu().numpy(), ref)


@pytest.mark.parametrize("n,s", [(200, 2), (256, 3), (256, 4), (500, 5), (333, 5), (1024, 6), (129, 6)])
def test_digit_product_accuracy(P, n, s):
    # a density-like operand: X = Q diag(x) Q^T with x in [0, 1]
    h = I.dense_hamiltonian(n, n // 2, 0.1, config=70, instance=n)
    X = (h.lmax * np.eye(n) - h.F) / (h.lmax - h.lmin)
    out = torch.empty((n, n), dtype=torch.float64, device="cuda")
    P.k_digit_product_f64(_cuda(X), _cuda(X), out, s, 0, 0)
    err = np.max(np.abs(out.cpu().numpy() - X @ X))
    # truncation of the digits: s digits carry 8 + 7 (s - 1) bits below 2^0;
    # the kept pairs reproduce the product to about sqrt(n) 2^-bits
    bits = 8 + 7 * (s - 1)
    assert err <= np.sqrt(n) * 2.0 ** (-bits + 3), err


@pytest.mark.parametrize("scheme", O.SCHEMES)
def test_mixed_purify_parity_n256(P, scheme):
    h = I.dense_hamiltonian(256, 128, 0.1, config=1)
    pur = P.Purifier(precision="mixed")
    pur.set_hamiltonian(h.F, nocc=h.nocc, mu=0.0, lmin=h.lmin, lmax=h.lmax, homo=h.homo,
                        lumo=h.lumo)
    code = pur.run(scheme, 1e-12, 200)
    D = pur.density()
    st = pur.stats()
    Do, r = O.purify(h.F, scheme, h.lmin, h.lmax, mu=0.0, homo=h.homo, lumo=h.lumo, tol=1e-12)
    assert code == P.OK
    assert st["iterations"] == r.iterations
    err = np.max(np.abs(D - Do))
    assert err <= 5e-8, err
    assert st["trace_err"] < 1e-6
    assert st["digit_max"] >= 4
    assert st["tensor_flops"] > 0


@pytest.mark.parametrize("n,nocc,gap", [(100, 3, 0.3), (333, 200, 0.02), (129, 64, 0.001),
                                        (65, 64, 0.1), (700, 350, 1e-4)])
@pytest.mark.parametrize("scheme", ["FIXED_MU_SF", "TC_SF", "TC_MONO"])
def test_mixed_purify_parity_ragged(P, n, nocc, gap, scheme):
    h = I.dense_hamiltonian(n, nocc, gap, config=71, instance=n)
    pur = P.Purifier(precision="mixed")
    pur.set_hamiltonian(h.F, nocc=h.nocc, mu=0.0, lmin=h.lmin, lmax=h.lmax, homo=h.homo,
                        lumo=h.lumo)
    assert pur.run(scheme, 1e-12, 300) == P.OK
    D = pur.density()
    Do, r = O.purify(h.F, scheme, h.lmin, h.lmax, mu=0.0, homo=h.homo, lumo=h.lumo, tol=1e-12)
    assert np.max(np.abs(D - Do)) <= 3e-7


def test_mixed_refine_and_fixed_digits(P):
    h = I.dense_hamiltonian(300, 120, 0.05, config=72)
    Do, _ = O.purify(h.F, "TC_SF", h.lmin, h.lmax, homo=h.homo, lumo=h.lumo, tol=1e-12)
    for kw in ({"digits": 6}, {"refine_squares": 1}, {"digits": 5, "refine_squares": 2}):
        pur = P.Purifier(precision="mixed", **kw)
        pur.set_hamiltonian(h.F, nocc=h.nocc, lmin=h.lmin, lmax=h.lmax, homo=h.homo, lumo=h.lumo)
        pur.run("TC_SF", 1e-12)
        st = pur.stats()
        assert st["refine_multiplications"] == 2 * kw.get("refine_squares", 0)
        assert np.max(np.abs(pur.density() - Do)) <= 1e-8
    # too few digits (15 bits) is visibly worse, but still near the right trace
    pur = P.Purifier(precision="mixed", digits=2)
    pur.set_hamiltonian(h.F, nocc=h.nocc, lmin=h.lmin, lmax=h.lmax, homo=h.homo, lumo=h.lumo)
    pur.run("TC_SF", 1e-12)
    assert np.max(np.abs(pur.density() - Do)) > 1e-6
    assert abs(pur.stats()["trace"] - h.nocc) < 0.1


@pytest.mark.parametrize("gap", [1e-2, 1e-4])
def test_mixed_full_size_vs_fp64(P, gap):
    # the workload of the throughput benchmark: n = 4096, max error vs the
    # float64 GPU path at the same schedule must stay below 1e-6
    h = I.dense_hamiltonian(4096, 2048, gap, config=2)
    F = _cuda(h.F)
    out = []
    for precision in ("mixed", "fp64"):
        pur = P.Purifier(precision=precision)
        pur.set_hamiltonian(F, nocc=h.nocc, mu=0.0, lmin=h.lmin, lmax=h.lmax, homo=h.homo,
                            lumo=h.lumo)
        assert pur.run("TC_SF", 1e-9, 200) == P.OK
        D = torch.empty((4096, 4096), dtype=torch.float64, device="cuda")
        pur.density(D)
        out.append(D)
        pur.close()
    err = float((out[0] - out[1]).abs().max())
    assert err <= 1e-6, err


@pytest.mark.parametrize("n,scheme", [(1000, "TC_SF"), (2200, "FIXED_MU_SF"), (4096, "TC_SF")])
def test_split_last_wave_matches_whole_tiles(P, n, scheme):
    # n_pad 1024: 36 tiles < 152 SMs, every tile in 4 k-ranges; n_pad 2304:
    # 171 tiles, the 19 of the second wave in 4; n 4096: 528 tiles, the last
    # 72 in 2.  Levels 0-2 are exact sums, so only the shared inexact level's
    # rounding moves (by ~2^-48 of the leading term per product, then
    # amplified near the gap like any rounding): both results stay within the
    # mixed tolerance of the exact density and the difference is of the size
    # of the path's own rounding error.
    h = I.dense_hamiltonian(n, n // 2, 0.01, config=71, instance=n)
    out = []
    for split in (True, False):
        pur = P.Purifier(precision="mixed", split_k=split)
        pur.set_hamiltonian(h.F, nocc=h.nocc, mu=0.0, lmin=h.lmin, lmax=h.lmax, homo=h.homo, lumo=h.lumo)
        pur.run(scheme, 1e-10, 200)
        out.append((pur.density(), pur.stats()))
        pur.close()
    (Ds, ss), (Dw, sw) = out
    assert ss["iterations"] == sw["iterations"]
    Dx = O.density_closed_form(h.Q, h.lam, 0.0)
    err_s, err_w = np.max(np.abs(Ds - Dx)), np.max(np.abs(Dw - Dx))
    assert err_s <= 3e-7 and err_w <= 3e-7, (err_s, err_w)
    assert np.max(np.abs(Ds - Dw)) <= max(err_s, err_w)
    assert np.array_equal(Ds, Ds.T)
    assert abs(ss["trace"] - h.nocc) < 1e-6
    # the same split is taken on every run: bitwise reproducible
    pur = P.Purifier(precision="mixed")
    pur.set_hamiltonian(h.F, nocc=h.nocc, mu=0.0, lmin=h.lmin, lmax=h.lmax, homo=h.homo, lumo=h.lumo)
    pur.run(scheme, 1e-10, 200)
    assert np.array_equal(pur.density(), Ds)
    pur.close()


@pytest.mark.parametrize("scale", [1e-25, 1e30])
def test_extreme_magnitudes_split_exactly(P, scale):
    # entries below 2^-74 take the split's float64 route, entries near 2^100
    # the top of its integer route; the density of s F with bounds s lambda is
    # that of F
    h = I.dense_hamiltonian(300, 120, 0.05, config=73)
    out = []
    for sc in (1.0, scale):
        pur = P.Purifier(precision="mixed")
        pur.set_hamiltonian(h.F * sc, nocc=h.nocc, mu=0.0, lmin=h.lmin * sc, lmax=h.lmax * sc,
                            homo=h.homo * sc, lumo=h.lumo * sc)
        pur.run("TC_SF", 1e-10, 200)
        out.append(pur.density())
        pur.close()
    assert np.max(np.abs(out[0] - out[1])) < 1e-9
    Dx = O.density_closed_form(h.Q, h.lam, 0.0)
    assert np.max(np.abs(out[1] - Dx)) < 3e-7


def test_fp64_refinement_sets_idempotency(P):
    # mixed run, then 0, 1 or 2 float64 McWeeny steps: the subspace (error
    # against the exact density) is that of the mixed run, the idempotency
    # error falls to float64 rounding
    h = I.dense_hamiltonian(512, 200, 0.01, config=74)
    Dx = O.density_closed_form(h.Q, h.lam, 0.0)
    res = []
    for R in (0, 1, 2):
        pur = P.Purifier(precision="mixed", refine_fp64=R)
        pur.set_hamiltonian(h.F, nocc=h.nocc, mu=0.0, lmin=h.lmin, lmax=h.lmax, homo=h.homo, lumo=h.lumo)
        pur.run("TC_SF", 1e-10, 200)
        D, st = pur.density(), pur.stats()
        pur.close()
        res.append((D, st, np.linalg.norm(D - D @ D)))
    (D0, s0, e0), (D1, s1, e1), (D2, s2, e2) = res
    for D, st, _ in res:
        assert np.max(np.abs(D - Dx)) <= 3e-7
        assert np.array_equal(D, D.T)
    assert s1["refine_multiplications"] == 2 and s2["refine_multiplications"] == 4
    assert s1["multiplications"] == s0["multiplications"] + 2
    assert e1 < 1e-11 < e0 and e2 < 1e-11
    # the reported idempotency error is that of the last refinement's input
    assert abs(s1["idem_err_fro"] - e0) <= 1e-3 * e0
    assert abs(s1["trace"] - h.nocc) < 1e-9


@pytest.mark.parametrize("scheme,gap_known", [("TC_MONO", False), ("TC_SF", True), ("TC_MONO", True)])
@pytest.mark.parametrize("host_schedule", [0, 1])
def test_trace_rule_on_the_mixed_path(P, scheme, gap_known, host_schedule):
    # Niklasson's trace rule: each branch from trace(X_{i-1}) versus nocc,
    # reduced in float64 by the previous product's epilogue; without gap
    # bounds the run stops when ||X - X^2||_F <= tol (reachable at the mixed
    # path's precision: 1e-5).  host_schedule = 0 decides every step on the
    # device and replays the steps from a CUDA graph; 1 takes one host round
    # trip per step.
    h = I.dense_hamiltonian(300, 110, 0.05, config=75)
    tol = 1e-9 if gap_known else 1e-5
    kw = dict(homo=h.homo, lumo=h.lumo) if gap_known else {}
    pur = P.Purifier(precision="mixed", branch_rule="trace")
    pur.set_options(host_schedule=host_schedule)
    pur.set_hamiltonian(h.F, nocc=h.nocc, lmin=h.lmin, lmax=h.lmax, **kw)
    pur.run(scheme, tol, 200)
    D, st = pur.density(), pur.stats()
    tr_hist, _ = pur.step_history()
    # a second run on the same handle replays the same graph
    pur.run(scheme, tol, 200)
    D2 = pur.density()
    pur.close()
    assert np.array_equal(D, D2)
    Do, r = O.purify_tc(h.F, h.lmin, h.lmax, tol=tol, scaled=scheme == "TC_SF", branch_rule="trace",
                        nocc=h.nocc, max_iter=200, **kw)
    assert r.converged
    assert st["iterations"] == r.iterations
    assert st["multiplications"] == r.multiplications
    assert np.max(np.abs(D - Do)) <= 3e-7
    assert abs(st["trace"] - h.nocc) < 1e-6
    np.testing.assert_allclose(tr_hist, r.traces, rtol=0, atol=300 * 5e-8)
    Dx = O.density_closed_form(h.Q, h.lam, 0.0)
    assert np.max(np.abs(D - Dx)) <= 3e-7 + (tol if not gap_known else 0.0)


@pytest.mark.parametrize("n", [256, 1024, 4096])
def test_trace_rule_device_schedule_equals_host_schedule(P, n):
    # the device-side schedule takes the same branches and digit counts as the
    # host one, with the same float64 operations except (1 + alpha)^2 (a
    # product there, the C library's pow here); a last-bit difference in a
    # coefficient moves digit roundings, so the densities agree to the mixed
    # path's own rounding level (~2^-36 per step, amplified near the gap),
    # far inside its 3e-7 tolerance
    h = I.dense_hamiltonian(n, n // 2 - 7, 1e-3, config=76, instance=n)
    out = []
    for host in (1, 0):
        pur = P.Purifier(precision="mixed", branch_rule="trace", host_schedule=host)
        pur.set_hamiltonian(h.F, nocc=h.nocc, mu=0.0, lmin=h.lmin, lmax=h.lmax, homo=h.homo, lumo=h.lumo)
        assert pur.run("TC_SF", 1e-9, 200) == P.OK
        out.append((pur.density(), pur.stats()["iterations"]))
        pur.close()
    assert out[0][1] == out[1][1]
    assert np.max(np.abs(out[0][0] - out[1][0])) <= 1e-9


@pytest.mark.parametrize("n,gap", [(300, 1e-2), (1000, 1e-3)])
def test_p33_fixed_mu_on_digit_planes(P, n, gap):
    # V and Q of P_{3,3} sit up to 7 bits above X_s: per-buffer exponents and
    # one more digit per iteration keep the result at the mixed tolerance
    h = I.dense_hamiltonian(n, n // 2 - 10, gap, config=89)
    pur = P.Purifier(precision="mixed")
    pur.set_hamiltonian(h.F, nocc=h.nocc, mu=0.0, lmin=h.lmin, lmax=h.lmax, homo=h.homo, lumo=h.lumo)
    pur.run("FIXED_MU_P33_SF", 1e-10, 200)
    D, st = pur.density(), pur.stats()
    pur.close()
    Do, r = O.purify_fixed_mu_pmm(h.F, h.lmin, h.lmax, 0.0, h.homo, h.lumo, m=3, tol=1e-10)
    assert st["iterations"] == r.iterations and st["multiplications"] == 5 * r.iterations
    assert np.max(np.abs(D - Do)) <= 3e-7
    assert abs(st["trace"] - h.nocc) < 1e-6


@pytest.mark.parametrize("scheme,ij", [("FIXED_MU_P13_SF", (1, 3)), ("FIXED_MU_P31_SF", (3, 1))])
def test_asymmetric_pij_on_digit_planes(P, scheme, ij):
    h = I.dense_hamiltonian(700, 300, 2e-3, config=91)
    pur = P.Purifier(precision="mixed")
    pur.set_hamiltonian(h.F, nocc=h.nocc, mu=0.0, lmin=h.lmin, lmax=h.lmax, homo=h.homo, lumo=h.lumo)
    pur.run(scheme, 1e-10, 200)
    D, st = pur.density(), pur.stats()
    pur.close()
    Do, r = O.purify_fixed_mu_pij(h.F, h.lmin, h.lmax, 0.0, h.homo, h.lumo, *ij, tol=1e-10)
    assert st["iterations"] == r.iterations and st["multiplications"] == r.multiplications
    assert np.max(np.abs(D - Do)) <= 3e-7
    assert abs(st["trace"] - h.nocc) < 1e-6


def test_autotuned_launch_shapes(P):
    # autotune: the first product of each digit count and size times the
    # candidate launch shapes (split of the last wave or whole tiles); the
    # chosen shape only reorders the inexact level's sums, so the density
    # stays within the mixed tolerance, and a second handle of the process
    # reuses the shapes: the same density bit for bit
    h = I.dense_hamiltonian(1200, 600, 0.01, config=73)
    out = []
    for _ in range(2):
        pur = P.Purifier(precision="mixed", autotune=True)
        pur.set_hamiltonian(h.F, nocc=h.nocc, mu=0.0, lmin=h.lmin, lmax=h.lmax, homo=h.homo, lumo=h.lumo)
        assert pur.run("TC_SF", 1e-10, 200) == P.OK
        out.append((pur.density(), pur.stats()))
        pur.close()
    (D0, s0), (D1, s1) = out
    assert np.array_equal(D0, D1)
    Dx = O.density_closed_form(h.Q, h.lam, 0.0)
    assert np.max(np.abs(D0 - Dx)) <= 3e-7
    assert s0["digit_kc"] == 32
    shape = P.tuned_shape(0, s0["digit_max"], 1200)
    assert shape is not None and shape[0] == 32 and shape[1] in (0, 1)


@pytest.mark.parametrize("scheme,refine", [("TC_SF", 0), ("FIXED_MU_SF", 0), ("TC_MONO", 1)])
def test_run_as_queue_launches_equals_per_product(P, scheme, refine):
    # n = 3200: 325 tiles per product, at least two waves on 152 SMs, so the
    # run goes through queue launches (products overlapping, an item waiting
    # on the device for the row panels it reads); with whole tiles the
    # per-product launches compute the same tiles with the same additions
    h = I.dense_hamiltonian(3200, 1300, 0.01, config=75)
    out = []
    for per_product in (False, True):
        pur = P.Purifier(precision="mixed", launch_per_product=per_product, split_k=False,
                         refine_squares=refine)
        pur.set_hamiltonian(h.F, nocc=h.nocc, mu=0.0, lmin=h.lmin, lmax=h.lmax, homo=h.homo, lumo=h.lumo)
        assert pur.run(scheme, 1e-10, 200) == P.OK
        out.append((pur.density(), pur.stats(), pur.step_history()))
        pur.close()
    (Dq, sq, hq), (Dp, sp, hp) = out
    assert np.array_equal(Dq, Dp)
    assert sq["multiplications"] == sp["multiplications"] and sq["iterations"] == sp["iterations"]
    assert sq["trace"] == pytest.approx(sp["trace"], abs=1e-9)
    assert np.allclose(hq[0], hp[0], rtol=0, atol=1e-9)
    Dx = O.density_closed_form(h.Q, h.lam, 0.0)
    assert np.max(np.abs(Dq - Dx)) <= 1e-6
