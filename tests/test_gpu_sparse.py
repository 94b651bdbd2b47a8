"""GPU tests of the block-sparse mixed path (Algorithm 2 with error-controlled
truncation of 32 x 32 blocks).

- tau = 0 drops only blocks that are exactly zero, and a product skips only
  k-chunks whose contributions are exactly zero: the result equals the dense
  mixed path bit for bit.
- tau > 0: the same iterations as the oracle's truncated recursion, the
  density within the mixed path's tolerance plus what a different drop
  decision at the budget's edge can move, and the distance to the exact
  density within the bound the truncation budget gives.
- The COO entry point gives what the dense entry point gives."""
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


def _lattice(L, instance=0):
    lat = I.lattice_hamiltonian(L, instance=instance)
    F = lat.dense()
    lo, hi = O.gershgorin(F)
    return lat, F, lo, hi


def _run(P, lat, lo, hi, tol, block_sparse, tau=0.0, coo=True, F=None, digits=0):
    # dense runs with whole tiles: block-sparse products are never split
    pur = P.Purifier(precision="mixed", block_sparse=block_sparse, trunc_tau=tau, digits=digits,
                     split_k=False)
    g = lat.gap_bound
    if coo:
        pur.set_hamiltonian_coo(lat.n, lat.rows, lat.cols, lat.vals, nocc=lat.nocc, mu=0.0, lmin=lo,
                                lmax=hi, homo=-g, lumo=g)
    else:
        pur.set_hamiltonian(F, nocc=lat.nocc, mu=0.0, lmin=lo, lmax=hi, homo=-g, lumo=g)
    pur.run("TC_SF", tol, 200)
    D = pur.density()
    st = pur.stats()
    hist = pur.block_history() if block_sparse else None
    pur.close()
    return D, st, hist


@pytest.mark.parametrize("L", [8, 12])
def test_tau_zero_is_the_dense_path(P, L):
    lat, F, lo, hi = _lattice(L)
    tol = 1e-9
    Dd, std, _ = _run(P, lat, lo, hi, tol, block_sparse=False, coo=False, F=F)
    Ds, sts, hist = _run(P, lat, lo, hi, tol, block_sparse=True, tau=0.0)
    assert sts["iterations"] == std["iterations"]
    assert np.array_equal(Ds, Dd), np.max(np.abs(Ds - Dd))
    assert len(hist) == sts["iterations"] + 1
    nb = (lat.n + 31) // 32
    assert hist[0] < nb * (nb + 1) // 2           # X_0 has the lattice's block pattern
    assert sts["nnz_blocks"] == hist[-1]
    # chunk lists skip work: fewer tensor flops than the dense product count
    assert sts["tensor_flops"] < std["tensor_flops"]


def test_coo_input_equals_dense_input(P):
    lat, F, lo, hi = _lattice(8, instance=1)
    D1, st1, h1 = _run(P, lat, lo, hi, 1e-9, block_sparse=True, tau=1e-6, coo=True)
    D2, st2, h2 = _run(P, lat, lo, hi, 1e-9, block_sparse=True, tau=1e-6, coo=False, F=F)
    assert np.array_equal(D1, D2)
    assert h1 == h2
    # bounds estimated on the device from the COO input equal those from the dense input
    pur = P.Purifier(precision="mixed")
    pur.set_hamiltonian_coo(lat.n, lat.rows, lat.cols, lat.vals, nocc=lat.nocc)
    a = pur.stats()
    pur.set_hamiltonian(F, nocc=lat.nocc)
    b = pur.stats()
    pur.close()
    # (the Lanczos reductions run in a fixed order: the estimate is reproducible)
    for k in ("lmin", "lmax", "homo", "lumo", "mu"):
        assert a[k] == b[k] or (np.isnan(a[k]) and np.isnan(b[k])), (k, a[k], b[k])


@pytest.mark.parametrize("L,tau", [(8, 1e-6), (8, 1e-4), (12, 1e-6), (12, 1e-5), (16, 1e-6)])
def test_truncated_vs_oracle(P, L, tau):
    lat, F, lo, hi = _lattice(L)
    g = lat.gap_bound
    tol = 1e-9
    Xo, r, hist_o = O.purify_tc_truncated(F, lo, hi, -g, g, tau, tol=tol)
    D, st, hist = _run(P, lat, lo, hi, tol, block_sparse=True, tau=tau)
    assert st["iterations"] == r.iterations
    assert hist[0] == hist_o[0]
    # The kept-block counts decide which blocks exist; the norms behind them
    # are computed in fp32 on the GPU and in float64 here, so a block at the
    # budget's edge may go either way.  With the same counts at every step the
    # two recursions drop the same blocks (the order is by norm), and D must
    # agree to the mixed path's own rounding (measured <= 1.3e-9 at n = 4096).
    # Otherwise each differing decision moves X by at most tau in the
    # Frobenius norm, amplified at most by 1 / (mapped gap).
    diff = np.max(np.abs(D - Xo))
    mapped_gap = 2 * g / (hi - lo)
    if hist == hist_o:
        assert diff <= 1e-8, diff
    else:
        assert diff <= 3e-7 + 2 * tau / mapped_gap, diff
        assert all(abs(a - b) <= max(4, 0.02 * b) for a, b in zip(hist, hist_o)), (hist, hist_o)
    Dx = O.density_by_eigh(F, 0.0)
    assert np.linalg.norm(D - Dx, 2) <= 3e-7 + (r.iterations + 1) * tau / mapped_gap
    assert abs(st["trace"] - lat.nocc) <= 1e-6 * lat.n + (r.iterations + 1) * tau * np.sqrt(lat.n)


def test_dense_input_through_block_sparse(P):
    # no zero blocks: every chunk list is "all chunks" and tau = 0 drops
    # nothing: the dense path's result
    h = I.dense_hamiltonian(300, 120, 0.02, config=70)
    out = []
    for bs in (False, True):
        pur = P.Purifier(precision="mixed", block_sparse=bs, trunc_tau=0.0, split_k=False)
        pur.set_hamiltonian(h.F, nocc=h.nocc, mu=0.0, lmin=h.lmin, lmax=h.lmax, homo=h.homo, lumo=h.lumo)
        pur.run("TC_SF", 1e-10, 200)
        out.append((pur.density(), pur.stats()))
        if bs:
            assert pur.block_history()[-1] == 10 * 11 // 2
        pur.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1]["iterations"] == out[1][1]["iterations"]


def test_block_sparse_unsupported_combinations(P):
    lat, F, lo, hi = _lattice(8)
    pur = P.Purifier(precision="fp64", block_sparse=True)
    pur.set_hamiltonian_coo(lat.n, lat.rows, lat.cols, lat.vals, nocc=lat.nocc)
    with pytest.raises(P.PurifyError):
        pur.run("TC_SF", 1e-9, 200)
    pur.close()
    pur = P.Purifier(precision="mixed", block_sparse=True)
    pur.set_hamiltonian_coo(lat.n, lat.rows, lat.cols, lat.vals, nocc=lat.nocc)
    with pytest.raises(P.PurifyError):
        pur.run("FIXED_MU_SF", 1e-9, 200)
    pur.close()
    with pytest.raises(P.PurifyError):
        P.Purifier(precision="mixed", block_sparse=True, trunc_tau=-1.0)


def test_coo_rejects_bad_indices(P):
    pur = P.Purifier(precision="mixed")
    with pytest.raises(P.PurifyError):
        pur.set_hamiltonian_coo(4, [0, 4], [0, 1], [1.0, 2.0], nocc=2)
    with pytest.raises(P.PurifyError):
        pur.set_hamiltonian_coo(4, [0, 1], [0, -1], [1.0, 2.0], nocc=2)
    with pytest.raises(P.PurifyError):                       # not symmetric
        pur.set_hamiltonian_coo(4, [0, 1], [1, 2], [1.0, 2.0], nocc=2)
    pur.close()


def test_full_size_lattice_invariants(P):
    # the 32^3 lattice (n = 32768) at tau = 1e-6: no oracle run at this size;
    # invariants of D on sampled columns, the trace, and the dense mixed path
    lat = I.lattice_hamiltonian(32)
    n, g = lat.n, lat.gap_bound
    rows = torch.from_numpy(lat.rows).cuda()
    cols = torch.from_numpy(lat.cols).cuda()
    vals = torch.from_numpy(lat.vals).cuda()
    js = torch.from_numpy(np.random.default_rng(5).integers(0, n, 8)).cuda()
    E = torch.zeros((n, 8), dtype=torch.float64, device="cuda")
    E[js, torch.arange(8, device="cuda")] = 1.0
    Ds = {}
    for bs in (True, False):
        pur = P.Purifier(precision="mixed", block_sparse=bs, trunc_tau=1e-6)
        pur.set_hamiltonian_coo(n, lat.rows, lat.cols, lat.vals, nocc=lat.nocc, mu=0.0, homo=-g, lumo=g)
        pur.run("TC_SF", 1e-9, 200)
        st = pur.stats()
        D = torch.empty((n, n), dtype=torch.float64, device="cuda")
        pur.density(D)
        if bs:
            hist = pur.block_history()
            assert len(hist) == st["iterations"] + 1 and hist[0] < hist[-1]
            # the pools hold at most every block of both iterates (12 KB each)
            nb = n // 32
            assert 0 < st["plane_pool_mib"] <= -(-2 * (nb * nb + 1) * 12288 // 2**20)
        else:
            assert st["plane_pool_mib"] == 0
        pur.close()
        assert abs(st["trace"] - lat.nocc) < 1e-4
        DE = D @ E
        assert (D @ DE - DE).abs().max().item() < 1e-6                  # idempotent
        # F applied to D's sampled columns and to the unit vectors, from COO
        FDE = torch.zeros((n, 8), dtype=torch.float64, device="cuda").index_add_(0, rows, vals[:, None] * DE[cols])
        FE = torch.zeros((n, 8), dtype=torch.float64, device="cuda").index_add_(0, rows, vals[:, None] * E[cols])
        assert (FDE - D @ FE).abs().max().item() < 1e-6                  # commutes with F
        assert torch.equal(D[:, js], D[js, :].T)                          # symmetric
        Ds[bs] = DE
        del D
        torch.cuda.empty_cache()
    # truncation at tau = 1e-6 per step moves the sampled columns little
    assert (Ds[True] - Ds[False]).abs().max().item() < 1e-6


@pytest.mark.parametrize("L,scheme", [(8, "TC_SF"), (8, "TC_MONO"), (12, "TC_SF")])
def test_truncation_budget_vs_oracle(P, L, scheme):
    # a total truncation budget: tau = budget / (m + 1) on both sides
    lat, F, lo, hi = _lattice(L)
    g = lat.gap_bound
    eps = 1e-4
    Xo, r, hist_o = O.purify_tc_truncated(F, lo, hi, -g, g, None, tol=1e-9, scaled=scheme == "TC_SF",
                                          tau_budget=eps)
    pur = P.Purifier(precision="mixed", block_sparse=True, trunc_budget=eps, split_k=False)
    pur.set_hamiltonian_coo(lat.n, lat.rows, lat.cols, lat.vals, nocc=lat.nocc, mu=0.0, lmin=lo, lmax=hi,
                            homo=-g, lumo=g)
    pur.run(scheme, 1e-9, 200)
    D, st, hist = pur.density(), pur.stats(), pur.block_history()
    pur.close()
    assert st["iterations"] == r.iterations
    assert hist[0] == hist_o[0]
    diff = np.max(np.abs(D - Xo))
    if hist == hist_o:
        assert diff <= 1e-8, diff
    else:
        assert diff <= 3e-7 + 2 * r.tau * (hi - lo) / (2 * g), diff


def test_density_blocks_expand_to_the_density(P):
    # the kept blocks of a block-sparse run, read as a block list, are the
    # nonzero blocks of the dense density (host and device outputs agree)
    lat, F, lo, hi = _lattice(12)
    g = lat.gap_bound
    pur = P.Purifier(precision="mixed", block_sparse=True, trunc_tau=1e-6)
    pur.set_hamiltonian_coo(lat.n, lat.rows, lat.cols, lat.vals, nocc=lat.nocc, mu=0.0, homo=-g, lumo=g)
    pur.run("TC_SF", 1e-9, 200)
    st = pur.stats()
    D = pur.density()
    Dd = torch.empty((lat.n, lat.n), dtype=torch.float64, device="cuda")
    pur.density(Dd)
    ij, vals = pur.density_blocks()
    assert pur.density_device_ptr() == 0
    pur.close()
    assert np.array_equal(Dd.cpu().numpy(), D)
    assert len(ij) == st["nnz_blocks"] and np.all(ij[:, 0] <= ij[:, 1])
    assert np.array_equal(ij, ij[np.lexsort((ij[:, 1], ij[:, 0]))])  # row-major order
    n, nb = lat.n, (lat.n + 127) // 128 * 4
    Dp = np.zeros((nb * 32, nb * 32))
    for (I_, J_), v in zip(ij, vals):
        Dp[32 * I_:32 * I_ + 32, 32 * J_:32 * J_ + 32] = v
        Dp[32 * J_:32 * J_ + 32, 32 * I_:32 * I_ + 32] = v.T
    assert np.array_equal(Dp[:n, :n], D)
    assert not Dp[n:, :].any() and not Dp[:, n:].any()
    assert abs(np.trace(D) - lat.nocc) < 1e-6


def test_csr_form_bounds_and_dense_paths(P):
    # a block-sparse handle keeps F as CSR: its estimated bounds agree with
    # the dense estimate to rounding, and a dense path asked for afterwards
    # (options changed to the dense mixed path) gets F from the CSR copy and
    # the same result as a handle loaded densely
    lat, F, lo, hi = _lattice(8, instance=2)
    g = lat.gap_bound
    a = P.Purifier(precision="mixed", block_sparse=True)
    a.set_hamiltonian_coo(lat.n, lat.rows, lat.cols, lat.vals, nocc=lat.nocc, mu=0.0, homo=-g, lumo=g)
    b = P.Purifier(precision="mixed")
    b.set_hamiltonian(F, nocc=lat.nocc, mu=0.0, homo=-g, lumo=g)
    sa, sb = a.stats(), b.stats()
    for k in ("lmin", "lmax"):
        assert abs(sa[k] - sb[k]) <= 1e-12 * (abs(sb[k]) + 1.0), (k, sa[k], sb[k])
    # the same bounds on both handles, then the dense mixed path on each
    for h in (a, b):
        h.set_options(block_sparse=False)
    a.set_hamiltonian_coo(lat.n, lat.rows, lat.cols, lat.vals, nocc=lat.nocc, mu=0.0, lmin=lo, lmax=hi,
                          homo=-g, lumo=g)
    b.set_hamiltonian(F, nocc=lat.nocc, mu=0.0, lmin=lo, lmax=hi, homo=-g, lumo=g)
    for h in (a, b):
        h.run("TC_SF", 1e-9, 200)
    assert np.array_equal(a.density(), b.density())
    # CSR form kept, dense path requested later: the same again
    c = P.Purifier(precision="mixed", block_sparse=True)
    c.set_hamiltonian_coo(lat.n, lat.rows, lat.cols, lat.vals, nocc=lat.nocc, mu=0.0, lmin=lo, lmax=hi,
                          homo=-g, lumo=g)
    c.set_options(block_sparse=False)
    c.run("TC_SF", 1e-9, 200)
    assert np.array_equal(c.density(), b.density())
    for h in (a, b, c):
        h.close()


def test_block_sparse_density_refuses_fp64_refinement(P):
    lat, F, lo, hi = _lattice(8)
    g = lat.gap_bound
    pur = P.Purifier(precision="mixed", block_sparse=True, refine_fp64=1)
    pur.set_hamiltonian_coo(lat.n, lat.rows, lat.cols, lat.vals, nocc=lat.nocc, mu=0.0, homo=-g, lumo=g)
    with pytest.raises(P.PurifyError):
        pur.run("TC_SF", 1e-9, 200)
    pur.close()


def _chain(n, seed):
    # a dimerised chain: onsite +-1.5 alternating, first-neighbour hopping
    # -1 + U(-0.1, 0.1), second-neighbour U(-0.05, 0.05); banded, with a gap
    # about 3 wide at mid spectrum
    rng = np.random.default_rng(seed)
    F = np.diag(np.where(np.arange(n) % 2 == 0, 1.5, -1.5))
    t1 = -1.0 + rng.uniform(-0.1, 0.1, n - 1)
    t2 = rng.uniform(-0.05, 0.05, n - 2)
    F += np.diag(t1, 1) + np.diag(t1, -1) + np.diag(t2, 2) + np.diag(t2, -2)
    return F


@pytest.mark.parametrize("kind", ["dense", "chain"])
def test_csr_form_at_a_ragged_size_equals_the_dense_path(P, kind):
    # n = 300 (not a multiple of 32): the CSR form's split (partial strips,
    # rows read from CSR) and the pooled density at tau = 0 give the dense
    # mixed path bit for bit; the banded chain has whole zero blocks, so its
    # products skip chunks
    n, nocc = 300, 150
    F = I.dense_hamiltonian(n, nocc, 0.05, config=71).F if kind == "dense" else _chain(n, 72)
    lam = np.linalg.eigvalsh(F)
    lo, hi, ho, lu = lam[0], lam[-1], lam[nocc - 1], lam[nocc]
    assert lu - ho > 1e-2
    rows, cols = np.nonzero(F)
    vals = F[rows, cols]
    out = {}
    for bs in (False, True):
        pur = P.Purifier(precision="mixed", block_sparse=bs, trunc_tau=0.0, split_k=False)
        if bs:
            pur.set_hamiltonian_coo(n, rows, cols, vals, nocc=nocc, mu=0.0, lmin=lo, lmax=hi, homo=ho, lumo=lu)
        else:
            pur.set_hamiltonian(F, nocc=nocc, mu=0.0, lmin=lo, lmax=hi, homo=ho, lumo=lu)
        pur.run("TC_SF", 1e-10, 200)
        out[bs] = (pur.density(), pur.stats())
        if bs:
            ij, vals_b = pur.density_blocks()
            assert len(ij) == out[bs][1]["nnz_blocks"]
        pur.close()
    assert np.array_equal(out[True][0], out[False][0])
    assert out[True][1]["iterations"] == out[False][1]["iterations"]
    if kind == "chain":
        assert out[True][1]["tensor_flops"] < out[False][1]["tensor_flops"]


def test_pooled_density_host_and_device_outputs_agree(P):
    # 24^3 at onsite +-6.0 (n = 13824): a host density goes through several
    # staging panels, and more kept blocks than one host staging pass holds;
    # host and device outputs of both readers are the same bits
    lat = I.lattice_hamiltonian(24, onsite=6.0)
    g = lat.gap_bound
    pur = P.Purifier(precision="mixed", block_sparse=True, trunc_tau=1e-6)
    pur.set_hamiltonian_coo(lat.n, lat.rows, lat.cols, lat.vals, nocc=lat.nocc, mu=0.0, homo=-g, lumo=g)
    pur.run("TC_SF", 1e-9, 300)
    st = pur.stats()
    n = lat.n
    assert n * n * 8 > 2 * (256 << 20)                  # at least three staging panels
    Dh = pur.density()
    Dd = torch.empty((n, n), dtype=torch.float64, device="cuda")
    pur.density(Dd)
    assert np.array_equal(Dh, Dd.cpu().numpy())
    del Dd
    ij_h, v_h = pur.density_blocks()
    ij_d, v_d = pur.density_blocks(device=True)
    pur.close()
    assert len(ij_h) == st["nnz_blocks"] > (256 << 20) // 8192  # more than one staging pass
    assert np.array_equal(ij_h, ij_d.cpu().numpy())
    assert np.array_equal(v_h, v_d.cpu().numpy())
    # the blocks are D's: spot-check a few against the dense output
    for k in np.random.default_rng(3).integers(0, len(ij_h), 16):
        I_, J_ = ij_h[k]
        assert np.array_equal(v_h[k], Dh[32 * I_:32 * I_ + 32, 32 * J_:32 * J_ + 32])
    torch.cuda.empty_cache()
