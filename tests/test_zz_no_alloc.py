"""The allocation-free Gershgorin entry point (static device scratch) gives
the same interval as the allocating one.

Some callers cannot allocate device memory: hosts whose device memory is all
handed to their own pool allocator, callers with a fully committed memory
budget, and loops that cannot absorb cudaFree's device synchronisation.  This
file is named so that pytest collects it last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    from paper_1101_0265_gb300 import build
    build.build()
    import paper_1101_0265_gb300 as P
    return P


def _sym(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    return torch.from_numpy(np.ascontiguousarray(0.5 * (A + A.T))).cuda()


def test_noalloc_gershgorin_matches_allocating_entry_point(P):
    # two calls in a row, different sizes: the shared static scratch still
    # holds the first call's partials when the second call runs
    for n, seed in ((1000, 1), (777, 2), (4096, 3)):
        F = _sym(n, seed)
        ref = torch.zeros(2, dtype=torch.float64, device="cuda")
        got = torch.zeros(2, dtype=torch.float64, device="cuda")
        P.k_gershgorin_f64(F, ref)
        assert P.k_gershgorin_f64_noalloc(F, got) == P.OK
        torch.cuda.synchronize()
        scale = float(F.abs().sum(dim=1).max())
        assert torch.allclose(got, ref, rtol=0.0, atol=1e-13 * scale), (n, got, ref)


def test_noalloc_gershgorin_rejects_oversize(P):
    F = _sym(8, 4)
    lohi = torch.full((2,), 7.0, dtype=torch.float64, device="cuda")
    code = P.k_gershgorin_f64_noalloc(F, lohi, n=P.GERSHGORIN_NOALLOC_MAX_N + 1, check=False)
    assert code == P.ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert torch.all(lohi == 7.0)        # nothing was launched


def test_noalloc_calls_queued_back_to_back_on_one_stream(P):
    # two sizes queued on one stream with no synchronisation in between: the
    # second call's kernels overwrite the shared scratch only after the first
    # call's kernels have read it (stream order), so both intervals are right
    F1, F2 = _sym(4096, 5), _sym(777, 6)
    got1 = torch.zeros(2, dtype=torch.float64, device="cuda")
    got2 = torch.zeros(2, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    assert P.k_gershgorin_f64_noalloc(F1, got1) == P.OK
    assert P.k_gershgorin_f64_noalloc(F2, got2) == P.OK
    assert P.k_gershgorin_f64_noalloc(F1, got1) == P.OK    # and the larger size again
    torch.cuda.synchronize()
    for F, got in ((F1, got1), (F2, got2)):
        ref = torch.zeros(2, dtype=torch.float64, device="cuda")
        P.k_gershgorin_f64(F, ref)
        torch.cuda.synchronize()
        scale = float(F.abs().sum(dim=1).max())
        assert torch.allclose(got, ref, rtol=0.0, atol=1e-13 * scale), (F.shape[0], got, ref)
