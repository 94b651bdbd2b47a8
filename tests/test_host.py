"""CPU-side checks of the library: it loads, exports what include/purify.h
declares, and its host logic (the scalar schedule and the tridiagonal
eigensolver used for Lanczos bounds) agrees with the oracle and the paper."""
import os
import re

import numpy as np
import pytest

import paper_1101_0265_gb300 as P
from oracle import purify_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _ensure_built():
    from paper_1101_0265_gb300 import build
    build.build()


def header_symbols():
    out = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            out += re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(purify_\w+)\s*\(", src, re.M)
    return sorted(set(out))


def test_library_exports_every_header_symbol():
    _ensure_built()
    lib = P.load()
    syms = header_symbols()
    assert len(syms) >= 16
    for s in syms:
        assert hasattr(lib, s), s
    # and the binding knows all of them
    assert set(P.EXPORTED) == set(syms)


@pytest.mark.parametrize("field,value", [
    ("digits", 7), ("digits", 1), ("split_k", 2), ("refine_fp64", 3), ("bits_floor", 15),
    ("bits_floor", 44), ("bits_gap", 15), ("bits_gap", 44), ("trunc_tau", -1.0),
    ("trunc_budget", float("nan")), ("precision", 5), ("lanczos_steps", -1), ("autotune", 2),
    ("wait_kcycles", -1), ("wait_kcycles", (1 << 21) + 1), ("host_schedule", 2)])
def test_invalid_options_rejected_before_the_device(field, value):
    # option checks come first: no device is touched, so this runs without a GPU
    import ctypes as C
    _ensure_built()
    lib = P.load()
    o = P._lib.Options()
    lib.purify_options_default(C.byref(o))
    setattr(o, field, value)
    h = C.c_void_p()
    assert lib.purify_create(C.byref(h), 0, None, C.byref(o)) == P.ERR_INVALID_ARG
    assert not h.value
    if field in ("digits", "bits_floor", "bits_gap"):
        b = C.c_void_p()
        assert lib.purify_batch_create(C.byref(b), 0, None, C.byref(o)) == P.ERR_INVALID_ARG


def test_tuned_shape_query_without_measurements():
    # nothing measured in this process: STATE; bad arguments: INVALID_ARG
    _ensure_built()
    assert P.tuned_shape(0, 5, 4096) is None
    with pytest.raises(P.PurifyError):
        P.tuned_shape(0, 9, 4096)


def test_strerror_names_codes():
    _ensure_built()
    for code in (P.OK, P.ERR_INVALID_ARG, P.ERR_BOUNDS, P.ERR_NOT_CONVERGED, P.ERR_OOM,
                 P.ERR_DEVICE_TIMEOUT, P.ERR_STATE, P.ERR_UNSUPPORTED, P.ERR_INTERNAL):
        assert P.strerror(code) and P.strerror(code) != "unknown status"


def _oracle_schedule(scheme, lmin, lmax, mu, homo, lumo, tol, max_iter):
    if scheme.startswith("FIXED_MU_P13") or scheme.startswith("FIXED_MU_P31"):
        i, j = (1, 3) if "P13" in scheme else (3, 1)
        c = O.pij_fixed_point(i, j)
        gamma = max((mu - lmin) / (1.0 - c), (lmax - mu) / c)
        b, bb = c - (lumo - mu) / gamma, c + (mu - homo) / gamma
        _, steps = O.pij_schedule(i, j, b, bb, tol, max_iter, scheme.endswith("_SF"))
        return (np.array([x[0] for x in steps]), np.zeros(len(steps), int),
                np.array([x[1] for x in steps]))
    if scheme.startswith("FIXED_MU_P33"):
        g = O.fixed_mu_gamma(lmin, lmax, mu)
        b = O.fixed_mu_beta0(g, mu, homo, lumo)
        al, be = O.pmm_schedule(3, b, tol, max_iter, scheme == "FIXED_MU_P33_SF")
        return np.array(al), np.zeros(len(al), int), np.array(be)
    if scheme.startswith("FIXED_MU"):
        g = O.fixed_mu_gamma(lmin, lmax, mu)
        b = O.fixed_mu_beta0(g, mu, homo, lumo)
        al, be = O.fixed_mu_schedule(b, tol, max_iter, scheme == "FIXED_MU_SF")
        return np.array(al), np.zeros(len(al), int), np.array(be)
    b, bb = O.tc_beta0(lmin, lmax, homo, lumo)
    s = O.tc_schedule(b, bb, tol, max_iter, scheme == "TC_SF")
    return (np.array([x[1] for x in s]), np.array([1 if x[0] == "P10" else 0 for x in s]),
            np.array([x[2] for x in s]))


CASES = [(-1.0, 1.0, 0.0, -g / 2, g / 2) for g in (1e-1, 1e-2, 1e-3, 1e-4)] + [
    (0.0, 1.0, mu, mu - 0.005, mu + 0.005) for mu in (0.1, 0.25, 0.5, 0.75, 0.9)] + [
    (-3.0, 2.0, -0.4, -0.45, -0.2), (-1.0, 1.0, 0.3, 0.25, 0.31)]


@pytest.mark.parametrize("scheme", O.SCHEMES + ("FIXED_MU_P33_SF", "FIXED_MU_P33_MONO", "FIXED_MU_P13_SF",
                                         "FIXED_MU_P13_MONO", "FIXED_MU_P31_SF", "FIXED_MU_P31_MONO"))
@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("tol", [1e-12, 1e-9, 1e-6])
def test_schedule_bitwise_equal_to_oracle(scheme, case, tol):
    _ensure_built()
    lmin, lmax, mu, homo, lumo = case
    s = P.schedule(scheme, lmin, lmax, mu, homo, lumo, tol, 500)
    al, br, be = _oracle_schedule(scheme, lmin, lmax, mu, homo, lumo, tol, 500)
    assert s["iterations"] == len(al)
    assert s["converged"]
    assert np.array_equal(s["alpha"], al)
    assert np.array_equal(s["branch"], br)
    assert np.array_equal(s["beta"], be)


def test_library_schedule_reproduces_golden_counts():
    # the library's own scalar schedule gives the stored multiplication counts
    # (tests/golden/scalar_counts.txt, from the oracle): Algorithm 1 two
    # products per iteration, Algorithm 2 one
    from test_oracle import golden_counts
    _ensure_built()
    for mu, xi, mm, ms, tm, ts in golden_counts():
        homo, lumo = mu - xi / 2, mu + xi / 2
        got = []
        for scheme, per in (("FIXED_MU_MONO", 2), ("FIXED_MU_SF", 2), ("TC_MONO", 1), ("TC_SF", 1)):
            sch = P.schedule(scheme, 0.0, 1.0, mu if scheme.startswith("FIXED") else float("nan"), homo, lumo,
                             1e-9, max_iter=10_000)
            got.append(per * len(sch["alpha"]))
        assert tuple(got) == (mm, ms, tm, ts), (mu, xi, got)


def test_schedule_not_converged_and_bad_bounds():
    _ensure_built()
    s = P.schedule("TC_SF", -1, 1, 0, -0.05, 0.05, 1e-12, max_iter=3)
    assert s["iterations"] == 3 and not s["converged"]
    with pytest.raises(P.PurifyError) as e:
        P.schedule("TC_SF", -1, 1, 0, 0.05, -0.05, 1e-12)
    assert e.value.code == P.ERR_BOUNDS
    with pytest.raises(P.PurifyError) as e:   # gap does not contain mu
        P.schedule("FIXED_MU_SF", -1, 1, 0.2, -0.05, 0.05, 1e-12)
    assert e.value.code == P.ERR_BOUNDS


@pytest.mark.parametrize("m", [1, 2, 5, 17, 40])
def test_tridiag_eig_against_lapack(m):
    _ensure_built()
    rng = np.random.default_rng(m)
    a = rng.normal(size=m)
    b = rng.uniform(0.1, 1.0, size=max(m - 1, 1))
    T = np.diag(a)
    if m > 1:
        T += np.diag(b[:m - 1], 1) + np.diag(b[:m - 1], -1)
    lam, V = np.linalg.eigh(T)
    w, last = P.tridiag_eig(a, b[:max(m - 1, 1)])
    assert np.max(np.abs(w - lam)) < 1e-12 * max(1.0, np.max(np.abs(lam)))
    assert np.max(np.abs(np.abs(last) - np.abs(V[-1, :]))) < 1e-10


def test_split_plan_invariants():
    # the product kernel's plan: whole waves stay whole, the last wave's tiles
    # are cut into at most 4 k-ranges of at least 4 chunks, never more parts
    # than CTAs (the split buffers' capacity), and the cut happens only when
    # the last wave leaves CTAs idle
    import ctypes as C
    _ensure_built()
    lib = P.load()
    b, w = C.c_int(), C.c_int()
    for ctas in (1, 2, 76, 148, 152):
        for T in range(1, 65):
            tiles = T * (T + 1) // 2
            for k_chunks in (4, 8, 16, 32, 64, 128, 256):
                assert lib.purify_k_split_plan(tiles, ctas, k_chunks, C.byref(b), C.byref(w)) == P.OK
                begin, ways = b.value, w.value
                assert 1 <= ways <= 4
                if ways == 1:
                    assert begin == tiles
                    continue
                assert begin % ctas == 0 and begin == tiles // ctas * ctas
                assert (tiles - begin) * ways <= ctas
                assert k_chunks // ways >= 4
    # n = 4096 on 152 SMs: 528 tiles, 3 whole waves, the last 72 tiles in 2
    assert lib.purify_k_split_plan(528, 152, 128, C.byref(b), C.byref(w)) == P.OK
    assert (b.value, w.value) == (456, 2)
    assert lib.purify_k_split_plan(0, 152, 128, C.byref(b), C.byref(w)) == P.ERR_INVALID_ARG


def test_options_struct_layout_matches_the_library():
    # the binding's Options mirrors purify_options field by field: the
    # library's defaults land in the right fields and nothing past the end of
    # the Python struct is written
    import ctypes as C
    _ensure_built()
    lib = P.load()
    size = C.sizeof(P._lib.Options)
    buf = (C.c_ubyte * (size + 64))(*([0xAB] * (size + 64)))
    lib.purify_options_default(C.cast(buf, C.POINTER(P._lib.Options)))
    assert bytes(buf[size:]) == b"\xab" * 64
    o = P._lib.Options.from_buffer(buf)
    assert o.precision == 0 and o.branch_rule == 0      # PURIFY_FP64, PURIFY_BRANCH_BETA
    assert o.lanczos_steps == 16 and o.refine_squares == 0 and o.digits == 0
    assert o.split_k == 1 and o.refine_fp64 == 0 and o.block_sparse == 0 and o.time_products == 0
    assert o.bits_floor == 0 and o.bits_gap == 0 and o.autotune == 0 and o.wait_kcycles == 0
    assert o.host_schedule == 0 and o.launch_per_product == 0
    assert o.reserved == 0
    assert o.trunc_tau == 1e-6 and o.trunc_budget == 0.0


def _header_struct(name):
    """(field, ctype name, count) of a struct in include/purify.h, in order."""
    src = open(os.path.join(ROOT, "include", "purify.h")).read()
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), src, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    out = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        typ, rest = decl.split(None, 1)
        for part in rest.split(","):
            part = part.strip()
            m = re.match(r"(\w+)(?:\[(\d+)\])?$", part)
            out.append((m.group(1), typ, int(m.group(2) or 1)))
    return out


@pytest.mark.parametrize("cname,pyname", [("purify_options", "Options"), ("purify_stats_t", "Stats"),
                                          ("purify_bounds", "Bounds")])
def test_binding_structs_follow_the_header(cname, pyname):
    import ctypes as C
    ctypes_of = {"int": C.c_int, "double": C.c_double, "int64_t": C.c_int64}
    fields = getattr(P._lib, pyname)._fields_
    hdr = _header_struct(cname)
    assert [f[0] for f in fields] == [h[0] for h in hdr]
    for (name, ct), (_, typ, cnt) in zip(fields, hdr):
        want = ctypes_of[typ] * cnt if cnt > 1 else ctypes_of[typ]
        assert C.sizeof(ct) == C.sizeof(want) and getattr(ct, "_type_", ct) == getattr(want, "_type_", want), name
