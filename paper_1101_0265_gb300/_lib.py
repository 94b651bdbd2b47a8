"""ctypes binding of libpurify's C ABI (include/purify.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Loading fails loudly if ``libpurify.so`` has not been built; there
is no fallback of any kind.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpurify.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_BOUNDS = -2
ERR_NOT_CONVERGED = -3
ERR_OOM = -4
ERR_CUDA = -5
ERR_DEVICE_TIMEOUT = -6
ERR_STATE = -7
ERR_UNSUPPORTED = -8
ERR_INTERNAL = -9

SCHEMES = {"FIXED_MU_SF": 0, "FIXED_MU_MONO": 1, "TC_SF": 2, "TC_MONO": 3, "FIXED_MU_P33_SF": 4,
           "FIXED_MU_P33_MONO": 5, "FIXED_MU_P13_SF": 6, "FIXED_MU_P13_MONO": 7, "FIXED_MU_P31_SF": 8,
           "FIXED_MU_P31_MONO": 9}
PRECISIONS = {"fp64": 0, "mixed": 1}
BRANCH_RULES = {"beta": 0, "trace": 1}

EXPORTED = (
    "purify_options_default", "purify_create", "purify_destroy", "purify_set_options",
    "purify_set_hamiltonian", "purify_set_hamiltonian_coo", "purify_block_history", "purify_get_density_blocks",
    "purify_estimate_gap",
    "purify_tuned_shape", "purify_k_split_plan",
    "purify_run", "purify_get_density", "purify_stats", "purify_step_history",
    "purify_density_device_ptr", "purify_strerror", "purify_schedule", "purify_tridiag_eig",
    "purify_k_symm_product_f64", "purify_k_step_f64", "purify_k_gershgorin_f64",
    "purify_k_lanczos_f64", "purify_k_digit_product_f64", "purify_k_gershgorin_f64_noalloc",
    "purify_batch_footprint", "purify_batch_create", "purify_batch_destroy", "purify_batch_add",
    "purify_batch_step", "purify_batch_advance", "purify_batch_run", "purify_batch_status", "purify_batch_get_density",
    "purify_batch_stats", "purify_batch_release", "purify_batch_bytes_in_use",
)


class Bounds(C.Structure):
    _fields_ = [("lmin", C.c_double), ("lmax", C.c_double), ("homo", C.c_double),
                ("lumo", C.c_double)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("branch_rule", C.c_int), ("lanczos_steps", C.c_int),
                ("refine_squares", C.c_int), ("digits", C.c_int), ("time_products", C.c_int),
                ("block_sparse", C.c_int), ("split_k", C.c_int), ("refine_fp64", C.c_int),
                ("bits_floor", C.c_int), ("bits_gap", C.c_int), ("autotune", C.c_int),
                ("wait_kcycles", C.c_int), ("host_schedule", C.c_int), ("launch_per_product", C.c_int),
                ("reserved", C.c_int),
                ("trunc_tau", C.c_double), ("trunc_budget", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("multiplications", C.c_int),
                ("refine_multiplications", C.c_int), ("err_bound", C.c_double),
                ("trace", C.c_double), ("trace_err", C.c_double), ("idem_err_fro", C.c_double),
                ("seconds", C.c_double), ("lmin", C.c_double), ("lmax", C.c_double),
                ("homo", C.c_double), ("lumo", C.c_double), ("mu", C.c_double),
                ("useful_flops", C.c_double), ("tensor_flops", C.c_double),
                ("digit_max", C.c_int), ("kernel_launches", C.c_int),
                ("product_launches", C.c_int), ("nnz_blocks", C.c_int), ("digit_kc", C.c_int),
                ("device_flag", C.c_int), ("plane_pool_mib", C.c_int), ("reserved", C.c_int),
                ("product_seconds", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class PurifyError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})" if what else f"{strerror(code)} ({code})")


_lib = None


def load(path: str = LIB_PATH):
    """Load libpurify.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1101_0265_gb300.build.build()")
    lib = C.CDLL(path)
    vp, i64, dbl, ip = C.c_void_p, C.c_int64, C.c_double, C.c_int
    dp = C.POINTER(C.c_double)
    sig = {
        "purify_options_default": (None, [C.POINTER(Options)]),
        "purify_create": (ip, [C.POINTER(vp), ip, vp, C.POINTER(Options)]),
        "purify_destroy": (ip, [vp]),
        "purify_set_options": (ip, [vp, C.POINTER(Options)]),
        "purify_set_hamiltonian": (ip, [vp, vp, i64, i64, i64, dbl, C.POINTER(Bounds)]),
        "purify_run": (ip, [vp, ip, dbl, ip]),
        "purify_set_hamiltonian_coo": (ip, [vp, i64, i64, vp, vp, vp, i64, dbl, C.POINTER(Bounds)]),
        "purify_block_history": (ip, [vp, C.POINTER(C.c_int), ip, C.POINTER(C.c_int)]),
        "purify_get_density_blocks": (ip, [vp, vp, vp, i64, C.POINTER(C.c_int64)]),
        "purify_tuned_shape": (ip, [ip, ip, i64, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "purify_k_split_plan": (ip, [ip, ip, ip, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "purify_estimate_gap": (ip, [vp, ip, dp, dp]),
        "purify_get_density": (ip, [vp, vp, i64]),
        "purify_stats": (ip, [vp, C.POINTER(Stats)]),
        "purify_step_history": (ip, [vp, dp, dp, ip, C.POINTER(C.c_int)]),
        "purify_density_device_ptr": (vp, [vp]),
        "purify_strerror": (C.c_char_p, [ip]),
        "purify_schedule": (ip, [ip, dbl, dbl, dbl, dbl, dbl, dbl, ip, dp, C.POINTER(C.c_int), dp,
                                 dp, C.POINTER(C.c_int)]),
        "purify_tridiag_eig": (ip, [dp, dp, ip, dp, dp]),
        "purify_k_symm_product_f64": (ip, [vp, vp, vp, i64, vp]),
        "purify_k_step_f64": (ip, [vp, vp, vp, vp, i64, dbl, dbl, dbl, dbl, dbl, vp, vp]),
        "purify_k_gershgorin_f64": (ip, [vp, i64, i64, vp, vp]),
        "purify_k_lanczos_f64": (ip, [vp, i64, ip, dp, dp, vp]),
        "purify_k_digit_product_f64": (ip, [vp, vp, vp, i64, ip, ip, ip, vp]),
        "purify_k_gershgorin_f64_noalloc": (ip, [vp, i64, i64, vp, vp]),
        "purify_batch_footprint": (i64, [i64]),
        "purify_batch_create": (ip, [C.POINTER(vp), ip, vp, C.POINTER(Options)]),
        "purify_batch_destroy": (ip, [vp]),
        "purify_batch_add": (ip, [vp, vp, i64, i64, i64, dbl, C.POINTER(Bounds), ip, dbl, ip,
                                  C.POINTER(C.c_int)]),
        "purify_batch_step": (ip, [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "purify_batch_advance": (ip, [vp, ip, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "purify_batch_run": (ip, [vp, ip]),
        "purify_batch_status": (ip, [vp, ip]),
        "purify_batch_get_density": (ip, [vp, ip, vp, i64]),
        "purify_batch_stats": (ip, [vp, ip, C.POINTER(Stats)]),
        "purify_batch_release": (ip, [vp, ip]),
        "purify_batch_bytes_in_use": (i64, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load().purify_strerror(code).decode()


def _check(code: int, what: str, allow=()):
    if code != OK and code not in allow:
        raise PurifyError(code, what)
    return code


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ptr(x) -> int:
    """Address of a numpy array or a torch tensor (host or device)."""
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return int(x.data_ptr())


def _stream_of(x=None) -> int | None:
    """torch's current stream on the current device (0 = legacy default)."""
    import torch
    return torch.cuda.current_stream().cuda_stream


def _caller_stream(stream):
    """The stream a handle is joined to: the given one, else torch's current
    stream when torch has CUDA, else the legacy default stream (None)."""
    if stream is not None:
        return int(stream) or None
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream or None
    except Exception:
        pass
    return None


def _nan(v):
    return float("nan") if v is None else float(v)


# ---------------------------------------------------------------------------
# Handle
# ---------------------------------------------------------------------------

class Purifier:
    """One libpurify handle on one device."""

    def __init__(self, device: int = 0, stream: int | None = None, precision: str = "fp64",
                 branch_rule: str = "beta", lanczos_steps: int = 16, refine_squares: int = 0,
                 digits: int = 0, time_products: bool = False, block_sparse: bool = False,
                 trunc_tau: float = 1e-6, split_k: bool = True, refine_fp64: int = 0,
                 trunc_budget: float = 0.0, bits_floor: int = 0, bits_gap: int = 0,
                 autotune: bool = False, wait_kcycles: int = 0, host_schedule: bool = False,
                 launch_per_product: bool = False):
        lib = load()
        self._lib = lib
        self.options = Options()
        lib.purify_options_default(C.byref(self.options))
        self.options.precision = PRECISIONS[precision]
        self.options.branch_rule = BRANCH_RULES[branch_rule]
        self.options.lanczos_steps = lanczos_steps
        self.options.refine_squares = refine_squares
        self.options.digits = digits
        self.options.time_products = int(time_products)
        self.options.block_sparse = int(block_sparse)
        self.options.split_k = int(split_k)
        self.options.refine_fp64 = int(refine_fp64)
        self.options.trunc_tau = float(trunc_tau)
        self.options.trunc_budget = float(trunc_budget)
        self.options.bits_floor = int(bits_floor)
        self.options.bits_gap = int(bits_gap)
        self.options.autotune = int(autotune)
        self.options.wait_kcycles = int(wait_kcycles)
        self.options.host_schedule = int(host_schedule)
        self.options.launch_per_product = int(launch_per_product)
        h = C.c_void_p()
        _check(lib.purify_create(C.byref(h), device, _caller_stream(stream), C.byref(self.options)),
               "purify_create")
        self._h = h
        self.n = 0
        self.device = int(device)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.purify_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_options(self, **kw):
        for k, v in kw.items():
            if k == "precision":
                v = PRECISIONS[v]
            elif k == "branch_rule":
                v = BRANCH_RULES[v]
            setattr(self.options, k, v)
        _check(self._lib.purify_set_options(self._h, C.byref(self.options)), "purify_set_options")

    def set_hamiltonian(self, F, nocc: int = -1, mu=None, lmin=None, lmax=None, homo=None,
                        lumo=None, ld: int | None = None):
        """F: (n, n) float64 numpy array or torch tensor (host or device)."""
        n = int(F.shape[0])
        if ld is None:
            ld = int(F.strides[0] // 8) if isinstance(F, np.ndarray) else int(F.stride(0))
        b = Bounds(_nan(lmin), _nan(lmax), _nan(homo), _nan(lumo))
        code = self._lib.purify_set_hamiltonian(self._h, _ptr(F), n, ld, int(nocc), _nan(mu),
                                                C.byref(b))
        _check(code, "purify_set_hamiltonian")
        self.n = n
        return code

    def set_hamiltonian_coo(self, n: int, rows, cols, vals, nocc: int = -1, mu=None, lmin=None,
                            lmax=None, homo=None, lumo=None):
        """Sparse symmetric F as COO triplets (host int64 / float64 arrays,
        both triangles, duplicates summed)."""
        r = np.ascontiguousarray(rows, dtype=np.int64)
        c = np.ascontiguousarray(cols, dtype=np.int64)
        v = np.ascontiguousarray(vals, dtype=np.float64)
        b = Bounds(_nan(lmin), _nan(lmax), _nan(homo), _nan(lumo))
        code = self._lib.purify_set_hamiltonian_coo(self._h, int(n), int(v.size), r.ctypes.data,
                                                    c.ctypes.data, v.ctypes.data, int(nocc), _nan(mu),
                                                    C.byref(b))
        _check(code, "purify_set_hamiltonian_coo")
        self.n = int(n)
        return code

    def estimate_gap(self, lanczos_steps: int = 40):
        """Inner estimates (homo, lumo) of the gap edges; they become the
        handle's gap bounds."""
        ho, lu = C.c_double(0.0), C.c_double(0.0)
        _check(self._lib.purify_estimate_gap(self._h, int(lanczos_steps), C.byref(ho), C.byref(lu)),
               "purify_estimate_gap")
        return ho.value, lu.value

    def block_history(self):
        cnt = C.c_int(0)
        _check(self._lib.purify_block_history(self._h, None, 0, C.byref(cnt)), "purify_block_history")
        buf = (C.c_int * max(cnt.value, 1))()
        _check(self._lib.purify_block_history(self._h, buf, cnt.value, C.byref(cnt)),
               "purify_block_history")
        return list(buf[:cnt.value])

    def run(self, scheme: str, tol: float = 1e-12, max_iter: int = 200, check: bool = True) -> int:
        code = self._lib.purify_run(self._h, SCHEMES[scheme], float(tol), int(max_iter))
        if check:
            _check(code, "purify_run", allow=(ERR_NOT_CONVERGED,))
        return code

    def density(self, out=None):
        """The density as a new host float64 array, or into `out` (numpy or
        torch, host or device, row-major with unit column stride)."""
        if out is None:
            out = np.empty((self.n, self.n), dtype=np.float64)
        ld = int(out.strides[0] // 8) if isinstance(out, np.ndarray) else int(out.stride(0))
        _check(self._lib.purify_get_density(self._h, _ptr(out), ld), "purify_get_density")
        return out

    def density_blocks(self, values: bool = True, device: bool = False):
        """The kept 32 x 32 blocks of a block-sparse run's density: an
        (m, 2) int32 array of (I, J), I <= J, and an (m, 32, 32) float64
        array of the blocks (None when values is False); numpy arrays, or
        torch tensors on the handle's device when `device`."""
        cnt = C.c_int64(0)
        _check(self._lib.purify_get_density_blocks(self._h, None, None, 0, C.byref(cnt)),
               "purify_get_density_blocks")
        m = cnt.value
        if device:
            import torch
            dev = torch.device("cuda", self.device)
            ij = torch.empty((max(m, 1), 2), dtype=torch.int32, device=dev)
            vals = torch.empty((max(m, 1), 32, 32), dtype=torch.float64, device=dev) if values else None
        else:
            ij = np.empty((max(m, 1), 2), dtype=np.int32)
            vals = np.empty((max(m, 1), 32, 32), dtype=np.float64) if values else None
        _check(self._lib.purify_get_density_blocks(self._h, _ptr(ij), _ptr(vals) if values else None, m,
                                                    C.byref(cnt)), "purify_get_density_blocks")
        return ij[:m], (vals[:m] if values else None)

    def density_device_ptr(self) -> int:
        return self._lib.purify_density_device_ptr(self._h) or 0

    def stats(self) -> dict:
        s = Stats()
        _check(self._lib.purify_stats(self._h, C.byref(s)), "purify_stats")
        return s.as_dict()

    def step_history(self):
        """Per-iteration reductions of the last run: (trace(X_i), ||X_{i-1} -
        X_{i-1}^2||_F) as two float64 arrays (the second NaN for fixed-mu)."""
        cnt = C.c_int(0)
        _check(self._lib.purify_step_history(self._h, None, None, 0, C.byref(cnt)), "purify_step_history")
        m = cnt.value
        tr = np.zeros(max(m, 1))
        idem = np.zeros(max(m, 1))
        _check(self._lib.purify_step_history(self._h, _dptr(tr), _dptr(idem), m, C.byref(cnt)),
               "purify_step_history")
        return tr[:m], idem[:m]


# ---------------------------------------------------------------------------
# Host-only entry points
# ---------------------------------------------------------------------------

def tuned_shape(device: int, digits: int, n: int):
    """The launch shape autotuning measured for products of `digits` digit
    planes at size n on `device` in this process: (kc, split_ways), or None."""
    lib = load()
    kc, ways = C.c_int(0), C.c_int(0)
    code = lib.purify_tuned_shape(int(device), int(digits), int(n), C.byref(kc), C.byref(ways))
    if code == ERR_STATE:
        return None
    _check(code, "purify_tuned_shape")
    return kc.value, ways.value


def schedule(scheme: str, lmin, lmax, mu, homo, lumo, tol, max_iter=500):
    lib = load()
    alpha = np.zeros(max_iter)
    beta = np.zeros(max_iter)
    betabar = np.zeros(max_iter)
    branch = (C.c_int * max(max_iter, 1))()
    it = C.c_int(0)
    code = lib.purify_schedule(SCHEMES[scheme], float(lmin), float(lmax), _nan(mu), float(homo),
                               float(lumo), float(tol), int(max_iter), _dptr(alpha), branch,
                               _dptr(beta), _dptr(betabar), C.byref(it))
    _check(code, "purify_schedule", allow=(ERR_NOT_CONVERGED,))
    m = it.value
    return {"alpha": alpha[:m].copy(), "branch": np.array(branch[:m], dtype=int),
            "beta": beta[:m].copy(), "betabar": betabar[:m].copy(), "iterations": m,
            "converged": code == OK}


def tridiag_eig(a, b):
    lib = load()
    a = np.ascontiguousarray(a, dtype=np.float64)
    m = a.size
    b = np.ascontiguousarray(b if m > 1 else np.zeros(1), dtype=np.float64)
    w = np.zeros(m)
    last = np.zeros(m)
    _check(lib.purify_tridiag_eig(_dptr(a), _dptr(b), m, _dptr(w), _dptr(last)), "tridiag_eig")
    return w, last


# ---------------------------------------------------------------------------
# Kernel-level entry points (torch CUDA tensors, current stream)
# ---------------------------------------------------------------------------

def _dev_f64(t, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
            and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")


def k_symm_product_f64(A, B, out):
    _dev_f64(A, "A"), _dev_f64(B, "B"), _dev_f64(out, "out")
    _check(load().purify_k_symm_product_f64(_ptr(A), _ptr(B), _ptr(out), int(A.shape[0]),
                                            _stream_of()), "k_symm_product_f64")
    return out


def k_step_f64(A, B, E, out, cP, cE, cI, dY=1.0, dI=0.0, red=None):
    for t, nm in ((A, "A"), (B, "B"), (out, "out")):
        _dev_f64(t, nm)
    if E is not None:
        _dev_f64(E, "E")
    _check(load().purify_k_step_f64(_ptr(A), _ptr(B), _ptr(E) if E is not None else None,
                                    _ptr(out), int(A.shape[0]), cP, cE, cI, dY, dI,
                                    _ptr(red) if red is not None else None, _stream_of()),
           "k_step_f64")
    return out


def k_gershgorin_f64(F, lohi):
    _dev_f64(lohi, "lohi")
    _check(load().purify_k_gershgorin_f64(_ptr(F), int(F.shape[0]), int(F.stride(0)), _ptr(lohi),
                                          _stream_of()), "k_gershgorin_f64")
    return lohi


def k_lanczos_f64(F, k: int):
    _dev_f64(F, "F")
    a = np.zeros(k)
    b = np.zeros(k)
    _check(load().purify_k_lanczos_f64(_ptr(F), int(F.shape[0]), int(k), _dptr(a), _dptr(b),
                                       _stream_of()), "k_lanczos_f64")
    return a, b


def k_digit_product_f64(A, B, out, digits: int, eA: int = 0, eB: int = 0):
    """out = A B through the digit-plane tensor-core product (see purify.h)."""
    for t, nm in ((A, "A"), (B, "B"), (out, "out")):
        _dev_f64(t, nm)
    _check(load().purify_k_digit_product_f64(_ptr(A), _ptr(B), _ptr(out), int(A.shape[0]),
                                             int(digits), int(eA), int(eB), _stream_of()),
           "k_digit_product_f64")
    return out


GERSHGORIN_NOALLOC_MAX_N = 65536


def k_gershgorin_f64_noalloc(F, lohi, n=None, check=True):
    """Gershgorin interval through the allocation-free entry point (static
    device scratch; see purify.h).  Returns the status code."""
    _dev_f64(lohi, "lohi")
    n = int(F.shape[0]) if n is None else int(n)
    code = load().purify_k_gershgorin_f64_noalloc(_ptr(F), n, max(n, int(F.stride(0))), _ptr(lohi),
                                                  _stream_of())
    if check:
        _check(code, "k_gershgorin_f64_noalloc")
    return code


# ---------------------------------------------------------------------------
# Batch (many Hamiltonians, grouped launches) and continuous batching
# ---------------------------------------------------------------------------

def batch_footprint(n: int) -> int:
    return int(load().purify_batch_footprint(int(n)))


class Batch:
    """A libpurify batch: many purifications of uneven size on one device."""

    def __init__(self, device: int = 0, stream: int | None = None, digits: int = 0, wait_kcycles: int = 0):
        lib = load()
        self._lib = lib
        o = Options()
        lib.purify_options_default(C.byref(o))
        o.digits = digits
        o.wait_kcycles = int(wait_kcycles)
        h = C.c_void_p()
        _check(lib.purify_batch_create(C.byref(h), device, _caller_stream(stream), C.byref(o)),
               "purify_batch_create")
        self._h = h
        self.sizes = {}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.purify_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, F, nocc, lmin, lmax, homo, lumo, scheme="TC_SF", tol=1e-9, max_iter=200, mu=None,
            ld=None) -> int:
        n = int(F.shape[0])
        if ld is None:
            ld = int(F.strides[0] // 8) if isinstance(F, np.ndarray) else int(F.stride(0))
        b = Bounds(float(lmin), float(lmax), float(homo), float(lumo))
        i = C.c_int(-1)
        _check(self._lib.purify_batch_add(self._h, _ptr(F), n, ld, int(nocc), _nan(mu), C.byref(b),
                                          SCHEMES[scheme], float(tol), int(max_iter), C.byref(i)),
               "purify_batch_add")
        self.sizes[i.value] = n
        return i.value

    def step(self):
        a, f = C.c_int(0), C.c_int(0)
        _check(self._lib.purify_batch_step(self._h, C.byref(a), C.byref(f)), "purify_batch_step")
        return a.value, f.value

    def advance(self, max_products: int = 4):
        """Advance every active instance by up to max_products products in one
        queue launch; returns (active, finished) like step()."""
        a, f = C.c_int(0), C.c_int(0)
        _check(self._lib.purify_batch_advance(self._h, int(max_products), C.byref(a), C.byref(f)),
               "purify_batch_advance")
        return a.value, f.value

    def run(self, use_graph: bool = True, rounds: bool = False):
        """Run every instance to completion: one queue launch in which each
        instance advances on its own (rounds=False), or one grouped launch
        per round (rounds=True); captured in a CUDA graph with use_graph."""
        mode = (1 if use_graph else 0) | (2 if rounds else 0)
        _check(self._lib.purify_batch_run(self._h, mode), "purify_batch_run")

    def done(self, i: int) -> bool:
        r = self._lib.purify_batch_status(self._h, int(i))
        if r < 0:
            raise PurifyError(r, "purify_batch_status")
        return r == 1

    def density(self, i: int, out=None):
        n = self.sizes[i]
        if out is None:
            out = np.empty((n, n), dtype=np.float64)
        ld = int(out.strides[0] // 8) if isinstance(out, np.ndarray) else int(out.stride(0))
        _check(self._lib.purify_batch_get_density(self._h, int(i), _ptr(out), ld),
               "purify_batch_get_density")
        return out

    def stats(self, i: int) -> dict:
        s = Stats()
        _check(self._lib.purify_batch_stats(self._h, int(i), C.byref(s)), "purify_batch_stats")
        return s.as_dict()

    def release(self, i: int):
        _check(self._lib.purify_batch_release(self._h, int(i)), "purify_batch_release")
        self.sizes.pop(i, None)

    def bytes_in_use(self) -> int:
        return int(self._lib.purify_batch_bytes_in_use(self._h))
