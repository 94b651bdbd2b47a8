"""Plain FP64 CPU oracle for recursive polynomial purification with the
non-monotonic scale-and-fold schemes of E. H. Rubensson, "Non-monotonic
recursive polynomial expansions for linear scaling calculation of the density
matrix" (arXiv:1101.0265).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` use it.  It shares no code with
the CUDA library and imports nothing from the product package.

Everything is float64 numpy.  Matrix products use ``@`` (a library primitive);
there is no blocking, fusion or reordering beyond the steps the paper states.
Each function names the passage it follows.

Two kinds of result (the paper's target function and its recursion):

* the plain definition D = theta(mu I - F) (the introduction's statement of
  the problem), by eigendecomposition or, for generated inputs, in closed
  form from the known eigenvectors;
* the recursion itself (Eq. 1 with the polynomials of Algorithm 1 and
  Algorithm 2), step by step, with the scalar schedule (alpha, beta, beta-bar)
  that accompanies it; needed for iteration counts, multiplication counts and
  parity at a fixed number of steps.

Readings where the paper is silent (each also listed in the design notes):

* Loop bound.  The algorithms loop "for i = 1, 2, ..., n" with no stop rule.
  In exact arithmetic the unoccupied eigenvalues of X_i lie in [0, beta_i] and
  the occupied ones in [beta-bar_i, 1] (Algorithm 1: beta-bar = 1 - beta by
  the symmetry P11(1 - x) = 1 - P11(x)), so ||X_i - D||_2 <= max(beta_i,
  1 - beta-bar_i), which is the accuracy measure of Fig. 3.  The loop stops
  once that bound is <= tol, or after max_iter iterations.
* Tie in Algorithm 2's branch test: the test is strict, (beta + beta-bar) > 1,
  evaluated in float64 in that order; a tie takes the P01 branch.
* Asymmetric gap in Algorithm 1 (the paper assumes the gap symmetric around
  mu): beta_0 = 1/2 - min(mu - homo, lumo - mu) / gamma, the nearer edge.
* Niklasson's trace rule (the alpha = 0 relative of Algorithm 2): take the
  P10 branch when trace(X_{i-1}) > nocc, otherwise P01.
* Multiplication count: Algorithm 1 uses two matrix products per iteration
  (X_s^2 and X_s^2 X_s), Algorithm 2 one (the square).
* Truncation (the paper leaves the scheme to future work and names control
  of the forward error): after every step, drop the 32 x 32 blocks of
  smallest Frobenius norm while the dropped mass sum ||B||_F^2 (blocks off
  the diagonal counted twice, for B and B^T) stays <= tau^2, so each step
  perturbs X by at most tau in the Frobenius (hence 2-) norm.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SCHEMES = ("FIXED_MU_SF", "FIXED_MU_MONO", "TC_SF", "TC_MONO")


# ---------------------------------------------------------------------------
# The P_{i,j} polynomials used by the schemes (paper: notation P_{i,j} of
# degree 1 + i + j with fixed points 0 and 1; P_{1,0} = x^2, P_{0,1} = 2x - x^2;
# Algorithm 1 uses P_{1,1} = 3x^2 - 2x^3).
# ---------------------------------------------------------------------------

def P10(x):
    return x * x


def P01(x):
    return 2.0 * x - x * x


def P11(x):
    return 3.0 * x * x - 2.0 * x * x * x


def P_ij(i: int, j: int, x):
    """P_{i,j}(x) = x^(i+1) sum_{k=0..j} C(i+k, k) (1-x)^k: the polynomial of
    degree 1 + i + j with fixed points 0 and 1 and i and j vanishing
    derivatives there (the tests check this closed form against that
    definition).  Evaluated with a Horner sum in t = 1 - x, then the power of x
    by repeated multiplication."""
    t = 1.0 - x
    acc = 0.0 * x
    for k in range(j, -1, -1):
        acc = acc * t + math.comb(i + k, k)
    p = x
    for _ in range(i):
        p = p * x
    return p * acc


def pmm_alpha(m: int, beta: float) -> float:
    """The alpha >= 1 with P_{m,m}(alpha (beta - 1/2) + 1/2) = P_{m,m}((1 - alpha)/2)
    (the scaling equation stated with Algorithm 1, for odd m): bisection on
    [1, 1 / (1 - 2 beta)], where the difference of the two sides goes from
    positive to negative, down to the last bit."""
    def g(a):
        return P_ij(m, m, a * (beta - 0.5) + 0.5) - P_ij(m, m, 0.5 * (1.0 - a))
    lo, hi = 1.0, 1.0 / (1.0 - 2.0 * beta)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid == lo or mid == hi:
            break
        if g(mid) > 0.0:
            lo = mid
        else:
            hi = mid
    return lo


# ---------------------------------------------------------------------------
# Result record
# ---------------------------------------------------------------------------

@dataclass
class Result:
    scheme: str
    iterations: int = 0
    multiplications: int = 0
    converged: bool = False
    alphas: list = field(default_factory=list)
    branches: list = field(default_factory=list)   # Algorithm 2: "P10" / "P01"
    betas: list = field(default_factory=list)      # beta after each iteration
    betabars: list = field(default_factory=list)   # beta-bar after each iteration
    traces: list = field(default_factory=list)     # trace(X_i) after each iteration
    idem: list = field(default_factory=list)       # ||X_{i-1} - X_{i-1}^2||_F (Algorithm 2)
    beta0: float = float("nan")
    betabar0: float = float("nan")
    f0: tuple = ()                                 # (c0, c1): X_0 = c0 I + c1 F
    tau: float = float("nan")                      # truncation per step (truncated runs)

    @property
    def err_bound(self) -> float:
        if not self.betas:
            return float("nan")
        return max(self.betas[-1], 1.0 - self.betabars[-1])


# ---------------------------------------------------------------------------
# Algorithm 1: McWeeny-based fixed-mu purification with scaling
# ---------------------------------------------------------------------------

def fixed_mu_gamma(lmin: float, lmax: float, mu: float) -> float:
    """Algorithm 1, first step: gamma = 2 max(lambda_max - mu, mu - lambda_min)."""
    return 2.0 * max(lmax - mu, mu - lmin)


def fixed_mu_beta0(gamma: float, mu: float, homo: float, lumo: float) -> float:
    """Algorithm 1, beta = 0.5 (1 - xi / gamma) for a gap xi centred on mu.
    For an off-centre gap the nearer edge is used (see module docstring)."""
    half = min(mu - homo, lumo - mu)
    return 0.5 - half / gamma


def fixed_mu_alpha(beta: float) -> float:
    """Algorithm 1: alpha = 3 / sqrt(12 beta^2 - 18 beta + 9), the alpha >= 1
    that solves Eq. 3 for P_{1,1}."""
    return 3.0 / math.sqrt(12.0 * beta * beta - 18.0 * beta + 9.0)


def fixed_mu_schedule(beta: float, tol: float, max_iter: int, scaled: bool = True):
    """Scalar part of Algorithm 1: the alpha of each iteration and the beta
    after it.  Stops once beta <= tol (module docstring) or at max_iter."""
    alphas, betas = [], []
    while beta > tol and len(alphas) < max_iter:
        alpha = fixed_mu_alpha(beta) if scaled else 1.0
        beta_s = alpha * (beta - 0.5) + 0.5
        beta = 3.0 * beta_s * beta_s - 2.0 * beta_s * beta_s * beta_s
        alphas.append(alpha)
        betas.append(beta)
    return alphas, betas


def purify_fixed_mu(F, lmin, lmax, mu, homo, lumo, tol=1e-12, max_iter=200, scaled=True):
    """Algorithm 1 on a dense symmetric F; scaled=False gives the regular
    grand-canonical McWeeny purification (alpha = 1), which the paper uses as
    its reference for this scheme."""
    F = np.asarray(F, dtype=np.float64)
    n = F.shape[0]
    I = np.eye(n)
    gamma = fixed_mu_gamma(lmin, lmax, mu)
    X = (mu * I - F) / gamma + 0.5 * I
    beta = fixed_mu_beta0(gamma, mu, homo, lumo)
    res = Result(scheme="FIXED_MU_SF" if scaled else "FIXED_MU_MONO", beta0=beta,
                 betabar0=1.0 - beta, f0=(mu / gamma + 0.5, -1.0 / gamma))
    alphas, betas = fixed_mu_schedule(beta, tol, max_iter, scaled)
    for alpha, beta_i in zip(alphas, betas):
        Xs = alpha * (X - 0.5 * I) + 0.5 * I
        Xs2 = Xs @ Xs
        X = 3.0 * Xs2 - 2.0 * (Xs2 @ Xs)
        res.alphas.append(alpha)
        res.betas.append(beta_i)
        res.betabars.append(1.0 - beta_i)
        res.traces.append(float(np.trace(X)))
        res.iterations += 1
        res.multiplications += 2
    res.converged = bool(betas) and betas[-1] <= tol or (not betas and beta <= tol)
    return X, res


def pmm_schedule(m: int, beta: float, tol: float, max_iter: int, scaled: bool = True):
    """Scalar part of the fixed-mu scheme with P_{m,m} (odd m): the alpha of
    each iteration and the beta after it, beta <- P_{m,m}(alpha (beta - 1/2)
    + 1/2); stops once beta <= tol or at max_iter."""
    alphas, betas = [], []
    while beta > tol and len(alphas) < max_iter:
        alpha = pmm_alpha(m, beta) if scaled else 1.0
        beta = P_ij(m, m, alpha * (beta - 0.5) + 0.5)
        alphas.append(alpha)
        betas.append(beta)
    return alphas, betas


# Matrix products per iteration of the fixed-mu scheme with P_{m,m} (a
# reading: the paper counts products only for m = 1): m = 1 as in Algorithm 1
# (X_s^2, then X_s^2 X_s); m = 3 for the evaluation order of
# P_{3,3}(x) = x^4 (35 - 84 x + 70 x^2 - 20 x^3): V = 70 X_s - 20 X_s^2,
# Q = X_s V - 84 X_s + 35 I, S = X_s^2, T = S^2, X = T Q.
PMM_PRODUCTS = {1: 2, 3: 5}


def purify_fixed_mu_pmm(F, lmin, lmax, mu, homo, lumo, m: int = 3, tol=1e-12, max_iter=200,
                        scaled=True):
    """Fixed-mu purification with f_i(X) = P_{m,m}(alpha (X - 1/2) + 1/2), m
    odd (the scheme stated with Algorithm 1 for general m; Algorithm 1 is
    m = 1).  X_0 and beta as in Algorithm 1."""
    F = np.asarray(F, dtype=np.float64)
    n = F.shape[0]
    I = np.eye(n)
    gamma = fixed_mu_gamma(lmin, lmax, mu)
    X = (mu * I - F) / gamma + 0.5 * I
    beta = fixed_mu_beta0(gamma, mu, homo, lumo)
    res = Result(scheme=f"FIXED_MU_P{m}{m}" + ("_SF" if scaled else "_MONO"), beta0=beta,
                 betabar0=1.0 - beta, f0=(mu / gamma + 0.5, -1.0 / gamma))
    alphas, betas = pmm_schedule(m, beta, tol, max_iter, scaled)
    for alpha, beta_i in zip(alphas, betas):
        Xs = alpha * (X - 0.5 * I) + 0.5 * I
        X = _matrix_P(m, m, Xs)
        res.alphas.append(alpha)
        res.betas.append(beta_i)
        res.betabars.append(1.0 - beta_i)
        res.traces.append(float(np.trace(X)))
        res.iterations += 1
        res.multiplications += PMM_PRODUCTS.get(m, 2 * m)
    res.converged = (bool(betas) and betas[-1] <= tol) or (not betas and beta <= tol)
    return X, res


def pij_fixed_point(i: int, j: int) -> float:
    """The unstable fixed point c in (0, 1) of P_{i,j} (i, j >= 1): P(x) - x is
    negative near 0 and positive near 1 and changes sign once; bisection."""
    lo, hi = 1e-12, 1.0 - 1e-12
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid == lo or mid == hi:
            break
        if P_ij(i, j, mid) - mid < 0.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _fold_root(g, lo: float, hi: float) -> float:
    """The alpha in [lo, hi] where g goes from positive to negative (bisection)."""
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid == lo or mid == hi:
            break
        if g(mid) > 0.0:
            lo = mid
        else:
            hi = mid
    return lo


def pij_alpha(i: int, j: int, c: float, beta: float, betabar: float) -> float:
    """Scaling about the unstable fixed point c for P_{i,j}, i and j odd: the
    unoccupied side folds at P(alpha (beta - c) + c) = P(c (1 - alpha)) (its
    lower end meets its edge), the occupied side at P(alpha (betabar - c) + c)
    = P(c + alpha (1 - c)); one alpha serves both, so the smaller.  With
    i = j, c = 1/2 and betabar = 1 - beta this is pmm_alpha."""
    a_u = _fold_root(lambda a: P_ij(i, j, a * (beta - c) + c) - P_ij(i, j, c * (1.0 - a)),
                     1.0, c / (c - beta))
    a_o = _fold_root(lambda a: P_ij(i, j, c + a * (1.0 - c)) - P_ij(i, j, a * (betabar - c) + c),
                     1.0, (1.0 - c) / (betabar - c))
    return min(a_u, a_o)


def pij_schedule(i: int, j: int, beta: float, betabar: float, tol: float, max_iter: int,
                 scaled: bool = True):
    """Scalar part of the fixed-mu scheme with P_{i,j} (i, j odd) scaled about
    its unstable fixed point c: per iteration alpha, then beta (upper bound of
    the unoccupied images: the larger of its edge's and its folded end's
    image) and betabar (lower bound of the occupied ones, likewise).  Stops
    once max(beta, 1 - betabar) <= tol."""
    c = pij_fixed_point(i, j)
    out = []
    while max(beta, 1.0 - betabar) > tol and len(out) < max_iter:
        a = pij_alpha(i, j, c, beta, betabar) if scaled else 1.0
        beta = max(P_ij(i, j, a * (beta - c) + c), P_ij(i, j, c * (1.0 - a)))
        betabar = min(P_ij(i, j, a * (betabar - c) + c), P_ij(i, j, c + a * (1.0 - c)))
        out.append((a, beta, betabar))
    return c, out


def purify_fixed_mu_pij(F, lmin, lmax, mu, homo, lumo, i: int, j: int, tol=1e-12, max_iter=200,
                        scaled=True):
    """Fixed-mu purification with f(X) = P_{i,j}(alpha (X - c I) + c I), i and
    j odd, c the unstable fixed point of P_{i,j}; X_0 maps mu to c and the
    spectrum into [0, 1]: X_0 = c I + (mu I - F) / gamma with gamma =
    max((mu - lmin) / (1 - c), (lmax - mu) / c); beta_0 = c - (lumo - mu) /
    gamma, betabar_0 = c + (mu - homo) / gamma."""
    F = np.asarray(F, dtype=np.float64)
    n = F.shape[0]
    Id = np.eye(n)
    c = pij_fixed_point(i, j)
    gamma = max((mu - lmin) / (1.0 - c), (lmax - mu) / c)
    X = c * Id + (mu * Id - F) / gamma
    beta, betabar = c - (lumo - mu) / gamma, c + (mu - homo) / gamma
    res = Result(scheme=f"FIXED_MU_P{i}{j}" + ("_SF" if scaled else "_MONO"), beta0=beta,
                 betabar0=betabar, f0=(c + mu / gamma, -1.0 / gamma))
    _, steps = pij_schedule(i, j, beta, betabar, tol, max_iter, scaled)
    for a, b, bb in steps:
        X = _matrix_P(i, j, a * (X - c * Id) + c * Id)
        res.alphas.append(a)
        res.betas.append(b)
        res.betabars.append(bb)
        res.traces.append(float(np.trace(X)))
        res.iterations += 1
        res.multiplications += PIJ_PRODUCTS.get((i, j), i + j + 1)
    res.converged = max(res.betas[-1], 1.0 - res.betabars[-1]) <= tol if steps else \
        max(beta, 1.0 - betabar) <= tol
    return X, res


# Products per iteration for these evaluation orders (a reading, as for
# P_{m,m}): P_{3,1} = x^4 (5 - 4x):
# S = X^2, T = S^2, X = 5 T - 4 T X; P_{1,3} = x^2 (10 - 20x + 15x^2 - 4x^3):
# V = 15 X - 4 X^2, Q = X V - 20 X + 10 I, S = X^2, X = S Q.
PIJ_PRODUCTS = {(1, 1): 2, (3, 3): 5, (3, 1): 3, (1, 3): 4}


def _matrix_P(i: int, j: int, Xs):
    """P_{i,j} of a symmetric matrix, from its definition as a polynomial:
    Xs^(i+1) (sum_k C(i+k, k) (I - Xs)^k), products in plain numpy."""
    n = Xs.shape[0]
    I = np.eye(n)
    T = I - Xs
    acc = np.zeros_like(Xs)
    for k in range(j, -1, -1):
        acc = acc @ T + math.comb(i + k, k) * I
    Pw = Xs.copy()
    for _ in range(i):
        Pw = Pw @ Xs
    return Pw @ acc


# ---------------------------------------------------------------------------
# Algorithm 2: P_{0,1} & P_{1,0} based varying-mu purification with scaling
# ---------------------------------------------------------------------------

def tc_f0(lmin: float, lmax: float):
    """Algorithm 2: X_0 = (lambda_max I - F) / (lambda_max - lambda_min),
    returned as (c0, c1) with X_0 = c0 I + c1 F."""
    w = lmax - lmin
    return lmax / w, -1.0 / w


def tc_beta0(lmin, lmax, homo, lumo):
    """Algorithm 2: beta = f_0(lambda_lumo), beta-bar = f_0(lambda_homo)."""
    w = lmax - lmin
    return (lmax - lumo) / w, (lmax - homo) / w


def tc_branch_by_beta(beta: float, betabar: float) -> str:
    """Algorithm 2's test: P10 when beta + beta-bar > 1 (strict), else P01."""
    return "P10" if (beta + betabar) > 1.0 else "P01"


def tc_alpha(branch: str, beta: float, betabar: float) -> float:
    """Algorithm 2: alpha = beta / (2 - beta) before x^2, alpha =
    (1 - beta-bar) / (1 + beta-bar) before 2x - x^2."""
    if branch == "P10":
        return beta / (2.0 - beta)
    return (1.0 - betabar) / (1.0 + betabar)


def tc_map(branch: str, alpha: float, x: float) -> float:
    """The scalar form of Eq. 4 (P10 branch) and Eq. 5 (P01 branch), used on
    beta and beta-bar."""
    if branch == "P10":
        y = (1.0 + alpha) * x - alpha
        return y * y
    return 2.0 * (1.0 + alpha) * x - (1.0 + alpha) ** 2 * x * x


def tc_schedule(beta: float, betabar: float, tol: float, max_iter: int, scaled: bool = True):
    """Scalar part of Algorithm 2 with the beta rule: per iteration the
    branch, alpha, and (beta, beta-bar) after it."""
    out = []
    while max(beta, 1.0 - betabar) > tol and len(out) < max_iter:
        branch = tc_branch_by_beta(beta, betabar)
        alpha = tc_alpha(branch, beta, betabar) if scaled else 0.0
        beta, betabar = tc_map(branch, alpha, beta), tc_map(branch, alpha, betabar)
        out.append((branch, alpha, beta, betabar))
    return out


def purify_tc(F, lmin, lmax, homo=None, lumo=None, tol=1e-12, max_iter=200, scaled=True,
              branch_rule="beta", nocc=None):
    """Algorithm 2 on a dense symmetric F.

    scaled=False is the alpha = 0 scheme the paper identifies with
    Niklasson's second-order trace-correcting purification (up to the branch
    rule).  branch_rule="trace" takes the branch from trace(X_{i-1}) versus
    nocc instead of from beta + beta-bar.  Without homo/lumo the loop stops
    when ||X_{i-1} - X_{i-1}^2||_F <= tol (trace rule only)."""
    F = np.asarray(F, dtype=np.float64)
    n = F.shape[0]
    I = np.eye(n)
    c0, c1 = tc_f0(lmin, lmax)
    X = (lmax * I - F) / (lmax - lmin)
    have_bounds = homo is not None and lumo is not None
    if not have_bounds and branch_rule != "trace":
        raise ValueError("the beta rule needs homo and lumo")
    if branch_rule == "trace" and nocc is None:
        raise ValueError("the trace rule needs nocc")
    beta, betabar = tc_beta0(lmin, lmax, homo, lumo) if have_bounds else (float("nan"),) * 2
    res = Result(scheme="TC_SF" if scaled else "TC_MONO", beta0=beta, betabar0=betabar,
                 f0=(c0, c1))
    while res.iterations < max_iter:
        if have_bounds and max(beta, 1.0 - betabar) <= tol:
            res.converged = True
            break
        if branch_rule == "trace":
            branch = "P10" if float(np.trace(X)) > nocc else "P01"
        else:
            branch = tc_branch_by_beta(beta, betabar)
        if scaled:
            alpha = tc_alpha(branch, beta, betabar)
        else:
            alpha = 0.0
        X2 = X @ X
        res.idem.append(float(np.linalg.norm(X - X2)))
        if branch == "P10":
            # ((1 + alpha) X - alpha I)^2 expanded over the square X^2
            X = (1.0 + alpha) ** 2 * X2 - 2.0 * alpha * (1.0 + alpha) * X + alpha * alpha * I
        else:
            X = 2.0 * (1.0 + alpha) * X - (1.0 + alpha) ** 2 * X2
        if have_bounds:
            beta, betabar = tc_map(branch, alpha, beta), tc_map(branch, alpha, betabar)
        res.alphas.append(alpha)
        res.branches.append(branch)
        res.betas.append(beta)
        res.betabars.append(betabar)
        res.traces.append(float(np.trace(X)))
        res.iterations += 1
        res.multiplications += 1
        if not have_bounds and res.idem[-1] <= tol:
            res.converged = True
            break
    else:
        if have_bounds and max(beta, 1.0 - betabar) <= tol:
            res.converged = True
    return X, res


def purify(F, scheme, lmin, lmax, mu=None, homo=None, lumo=None, nocc=None, tol=1e-12,
           max_iter=200, branch_rule="beta"):
    """Dispatch on the four scheme names used by the library."""
    if scheme == "FIXED_MU_SF" or scheme == "FIXED_MU_MONO":
        if mu is None:
            mu = 0.5 * (homo + lumo)
        return purify_fixed_mu(F, lmin, lmax, mu, homo, lumo, tol, max_iter,
                               scaled=scheme == "FIXED_MU_SF")
    if scheme == "TC_SF" or scheme == "TC_MONO":
        return purify_tc(F, lmin, lmax, homo, lumo, tol, max_iter, scaled=scheme == "TC_SF",
                         branch_rule=branch_rule, nocc=nocc)
    raise ValueError(scheme)


# ---------------------------------------------------------------------------
# The plain definition D = theta(mu I - F)
# ---------------------------------------------------------------------------

def density_by_eigh(F, mu: float):
    """D = theta(mu I - F): the sum of v v^T over eigenpairs with lambda < mu."""
    lam, V = np.linalg.eigh(np.asarray(F, dtype=np.float64))
    occ = V[:, lam < mu]
    return occ @ occ.T


def density_closed_form(Q, lam, mu: float):
    """D = Q_occ Q_occ^T for F = Q diag(lam) Q^T."""
    occ = np.asarray(Q)[:, np.asarray(lam) < mu]
    return occ @ occ.T


# ---------------------------------------------------------------------------
# Spectral bounds lambda_min, lambda_max ("extremal eigenvalues of F or
# bounds thereof", the inputs of Algorithms 1 and 2)
# ---------------------------------------------------------------------------

def gershgorin(F):
    """Gershgorin's circle theorem: every eigenvalue lies in
    [min_i (F_ii - R_i), max_i (F_ii + R_i)], R_i = sum_{j != i} |F_ij|."""
    F = np.asarray(F, dtype=np.float64)
    d = np.diag(F)
    R = np.abs(F).sum(axis=1) - np.abs(d)
    return float(np.min(d - R)), float(np.max(d + R))


_GOLDEN = 0x9E3779B97F4A7C15
_MASK = (1 << 64) - 1
LANCZOS_KEY = 0x11010265


def _splitmix64(x: int) -> int:
    # SplitMix64 (Steele, Lea, Flood 2014): one step from state x.
    z = (x + _GOLDEN) & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def lanczos_start(n: int, key: int = LANCZOS_KEY):
    """Counter-based start vector: q_i = 2 u_i - 1 with u_i the top 53 bits of
    SplitMix64 at state key + i * golden, as a fraction of 2^53."""
    q = np.empty(n)
    for i in range(n):
        z = _splitmix64((key + i * _GOLDEN) & _MASK)
        q[i] = 2.0 * ((z >> 11) * (1.0 / 9007199254740992.0)) - 1.0
    return q


def lanczos(F, k: int, q):
    """k steps of the symmetric Lanczos three-term recurrence from q (no
    reorthogonalisation).  Returns the diagonal a[0..m) and off-diagonal
    b[0..m) of the tridiagonal T_m (m <= k; b[m-1] is the residual norm)."""
    F = np.asarray(F, dtype=np.float64)
    v = np.asarray(q, dtype=np.float64) / np.linalg.norm(q)
    v_prev = np.zeros_like(v)
    b_prev = 0.0
    a, b = [], []
    for _ in range(k):
        w = F @ v - b_prev * v_prev
        aj = float(w @ v)
        w = w - aj * v
        bj = float(np.linalg.norm(w))
        a.append(aj)
        b.append(bj)
        if bj == 0.0:
            break
        v_prev, v, b_prev = v, w / bj, bj
    return np.array(a), np.array(b)


def lanczos_bounds(F, k: int, q=None):
    """Extremal Ritz values of T_k widened by their residual norms
    |b_k y_k|, intersected with the Gershgorin interval."""
    F = np.asarray(F, dtype=np.float64)
    if q is None:
        q = lanczos_start(F.shape[0])
    a, b = lanczos(F, k, q)
    m = a.size
    T = np.diag(a) + np.diag(b[:m - 1], 1) + np.diag(b[:m - 1], -1)
    theta, Y = np.linalg.eigh(T)
    r_lo = abs(b[m - 1] * Y[m - 1, 0])
    r_hi = abs(b[m - 1] * Y[m - 1, -1])
    g_lo, g_hi = gershgorin(F)
    return max(g_lo, theta[0] - r_lo), min(g_hi, theta[-1] + r_hi)


# ---------------------------------------------------------------------------
# Gap edges from the purification (the paper asks for a lower bound of the
# gap's lower edge and an upper bound of its upper edge, obtainable by a
# technique for interior eigenvalues)
# ---------------------------------------------------------------------------

def lanczos_top(apply, n: int, k: int, q):
    """k plain Lanczos steps with the operator `apply` (v -> A v) from q.
    Returns the largest Ritz value, its Ritz vector and residual norm
    |b_m z_{m-1}|."""
    v = np.asarray(q, dtype=np.float64) / np.linalg.norm(q)
    v_prev = np.zeros(n)
    b_prev = 0.0
    a, b, V = [], [], []
    for _ in range(k):
        V.append(v)
        w = apply(v) - b_prev * v_prev
        aj = float(w @ v)
        w = w - aj * v
        bj = float(np.linalg.norm(w))
        a.append(aj)
        b.append(bj)
        if bj == 0.0:
            break
        v_prev, v, b_prev = v, w / bj, bj
    m = len(a)
    T = np.diag(a) + np.diag(b[:m - 1], 1) + np.diag(b[:m - 1], -1)
    theta, Z = np.linalg.eigh(T)
    return float(theta[-1]), np.array(V).T @ Z[:, -1], float(abs(b[m - 1] * Z[m - 1, -1]))


GAP_FILTER_POWER = 4


def _solve_monotone(g, target, lo, hi):
    """x in [lo, hi] with g(x) = target for g monotone on [lo, hi] (bisection
    to the last bit); the end nearer the target when it lies outside."""
    glo, ghi = g(lo), g(hi)
    inc = ghi > glo
    if (target <= min(glo, ghi)):
        return lo if inc else hi
    if (target >= max(glo, ghi)):
        return hi if inc else lo
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid in (lo, hi):
            break
        if (g(mid) < target) == inc:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def estimate_gap(F, lmin, lmax, nocc, k: int = 40, max_steps: int = 100, q=None):
    """Inner estimates (homo_est >= homo, lumo_est <= lumo) of the gap edges.

    1. X_0 = (lmax I - F) / (lmax - lmin) (Algorithm 2's f_0: occupied near 1),
       then steps of the alpha = 0 scheme with the trace rule, recording the
       branches; every map keeps the order of the eigenvalues.
    2. Once ||X - X^2||_F < 1 / (4 sqrt(n)) and round(trace X) = nocc, exactly
       the nocc occupied eigenvalues lie above 1/2 (|trace X - #{x > 1/2}|
       <= sum min(x, 1 - x) <= 2 sqrt(n) ||X - X^2||_F), and every eigenvalue
       has x (1 - x) < 1/16 (x > 0.93 or x < 0.07).
    3. Lanczos on X^p (I - X) (p = 4): its largest eigenvalue belongs to the
       occupied eigenvalue nearest 1/2 (x^p (1 - x) falls for x > p / (p + 1)
       and the unoccupied side is suppressed to x^p); on X (I - X)^p likewise
       for the unoccupied side.  The top Ritz vector's Rayleigh quotient with
       X must lie on the expected side of 1/2 (else one more step is taken).
       Raising each top Ritz value by its residual norm and solving for x on
       the monotone branch gives images no farther from 1/2 than the edges'.
    4. The inverse of the recorded steps (x^2 -> sqrt; 2x - x^2 -> 1 -
       sqrt(1 - y)) and of f_0 map the two images back to the spectrum of F;
       64 ulps of lmax - lmin towards the gap's centre cover the rounding of
       that map.
    Returns (homo_est, lumo_est, steps taken)."""
    F = np.asarray(F, dtype=np.float64)
    n = F.shape[0]
    w = lmax - lmin
    margin = 64.0 * np.finfo(np.float64).eps * w
    p = GAP_FILTER_POWER
    X = (lmax * np.eye(n) - F) / w
    branches = []
    if q is None:
        q = lanczos_start(n)
    for step in range(max_steps + 1):
        S = X @ X
        idem = float(np.linalg.norm(X - S))
        if idem < 1.0 / (4.0 * np.sqrt(n)) and round(float(np.trace(X))) == nocc:
            def occ_filter(v):
                t = v
                for _ in range(p):
                    t = X @ t
                return t - X @ t

            def unocc_filter(v):
                t = v
                for _ in range(p):
                    t = t - X @ t
                return X @ t
            th_o, u_o, r_o = lanczos_top(occ_filter, n, k, q)
            th_u, u_u, r_u = lanczos_top(unocc_filter, n, k, q)
            if float(u_o @ X @ u_o) / float(u_o @ u_o) > 0.5 > float(u_u @ X @ u_u) / float(u_u @ u_u):
                x_h = _solve_monotone(lambda x: x ** p * (1.0 - x), th_o + r_o, p / (p + 1.0), 1.0)
                x_l = _solve_monotone(lambda x: x * (1.0 - x) ** p, th_u + r_u, 0.0, 1.0 / (p + 1.0))
                for br in reversed(branches):
                    if br == "P10":
                        x_h, x_l = np.sqrt(x_h), np.sqrt(x_l)
                    else:
                        x_h, x_l = 1.0 - np.sqrt(1.0 - x_h), 1.0 - np.sqrt(1.0 - x_l)
                return lmax - w * x_h + margin, lmax - w * x_l - margin, step
        if step == max_steps or idem == 0.0:
            break
        if float(np.trace(X)) > nocc:
            X, br = S, "P10"
        else:
            X, br = 2.0 * X - S, "P01"
        branches.append(br)
    raise RuntimeError("gap edges not resolved within max_steps")


# ---------------------------------------------------------------------------
# Invariants
# ---------------------------------------------------------------------------

def idempotency_error(X):
    X = np.asarray(X)
    return float(np.linalg.norm(X - X @ X))


def commutator_norm(X, F):
    X = np.asarray(X)
    F = np.asarray(F)
    return float(np.linalg.norm(X @ F - F @ X))


# ---------------------------------------------------------------------------
# Block truncation (sparsity discussion: drop small elements, controlling the
# error each step adds)
# ---------------------------------------------------------------------------

def block_norms(X, bs: int = 32):
    """Frobenius norms of the bs x bs blocks of X (n a multiple of bs)."""
    X = np.asarray(X, dtype=np.float64)
    nb = X.shape[0] // bs
    B = X.reshape(nb, bs, nb, bs)
    return np.sqrt(np.einsum("ikjl,ikjl->ij", B, B))


def truncation_mask(X, tau: float, bs: int = 32):
    """Blocks kept (boolean nb x nb, symmetric): blocks (I <= J) sorted by
    ascending norm (ties by row, then column) are dropped while the dropped
    mass, counting off-diagonal blocks twice, stays <= tau^2; a block of norm
    exactly zero is always dropped."""
    N = block_norms(X, bs)
    nb = N.shape[0]
    I, J = np.triu_indices(nb)
    w = np.where(I == J, 1.0, 2.0)
    order = np.lexsort((J, I, N[I, J]))
    keep = np.ones((nb, nb), dtype=bool)
    budget = tau * tau
    acc = 0.0
    for k in order:
        m = w[k] * N[I[k], J[k]] ** 2
        if m > 0.0 and acc + m > budget:
            break
        acc += m
        keep[I[k], J[k]] = keep[J[k], I[k]] = False
    return keep


def truncate_blocks(X, tau: float, bs: int = 32):
    keep = truncation_mask(X, tau, bs)
    mask = np.repeat(np.repeat(keep, bs, axis=0), bs, axis=1)
    return np.where(mask, X, 0.0), keep


def purify_tc_truncated(F, lmin, lmax, homo, lumo, tau, tol=1e-9, max_iter=200, scaled=True,
                        bs: int = 32, tau_budget=None):
    """Algorithm 2 with the truncation above applied to every iterate
    (X_0 included).  Returns X, the Result and the kept-block counts (blocks
    I <= J) after each truncation.

    tau_budget: a total budget for all truncations instead of tau, spread
    evenly over X_0 and the m scheduled iterations (tau = budget / (m + 1)),
    so that a schedule with fewer iterations truncates harder at the same
    bound on the accumulated truncation (closing discussion: fewer iterations
    allow more aggressive truncation in each)."""
    F = np.asarray(F, dtype=np.float64)
    n = F.shape[0]
    I = np.eye(n)
    beta, betabar = tc_beta0(lmin, lmax, homo, lumo)
    steps = list(tc_schedule(beta, betabar, tol, max_iter, scaled))
    if tau_budget is not None:
        tau = tau_budget / (len(steps) + 1)
    X = (lmax * I - F) / (lmax - lmin)
    X, keep = truncate_blocks(X, tau, bs)
    nnzb = [int(np.triu(keep).sum())]
    res = Result(scheme="TC_SF" if scaled else "TC_MONO", beta0=beta, betabar0=betabar,
                 f0=tc_f0(lmin, lmax))
    res.tau = tau
    for branch, alpha, b, bb in steps:
        X2 = X @ X
        res.idem.append(float(np.linalg.norm(X - X2)))
        if branch == "P10":
            X = (1.0 + alpha) ** 2 * X2 - 2.0 * alpha * (1.0 + alpha) * X + alpha * alpha * I
        else:
            X = 2.0 * (1.0 + alpha) * X - (1.0 + alpha) ** 2 * X2
        X, keep = truncate_blocks(X, tau, bs)
        nnzb.append(int(np.triu(keep).sum()))
        res.alphas.append(alpha)
        res.branches.append(branch)
        res.betas.append(b)
        res.betabars.append(bb)
        res.traces.append(float(np.trace(X)))
        res.iterations += 1
        res.multiplications += 1
    res.converged = bool(res.betas) and max(res.betas[-1], 1.0 - res.betabars[-1]) <= tol
    return X, res, nnzb
