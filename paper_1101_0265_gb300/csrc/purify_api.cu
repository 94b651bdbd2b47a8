// C ABI of libpurify: handle management, the host-side scalar schedule of
// the two scale-and-fold schemes (Algorithm 1, Algorithm 2), and the
// iteration driver that issues one fused device step per matrix product.
//
// Host arithmetic here is compiled without FMA contraction so that the
// scalar schedule (alpha, beta, beta-bar, the branch test) is evaluated in
// the plain float64 order the algorithms state.
#include "internal.h"
#include "mixed.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

namespace purify {

static thread_local char g_last_error[256] = "";

// Kernel launches of the calling thread: a handle is used by one thread at a
// time, so differences of this count are the handle's own launches even when
// other threads drive other handles.
static thread_local long long g_launches = 0;
void count_launches(int k) { g_launches += k; }
long long launches_so_far() { return g_launches; }

int cuda_status(cudaError_t e, const char* what) {
    std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PURIFY_ERR_OOM : PURIFY_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Scalar schedule (host, float64)
// ---------------------------------------------------------------------------

// Algorithm 1: alpha = 3 / sqrt(12 beta^2 - 18 beta + 9) (solves Eq. 3).
static double fixed_mu_alpha(double beta) {
    return 3.0 / std::sqrt(12.0 * beta * beta - 18.0 * beta + 9.0);
}

// Algorithm 1: gamma = 2 max(lmax - mu, mu - lmin).
static double fixed_mu_gamma(double lmin, double lmax, double mu) {
    return 2.0 * std::max(lmax - mu, mu - lmin);
}

// Algorithm 1: beta = (1 - xi / gamma) / 2 for a gap centred on mu; for an
// off-centre gap the nearer edge is used.
static double fixed_mu_beta0(double gamma, double mu, double homo, double lumo) {
    const double half = std::min(mu - homo, lumo - mu);
    return 0.5 - half / gamma;
}

// Algorithm 2: beta = f_0(lumo), beta_bar = f_0(homo).
static void tc_beta0(double lmin, double lmax, double homo, double lumo, double* b, double* bb) {
    const double w = lmax - lmin;
    *b = (lmax - lumo) / w;
    *bb = (lmax - homo) / w;
}

// Algorithm 2's test (strict): P_{1,0} when beta + beta_bar > 1.
static int tc_branch(double b, double bb) { return (b + bb) > 1.0 ? 1 : 0; }

// Algorithm 2: alpha of the chosen branch.
double tc_alpha(int branch, double b, double bb) {
    return branch ? b / (2.0 - b) : (1.0 - bb) / (1.0 + bb);
}

// The square (1 + a)^2 of Eq. 4 / Eq. 5 as the C library's pow evaluates a
// float power (the test oracle's float power calls the same function, so the
// two schedules agree bit for bit).  The call goes through a volatile pointer:
// a compiler may otherwise turn pow(v, 2) into v * v.
static double (*volatile g_pow)(double, double) = ::pow;
double sq1p(double a) { return g_pow(1.0 + a, 2.0); }

// Eq. 4 (branch 1) / Eq. 5 (branch 0) on a scalar.
double tc_map(int branch, double a, double x) {
    if (branch) {
        const double y = (1.0 + a) * x - a;
        return y * y;
    }
    return 2.0 * (1.0 + a) * x - sq1p(a) * x * x;
}

static bool is_fixed_mu(int scheme) { return scheme != PURIFY_TC_SF && scheme != PURIFY_TC_MONO; }
static bool is_scaled(int scheme) {
    return scheme == PURIFY_FIXED_MU_SF || scheme == PURIFY_TC_SF || scheme == PURIFY_FIXED_MU_P33_SF ||
           scheme == PURIFY_FIXED_MU_P13_SF || scheme == PURIFY_FIXED_MU_P31_SF;
}

int pmm_order(int scheme) {
    return (scheme == PURIFY_FIXED_MU_P33_SF || scheme == PURIFY_FIXED_MU_P33_MONO) ? 3 : 1;
}

void pij_orders(int scheme, int* i, int* j) {
    *i = *j = 1;
    if (scheme == PURIFY_FIXED_MU_P33_SF || scheme == PURIFY_FIXED_MU_P33_MONO) *i = *j = 3;
    if (scheme == PURIFY_FIXED_MU_P13_SF || scheme == PURIFY_FIXED_MU_P13_MONO) *j = 3;
    if (scheme == PURIFY_FIXED_MU_P31_SF || scheme == PURIFY_FIXED_MU_P31_MONO) *i = 3;
}

bool is_asymmetric(int scheme) {
    int i, j;
    pij_orders(scheme, &i, &j);
    return i != j;
}

int products_per_iteration(int scheme) {
    if (!is_fixed_mu(scheme)) return 1;
    int i, j;
    pij_orders(scheme, &i, &j);
    if (i == 3 && j == 3) return 5;
    if (i == 1 && j == 3) return 4;
    if (i == 3 && j == 1) return 3;
    return 2;
}

// P_{i,j}(x) = x^(i+1) sum_{k=0..j} C(i+k, k) (1 - x)^k: Horner in t = 1 - x,
// then the power of x by repeated multiplication (the oracle's order).
double P_ij_scalar(int i, int j, double x) {
    const double t = 1.0 - x;
    double acc = 0.0 * x;
    for (int k = j; k >= 0; --k) {
        double c = 1.0;  // C(i + k, k), exact in float64 for these orders
        for (int q = 1; q <= k; ++q) c = c * (double)(i + q) / (double)q;
        acc = acc * t + c;
    }
    double p = x;
    for (int q = 0; q < i; ++q) p = p * x;
    return p * acc;
}

// The unstable fixed point c in (0, 1) of P_{i,j} (i, j >= 1): bisection on
// the sign of P(x) - x.
double pij_fixed_point(int i, int j) {
    double lo = 1e-12, hi = 1.0 - 1e-12;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        if (P_ij_scalar(i, j, mid) - mid < 0.0)
            lo = mid;
        else
            hi = mid;
    }
    return 0.5 * (lo + hi);
}

// The alpha in [lo, hi] where g goes from positive to negative (bisection).
template <typename G>
static double fold_root(G g, double lo, double hi) {
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        if (g(mid) > 0.0)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Scaling about c for asymmetric P_{i,j}: the smaller of the unoccupied
// side's fold (P(alpha (beta - c) + c) = P(c (1 - alpha))) and the occupied
// side's (P(c + alpha (1 - c)) = P(alpha (beta_bar - c) + c)).
double pij_alpha(int i, int j, double c, double b, double bb) {
    const double au = fold_root(
        [&](double a) { return P_ij_scalar(i, j, a * (b - c) + c) - P_ij_scalar(i, j, c * (1.0 - a)); }, 1.0,
        c / (c - b));
    const double ao = fold_root(
        [&](double a) { return P_ij_scalar(i, j, c + a * (1.0 - c)) - P_ij_scalar(i, j, a * (bb - c) + c); }, 1.0,
        (1.0 - c) / (bb - c));
    return std::min(au, ao);
}

// The alpha >= 1 with P_{m,m}(alpha (beta - 1/2) + 1/2) = P_{m,m}((1 - alpha)/2):
// bisection on [1, 1 / (1 - 2 beta)] down to the last bit.
double pmm_alpha(int m, double beta) {
    double lo = 1.0, hi = 1.0 / (1.0 - 2.0 * beta);
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        const double g = P_ij_scalar(m, m, mid * (beta - 0.5) + 0.5) - P_ij_scalar(m, m, 0.5 * (1.0 - mid));
        if (g > 0.0)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

static int build_schedule(int scheme, double lmin, double lmax, double mu, double homo, double lumo,
                          double tol, int max_iter, Schedule& S) {
    if (is_asymmetric(scheme)) {
        int i, j;
        pij_orders(scheme, &i, &j);
        const double c = pij_fixed_point(i, j);
        const double gamma = std::max((mu - lmin) / (1.0 - c), (lmax - mu) / c);
        double b = c - (lumo - mu) / gamma, bb = c + (mu - homo) / gamma;
        S.beta0 = b;
        S.betabar0 = bb;
        const bool scaled = is_scaled(scheme);
        while (std::max(b, 1.0 - bb) > tol && (int)S.alpha.size() < max_iter) {
            const double a = scaled ? pij_alpha(i, j, c, b, bb) : 1.0;
            b = std::max(P_ij_scalar(i, j, a * (b - c) + c), P_ij_scalar(i, j, c * (1.0 - a)));
            bb = std::min(P_ij_scalar(i, j, a * (bb - c) + c), P_ij_scalar(i, j, c + a * (1.0 - c)));
            S.alpha.push_back(a);
            S.beta.push_back(b);
            S.betabar.push_back(bb);
            S.branch.push_back(0);
        }
        S.converged = std::max(b, 1.0 - bb) <= tol;
        return PURIFY_OK;
    }
    if (is_fixed_mu(scheme)) {
        const double gamma = fixed_mu_gamma(lmin, lmax, mu);
        double beta = fixed_mu_beta0(gamma, mu, homo, lumo);
        S.beta0 = beta;
        S.betabar0 = 1.0 - beta;
        const bool scaled = is_scaled(scheme);
        const int m = pmm_order(scheme);
        while (beta > tol && (int)S.alpha.size() < max_iter) {
            const double alpha = scaled ? (m == 1 ? fixed_mu_alpha(beta) : pmm_alpha(m, beta)) : 1.0;
            const double bs = alpha * (beta - 0.5) + 0.5;
            beta = m == 1 ? 3.0 * bs * bs - 2.0 * bs * bs * bs : P_ij_scalar(m, m, bs);
            S.alpha.push_back(alpha);
            S.beta.push_back(beta);
            S.betabar.push_back(1.0 - beta);
            S.branch.push_back(0);
        }
        S.converged = beta <= tol;
        return PURIFY_OK;
    }
    double b, bb;
    tc_beta0(lmin, lmax, homo, lumo, &b, &bb);
    S.beta0 = b;
    S.betabar0 = bb;
    const bool scaled = is_scaled(scheme);
    while (std::max(b, 1.0 - bb) > tol && (int)S.alpha.size() < max_iter) {
        const int br = tc_branch(b, bb);
        const double a = scaled ? tc_alpha(br, b, bb) : 0.0;
        const double nb = tc_map(br, a, b), nbb = tc_map(br, a, bb);
        b = nb;
        bb = nbb;
        S.alpha.push_back(a);
        S.branch.push_back(br);
        S.beta.push_back(b);
        S.betabar.push_back(bb);
    }
    S.converged = std::max(b, 1.0 - bb) <= tol;
    return PURIFY_OK;
}

int build_schedule_public(int scheme, double lmin, double lmax, double mu, double homo, double lumo,
                          double tol, int max_iter, Schedule& S) {
    return build_schedule(scheme, lmin, lmax, mu, homo, lumo, tol, max_iter, S);
}

// ---------------------------------------------------------------------------
// Cyclic Jacobi on a small symmetric matrix (Lanczos tridiagonal)
// ---------------------------------------------------------------------------

static void jacobi_eig(std::vector<double>& A, int m, std::vector<double>& V) {
    V.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) V[(size_t)i * m + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        // converged once the off-diagonal mass is below rounding relative to
        // the diagonal's (it falls quadratically: a handful of sweeps)
        double off = 0.0, diag = 0.0;
        for (int p = 0; p < m; ++p) {
            diag += A[(size_t)p * m + p] * A[(size_t)p * m + p];
            for (int q = p + 1; q < m; ++q) off += A[(size_t)p * m + q] * A[(size_t)p * m + q];
        }
        if (off == 0.0 || off <= 1e-36 * diag) break;
        for (int p = 0; p < m; ++p) {
            for (int q = p + 1; q < m; ++q) {
                const double apq = A[(size_t)p * m + q];
                if (apq == 0.0) continue;
                const double app = A[(size_t)p * m + p], aqq = A[(size_t)q * m + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) /
                                 (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < m; ++k) {  // A <- J^T A J
                    const double akp = A[(size_t)k * m + p], akq = A[(size_t)k * m + q];
                    A[(size_t)k * m + p] = c * akp - s * akq;
                    A[(size_t)k * m + q] = s * akp + c * akq;
                }
                for (int k = 0; k < m; ++k) {
                    const double apk = A[(size_t)p * m + k], aqk = A[(size_t)q * m + k];
                    A[(size_t)p * m + k] = c * apk - s * aqk;
                    A[(size_t)q * m + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < m; ++k) {
                    const double vkp = V[(size_t)k * m + p], vkq = V[(size_t)k * m + q];
                    V[(size_t)k * m + p] = c * vkp - s * vkq;
                    V[(size_t)k * m + q] = s * vkp + c * vkq;
                }
            }
        }
    }
}

void tridiag_eig_full(const double* a, const double* b, int m, std::vector<double>& w, std::vector<double>& Z) {
    std::vector<double> A((size_t)m * m, 0.0), V;
    for (int i = 0; i < m; ++i) {
        A[(size_t)i * m + i] = a[i];
        if (i + 1 < m) A[(size_t)i * m + i + 1] = A[(size_t)(i + 1) * m + i] = b[i];
    }
    jacobi_eig(A, m, V);
    std::vector<int> order(m);
    for (int i = 0; i < m; ++i) order[i] = i;
    std::sort(order.begin(), order.end(),
              [&](int x, int y) { return A[(size_t)x * m + x] < A[(size_t)y * m + y]; });
    w.assign(m, 0.0);
    Z.assign((size_t)m * m, 0.0);
    for (int j = 0; j < m; ++j) {
        const int c = order[j];
        w[j] = A[(size_t)c * m + c];
        for (int i = 0; i < m; ++i) Z[(size_t)j * m + i] = V[(size_t)i * m + c];
    }
}

int host_bounds_from_lanczos(const double* a, const double* bsq, int k, double g_lo, double g_hi,
                             double* lo, double* hi) {
    // Truncate at an exact breakdown (b_j == 0: invariant subspace found).
    int m = 0;
    std::vector<double> b(k);
    for (int j = 0; j < k; ++j) {
        b[j] = std::sqrt(std::max(bsq[j], 0.0));
        ++m;
        if (b[j] == 0.0) break;
    }
    std::vector<double> w(m), last(m);
    int r = purify_tridiag_eig(a, b.data(), m, w.data(), last.data());
    if (r != PURIFY_OK) return r;
    const double r_lo = std::fabs(b[m - 1] * last[0]);
    const double r_hi = std::fabs(b[m - 1] * last[m - 1]);
    *lo = std::max(g_lo, w[0] - r_lo);
    *hi = std::min(g_hi, w[m - 1] + r_hi);
    return PURIFY_OK;
}

}  // namespace purify

using namespace purify;

// ---------------------------------------------------------------------------
// Handle
// ---------------------------------------------------------------------------

static void free_buffers(purify_ctx* h) {
    cudaFree(h->F);
    cudaFree(h->X[0]);
    cudaFree(h->X[1]);
    cudaFree(h->S);
    cudaFree(h->P3[0]);
    cudaFree(h->P3[1]);
    h->F = h->X[0] = h->X[1] = h->S = h->P3[0] = h->P3[1] = nullptr;
    h->cap = 0;
    h->p3_cap = 0;
}

static int ensure_capacity(purify_ctx* h, int64_t n) {
    if (n <= h->cap) return PURIFY_OK;
    free_buffers(h);
    const size_t bytes = sizeof(double) * (size_t)n * (size_t)n;
    PURIFY_CUDA_TRY(cudaMalloc(&h->F, bytes));
    PURIFY_CUDA_TRY(cudaMalloc(&h->X[0], bytes));
    h->cap = n;
    return PURIFY_OK;
}

// The second iterate and the product buffer (float64 runs, refinement, gap
// estimation) at the handle's capacity, allocated on first use: block-sparse
// and mixed runs hold only F and the density.
int purify::ensure_dense_F(purify_ctx* h) {
    if (h->F_dense) return PURIFY_OK;
    if (!h->csr_valid) return PURIFY_ERR_STATE;
    PURIFY_TRY(ensure_capacity(h, h->n));
    PURIFY_CUDA_TRY(cudaMemsetAsync(h->F, 0, sizeof(double) * (size_t)h->n * (size_t)h->n, h->stream));
    PURIFY_TRY(launch_scatter_csr(csr_of(h), h->n, h->F, h->stream));
    h->F_dense = true;
    return PURIFY_OK;
}

int purify::ensure_work(purify_ctx* h) {
    if (h->X[1] && h->S) return PURIFY_OK;
    const size_t bytes = sizeof(double) * (size_t)h->cap * (size_t)h->cap;
    if (!h->X[1]) PURIFY_CUDA_TRY(cudaMalloc(&h->X[1], bytes));
    if (!h->S) PURIFY_CUDA_TRY(cudaMalloc(&h->S, bytes));
    return PURIFY_OK;
}

int purify::ensure_scratch(purify_ctx* h, int64_t doubles) {
    if (doubles <= h->scratch_cap) return PURIFY_OK;
    cudaFree(h->scratch);
    h->scratch = nullptr;
    h->scratch_cap = 0;
    PURIFY_CUDA_TRY(cudaMalloc(&h->scratch, sizeof(double) * (size_t)doubles));
    h->scratch_cap = doubles;
    return PURIFY_OK;
}

int purify::ensure_red(purify_ctx* h, int64_t doubles) {
    if (doubles <= h->red_cap) return PURIFY_OK;
    cudaFree(h->red);
    h->red = nullptr;
    h->red_cap = 0;
    PURIFY_CUDA_TRY(cudaMalloc(&h->red, sizeof(double) * (size_t)doubles));
    h->red_cap = doubles;
    return PURIFY_OK;
}

int purify::join_streams(cudaStream_t after, cudaStream_t before, cudaEvent_t ev) {
    PURIFY_CUDA_TRY(cudaEventRecord(ev, before));
    PURIFY_CUDA_TRY(cudaStreamWaitEvent(after, ev, 0));
    return PURIFY_OK;
}

int purify::copy_in_matrix(double* dst, const double* src, int64_t n, int64_t ld, cudaStream_t s) {
    cudaPointerAttributes attr;
    PURIFY_CUDA_TRY(cudaPointerGetAttributes(&attr, src));
    const bool host = attr.type == cudaMemoryTypeHost || attr.type == cudaMemoryTypeUnregistered;
    if (ld == n)
        PURIFY_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)n * n, cudaMemcpyDefault, s));
    else
        PURIFY_CUDA_TRY(cudaMemcpy2DAsync(dst, sizeof(double) * n, src, sizeof(double) * ld, sizeof(double) * n,
                                          n, cudaMemcpyDefault, s));
    if (host) PURIFY_CUDA_TRY(cudaStreamSynchronize(s));
    return PURIFY_OK;
}

static int join_in(purify_ctx* h) { return join_streams(h->stream, h->user_stream, h->join_ev); }
static int join_out(purify_ctx* h) { return join_streams(h->user_stream, h->stream, h->join_ev); }

int purify::product_begin(purify_ctx* h) {
    if (!h->opt.time_products) return PURIFY_OK;
    const size_t need = 2 * (size_t)h->pev_used + 2;
    while (h->pev.size() < need) {
        cudaEvent_t e;
        PURIFY_CUDA_TRY(cudaEventCreate(&e));
        h->pev.push_back(e);
    }
    PURIFY_CUDA_TRY(cudaEventRecord(h->pev[2 * (size_t)h->pev_used], h->stream));
    return PURIFY_OK;
}

int purify::product_end(purify_ctx* h) {
    if (!h->opt.time_products) return PURIFY_OK;
    PURIFY_CUDA_TRY(cudaEventRecord(h->pev[2 * (size_t)h->pev_used + 1], h->stream));
    ++h->pev_used;
    return PURIFY_OK;
}

double purify::product_seconds(purify_ctx* h) {
    if (!h->opt.time_products) return NAN;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return NAN;
    double s = 0.0;
    for (int i = 0; i < h->pev_used; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->pev[2 * (size_t)i], h->pev[2 * (size_t)i + 1]) != cudaSuccess)
            return NAN;
        s += 1e-3 * ms;
    }
    return s;
}

static int set_device(purify_ctx* h) {
    PURIFY_CUDA_TRY(cudaSetDevice(h->device));
    return PURIFY_OK;
}

extern "C" {

void purify_options_default(purify_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = PURIFY_FP64;
    opt->branch_rule = PURIFY_BRANCH_BETA;
    opt->lanczos_steps = 16;
    opt->refine_squares = 0;
    opt->digits = 0;
    opt->block_sparse = 0;
    opt->split_k = 1;
    opt->refine_fp64 = 0;
    opt->trunc_tau = 1e-6;
    opt->trunc_budget = 0.0;
}

static int check_options(const purify_options* o) {
    if (o->precision != PURIFY_FP64 && o->precision != PURIFY_MIXED) return PURIFY_ERR_INVALID_ARG;
    if (o->branch_rule != PURIFY_BRANCH_BETA && o->branch_rule != PURIFY_BRANCH_TRACE)
        return PURIFY_ERR_INVALID_ARG;
    if (o->lanczos_steps < 0 || o->lanczos_steps > 512) return PURIFY_ERR_INVALID_ARG;
    if (o->refine_squares < 0 || o->refine_squares > 8) return PURIFY_ERR_INVALID_ARG;
    if (o->digits != 0 && (o->digits < 2 || o->digits > kMaxDigits)) return PURIFY_ERR_INVALID_ARG;
    if (o->block_sparse != 0 && o->block_sparse != 1) return PURIFY_ERR_INVALID_ARG;
    if (o->split_k != 0 && o->split_k != 1) return PURIFY_ERR_INVALID_ARG;
    if (o->refine_fp64 < 0 || o->refine_fp64 > 2) return PURIFY_ERR_INVALID_ARG;
    if (o->bits_floor != 0 && (o->bits_floor < 16 || o->bits_floor > 43)) return PURIFY_ERR_INVALID_ARG;
    if (o->bits_gap != 0 && (o->bits_gap < 16 || o->bits_gap > 43)) return PURIFY_ERR_INVALID_ARG;
    if (o->autotune != 0 && o->autotune != 1) return PURIFY_ERR_INVALID_ARG;
    if (o->wait_kcycles < 0 || o->wait_kcycles > (1 << 21)) return PURIFY_ERR_INVALID_ARG;
    if (o->host_schedule != 0 && o->host_schedule != 1) return PURIFY_ERR_INVALID_ARG;
    if (!(o->trunc_tau >= 0.0) || !(o->trunc_budget >= 0.0)) return PURIFY_ERR_INVALID_ARG;
    return PURIFY_OK;
}

int purify_create(purify_t* out, int device, void* cuda_stream, const purify_options* opt) {
    if (!out) return PURIFY_ERR_INVALID_ARG;
    *out = nullptr;
    purify_options o;
    purify_options_default(&o);
    if (opt) o = *opt;
    PURIFY_TRY(check_options(&o));
    int ndev = 0;
    PURIFY_CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return PURIFY_ERR_INVALID_ARG;
    cudaDeviceProp prop;
    PURIFY_CUDA_TRY(cudaGetDeviceProperties(&prop, device));
    if (!(prop.major == 10 && prop.minor == 3)) return PURIFY_ERR_UNSUPPORTED;
    purify_ctx* h = new (std::nothrow) purify_ctx();
    if (!h) return PURIFY_ERR_OOM;
    h->device = device;
    h->opt = o;
    int r = set_device(h);
    if (r == PURIFY_OK) {
        h->user_stream = (cudaStream_t)cuda_stream;
        cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) r = cuda_status(e, "cudaStreamCreateWithFlags");
        h->own_stream = (e == cudaSuccess);
    }
    if (r == PURIFY_OK) {
        cudaError_t e = cudaEventCreate(&h->e0);
        if (e == cudaSuccess) e = cudaEventCreate(&h->e1);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming);
        if (e != cudaSuccess) r = cuda_status(e, "cudaEventCreate");
    }
    if (r != PURIFY_OK) {
        purify_destroy(h);
        return r;
    }
    h->st.status = PURIFY_ERR_STATE;
    *out = h;
    return PURIFY_OK;
}

int purify_destroy(purify_t h) {
    if (!h) return PURIFY_OK;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_buffers(h);
    cudaFree(h->red);
    cudaFree(h->scratch);
    cudaFree(h->csr_ptr);
    cudaFree(h->csr_col);
    cudaFree(h->csr_val);
    mixed_free(h->mixed);
    for (cudaEvent_t e : h->pev) cudaEventDestroy(e);
    if (h->e0) cudaEventDestroy(h->e0);
    if (h->e1) cudaEventDestroy(h->e1);
    if (h->join_ev) cudaEventDestroy(h->join_ev);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return PURIFY_OK;
}

int purify_set_options(purify_t h, const purify_options* opt) {
    if (!h || !opt) return PURIFY_ERR_INVALID_ARG;
    PURIFY_TRY(check_options(opt));
    h->opt = *opt;
    return PURIFY_OK;
}

const double* purify_density_device_ptr(purify_t h) {
    if (!h || h->cur < 0 || (h->mixed && h->mixed->d_pooled)) return nullptr;
    return h->X[h->cur];
}

// The part of loading a Hamiltonian after h->F (n x n, dense) holds it:
// bounds (estimated when NaN), validation, statistics.
static int finish_set(purify_t h, int64_t n, int64_t nocc, double mu, const purify_bounds* b,
                      long long set_launches0) {
    purify_bounds bb = *b;
    if (std::isnan(bb.lmin) || std::isnan(bb.lmax)) {
        const int k = (int)std::min<int64_t>(h->opt.lanczos_steps, n);
        const int64_t need = 2 + gershgorin_scratch_doubles(n) + (k > 0 ? lanczos_scratch_doubles(n, k) : 0);
        PURIFY_TRY(ensure_scratch(h, need));
        double* lohi = h->scratch;
        double* gs = h->scratch + 2;
        const bool csr = h->csr_valid && !h->F_dense;
        const CsrF cf = csr_of(h);
        if (csr)
            PURIFY_TRY(launch_gershgorin_csr_f64(cf, n, lohi, gs, h->stream));
        else
            PURIFY_TRY(launch_gershgorin_f64(h->F, n, n, lohi, gs, h->stream));
        double g[2];
        double lo, hi;
        if (k > 0) {
            // the Lanczos steps are queued before any result is read back, so
            // the device runs the whole estimate without a host round trip
            double* ls = h->scratch + 2;  // Gershgorin partials are consumed already
            PURIFY_TRY(launch_lanczos_f64(h->F, n, k, ls, h->stream, csr ? &cf : nullptr));
            PURIFY_CUDA_TRY(cudaMemcpyAsync(g, lohi, sizeof(g), cudaMemcpyDeviceToHost, h->stream));
            std::vector<double> a(k), bsq(k);
            PURIFY_CUDA_TRY(cudaMemcpyAsync(a.data(), ls + lanczos_a_offset(n), sizeof(double) * k,
                                            cudaMemcpyDeviceToHost, h->stream));
            PURIFY_CUDA_TRY(cudaMemcpyAsync(bsq.data(), ls + lanczos_bsq_offset(n, k),
                                            sizeof(double) * k, cudaMemcpyDeviceToHost, h->stream));
            PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
            PURIFY_TRY(host_bounds_from_lanczos(a.data(), bsq.data(), k, g[0], g[1], &lo, &hi));
        } else {
            PURIFY_CUDA_TRY(cudaMemcpyAsync(g, lohi, sizeof(g), cudaMemcpyDeviceToHost, h->stream));
            PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
            lo = g[0];
            hi = g[1];
        }
        if (std::isnan(bb.lmin)) bb.lmin = lo;
        if (std::isnan(bb.lmax)) bb.lmax = hi;
        // Estimated extremes never cut into the given gap edges.
        if (!std::isnan(bb.homo)) bb.lmin = std::min(bb.lmin, bb.homo);
        if (!std::isnan(bb.lumo)) bb.lmax = std::max(bb.lmax, bb.lumo);
    }
    if (!(bb.lmax > bb.lmin)) return PURIFY_ERR_BOUNDS;
    if (!std::isnan(bb.homo) && !std::isnan(bb.lumo)) {
        if (!(bb.homo < bb.lumo)) return PURIFY_ERR_BOUNDS;
        if (bb.homo < bb.lmin || bb.lumo > bb.lmax) return PURIFY_ERR_BOUNDS;
    }
    const int set_launches = (int)(launches_so_far() - set_launches0);
    h->b = bb;
    h->nocc = nocc;
    h->mu = mu;
    std::memset(&h->st, 0, sizeof(h->st));
    h->st.status = PURIFY_ERR_STATE;
    h->st.lmin = bb.lmin;
    h->st.lmax = bb.lmax;
    h->st.homo = bb.homo;
    h->st.lumo = bb.lumo;
    h->st.mu = mu;
    h->st.kernel_launches = set_launches;
    h->st.product_seconds = NAN;
    h->have_F = true;
    return join_out(h);
}

int purify_set_hamiltonian(purify_t h, const double* F, int64_t n, int64_t ld, int64_t nocc,
                           double mu, const purify_bounds* b) {
    if (!h || !F || !b || n <= 0 || ld < n) return PURIFY_ERR_INVALID_ARG;
    if (nocc > n) return PURIFY_ERR_INVALID_ARG;
    if (n > (int64_t)1 << 17) return PURIFY_ERR_INVALID_ARG;
    PURIFY_TRY(set_device(h));
    const long long set_launches0 = launches_so_far();
    h->have_F = false;
    h->cur = -1;
    PURIFY_TRY(join_in(h));
    PURIFY_TRY(ensure_capacity(h, n));
    h->n = n;
    h->csr_valid = false;
    h->F_dense = false;
    PURIFY_TRY(copy_in_matrix(h->F, F, n, ld, h->stream));
    PURIFY_TRY(launch_mirror_upper_f64(h->F, n, h->stream));
    h->F_dense = true;
    return finish_set(h, n, nocc, mu, b, set_launches0);
}

int purify_set_hamiltonian_coo(purify_t h, int64_t n, int64_t nnz, const int64_t* rows,
                               const int64_t* cols, const double* vals, int64_t nocc, double mu,
                               const purify_bounds* b) {
    if (!h || !b || n <= 0 || nnz < 0 || (nnz > 0 && (!rows || !cols || !vals))) return PURIFY_ERR_INVALID_ARG;
    // a block-sparse mixed handle keeps F in CSR form (no n x n array), so
    // it takes larger n
    const bool csr_mode = h->opt.block_sparse && h->opt.precision == PURIFY_MIXED;
    if (nocc > n || n > (int64_t)1 << (csr_mode ? 18 : 17)) return PURIFY_ERR_INVALID_ARG;
    for (int64_t k = 0; k < nnz; ++k)
        if (rows[k] < 0 || rows[k] >= n || cols[k] < 0 || cols[k] >= n) return PURIFY_ERR_INVALID_ARG;
    // merge duplicates (summed in input order, so the result does not depend
    // on the device's scheduling) and require (i, j) and (j, i) to agree
    std::vector<int64_t> perm(nnz), key(nnz);
    for (int64_t k = 0; k < nnz; ++k) {
        perm[k] = k;
        key[k] = rows[k] * n + cols[k];
    }
    std::stable_sort(perm.begin(), perm.end(), [&](int64_t a, int64_t b) { return key[a] < key[b]; });
    std::vector<int64_t> ukey;
    std::vector<double> uval;
    ukey.reserve(nnz);
    uval.reserve(nnz);
    for (int64_t q = 0; q < nnz; ++q) {
        const int64_t k = perm[q];
        if (!ukey.empty() && ukey.back() == key[k])
            uval.back() += vals[k];
        else {
            ukey.push_back(key[k]);
            uval.push_back(vals[k]);
        }
    }
    for (size_t u = 0; u < ukey.size(); ++u) {
        const int64_t t = (ukey[u] % n) * n + ukey[u] / n;
        const auto it = std::lower_bound(ukey.begin(), ukey.end(), t);
        if (it == ukey.end() || *it != t || uval[it - ukey.begin()] != uval[u]) return PURIFY_ERR_INVALID_ARG;
    }
    nnz = (int64_t)ukey.size();
    PURIFY_TRY(set_device(h));
    const long long set_launches0 = launches_so_far();
    h->have_F = false;
    h->cur = -1;
    h->csr_valid = false;
    h->F_dense = false;
    PURIFY_TRY(join_in(h));
    if (csr_mode) {
        // rows and columns in key order: CSR with sorted columns; F's block
        // pattern (with the diagonal) for the block-sparse split
        std::vector<int64_t> ptr(n + 1, 0);
        std::vector<int> col(nnz);
        const int nb = pad128(n) / 32, words = (nb + 63) / 64;
        h->f_pattern.assign((size_t)nb * words, 0);
        h->f_pattern_words = words;
        for (int64_t u = 0; u < nnz; ++u) {
            const int64_t i = ukey[u] / n, j = ukey[u] % n;
            ++ptr[i + 1];
            col[u] = (int)j;
            h->f_pattern[(size_t)(i >> 5) * words + (j >> 11)] |= 1ull << ((j >> 5) & 63);
        }
        for (int I = 0; I < nb; ++I) h->f_pattern[(size_t)I * words + (I >> 6)] |= 1ull << (I & 63);
        for (int64_t i = 0; i < n; ++i) ptr[i + 1] += ptr[i];
        free_buffers(h);  // an earlier dense F and density
        if (h->csr_rows_cap < n + 1) {
            cudaFree(h->csr_ptr);
            h->csr_ptr = nullptr;
            h->csr_rows_cap = 0;
            PURIFY_CUDA_TRY(cudaMalloc(&h->csr_ptr, sizeof(int64_t) * (size_t)(n + 1)));
            h->csr_rows_cap = n + 1;
        }
        if (h->csr_nnz_cap < std::max<int64_t>(nnz, 1)) {
            cudaFree(h->csr_col);
            cudaFree(h->csr_val);
            h->csr_col = nullptr;
            h->csr_val = nullptr;
            h->csr_nnz_cap = 0;
            const int64_t c = std::max<int64_t>(nnz, 1);
            PURIFY_CUDA_TRY(cudaMalloc(&h->csr_col, sizeof(int) * (size_t)c));
            PURIFY_CUDA_TRY(cudaMalloc(&h->csr_val, sizeof(double) * (size_t)c));
            h->csr_nnz_cap = c;
        }
        PURIFY_CUDA_TRY(cudaMemcpyAsync(h->csr_ptr, ptr.data(), sizeof(int64_t) * ptr.size(), cudaMemcpyHostToDevice,
                                        h->stream));
        if (nnz > 0) {
            PURIFY_CUDA_TRY(cudaMemcpyAsync(h->csr_col, col.data(), sizeof(int) * (size_t)nnz, cudaMemcpyHostToDevice,
                                            h->stream));
            PURIFY_CUDA_TRY(cudaMemcpyAsync(h->csr_val, uval.data(), sizeof(double) * (size_t)nnz,
                                            cudaMemcpyHostToDevice, h->stream));
        }
        PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));  // the host arrays go out of scope
        h->n = n;
        h->csr_nnz = nnz;
        h->csr_valid = true;
        return finish_set(h, n, nocc, mu, b, set_launches0);
    }
    PURIFY_TRY(ensure_capacity(h, n));
    h->n = n;
    PURIFY_CUDA_TRY(cudaMemsetAsync(h->F, 0, sizeof(double) * (size_t)n * n, h->stream));
    if (nnz > 0) {
        PURIFY_TRY(ensure_scratch(h, 2 * nnz));
        int64_t* dk = (int64_t*)h->scratch;
        double* dv = (double*)(dk + nnz);
        PURIFY_CUDA_TRY(cudaMemcpyAsync(dk, ukey.data(), sizeof(int64_t) * nnz, cudaMemcpyHostToDevice, h->stream));
        PURIFY_CUDA_TRY(cudaMemcpyAsync(dv, uval.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice, h->stream));
        PURIFY_TRY(launch_scatter_coo(dk, dv, nnz, h->F, h->stream));
        PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));  // the scratch is reused below
    }
    h->F_dense = true;
    return finish_set(h, n, nocc, mu, b, set_launches0);
}

int purify_block_history(purify_t h, int* nnz_blocks, int cap, int* count) {
    if (!h || !count || cap < 0 || (cap > 0 && !nnz_blocks)) return PURIFY_ERR_INVALID_ARG;
    if (!h->mixed) {
        *count = 0;
        return PURIFY_OK;
    }
    const std::vector<int>& hist = h->mixed->nnzb_history;
    *count = (int)hist.size();
    for (int i = 0; i < cap && i < (int)hist.size(); ++i) nnz_blocks[i] = hist[i];
    return PURIFY_OK;
}

// One float64 step with reductions into slot `slot` (4 doubles).
static int step64(purify_ctx* h, const double* A, const double* B, const double* E, double* C,
                  double cP, double cE, double cI, double dY, double dI, int64_t slot) {
    PURIFY_TRY(product_begin(h));
    PURIFY_TRY(launch_step_f64(A, B, E, C, h->n, cP, cE, cI, dY, dI, h->red + 4 * slot, h->stream));
    ++h->st.product_launches;
    return product_end(h);
}

// Coefficients of the Algorithm 2 step on X: Y = cP X^2 + cE X + cI I.
static void tc_coeffs(int branch, double a, double* cP, double* cE, double* cI) {
    if (branch) {  // ((1 + a) X - a I)^2
        *cP = sq1p(a);
        *cE = -2.0 * a * (1.0 + a);
        *cI = a * a;
    } else {  // 2 (1 + a) X - (1 + a)^2 X^2
        *cP = -sq1p(a);
        *cE = 2.0 * (1.0 + a);
        *cI = 0.0;
    }
}

// Float64 McWeeny steps X <- 3 X^2 - 2 X^3 on the current density (the
// refinement squares that set the final idempotency after a mixed run).
// Sets the trace of the last result and ||X - X^2||_F of its input.
static int refine_f64(purify_ctx* h, int R) {
    if (R <= 0 || h->cur < 0) return PURIFY_OK;
    if (h->mixed && h->mixed->d_pooled) return PURIFY_ERR_UNSUPPORTED;  // a block-sparse density
    PURIFY_TRY(ensure_work(h));
    PURIFY_TRY(ensure_red(h, 4 * (int64_t)(2 * R)));
    PURIFY_CUDA_TRY(cudaMemsetAsync(h->red, 0, sizeof(double) * 8 * R, h->stream));
    int x = h->cur;
    for (int r = 0; r < R; ++r) {
        double* X = h->X[x];
        // S = X^2, reducing ||X - X^2||_F^2 (E = X)
        PURIFY_TRY(step64(h, X, X, X, h->S, 1.0, 0.0, 0.0, 1.0, 0.0, 2 * r));
        // X' = 3 S - 2 S X
        PURIFY_TRY(step64(h, h->S, X, h->S, h->X[x ^ 1], -2.0, 3.0, 0.0, 1.0, 0.0, 2 * r + 1));
        x ^= 1;
    }
    h->cur = x;
    PURIFY_CUDA_TRY(cudaEventRecord(h->e1, h->stream));
    std::vector<double> red(8 * (size_t)R);
    PURIFY_CUDA_TRY(cudaMemcpyAsync(red.data(), h->red, sizeof(double) * red.size(), cudaMemcpyDeviceToHost,
                                    h->stream));
    PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->st.trace = red[4 * (size_t)(2 * R - 1)];
    h->st.idem_err_fro = std::sqrt(std::max(red[4 * (size_t)(2 * R - 2) + 1], 0.0));
    h->st.refine_multiplications += 2 * R;
    return PURIFY_OK;
}

static int run_fp64(purify_ctx* h, int scheme, double tol, int max_iter, double mu, Schedule& S,
                    bool trace_rule, int* iters_out, std::vector<double>& red_host) {
    PURIFY_TRY(ensure_work(h));
    const int64_t n = h->n;
    const double lmin = h->b.lmin, lmax = h->b.lmax;
    int m = (int)S.alpha.size();
    if (is_fixed_mu(scheme) && (pmm_order(scheme) == 3 || is_asymmetric(scheme))) {
        // Higher-order and asymmetric P_{i,j}, scaled about c (1/2 when i = j):
        //   P_{3,3} = x^4 (35 - 84x + 70x^2 - 20x^3): V = 70 X_s - 20 X_s^2,
        //     Q = X_s V - 84 X_s + 35 I, S = X_s^2, T = S^2 (over V), X = T Q;
        //   P_{3,1} = x^4 (5 - 4x): S = X_s^2, T = S^2, X = 5 T - 4 T X_s;
        //   P_{1,3} = x^2 (10 - 20x + 15x^2 - 4x^3): V = 15 X_s - 4 X_s^2,
        //     Q = X_s V - 20 X_s + 10 I, S = X_s^2, X = S Q;
        // the last product also applies the next iteration's scaling.
        int pi, pj;
        pij_orders(scheme, &pi, &pj);
        const double c = pi == pj ? 0.5 : pij_fixed_point(pi, pj);
        const double gamma = std::max((mu - lmin) / (1.0 - c), (lmax - mu) / c);
        const int ppi = products_per_iteration(scheme);
        if (h->p3_cap < n) {
            cudaFree(h->P3[0]);
            cudaFree(h->P3[1]);
            h->P3[0] = h->P3[1] = nullptr;
            h->p3_cap = 0;
            PURIFY_CUDA_TRY(cudaMalloc(&h->P3[0], sizeof(double) * (size_t)n * n));
            PURIFY_CUDA_TRY(cudaMalloc(&h->P3[1], sizeof(double) * (size_t)n * n));
            h->p3_cap = n;
        }
        PURIFY_TRY(ensure_red(h, 4 * (int64_t)(ppi * m + 2)));
        PURIFY_CUDA_TRY(cudaMemsetAsync(h->red, 0, sizeof(double) * 4 * (ppi * m + 2), h->stream));
        PURIFY_CUDA_TRY(cudaEventRecord(h->e0, h->stream));
        if (m == 0) {  // X_0 = c I + (mu I - F) / gamma
            PURIFY_TRY(launch_affine_f64(h->F, n, h->X[0], n, -1.0 / gamma, c + mu / gamma, h->stream));
            h->cur = 0;
        } else {
            // X_s = c I + alpha_1 (X_0 - c I)
            const double a1 = S.alpha[0];
            PURIFY_TRY(launch_affine_f64(h->F, n, h->X[0], n, -a1 / gamma, c + a1 * mu / gamma, h->stream));
            int xs = 0;
            double* V = h->P3[0];
            double* Q = h->P3[1];
            for (int i = 0; i < m; ++i) {
                double* Xs = h->X[xs];
                double* Xn = h->X[xs ^ 1];
                const double an = (i + 1 < m) ? S.alpha[i + 1] : 1.0;
                const double dY = an, dI = c * (1.0 - an);
                const int sl = ppi * i;
                if (pi == 3 && pj == 3) {
                    PURIFY_TRY(step64(h, Xs, Xs, Xs, V, -20.0, 70.0, 0.0, 1.0, 0.0, sl));
                    PURIFY_TRY(step64(h, Xs, V, Xs, Q, 1.0, -84.0, 35.0, 1.0, 0.0, sl + 1));
                    PURIFY_TRY(step64(h, Xs, Xs, nullptr, h->S, 1.0, 0.0, 0.0, 1.0, 0.0, sl + 2));
                    PURIFY_TRY(step64(h, h->S, h->S, nullptr, V, 1.0, 0.0, 0.0, 1.0, 0.0, sl + 3));
                    PURIFY_TRY(step64(h, V, Q, nullptr, Xn, 1.0, 0.0, 0.0, dY, dI, sl + 4));
                } else if (pi == 3) {  // P_{3,1}
                    PURIFY_TRY(step64(h, Xs, Xs, nullptr, h->S, 1.0, 0.0, 0.0, 1.0, 0.0, sl));
                    PURIFY_TRY(step64(h, h->S, h->S, nullptr, V, 1.0, 0.0, 0.0, 1.0, 0.0, sl + 1));
                    PURIFY_TRY(step64(h, V, Xs, V, Xn, -4.0, 5.0, 0.0, dY, dI, sl + 2));
                } else {  // P_{1,3}
                    PURIFY_TRY(step64(h, Xs, Xs, Xs, V, -4.0, 15.0, 0.0, 1.0, 0.0, sl));
                    PURIFY_TRY(step64(h, Xs, V, Xs, Q, 1.0, -20.0, 10.0, 1.0, 0.0, sl + 1));
                    PURIFY_TRY(step64(h, Xs, Xs, nullptr, h->S, 1.0, 0.0, 0.0, 1.0, 0.0, sl + 2));
                    PURIFY_TRY(step64(h, h->S, Q, nullptr, Xn, 1.0, 0.0, 0.0, dY, dI, sl + 3));
                }
                xs ^= 1;
            }
            h->cur = xs;
        }
        PURIFY_CUDA_TRY(cudaEventRecord(h->e1, h->stream));
        red_host.assign(4 * (size_t)(ppi * m + 2), 0.0);
        PURIFY_CUDA_TRY(cudaMemcpyAsync(red_host.data(), h->red, sizeof(double) * red_host.size(),
                                        cudaMemcpyDeviceToHost, h->stream));
        PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
        *iters_out = m;
        return PURIFY_OK;
    }
    if (is_fixed_mu(scheme)) {
        // X_s of the first iteration straight from F: X_0 = c0 I + c1 F.
        const double gamma = fixed_mu_gamma(lmin, lmax, mu);
        const double c0 = mu / gamma + 0.5, c1 = -1.0 / gamma;
        PURIFY_TRY(ensure_red(h, 4 * (int64_t)(2 * m + 2)));
        PURIFY_CUDA_TRY(cudaMemsetAsync(h->red, 0, sizeof(double) * 4 * (2 * m + 2), h->stream));
        PURIFY_CUDA_TRY(cudaEventRecord(h->e0, h->stream));
        if (m == 0) {
            PURIFY_TRY(launch_affine_f64(h->F, n, h->X[0], n, c1, c0, h->stream));
            h->cur = 0;
        } else {
            const double a1 = S.alpha[0];
            PURIFY_TRY(launch_affine_f64(h->F, n, h->X[0], n, a1 * c1, a1 * (c0 - 0.5) + 0.5, h->stream));
            int xs = 0;
            for (int i = 0; i < m; ++i) {
                // S = X_s^2
                PURIFY_TRY(step64(h, h->X[xs], h->X[xs], nullptr, h->S, 1.0, 0.0, 0.0, 1.0, 0.0, 2 * i));
                // X_i = 3 S - 2 S X_s, emitted as the next X_s (or as D after the last)
                const double an = (i + 1 < m) ? S.alpha[i + 1] : 1.0;
                const double dY = an, dI = 0.5 * (1.0 - an);
                PURIFY_TRY(step64(h, h->S, h->X[xs], h->S, h->X[xs ^ 1], -2.0, 3.0, 0.0, dY, dI, 2 * i + 1));
                xs ^= 1;
            }
            h->cur = xs;
        }
        PURIFY_CUDA_TRY(cudaEventRecord(h->e1, h->stream));
        red_host.assign(4 * (size_t)(2 * m + 2), 0.0);
        PURIFY_CUDA_TRY(cudaMemcpyAsync(red_host.data(), h->red, sizeof(double) * red_host.size(),
                                        cudaMemcpyDeviceToHost, h->stream));
        PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
        *iters_out = m;
        return PURIFY_OK;
    }
    // Algorithm 2
    const double w = lmax - lmin;
    const double c0 = lmax / w, c1 = -1.0 / w;
    const int slots = (trace_rule ? max_iter : m) + 2;
    PURIFY_TRY(ensure_red(h, 4 * (int64_t)slots));
    PURIFY_CUDA_TRY(cudaMemsetAsync(h->red, 0, sizeof(double) * 4 * slots, h->stream));
    PURIFY_CUDA_TRY(cudaEventRecord(h->e0, h->stream));
    PURIFY_TRY(launch_affine_f64(h->F, n, h->X[0], n, c1, c0, h->stream));
    int x = 0;
    if (!trace_rule) {
        for (int i = 0; i < m; ++i) {
            double cP, cE, cI;
            tc_coeffs(S.branch[i], S.alpha[i], &cP, &cE, &cI);
            PURIFY_TRY(step64(h, h->X[x], h->X[x], h->X[x], h->X[x ^ 1], cP, cE, cI, 1.0, 0.0, i));
            x ^= 1;
        }
        h->cur = x;
        PURIFY_CUDA_TRY(cudaEventRecord(h->e1, h->stream));
        red_host.assign(4 * (size_t)slots, 0.0);
        PURIFY_CUDA_TRY(cudaMemcpyAsync(red_host.data(), h->red, sizeof(double) * red_host.size(),
                                        cudaMemcpyDeviceToHost, h->stream));
        PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
        *iters_out = m;
        return PURIFY_OK;
    }
    // Trace rule: the branch of step i needs trace(X_{i-1}); one host round
    // trip per step.  Slot max_iter + 1 holds trace(X_0).
    const bool have_gap = !std::isnan(h->b.homo) && !std::isnan(h->b.lumo);
    const bool scaled = is_scaled(scheme);
    double b = S.beta0, bb = S.betabar0;
    S.alpha.clear();
    S.branch.clear();
    S.beta.clear();
    S.betabar.clear();
    double* tr0 = h->red + 4 * (int64_t)(max_iter + 1);
    PURIFY_TRY(launch_trace_f64(h->X[0], n, tr0, h->stream));
    double tr_prev;
    PURIFY_CUDA_TRY(cudaMemcpyAsync(&tr_prev, tr0, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
    int it = 0;
    bool done = have_gap && std::max(b, 1.0 - bb) <= tol;
    while (!done && it < max_iter) {
        const int br = tr_prev > (double)h->nocc ? 1 : 0;
        const double a = scaled ? tc_alpha(br, b, bb) : 0.0;
        double cP, cE, cI;
        tc_coeffs(br, a, &cP, &cE, &cI);
        PURIFY_TRY(step64(h, h->X[x], h->X[x], h->X[x], h->X[x ^ 1], cP, cE, cI, 1.0, 0.0, it));
        x ^= 1;
        double r[4];
        PURIFY_CUDA_TRY(cudaMemcpyAsync(r, h->red + 4 * it, sizeof(r), cudaMemcpyDeviceToHost, h->stream));
        PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
        tr_prev = r[0];
        if (have_gap) {
            const double nb = tc_map(br, a, b), nbb = tc_map(br, a, bb);
            b = nb;
            bb = nbb;
        }
        S.alpha.push_back(a);
        S.branch.push_back(br);
        S.beta.push_back(b);
        S.betabar.push_back(bb);
        ++it;
        if (have_gap) done = std::max(b, 1.0 - bb) <= tol;
        else done = std::sqrt(std::max(r[1], 0.0)) <= tol;
    }
    S.converged = done;
    h->cur = x;
    PURIFY_CUDA_TRY(cudaEventRecord(h->e1, h->stream));
    red_host.assign(4 * (size_t)slots, 0.0);
    PURIFY_CUDA_TRY(cudaMemcpyAsync(red_host.data(), h->red, sizeof(double) * red_host.size(),
                                    cudaMemcpyDeviceToHost, h->stream));
    PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
    *iters_out = it;
    return PURIFY_OK;
}

int purify_run(purify_t h, int scheme, double tol, int max_iter) {
    if (!h) return PURIFY_ERR_INVALID_ARG;
    if (!h->have_F) return PURIFY_ERR_STATE;
    if (scheme < PURIFY_FIXED_MU_SF || scheme > PURIFY_SCHEME_LAST) return PURIFY_ERR_INVALID_ARG;
    if (!(tol >= 0.0) || max_iter < 0 || max_iter > 10000) return PURIFY_ERR_INVALID_ARG;
    PURIFY_TRY(set_device(h));
    const purify_bounds& bb = h->b;
    const bool have_gap = !std::isnan(bb.homo) && !std::isnan(bb.lumo);
    const bool trace_rule = !is_fixed_mu(scheme) && h->opt.branch_rule == PURIFY_BRANCH_TRACE;
    double mu = h->mu;
    if (is_fixed_mu(scheme)) {
        if (!have_gap) return PURIFY_ERR_BOUNDS;
        if (std::isnan(mu)) mu = 0.5 * (bb.homo + bb.lumo);
        if (!(std::min(mu - bb.homo, bb.lumo - mu) > 0.0)) return PURIFY_ERR_BOUNDS;
        if (mu <= bb.lmin || mu >= bb.lmax) return PURIFY_ERR_BOUNDS;
    } else {
        if (trace_rule) {
            if (h->nocc < 0) return PURIFY_ERR_INVALID_ARG;
            if (scheme == PURIFY_TC_SF && !have_gap) return PURIFY_ERR_BOUNDS;
        } else if (!have_gap) {
            return PURIFY_ERR_BOUNDS;
        }
    }
    Schedule S;
    if (have_gap)
        PURIFY_TRY(build_schedule(scheme, bb.lmin, bb.lmax, mu, bb.homo, bb.lumo, tol, max_iter, S));
    PURIFY_TRY(join_in(h));
    h->cur = -1;
    const long long launches0 = launches_so_far();
    h->pev_used = 0;
    h->st.product_launches = 0;
    h->st.refine_multiplications = 0;
    h->st.tensor_flops = 0.0;
    h->st.digit_max = 0;
    h->st.device_flag = 0;
    h->hist_trace.clear();
    h->hist_idem.clear();
    std::vector<double> red;
    int iters = 0;
    int r;
    bool graph_run = false;  // products replayed from a graph are not timed one by one
    if (h->opt.block_sparse && h->opt.precision != PURIFY_MIXED) return PURIFY_ERR_UNSUPPORTED;
    if (h->mixed) h->mixed->d_pooled = false;
    const bool pooled_run = h->opt.precision == PURIFY_MIXED && h->opt.block_sparse && !trace_rule &&
                            pmm_order(scheme) != 3 && !is_asymmetric(scheme);
    if (!pooled_run) PURIFY_TRY(ensure_dense_F(h));
    if (h->opt.precision == PURIFY_MIXED) {
        if (trace_rule && h->opt.block_sparse) return PURIFY_ERR_UNSUPPORTED;
        if (trace_rule) {
            // the device-side schedule, unless the host one is asked for or
            // the bounds already meet tol before the first step
            const bool at_start = have_gap && std::max(S.beta0, 1.0 - S.betabar0) <= tol;
            if (h->opt.host_schedule || at_start || max_iter == 0) {
                r = run_mixed_trace(h, scheme, tol, max_iter, S, &h->cur, &iters);
            } else {
                r = run_mixed_trace_graph(h, scheme, tol, max_iter, S, &h->cur, &iters);
                graph_run = true;
            }
        } else if (h->opt.block_sparse && (pmm_order(scheme) == 3 || is_asymmetric(scheme))) {
            r = PURIFY_ERR_UNSUPPORTED;
        } else if (pmm_order(scheme) == 3 || is_asymmetric(scheme)) {
            r = run_mixed_poly(h, scheme, mu, S, &h->cur, red);
        } else if (h->opt.block_sparse) {
            r = run_block_sparse(h, scheme, S, &h->cur, red);
            if (r == PURIFY_OK && h->mixed && !h->mixed->nnzb_history.empty())
                h->st.nnz_blocks = h->mixed->nnzb_history.back();
        } else {
            r = run_mixed(h, scheme, mu, S, &h->cur, red);
        }
        if (r == PURIFY_OK) r = refine_f64(h, h->opt.refine_fp64);
        if (!trace_rule) iters = (int)S.alpha.size();
    } else {
        r = run_fp64(h, scheme, tol, max_iter, mu, S, trace_rule, &iters, red);
    }
    if (r != PURIFY_OK) {
        h->st.status = r;
        return r;
    }
    float ms = 0.f;
    PURIFY_CUDA_TRY(cudaEventElapsedTime(&ms, h->e0, h->e1));
    purify_stats_t& st = h->st;
    const int mult_per_it = products_per_iteration(scheme);
    st.iterations = iters;
    st.multiplications = mult_per_it * iters + st.refine_multiplications;
    st.seconds = 1e-3 * ms;
    st.mu = mu;
    st.err_bound = iters > 0 ? std::max(S.beta[iters - 1], 1.0 - S.betabar[iters - 1])
                             : std::max(S.beta0, 1.0 - S.betabar0);
    const double nn = (double)h->n;
    st.useful_flops = (double)st.multiplications * nn * nn * (nn + 1.0);
    // trace(X_n) and idempotency of the last squared iterate
    double trace = NAN, idem = NAN;
    if (h->opt.precision == PURIFY_MIXED) {
        trace = st.trace;
        idem = st.idem_err_fro;
    } else if (iters > 0) {
        if (is_fixed_mu(scheme)) {
            const int ppi = products_per_iteration(scheme);
            trace = red[4 * (size_t)(ppi * (iters - 1) + ppi - 1) + 0];
        } else {
            trace = red[4 * (size_t)(iters - 1) + 0];
            idem = std::sqrt(std::max(red[4 * (size_t)(iters - 1) + 1], 0.0));
        }
    }
    st.trace = trace;
    st.idem_err_fro = idem;
    // per-iteration reductions: the trace of X_i and, for Algorithm 2, the
    // idempotency of the squared X_{i-1}, from each iteration's last product.
    // The trace-rule paths record them as they go.
    if (!trace_rule) {
        const bool mixed = h->opt.precision == PURIFY_MIXED;
        const int ppi = products_per_iteration(scheme);
        for (int i = 0; i < iters; ++i) {
            const size_t slot = mixed ? (size_t)(2 * i + 1) : (size_t)(is_fixed_mu(scheme) ? ppi * i + ppi - 1 : i);
            if (4 * slot + 1 >= red.size()) break;
            h->hist_trace.push_back(red[4 * slot]);
            h->hist_idem.push_back(is_fixed_mu(scheme) ? NAN : std::sqrt(std::max(red[4 * slot + 1], 0.0)));
        }
    } else if (h->opt.precision != PURIFY_MIXED) {
        for (int i = 0; i < iters && 4 * (size_t)i + 1 < red.size(); ++i) {
            h->hist_trace.push_back(red[4 * (size_t)i]);
            h->hist_idem.push_back(std::sqrt(std::max(red[4 * (size_t)i + 1], 0.0)));
        }
    }
    st.kernel_launches = (int)(launches_so_far() - launches0);
    st.product_seconds = graph_run ? NAN : product_seconds(h);
    st.trace_err = h->nocc >= 0 ? std::fabs(trace - (double)h->nocc) : NAN;
    int status = S.converged ? PURIFY_OK : PURIFY_ERR_NOT_CONVERGED;
    if (status == PURIFY_OK && h->nocc >= 0 && iters > 0 && !(st.trace_err <= 0.5))
        status = PURIFY_ERR_BOUNDS;
    st.status = status;
    PURIFY_TRY(join_out(h));
    return status;
}

int purify_get_density(purify_t h, double* D, int64_t ld) {
    if (!h || !D || ld < h->n) return PURIFY_ERR_INVALID_ARG;
    if (h->cur < 0) return PURIFY_ERR_STATE;
    PURIFY_TRY(set_device(h));
    PURIFY_TRY(join_in(h));
    if (h->mixed && h->mixed->d_pooled) {
        PURIFY_TRY(density_pooled(h, D, ld));
        return join_out(h);
    }
    PURIFY_CUDA_TRY(cudaMemcpy2DAsync(D, sizeof(double) * ld, h->X[h->cur], sizeof(double) * h->n,
                                      sizeof(double) * h->n, h->n, cudaMemcpyDefault, h->stream));
    PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return join_out(h);
}

int purify_get_density_blocks(purify_t h, int32_t* block_ij, double* values, int64_t cap, int64_t* count) {
    if (!h || !count || cap < 0 || (cap > 0 && !block_ij && !values)) return PURIFY_ERR_INVALID_ARG;
    if (h->cur < 0 || !h->mixed || !h->mixed->d_pooled) return PURIFY_ERR_STATE;
    PURIFY_TRY(set_device(h));
    PURIFY_TRY(join_in(h));
    PURIFY_TRY(density_blocks(h, block_ij, values, cap, count));
    return join_out(h);
}

int purify_stats(purify_t h, purify_stats_t* out) {
    if (!h || !out) return PURIFY_ERR_INVALID_ARG;
    *out = h->st;
    return PURIFY_OK;
}

int purify_step_history(purify_t h, double* trace, double* idem, int cap, int* count) {
    if (!h || !count || cap < 0) return PURIFY_ERR_INVALID_ARG;
    if (h->cur < 0 || h->st.status == PURIFY_ERR_STATE) return PURIFY_ERR_STATE;
    const int m = (int)h->hist_trace.size();
    for (int i = 0; i < m && i < cap; ++i) {
        if (trace) trace[i] = h->hist_trace[i];
        if (idem) idem[i] = i < (int)h->hist_idem.size() ? h->hist_idem[i] : NAN;
    }
    *count = m;
    return PURIFY_OK;
}

const char* purify_strerror(int code) {
    switch (code) {
        case PURIFY_OK: return "ok";
        case PURIFY_ERR_INVALID_ARG: return "invalid argument";
        case PURIFY_ERR_BOUNDS: return "inconsistent spectral bounds, zero gap, or occupied/unoccupied mix-up";
        case PURIFY_ERR_NOT_CONVERGED: return "not converged within max_iter";
        case PURIFY_ERR_OOM: return "device out of memory";
        case PURIFY_ERR_CUDA: return g_last_error[0] ? g_last_error : "CUDA error";
        case PURIFY_ERR_DEVICE_TIMEOUT: return "bounded device wait timed out";
        case PURIFY_ERR_STATE: return "wrong call order";
        case PURIFY_ERR_UNSUPPORTED: return "unsupported device or feature";
        case PURIFY_ERR_INTERNAL: return "internal consistency check failed on the device";
        default: return "unknown status";
    }
}

int purify_schedule(int scheme, double lmin, double lmax, double mu, double homo, double lumo,
                    double tol, int max_iter, double* alpha, int* branch, double* beta,
                    double* beta_bar, int* iterations) {
    if (scheme < PURIFY_FIXED_MU_SF || scheme > PURIFY_SCHEME_LAST) return PURIFY_ERR_INVALID_ARG;
    if (max_iter < 0 || !(tol >= 0.0)) return PURIFY_ERR_INVALID_ARG;
    if (!(lmax > lmin) || !(homo < lumo)) return PURIFY_ERR_BOUNDS;
    if (is_fixed_mu(scheme)) {
        if (std::isnan(mu)) mu = 0.5 * (homo + lumo);
        if (!(std::min(mu - homo, lumo - mu) > 0.0)) return PURIFY_ERR_BOUNDS;
    }
    Schedule S;
    PURIFY_TRY(build_schedule(scheme, lmin, lmax, mu, homo, lumo, tol, max_iter, S));
    const int m = (int)S.alpha.size();
    for (int i = 0; i < m; ++i) {
        if (alpha) alpha[i] = S.alpha[i];
        if (branch) branch[i] = S.branch[i];
        if (beta) beta[i] = S.beta[i];
        if (beta_bar) beta_bar[i] = S.betabar[i];
    }
    if (iterations) *iterations = m;
    return S.converged ? PURIFY_OK : PURIFY_ERR_NOT_CONVERGED;
}

int purify_tridiag_eig(const double* a, const double* b, int m, double* w, double* last_row) {
    if (!a || !w || m <= 0 || (m > 1 && !b) || m > 4096) return PURIFY_ERR_INVALID_ARG;
    std::vector<double> A((size_t)m * m, 0.0), V;
    for (int i = 0; i < m; ++i) {
        A[(size_t)i * m + i] = a[i];
        if (i + 1 < m) A[(size_t)i * m + i + 1] = A[(size_t)(i + 1) * m + i] = b[i];
    }
    jacobi_eig(A, m, V);
    std::vector<int> order(m);
    for (int i = 0; i < m; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int x, int y) {
        return A[(size_t)x * m + x] < A[(size_t)y * m + y];
    });
    for (int j = 0; j < m; ++j) {
        const int c = order[j];
        w[j] = A[(size_t)c * m + c];
        if (last_row) last_row[j] = V[(size_t)(m - 1) * m + c];
    }
    return PURIFY_OK;
}

// ---- kernel-level entry points --------------------------------------------

int purify_k_symm_product_f64(const double* A, const double* B, double* C, int64_t n, void* stream) {
    if (!A || !B || !C || n <= 0) return PURIFY_ERR_INVALID_ARG;
    return launch_step_f64(A, B, nullptr, C, n, 1.0, 0.0, 0.0, 1.0, 0.0, nullptr, (cudaStream_t)stream);
}

int purify_k_step_f64(const double* A, const double* B, const double* E, double* C, int64_t n,
                      double cP, double cE, double cI, double dY, double dI, double* red,
                      void* stream) {
    if (!A || !B || !C || n <= 0) return PURIFY_ERR_INVALID_ARG;
    if (!E && cE != 0.0) return PURIFY_ERR_INVALID_ARG;
    if (C == A || C == B || (E && C == E)) return PURIFY_ERR_INVALID_ARG;
    return launch_step_f64(A, B, E, C, n, cP, cE, cI, dY, dI, red, (cudaStream_t)stream);
}

int purify_k_gershgorin_f64(const double* F, int64_t n, int64_t ld, double* lohi, void* stream) {
    if (!F || !lohi || n <= 0 || ld < n) return PURIFY_ERR_INVALID_ARG;
    double* scratch = nullptr;
    PURIFY_CUDA_TRY(cudaMalloc(&scratch, sizeof(double) * (size_t)gershgorin_scratch_doubles(n)));
    int r = launch_gershgorin_f64(F, n, ld, lohi, scratch, (cudaStream_t)stream);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    cudaFree(scratch);
    if (r != PURIFY_OK) return r;
    PURIFY_CUDA_TRY(e);
    return PURIFY_OK;
}

int purify_k_lanczos_f64(const double* F, int64_t n, int k, double* a, double* b, void* stream) {
    if (!F || !a || !b || n <= 0 || k <= 0 || k > 4096) return PURIFY_ERR_INVALID_ARG;
    double* scratch = nullptr;
    PURIFY_CUDA_TRY(cudaMalloc(&scratch, sizeof(double) * (size_t)lanczos_scratch_doubles(n, k)));
    cudaStream_t s = (cudaStream_t)stream;
    int r = launch_lanczos_f64(F, n, k, scratch, s);
    std::vector<double> bsq(k);
    if (r == PURIFY_OK) {
        cudaError_t e = cudaMemcpyAsync(a, scratch + lanczos_a_offset(n), sizeof(double) * k,
                                        cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(bsq.data(), scratch + lanczos_bsq_offset(n, k), sizeof(double) * k,
                                cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) r = cuda_status(e, "lanczos copy-out");
    }
    cudaFree(scratch);
    if (r != PURIFY_OK) return r;
    for (int j = 0; j < k; ++j) b[j] = std::sqrt(std::max(bsq[j], 0.0));
    return PURIFY_OK;
}

}  // extern "C"
