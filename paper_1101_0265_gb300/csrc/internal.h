// Internal declarations shared by the libpurify translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <vector>

#include "../../include/purify.h"

namespace purify {

// Record the failing call for purify_strerror-style diagnostics and map a
// CUDA error to PURIFY_ERR_CUDA / PURIFY_ERR_OOM.
int cuda_status(cudaError_t e, const char* what);

#define PURIFY_CUDA_TRY(call)                                                  \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) return ::purify::cuda_status(e_, #call);        \
    } while (0)

#define PURIFY_TRY(call)                                                       \
    do {                                                                       \
        int r_ = (call);                                                       \
        if (r_ != PURIFY_OK) return r_;                                        \
    } while (0)

// Status of a product kernel's device error flag: bit 8 is the internal check
// that a tile's k-chunk count matches its bitmask (a library bug, not a
// timeout); the other bits name bounded waits that gave up.
constexpr int kDeviceFlagPlan = 8;
inline int device_flag_status(int flag) {
    if (flag == 0) return PURIFY_OK;
    return (flag & kDeviceFlagPlan) ? PURIFY_ERR_INTERNAL : PURIFY_ERR_DEVICE_TIMEOUT;
}

// Number of upper-triangle tiles (ti <= tj) for a T x T tile grid.
inline int64_t upper_tiles(int64_t T) { return T * (T + 1) / 2; }

// ---- float64 SIMT kernels (kernels_fp64.cu) -------------------------------
// Fused scheme step, see purify_k_step_f64 in purify.h.
int launch_step_f64(const double* A, const double* B, const double* E, double* C, int64_t n,
                    double cP, double cE, double cI, double dY, double dI, double* red,
                    cudaStream_t s);
// out = a F + b I on an n x n matrix (ld_out = n, ld_f = ldf).
int launch_affine_f64(const double* F, int64_t ldf, double* out, int64_t n, double a, double b,
                      cudaStream_t s);
// Copy the upper triangle onto the lower one in place (n x n, ld n).
int launch_mirror_upper_f64(double* X, int64_t n, cudaStream_t s);
// red[0] += trace(X)
int launch_trace_f64(const double* X, int64_t n, double* red, cudaStream_t s);

// ---- bounds (kernels_bounds.cu) ------------------------------------------
// F in CSR storage (device arrays): row pointers ptr[n + 1], column indices
// sorted within each row, values.
struct CsrF {
    const int64_t* ptr = nullptr;
    const int* col = nullptr;
    const double* val = nullptr;
};
int launch_gershgorin_f64(const double* F, int64_t n, int64_t ld, double* lohi,
                          double* scratch, cudaStream_t s);
// The same discs from CSR storage (scratch as above).
int launch_gershgorin_csr_f64(const CsrF& F, int64_t n, double* lohi, double* scratch, cudaStream_t s);
int64_t gershgorin_scratch_doubles(int64_t n);
// k Lanczos steps; scratch holds lanczos_scratch_doubles(n, k) doubles.
// Writes a[0..k), bsq[0..k) (squared off-diagonals) into scratch tail; the
// host copies them out (see purify_k_lanczos_f64).  csr set: the matvecs
// read F from CSR storage and F (dense) is not used.
int launch_lanczos_f64(const double* F, int64_t n, int k, double* scratch, cudaStream_t s,
                       const CsrF* csr = nullptr);
int64_t lanczos_scratch_doubles(int64_t n, int k);
// Offsets of the a / bsq arrays inside the Lanczos scratch.
inline int64_t lanczos_a_offset(int64_t n) { return 3 * n + 1; }
inline int64_t lanczos_bsq_offset(int64_t n, int k) { return 3 * n + 1 + k; }

// Host-side helpers (purify_api.cu)
int host_bounds_from_lanczos(const double* a, const double* bsq, int k, double g_lo, double g_hi,
                             double* lo, double* hi);

// Count kernels launched by the library (for the statistics).
void count_launches(int k);
long long launches_so_far();

// Scalar schedule of one run (Algorithm 1: alpha, beta; Algorithm 2:
// branch, alpha, beta, beta_bar), computed on the host.
struct Schedule {
    std::vector<double> alpha, beta, betabar;
    std::vector<int> branch;
    double beta0 = NAN, betabar0 = NAN;
    bool converged = false;
};

// Eigenpairs of the symmetric tridiagonal matrix (diagonal a[0..m),
// off-diagonal b[0..m-1)) by cyclic Jacobi: w ascending, Z[j * m + i] the i-th
// component of the j-th normalised eigenvector (host).
void tridiag_eig_full(const double* a, const double* b, int m, std::vector<double>& w, std::vector<double>& Z);

// Algorithm 2's scalar pieces (float64, host): alpha of a branch (1 = P_{1,0},
// 0 = P_{0,1}) and the branch's map of a scalar (Eq. 4 / Eq. 5).
double tc_alpha(int branch, double b, double bb);
// (1 + a)^2 of Eq. 4 / Eq. 5, evaluated by the C library's pow.
double sq1p(double a);
double tc_map(int branch, double a, double x);
// The fixed-mu polynomial order of a scheme (1: P_{1,1}, 3: P_{3,3}), its
// products per iteration, P_{i,j} on a scalar and the P_{m,m} scaling alpha.
int pmm_order(int scheme);
void pij_orders(int scheme, int* i, int* j);
bool is_asymmetric(int scheme);
int products_per_iteration(int scheme);
double P_ij_scalar(int i, int j, double x);
double pmm_alpha(int m, double beta);
double pij_fixed_point(int i, int j);
double pij_alpha(int i, int j, double c, double b, double bb);

struct MixedState;

}  // namespace purify

// The handle behind purify_t.
struct purify_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;       // private, non-blocking: all library work
    cudaStream_t user_stream = nullptr;  // the caller's stream (null = legacy default)
    cudaEvent_t join_ev = nullptr;
    bool own_stream = false;
    purify_options opt{};
    int64_t n = 0, cap = 0;
    double* F = nullptr;
    double* X[2] = {nullptr, nullptr};
    double* S = nullptr;
    double* P3[2] = {nullptr, nullptr};  // float64 P_{3,3} intermediates, allocated on use
    int64_t p3_cap = 0;
    double* red = nullptr;
    int64_t red_cap = 0;  // doubles
    double* scratch = nullptr;
    int64_t scratch_cap = 0;  // doubles
    int cur = -1;
    bool have_F = false;
    // F loaded from COO for a block-sparse handle: CSR in device memory, and
    // F (dense) allocated and filled only when a dense path asks for it
    int64_t* csr_ptr = nullptr;
    int* csr_col = nullptr;
    double* csr_val = nullptr;
    int64_t csr_rows_cap = 0, csr_nnz_cap = 0, csr_nnz = 0;
    bool csr_valid = false;  // csr_* hold the current F
    bool F_dense = false;    // F holds the current F
    // with csr_valid: F's 32 x 32 block pattern and the diagonal, nb rows of
    // f_pattern_words 64-bit words (nb = padded n / 32)
    std::vector<uint64_t> f_pattern;
    int f_pattern_words = 0;
    int64_t nocc = -1;
    double mu = NAN;
    purify_bounds b{NAN, NAN, NAN, NAN};
    purify_stats_t st{};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::vector<cudaEvent_t> pev;  // product timing events (pairs)
    int pev_used = 0;
    purify::MixedState* mixed = nullptr;
    // per-iteration reductions of the last run (purify_step_history)
    std::vector<double> hist_trace, hist_idem;
};

namespace purify {
// Order `work` after what the caller queued on `user` (join_in) and the
// caller's stream after the library's work (join_out).
int join_streams(cudaStream_t after, cudaStream_t before, cudaEvent_t ev);
// Copy an n x n float64 matrix (leading dimension ld, host or device) into
// dst (leading dimension n) on `s`.  A host source has been read when this
// returns (the caller may reuse it); a device source is read in stream order.
int copy_in_matrix(double* dst, const double* src, int64_t n, int64_t ld, cudaStream_t s);
// Product timing: bracket one product launch with events when requested.
int product_begin(purify_ctx* h);
int product_end(purify_ctx* h);
// Sum of the bracketed product times of the last run (seconds), NaN if off.
double product_seconds(purify_ctx* h);
int ensure_red(purify_ctx* h, int64_t doubles);
// Allocate the handle's second float64 iterate X[1] and product buffer S (at
// its capacity) if they are not yet allocated.
int ensure_work(purify_ctx* h);
// The handle's float64 scratch holds at least `doubles` doubles.
int ensure_scratch(purify_ctx* h, int64_t doubles);
// Make the dense F (and the density buffer X[0]) valid: from the CSR copy
// when the Hamiltonian was loaded in block-sparse form.
int ensure_dense_F(purify_ctx* h);
// The current F as CSR (csr_valid) for the bounds and the block-sparse split.
inline CsrF csr_of(const purify_ctx* h) {
    CsrF c;
    c.ptr = h->csr_ptr;
    c.col = h->csr_col;
    c.val = h->csr_val;
    return c;
}
}  // namespace purify
