// Gap edges (homo, lumo) of F from the purification itself.  Algorithms 1
// and 2 require a lower bound of the gap's lower edge and an upper bound of
// its upper edge; the paper points to techniques for interior eigenvalues.
// Here the edges come from a few steps of the alpha = 0 scheme with the trace
// rule, which needs no gap and keeps the order of the eigenvalues:
//
//   1. X_0 = (lmax I - F) / (lmax - lmin), then trace-rule steps
//      (trace(X) > nocc -> X^2, else 2X - X^2), each iterate also written in
//      float64, until ||X - X^2||_F < 1 / (4 sqrt(n)) and round(trace X) =
//      nocc: then exactly the nocc occupied eigenvalues lie above 1/2
//      (|trace X - #{x > 1/2}| <= sum min(x, 1 - x) <= 2 sqrt(n) ||X - X^2||_F)
//      and every eigenvalue has x (1 - x) < 1/16;
//   2. Lanczos on X^4 (I - X) and on X (I - X)^4: the largest eigenvalue of
//      the first belongs to the occupied eigenvalue nearest 1/2 (the image of
//      homo), of the second to the unoccupied one nearest 1/2 (lumo); the top
//      Ritz vector's Rayleigh quotient with X confirms the side;
//   3. each top Ritz value raised by its residual norm (and an allowance for
//      the iterate's rounding) is solved for x on the filter's monotone
//      branch; the inverse of the recorded steps and of X_0's map carry x
//      back to the spectrum of F.  The estimates lie inside the gap.
// All of it runs on the device except the scalar work (tridiagonal
// eigenproblem, bisection, inverse maps).  Reductions use per-block partials
// summed in a fixed order.
#include <algorithm>
#include <cmath>
#include <vector>

#include "digits_tc.h"
#include "internal.h"
#include "mixed.h"

namespace purify {
namespace {

constexpr int kFilterPower = 4;
constexpr int kVecBlocks = 152 * 4;
constexpr int kRowsPerCta = 8;  // one warp per row
constexpr unsigned long long kGolden = 0x9E3779B97F4A7C15ull;
constexpr unsigned long long kStartKey = 0x11010265ull;  // the bounds' Lanczos start
// Allowance on a filter's Ritz value for the rounding of a mixed-precision
// iterate (the mixed path's densities are within 3e-7 of the exact ones).
constexpr double kMixedAllowance = 1e-7;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over a 256-thread block in a fixed order, valid in every thread.
__device__ double block_sum256(double v) {
    __shared__ double ws[8];
    __shared__ double total;
    v = warp_sum_d(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += ws[q];
        total = t;
    }
    __syncthreads();
    return total;
}

__device__ double sum_parts256(const double* __restrict__ p, int count) {
    double s = 0.0;
    for (int q = threadIdx.x; q < count; q += 256) s += p[q];
    return block_sum256(s);
}

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    unsigned long long z = x + kGolden;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// y = alpha (X v) + beta z (z may be null), one warp per row of X (n x n).
__global__ void __launch_bounds__(256)
filter_matvec_kernel(const double* __restrict__ X, int64_t n, const double* __restrict__ v, double alpha,
                     double beta, const double* __restrict__ z, double* __restrict__ y) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * kRowsPerCta + warp;
    if (i >= n) return;
    const double* row = X + i * n;
    double s = 0.0;
    for (int64_t j = lane; j < n; j += 32) s = fma(row[j], v[j], s);
    s = warp_sum_d(s);
    if (lane == 0) y[i] = alpha * s + (z ? beta * z[i] : 0.0);
}

// q_i = 2 u_i - 1 with u_i the top 53 bits of SplitMix64 at key + i golden;
// pb[block] = the block's share of q . q.
__global__ void __launch_bounds__(256) start_kernel(double* q, int64_t n, double* pb) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long z = splitmix64(kStartKey + (unsigned long long)i * kGolden);
        const double x = 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
        q[i] = x;
        s += x * x;
    }
    s = block_sum256(s);
    if (threadIdx.x == 0) pb[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) normalize_kernel(double* q, int64_t n, const double* pb, int parts) {
    const double inv = 1.0 / sqrt(sum_parts256(pb, parts));
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        q[i] *= inv;
}

// w = t - b_{j-1} v_{j-1}; pa[block] = the block's share of w . v_j
__global__ void __launch_bounds__(256)
lanczos_w_kernel(const double* __restrict__ t, const double* __restrict__ v, const double* __restrict__ vprev,
                 const double* bsq_prev, int64_t n, double* __restrict__ w, double* pa) {
    const double b = bsq_prev ? sqrt(*bsq_prev) : 0.0;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double wi = t[i] - (vprev ? b * vprev[i] : 0.0);
        w[i] = wi;
        s += wi * v[i];
    }
    s = block_sum256(s);
    if (threadIdx.x == 0) pa[blockIdx.x] = s;
}

// a_j = sum pa; w -= a_j v_j; pb[block] = the block's share of w . w
__global__ void __launch_bounds__(256)
lanczos_orth2_kernel(double* __restrict__ w, const double* __restrict__ v, int64_t n, const double* pa, int parts,
                     double* a_j, double* pb) {
    const double a = sum_parts256(pa, parts);
    if (blockIdx.x == 0 && threadIdx.x == 0) *a_j = a;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double wi = w[i] - a * v[i];
        w[i] = wi;
        s += wi * wi;
    }
    s = block_sum256(s);
    if (threadIdx.x == 0) pb[blockIdx.x] = s;
}

// b_j^2 = sum pb; v_{j+1} = w / b_j (0 on breakdown)
__global__ void __launch_bounds__(256)
lanczos_next_kernel(const double* __restrict__ w, int64_t n, const double* pb, int parts, double* bsq_j,
                    double* __restrict__ vnext) {
    const double b2 = sum_parts256(pb, parts);
    if (blockIdx.x == 0 && threadIdx.x == 0) *bsq_j = b2;
    const double b = sqrt(b2);
    const double inv = b > 0.0 ? 1.0 / b : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        vnext[i] = w[i] * inv;
}

// u = sum_j z_j V_j (V: m rows of n)
__global__ void __launch_bounds__(256)
combine_kernel(const double* __restrict__ V, int m, int64_t n, const double* __restrict__ z, double* __restrict__ u) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < m; ++j) s = fma(z[j], V[(size_t)j * n + i], s);
        u[i] = s;
    }
}

// parts[block] = the block's share of a . b
__global__ void __launch_bounds__(256)
dot_kernel(const double* __restrict__ a, const double* __restrict__ b, int64_t n, double* parts) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += a[i] * b[i];
    s = block_sum256(s);
    if (threadIdx.x == 0) parts[blockIdx.x] = s;
}

unsigned vec_grid(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, kVecBlocks)); }

// Device work space of one estimate.
struct GapWork {
    double* V = nullptr;  // (k + 1) x n Lanczos basis
    double* t = nullptr;  // filter output
    double* w = nullptr;
    double* t1 = nullptr;  // filter temporaries
    double* t2 = nullptr;
    double* u = nullptr;   // Ritz vector
    double* parts = nullptr;  // 2 x kVecBlocks partials
    double* ab = nullptr;     // a[k] | bsq[k] | z[k]
};

int matvec(const double* X, int64_t n, const double* v, double alpha, double beta, const double* z, double* y,
           cudaStream_t s) {
    filter_matvec_kernel<<<(unsigned)((n + kRowsPerCta - 1) / kRowsPerCta), 32 * kRowsPerCta, 0, s>>>(X, n, v, alpha,
                                                                                                   beta, z, y);
    PURIFY_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return PURIFY_OK;
}

// t = X^p (I - X) v (occupied side) or X (I - X)^p v (unoccupied side).
int apply_filter(const double* X, int64_t n, bool occupied, const double* v, GapWork& g, cudaStream_t s) {
    const double* cur = v;
    double* buf[2] = {g.t1, g.t2};
    for (int q = 0; q < kFilterPower; ++q) {
        if (occupied)
            PURIFY_TRY(matvec(X, n, cur, 1.0, 0.0, nullptr, buf[q & 1], s));
        else
            PURIFY_TRY(matvec(X, n, cur, -1.0, 1.0, cur, buf[q & 1], s));
        cur = buf[q & 1];
    }
    if (occupied) return matvec(X, n, cur, -1.0, 1.0, cur, g.t, s);
    return matvec(X, n, cur, 1.0, 0.0, nullptr, g.t, s);
}

// Fixed-order dot product through device partials.
int dot(const double* a, const double* b, int64_t n, GapWork& g, cudaStream_t s, double* out) {
    const unsigned vb = vec_grid(n);
    dot_kernel<<<vb, 256, 0, s>>>(a, b, n, g.parts);
    PURIFY_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    std::vector<double> p(vb);
    PURIFY_CUDA_TRY(cudaMemcpyAsync(p.data(), g.parts, sizeof(double) * vb, cudaMemcpyDeviceToHost, s));
    PURIFY_CUDA_TRY(cudaStreamSynchronize(s));
    double t = 0.0;
    for (double x : p) t += x;
    *out = t;
    return PURIFY_OK;
}

// k Lanczos steps on one filter of X; the top Ritz value, its residual norm
// and the Ritz vector's Rayleigh quotient with X.
int lanczos_top(const double* X, int64_t n, bool occupied, int k, GapWork& g, cudaStream_t s, double* theta,
                double* resid, double* rq) {
    const unsigned vb = vec_grid(n);
    double* pa = g.parts;
    double* pb = g.parts + kVecBlocks;
    double* a = g.ab;
    double* bsq = g.ab + k;
    start_kernel<<<vb, 256, 0, s>>>(g.V, n, pb);
    normalize_kernel<<<vb, 256, 0, s>>>(g.V, n, pb, (int)vb);
    PURIFY_CUDA_TRY(cudaGetLastError());
    count_launches(2);
    for (int j = 0; j < k; ++j) {
        const double* v = g.V + (size_t)j * n;
        PURIFY_TRY(apply_filter(X, n, occupied, v, g, s));
        lanczos_w_kernel<<<vb, 256, 0, s>>>(g.t, v, j ? g.V + (size_t)(j - 1) * n : nullptr, j ? bsq + j - 1 : nullptr,
                                            n, g.w, pa);
        lanczos_orth2_kernel<<<vb, 256, 0, s>>>(g.w, v, n, pa, (int)vb, a + j, pb);
        lanczos_next_kernel<<<vb, 256, 0, s>>>(g.w, n, pb, (int)vb, bsq + j, g.V + (size_t)(j + 1) * n);
        PURIFY_CUDA_TRY(cudaGetLastError());
        count_launches(3);
    }
    std::vector<double> ha(k), hb(k);
    PURIFY_CUDA_TRY(cudaMemcpyAsync(ha.data(), a, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
    PURIFY_CUDA_TRY(cudaMemcpyAsync(hb.data(), bsq, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
    PURIFY_CUDA_TRY(cudaStreamSynchronize(s));
    int m = k;
    for (int j = 0; j < k; ++j)
        if (!(hb[j] > 0.0)) {  // breakdown: an invariant subspace
            m = j + 1;
            break;
        }
    std::vector<double> off(m > 1 ? m - 1 : 1), w, Z;
    for (int j = 0; j + 1 < m; ++j) off[j] = std::sqrt(hb[j]);
    tridiag_eig_full(ha.data(), off.data(), m, w, Z);
    const double* z = &Z[(size_t)(m - 1) * m];  // eigenvector of the largest
    *theta = w[m - 1];
    *resid = std::fabs(std::sqrt(std::max(hb[m - 1], 0.0)) * z[m - 1]);
    double* dz = g.ab + 2 * k;
    PURIFY_CUDA_TRY(cudaMemcpyAsync(dz, z, sizeof(double) * m, cudaMemcpyHostToDevice, s));
    combine_kernel<<<vb, 256, 0, s>>>(g.V, m, n, dz, g.u);
    PURIFY_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    PURIFY_TRY(matvec(X, n, g.u, 1.0, 0.0, nullptr, g.t, s));
    double uxu = 0.0, uu = 0.0;
    PURIFY_TRY(dot(g.u, g.t, n, g, s, &uxu));
    PURIFY_TRY(dot(g.u, g.u, n, g, s, &uu));
    *rq = uu > 0.0 ? uxu / uu : 0.5;
    return PURIFY_OK;
}

// x in [lo, hi] with g(x) = target, g monotone there (bisection); the end
// nearer the target when it lies outside g's range.
template <typename G>
double solve_monotone(G g, double target, double lo, double hi) {
    const double glo = g(lo), ghi = g(hi);
    const bool inc = ghi > glo;
    if (target <= std::min(glo, ghi)) return inc ? lo : hi;
    if (target >= std::max(glo, ghi)) return inc ? hi : lo;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        if ((g(mid) < target) == inc)
            lo = mid;
        else
            hi = mid;
    }
    return 0.5 * (lo + hi);
}

}  // namespace
}  // namespace purify

using namespace purify;

extern "C" int purify_estimate_gap(purify_t h, int lanczos_steps, double* homo_out, double* lumo_out) {
    if (!h || !homo_out || !lumo_out || lanczos_steps < 4 || lanczos_steps > 512) return PURIFY_ERR_INVALID_ARG;
    if (!h->have_F) return PURIFY_ERR_STATE;
    if (h->nocc <= 0 || h->nocc >= h->n) return PURIFY_ERR_INVALID_ARG;
    PURIFY_CUDA_TRY(cudaSetDevice(h->device));
    PURIFY_TRY(join_streams(h->stream, h->user_stream, h->join_ev));
    cudaStream_t s = h->stream;
    const int64_t n = h->n;
    const int k = lanczos_steps;
    const int max_steps = 200;
    const bool mixed = h->opt.precision == PURIFY_MIXED;
    const double lmin = h->b.lmin, lmax = h->b.lmax, wdt = lmax - lmin;
    const double c0 = lmax / wdt, c1 = -1.0 / wdt;
    PURIFY_TRY(ensure_red(h, 4 * (int64_t)(max_steps + 1)));
    PURIFY_CUDA_TRY(cudaMemsetAsync(h->red, 0, sizeof(double) * 4 * (max_steps + 1), s));
    double* trF = h->red + 4 * (int64_t)max_steps;
    PURIFY_TRY(ensure_dense_F(h));
    PURIFY_TRY(launch_trace_f64(h->F, n, trF, s));
    double tf = 0.0;
    PURIFY_CUDA_TRY(cudaMemcpyAsync(&tf, trF, sizeof(double), cudaMemcpyDeviceToHost, s));
    PURIFY_CUDA_TRY(cudaStreamSynchronize(s));
    double tr_prev = c0 * (double)n + c1 * tf;
    // iterates in float64: X_i in Xf[(i + 1) & 1] (X_0 in Xf[1])
    PURIFY_TRY(ensure_work(h));
    double* Xf[2] = {h->X[0], h->X[1]};
    int x = 0;
    const int n_pad = pad128(n);
    const int rb = remainder_bits(n_pad);
    if (mixed) {
        PURIFY_TRY(ensure_mixed(h, n_pad));
        PURIFY_TRY(launch_split(h->F, n, (int)n, n_pad, c1, c0, 0, kMaxDigitPlanes, rb, h->mixed->Xd[0], nullptr, s));
        PURIFY_CUDA_TRY(cudaMemsetAsync(h->mixed->err, 0, sizeof(int), s));
    } else {
        PURIFY_TRY(launch_affine_f64(h->F, n, Xf[1], n, c1, c0, s));
    }
    std::vector<int> branches;
    const double thr = 1.0 / (4.0 * std::sqrt((double)n));
    GapWork g;
    std::vector<void*> allocs;
    auto alloc = [&](double** p, size_t count) {
        if (cudaMalloc(p, sizeof(double) * count) != cudaSuccess) return false;
        allocs.push_back(*p);
        return true;
    };
    auto release = [&]() {
        for (void* p : allocs) cudaFree(p);
    };
    if (!alloc(&g.V, (size_t)(k + 1) * n) || !alloc(&g.t, n) || !alloc(&g.w, n) || !alloc(&g.t1, n) ||
        !alloc(&g.t2, n) || !alloc(&g.u, n) || !alloc(&g.parts, 2 * kVecBlocks) || !alloc(&g.ab, 3 * (size_t)k)) {
        release();
        return PURIFY_ERR_OOM;
    }
    int rc = PURIFY_ERR_NOT_CONVERGED;
    double homo = NAN, lumo = NAN;
    for (int i = 0; i < max_steps; ++i) {
        // step i: X_{i+1} from X_i, reducing trace(X_{i+1}) and ||X_i - X_i^2||_F
        const int br = tr_prev > (double)h->nocc ? 1 : 0;
        const double cP = br ? 1.0 : -1.0, cE = br ? 0.0 : 2.0;
        double* red = h->red + 4 * (int64_t)i;
        int r;
        if (mixed) {
            MixedState* ms = h->mixed;
            DigitStep st;
            st.n = (int)n;
            st.n_pad = n_pad;
            st.rbits = rb;
            st.A = st.B = ms->Xd[x];
            st.s_in = kMaxDigitPlanes;
            st.use_E = 1;
            st.cP = cP;
            st.cE = cE;
            st.out = ms->Xd[x ^ 1];
            st.s_out = kMaxDigitPlanes;
            st.out64 = Xf[i & 1];
            st.red = red;
            st.err = ms->err;
            st.scratch = ms->scratch;
            st.max_ctas = ms->ctas;
            if (h->opt.split_k) {
                st.partial = ms->partial;
                st.split_cnt = ms->split_cnt;
            }
            st.wait_cycles = 1000ll * h->opt.wait_kcycles;
            r = launch_digit_step(st, s);
        } else {
            const double* Xi = Xf[(i + 1) & 1];
            r = launch_step_f64(Xi, Xi, Xi, Xf[i & 1], n, cP, cE, 0.0, 1.0, 0.0, red, s);
        }
        if (r != PURIFY_OK) {
            release();
            return r;
        }
        double rr[4];
        if (cudaMemcpyAsync(rr, red, sizeof(rr), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            release();
            return PURIFY_ERR_CUDA;
        }
        const double idem_in = std::sqrt(std::max(rr[1], 0.0));
        if (i > 0 && idem_in < thr && std::llround(tr_prev) == h->nocc) {
            // X_i satisfies the switch condition: filtered Lanczos on it
            const double* Xs = Xf[(i + 1) & 1];
            double th_o, r_o, rq_o, th_u, r_u, rq_u;
            r = lanczos_top(Xs, n, true, k, g, s, &th_o, &r_o, &rq_o);
            if (r == PURIFY_OK) r = lanczos_top(Xs, n, false, k, g, s, &th_u, &r_u, &rq_u);
            if (r != PURIFY_OK) {
                release();
                return r;
            }
            if (rq_o > 0.5 && rq_u < 0.5) {
                const double allow = mixed ? kMixedAllowance : 0.0;
                const double p = kFilterPower;
                double xh = solve_monotone([&](double v) { return std::pow(v, p) * (1.0 - v); }, th_o + r_o + allow,
                                           p / (p + 1.0), 1.0);
                double xl = solve_monotone([&](double v) { return v * std::pow(1.0 - v, p); }, th_u + r_u + allow, 0.0,
                                           1.0 / (p + 1.0));
                for (int q = (int)branches.size() - 1; q >= 0; --q) {
                    if (branches[q]) {
                        xh = std::sqrt(xh);
                        xl = std::sqrt(xl);
                    } else {
                        xh = 1.0 - std::sqrt(1.0 - xh);
                        xl = 1.0 - std::sqrt(1.0 - xl);
                    }
                }
                const double margin = 64.0 * 2.220446049250313e-16 * wdt;
                homo = lmax - wdt * xh + margin;
                lumo = lmax - wdt * xl - margin;
                rc = homo < lumo ? PURIFY_OK : PURIFY_ERR_BOUNDS;
                break;
            }
            // the filters did not separate the sides yet: one more step
        }
        branches.push_back(br);
        tr_prev = rr[0];
        x ^= 1;
    }
    release();
    int err = 0;
    if (mixed) {
        PURIFY_CUDA_TRY(cudaMemcpyAsync(&err, h->mixed->err, sizeof(int), cudaMemcpyDeviceToHost, s));
        PURIFY_CUDA_TRY(cudaStreamSynchronize(s));
    }
    h->st.device_flag = err;
    if (err) return device_flag_status(err);
    if (rc == PURIFY_OK) {
        h->b.homo = homo;
        h->b.lumo = lumo;
        h->st.homo = homo;
        h->st.lumo = lumo;
        *homo_out = homo;
        *lumo_out = lumo;
    }
    h->cur = -1;  // the iterates in the float64 buffers are not a density
    PURIFY_TRY(join_streams(h->user_stream, h->stream, h->join_ev));
    return rc;
}
