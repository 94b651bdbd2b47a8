// Spectral bounds lambda_min, lambda_max of F, the inputs that Algorithm 1
// and Algorithm 2 require ("the extremal eigenvalues of F or bounds
// thereof"): Gershgorin discs, tightened by a few float64 Lanczos steps.
//
// Both kernels stream F once per pass and are bound by HBM bandwidth: one
// warp per row reads the row with coalesced 8-byte loads.
#include <cuda.h>

#include "internal.h"

#include <cmath>
#include <mutex>

namespace purify {

namespace {

constexpr int ROWS_PER_CTA = 8;  // Gershgorin: one warp per row
constexpr int LZ_ROWS = 4;       // Lanczos matvec: one warp per row, 6-7 CTAs per SM at n = 4096
constexpr unsigned long long GOLDEN = 0x9E3779B97F4A7C15ull;
constexpr unsigned long long LANCZOS_KEY = 0x11010265ull;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// |x| by clearing the sign bit (an integer operation: GB300's float64 pipe is
// the bound of this pass, and it then carries only the additions).
__device__ __forceinline__ double abs_bits(double x) {
    // the sign bit of the high 32-bit half (64-bit integer operations would
    // run on the float64 pipe too)
    return __hiloint2double(__double2hiint(x) & 0x7FFFFFFF, __double2loint(x));
}

// Per-CTA partial (min lo, max hi) of the Gershgorin interval.
__global__ void __launch_bounds__(256)
gershgorin_rows_kernel(const double* __restrict__ F, int64_t n, int64_t ld, double* __restrict__ part) {
    __shared__ double slo[ROWS_PER_CTA], shi[ROWS_PER_CTA];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // 32-bit row and column indices (any n whose n x n matrix fits in memory
    // is below 2^31): 64-bit integer arithmetic
    // would share the float64 pipe that bounds this pass
    const int nn = (int)n;
    const int i = (int)blockIdx.x * ROWS_PER_CTA + warp;
    double lo = INFINITY, hi = -INFINITY;
    if (i < nn) {
        // four independent partial sums per lane keep the float64 pipe fed
        const double* row = F + (int64_t)i * ld;
        double r0 = 0.0, r1 = 0.0, r2 = 0.0, r3 = 0.0;
        int j = lane;
        for (; j + 96 < nn; j += 128) {  // the disc radius leaves out the diagonal
            r0 += (j == i) ? 0.0 : abs_bits(row[j]);
            r1 += (j + 32 == i) ? 0.0 : abs_bits(row[j + 32]);
            r2 += (j + 64 == i) ? 0.0 : abs_bits(row[j + 64]);
            r3 += (j + 96 == i) ? 0.0 : abs_bits(row[j + 96]);
        }
        for (; j < nn; j += 32) r0 += (j == i) ? 0.0 : abs_bits(row[j]);
        const double r = warp_sum((r0 + r1) + (r2 + r3));
        const double d = row[i];
        lo = d - r;
        hi = d + r;
    }
    if (lane == 0) {
        slo[warp] = lo;
        shi[warp] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < ROWS_PER_CTA; ++w) {
            lo = fmin(lo, slo[w]);
            hi = fmax(hi, shi[w]);
        }
        part[2 * blockIdx.x] = lo;
        part[2 * blockIdx.x + 1] = hi;
    }
}

// The same discs from CSR storage (one warp per row; the diagonal entry is
// the disc's centre, the other entries' magnitudes its radius).
__global__ void __launch_bounds__(256)
gershgorin_csr_kernel(const int64_t* __restrict__ ptr, const int* __restrict__ col, const double* __restrict__ val,
                      int n, double* __restrict__ part) {
    __shared__ double slo[ROWS_PER_CTA], shi[ROWS_PER_CTA];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = (int)blockIdx.x * ROWS_PER_CTA + warp;
    double lo = INFINITY, hi = -INFINITY;
    if (i < n) {
        double r = 0.0, d = 0.0;
        const int64_t p1 = ptr[i + 1];
        for (int64_t k = ptr[i] + lane; k < p1; k += 32) {
            const double v = val[k];
            if (col[k] == i)
                d = v;
            else
                r += abs_bits(v);
        }
        r = warp_sum(r);
        d = warp_sum(d);  // one lane holds the diagonal entry, the others 0
        lo = d - r;
        hi = d + r;
    }
    if (lane == 0) {
        slo[warp] = lo;
        shi[warp] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < ROWS_PER_CTA; ++w) {
            lo = fmin(lo, slo[w]);
            hi = fmax(hi, shi[w]);
        }
        part[2 * blockIdx.x] = lo;
        part[2 * blockIdx.x + 1] = hi;
    }
}

__global__ void minmax_reduce_kernel(const double* __restrict__ part, int64_t m, double* lohi) {
    __shared__ double slo[32], shi[32];
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t q = threadIdx.x; q < m; q += blockDim.x) {
        lo = fmin(lo, part[2 * q]);
        hi = fmax(hi, part[2 * q + 1]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        slo[warp] = lo;
        shi[warp] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int w = 1; w < nw; ++w) {
            lo = fmin(lo, slo[w]);
            hi = fmax(hi, shi[w]);
        }
        lohi[0] = fmin(slo[0], lo);
        lohi[1] = fmax(shi[0], hi);
    }
}

// ---- Lanczos ---------------------------------------------------------------
// Scratch layout (doubles): v_prev[n] | v[n] | w[n] | qnorm2 | a[k] | bsq[k] |
// pa[rows] | pb[kVecBlocksMax].  Every reduction goes through per-block
// partials summed in a fixed order, so the coefficients (and the bounds built
// from them) are the same on every run.

constexpr int kVecBlocksMax = 152 * 4;

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    unsigned long long z = x + GOLDEN;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Sum over a 256-thread block in a fixed order; the result is valid in every
// thread.
__device__ double block_sum256(double v) {
    __shared__ double ws[8];
    __shared__ double total;
    v = warp_sum(v);
    __syncthreads();  // ws and total may still be read from a previous call
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

// Fixed-order sum of count partials (256-thread block).
__device__ double sum_parts256(const double* __restrict__ p, int64_t count) {
    double s = 0.0;
    for (int64_t q = threadIdx.x; q < count; q += 256) s += p[q];
    return block_sum256(s);
}

__global__ void __launch_bounds__(256)
lanczos_start_kernel(double* v, double* vprev, int64_t n, double* pb) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long z = splitmix64(LANCZOS_KEY + (unsigned long long)i * GOLDEN);
        const double q = 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
        v[i] = q;
        vprev[i] = 0.0;
        s += q * q;
    }
    s = block_sum256(s);
    if (threadIdx.x == 0) pb[blockIdx.x] = s;
}

// v <- v / ||v|| with ||v||^2 the sum of the start kernel's partials
__global__ void __launch_bounds__(256)
scale_by_norm_kernel(double* v, int64_t n, const double* pb, int parts, double* qnorm2) {
    const double q2 = sum_parts256(pb, parts);
    if (blockIdx.x == 0 && threadIdx.x == 0) *qnorm2 = q2;
    const double inv = 1.0 / sqrt(q2);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        v[i] *= inv;
}

// w = F v - b_{j-1} v_prev; pa[block] = this block's share of w . v
// (one warp per row)
__global__ void __launch_bounds__(256)
lanczos_matvec_kernel(const double* __restrict__ F, int64_t n, const double* __restrict__ v,
                      const double* __restrict__ vprev, double* __restrict__ w,
                      const double* bsq_prev, double* pa) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // 32-bit indices (n below 2^31): 64-bit integer arithmetic would share the
    // float64 pipe that bounds this pass
    const int nn = (int)n;
    const int i = (int)blockIdx.x * LZ_ROWS + warp;
    __shared__ double sdot[LZ_ROWS];
    double dot = 0.0;
    if (i < nn) {
        // four independent chains per lane keep the float64 pipe fed
        const double* row = F + (int64_t)i * nn;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int j = lane;
        for (; j + 96 < nn; j += 128) {
            s0 = fma(row[j], v[j], s0);
            s1 = fma(row[j + 32], v[j + 32], s1);
            s2 = fma(row[j + 64], v[j + 64], s2);
            s3 = fma(row[j + 96], v[j + 96], s3);
        }
        for (; j < nn; j += 32) s0 = fma(row[j], v[j], s0);
        const double s = warp_sum((s0 + s1) + (s2 + s3));
        const double bprev = bsq_prev ? sqrt(*bsq_prev) : 0.0;
        const double wi = s - bprev * vprev[i];
        if (lane == 0) w[i] = wi;
        dot = wi * v[i];
    }
    if (lane == 0) sdot[warp] = dot;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < LZ_ROWS; ++q) t += sdot[q];
        pa[blockIdx.x] = t;
    }
}

// The matvec from CSR storage (one warp per row).
__global__ void __launch_bounds__(256)
lanczos_matvec_csr_kernel(const int64_t* __restrict__ ptr, const int* __restrict__ col,
                          const double* __restrict__ val, int n, const double* __restrict__ v,
                          const double* __restrict__ vprev, double* __restrict__ w, const double* bsq_prev,
                          double* pa) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = (int)blockIdx.x * LZ_ROWS + warp;
    __shared__ double sdot[LZ_ROWS];
    double dot = 0.0;
    if (i < n) {
        double s0 = 0.0;
        const int64_t p1 = ptr[i + 1];
        for (int64_t k = ptr[i] + lane; k < p1; k += 32) s0 = fma(val[k], v[col[k]], s0);
        const double s = warp_sum(s0);
        const double bprev = bsq_prev ? sqrt(*bsq_prev) : 0.0;
        const double wi = s - bprev * vprev[i];
        if (lane == 0) w[i] = wi;
        dot = wi * v[i];
    }
    if (lane == 0) sdot[warp] = dot;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < LZ_ROWS; ++q) t += sdot[q];
        pa[blockIdx.x] = t;
    }
}

// a_j = sum of the matvec partials; w -= a_j v; pb[block] = share of w . w
__global__ void __launch_bounds__(256)
lanczos_orth_kernel(double* __restrict__ w, const double* __restrict__ v, int64_t n, const double* pa,
                    int64_t rows, double* a_j, double* pb) {
    const double a = sum_parts256(pa, rows);
    if (blockIdx.x == 0 && threadIdx.x == 0) *a_j = a;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double wi = w[i] - a * v[i];
        w[i] = wi;
        s += wi * wi;
    }
    s = block_sum256(s);
    if (threadIdx.x == 0) pb[blockIdx.x] = s;
}

// b_j^2 = sum of the orth partials; v_prev <- v; v <- w / b_j
// (v <- 0 on breakdown b_j == 0)
__global__ void __launch_bounds__(256)
lanczos_shift_kernel(double* __restrict__ vprev, double* __restrict__ v, const double* __restrict__ w,
                     int64_t n, const double* pb, int parts, double* bsq_j) {
    const double b2 = sum_parts256(pb, parts);
    if (blockIdx.x == 0 && threadIdx.x == 0) *bsq_j = b2;
    const double b = sqrt(b2);
    const double inv = b > 0.0 ? 1.0 / b : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        vprev[i] = v[i];
        v[i] = w[i] * inv;
    }
}

unsigned vec_blocks(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > kVecBlocksMax) b = kVecBlocksMax;
    if (b < 1) b = 1;
    return (unsigned)b;
}

}  // namespace

int64_t gershgorin_scratch_doubles(int64_t n) {
    return 2 * ((n + ROWS_PER_CTA - 1) / ROWS_PER_CTA);
}

int launch_gershgorin_f64(const double* F, int64_t n, int64_t ld, double* lohi, double* scratch,
                          cudaStream_t s) {
    if (n <= 0 || ld < n) return PURIFY_ERR_INVALID_ARG;
    const int64_t ctas = (n + ROWS_PER_CTA - 1) / ROWS_PER_CTA;
    gershgorin_rows_kernel<<<(unsigned)ctas, 32 * ROWS_PER_CTA, 0, s>>>(F, n, ld, scratch);
    PURIFY_CUDA_TRY(cudaGetLastError());
    minmax_reduce_kernel<<<1, 1024, 0, s>>>(scratch, ctas, lohi);
    PURIFY_CUDA_TRY(cudaGetLastError());
    count_launches(2);
    return PURIFY_OK;
}

int launch_gershgorin_csr_f64(const CsrF& F, int64_t n, double* lohi, double* scratch, cudaStream_t s) {
    if (n <= 0 || !F.ptr) return PURIFY_ERR_INVALID_ARG;
    const int64_t ctas = (n + ROWS_PER_CTA - 1) / ROWS_PER_CTA;
    gershgorin_csr_kernel<<<(unsigned)ctas, 32 * ROWS_PER_CTA, 0, s>>>(F.ptr, F.col, F.val, (int)n, scratch);
    PURIFY_CUDA_TRY(cudaGetLastError());
    minmax_reduce_kernel<<<1, 1024, 0, s>>>(scratch, ctas, lohi);
    PURIFY_CUDA_TRY(cudaGetLastError());
    count_launches(2);
    return PURIFY_OK;
}

int64_t lanczos_scratch_doubles(int64_t n, int k) {
    return 3 * n + 1 + 2 * (int64_t)k + (n + LZ_ROWS - 1) / LZ_ROWS + kVecBlocksMax;
}

int launch_lanczos_f64(const double* F, int64_t n, int k, double* scratch, cudaStream_t s, const CsrF* csr) {
    if (n <= 0 || k <= 0 || (!F && !csr)) return PURIFY_ERR_INVALID_ARG;
    double* vprev = scratch;
    double* v = scratch + n;
    double* w = scratch + 2 * n;
    double* qn = scratch + 3 * n;
    double* a = scratch + lanczos_a_offset(n);
    double* bsq = scratch + lanczos_bsq_offset(n, k);
    const int64_t rows = (n + LZ_ROWS - 1) / LZ_ROWS;
    double* pa = bsq + k;
    double* pb = pa + rows;
    const unsigned vb = vec_blocks(n);
    lanczos_start_kernel<<<vb, 256, 0, s>>>(v, vprev, n, pb);
    scale_by_norm_kernel<<<vb, 256, 0, s>>>(v, n, pb, (int)vb, qn);
    for (int j = 0; j < k; ++j) {
        if (csr)
            lanczos_matvec_csr_kernel<<<(unsigned)rows, 32 * LZ_ROWS, 0, s>>>(
                csr->ptr, csr->col, csr->val, (int)n, v, vprev, w, j ? bsq + j - 1 : nullptr, pa);
        else
            lanczos_matvec_kernel<<<(unsigned)rows, 32 * LZ_ROWS, 0, s>>>(F, n, v, vprev, w,
                                                                            j ? bsq + j - 1 : nullptr, pa);
        lanczos_orth_kernel<<<vb, 256, 0, s>>>(w, v, n, pa, rows, a + j, pb);
        lanczos_shift_kernel<<<vb, 256, 0, s>>>(vprev, v, w, n, pb, (int)vb, bsq + j);
    }
    PURIFY_CUDA_TRY(cudaGetLastError());
    count_launches(2 + 3 * k);
    return PURIFY_OK;
}

}  // namespace purify

// ---------------------------------------------------------------------------
// Allocation-free Gershgorin entry point: the per-block partials of the bound
// kernel live in a file-scope device array instead of caller- or
// library-allocated memory.  Host code may only use the array's name with
// cudaGetSymbolAddress: on the host the name is a stand-in, not a device
// address.
// ---------------------------------------------------------------------------

namespace purify {
namespace {

constexpr int64_t kNoAllocMaxN = PURIFY_GERSHGORIN_NOALLOC_MAX_N;
static __device__ __align__(256) double g_gershgorin_scratch[2 * ((kNoAllocMaxN + ROWS_PER_CTA - 1) / ROWS_PER_CTA)];

std::mutex g_scratch_mu;
constexpr int kMaxDevices = 64;
// Per device: the context the address was looked up in (its unique ID) and
// the address.  A device reset or a recreated primary context gives a new
// context ID, so the lookup is repeated instead of reusing a dead address.
struct ScratchAddr {
    unsigned long long ctx_id;
    double* ptr;
};
ScratchAddr g_scratch_dev[kMaxDevices] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Unique ID of the calling thread's current context (driver entry points
// fetched through the runtime, so the library links no driver library);
// *have = false when no context is current yet.
int current_context_id(unsigned long long* id, bool* have) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (CtxGetCurrentFn)p;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (CtxGetIdFn)p;
    });
    if (!get_current || !get_id) return PURIFY_ERR_UNSUPPORTED;
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS) return PURIFY_ERR_CUDA;
    *have = ctx != nullptr;
    if (ctx && get_id(ctx, id) != CUDA_SUCCESS) return PURIFY_ERR_CUDA;
    return PURIFY_OK;
}

// Device address of the static scratch on the current device, looked up once
// per device and context.
int noalloc_scratch(double** out) {
    int dev = 0;
    PURIFY_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return PURIFY_ERR_UNSUPPORTED;
    unsigned long long id = 0;
    bool have = false;
    PURIFY_TRY(current_context_id(&id, &have));
    std::lock_guard<std::mutex> g(g_scratch_mu);
    ScratchAddr& a = g_scratch_dev[dev];
    if (!have || !a.ptr || a.ctx_id != id) {
        // the lookup makes the device's primary context current if none was
        void* p = nullptr;
        PURIFY_CUDA_TRY(cudaGetSymbolAddress(&p, g_gershgorin_scratch));
        PURIFY_TRY(current_context_id(&id, &have));
        if (!have) return PURIFY_ERR_CUDA;
        a.ptr = (double*)p;
        a.ctx_id = id;
    }
    *out = a.ptr;
    return PURIFY_OK;
}

}  // namespace

}  // namespace purify

extern "C" int purify_k_gershgorin_f64_noalloc(const double* F, int64_t n, int64_t ld, double* lohi,
                                               void* stream) {
    using namespace purify;
    if (!F || !lohi || n <= 0 || ld < n) return PURIFY_ERR_INVALID_ARG;
    if (n > kNoAllocMaxN) return PURIFY_ERR_INVALID_ARG;
    double* scratch = nullptr;
    PURIFY_TRY(noalloc_scratch(&scratch));
    return launch_gershgorin_f64(F, n, ld, lohi, scratch, (cudaStream_t)stream);
}
