// Float64 SIMT kernels: the symmetric product of one purification step with
// its fused polynomial epilogue (Eq. 1 with the f_i of Algorithm 1 and
// Algorithm 2), the affine start f_0, and small helpers.
//
// GB300's float64 rate is about 1.1 TFLOP/s for the whole chip (roughly two
// float64 FMAs per clock per SM), so this path is bound by the FMA pipe, not
// by memory: a 64 x 64 output tile per 256-thread CTA with 4 x 4 outputs per
// thread keeps the pipe fed from shared memory, and only tiles on or above
// the diagonal are computed (a symmetric product needs n^2 (n + 1) flops).
#include "internal.h"

#include <cstdio>

namespace purify {

namespace {

constexpr int BM = 64;   // tile edge (rows = cols)
constexpr int BK = 16;   // k-slab staged in shared memory
constexpr int NT = 256;  // threads per CTA (16 x 16)

// Tile number t in J-major order, t = tj (tj + 1) / 2 + ti with ti <= tj.
__device__ __forceinline__ void decode_upper(int64_t t, int& ti, int& tj) {
    int64_t j = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((j + 1) * (j + 2) / 2 <= t) ++j;
    while (j * (j + 1) / 2 > t) --j;
    tj = (int)j;
    ti = (int)(t - j * (j + 1) / 2);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(NT)
step_f64_kernel(const double* __restrict__ A, const double* __restrict__ B,
                const double* __restrict__ E, double* __restrict__ C, int64_t n,
                double cP, double cE, double cI, double dY, double dI, double* red) {
    __shared__ double As[2][BK][BM + 1];
    __shared__ double Bs[2][BK][BM];
    __shared__ double rsum[3][NT / 32];

    int ti, tj;
    decode_upper(blockIdx.x, ti, tj);
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t row0 = (int64_t)ti * BM, col0 = (int64_t)tj * BM;

    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;

    double ra[4], rb[4];
    auto load_regs = [&](int64_t k0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int idx = tid + NT * q;
            int r = idx >> 4, k = idx & 15;            // A: 64 rows x 16 k
            int64_t gr = row0 + r, gk = k0 + k;
            ra[q] = (gr < n && gk < n) ? A[gr * n + gk] : 0.0;
            int kb = idx >> 6, c = idx & 63;           // B: 16 k x 64 cols
            int64_t gkb = k0 + kb, gc = col0 + c;
            rb[q] = (gkb < n && gc < n) ? B[gkb * n + gc] : 0.0;
        }
    };
    auto store_smem = [&](int buf) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int idx = tid + NT * q;
            As[buf][idx & 15][idx >> 4] = ra[q];
            Bs[buf][idx >> 6][idx & 63] = rb[q];
        }
    };

    const int64_t nk = (n + BK - 1) / BK;
    load_regs(0);
    store_smem(0);
    __syncthreads();
    for (int64_t kt = 0; kt < nk; ++kt) {
        const int buf = (int)(kt & 1);
        if (kt + 1 < nk) load_regs((kt + 1) * BK);
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            double av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[buf][k][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[buf][k][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
        if (kt + 1 < nk) store_smem(buf ^ 1);
        __syncthreads();
    }

    // Fused epilogue: Y = cP P + cE E + cI I; C = dY Y + dI I (with mirror).
    // Only entries with i <= j are formed; each off-diagonal one is written
    // twice and counts twice in the Frobenius sums, so C is exactly symmetric.
    const bool diag_tile = (ti == tj);
    double s_tr = 0.0, s_idem = 0.0, s_fro = 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t i = row0 + ty + 16 * a;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t j = col0 + tx + 16 * b;
            if (i < n && j < n && (!diag_tile || i <= j)) {
                const double w = (i == j) ? 1.0 : 2.0;
                const double p = acc[a][b];
                const double e = E ? E[i * n + j] : 0.0;
                double y = cP * p + cE * e;
                if (i == j) y += cI;
                double c = dY * y;
                if (i == j) {
                    c += dI;
                    s_tr += y;
                }
                C[i * n + j] = c;
                if (i != j) C[j * n + i] = c;
                const double d = e - p;
                s_idem += w * d * d;
                s_fro += w * y * y;
            }
        }
    }
    if (red) {
        s_tr = warp_sum(s_tr);
        s_idem = warp_sum(s_idem);
        s_fro = warp_sum(s_fro);
        const int wid = tid >> 5, lane = tid & 31;
        if (lane == 0) {
            rsum[0][wid] = s_tr;
            rsum[1][wid] = s_idem;
            rsum[2][wid] = s_fro;
        }
        __syncthreads();
        if (tid < 3) {
            double v = 0.0;
            for (int q = 0; q < NT / 32; ++q) v += rsum[tid][q];
            atomicAdd(&red[tid], v);
        }
    }
}

// Rows over the grid, columns over the threads (no 64-bit division: that runs
// on the float64 pipe).
__global__ void affine_f64_kernel(const double* __restrict__ F, int64_t ldf, double* __restrict__ out,
                                  int64_t n, double a, double b) {
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x)
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
            double v = a * F[i * ldf + j];
            if (i == j) v += b;
            out[i * n + j] = v;
        }
}

// Copy the upper triangle onto the lower one, 32 x 32 tiles through shared
// memory so both the read and the transposed write are coalesced.
__global__ void mirror_upper_kernel(double* X, int64_t n) {
    __shared__ double t[32][33];
    const int64_t T = (n + 31) / 32;
    int ti, tj;
    decode_upper(blockIdx.x, ti, tj);
    if (ti == tj) {
        // diagonal tile: lower part from upper part of the same tile
        const int64_t base = (int64_t)ti * 32;
        for (int r = threadIdx.y; r < 32; r += blockDim.y) {
            const int64_t i = base + r, j = base + threadIdx.x;
            if (i < n && j < n) t[r][threadIdx.x] = X[i * n + j];
        }
        __syncthreads();
        for (int r = threadIdx.y; r < 32; r += blockDim.y) {
            const int64_t i = base + r, j = base + threadIdx.x;
            if (i < n && j < n && j < i) X[i * n + j] = t[threadIdx.x][r];
        }
        return;
    }
    (void)T;
    const int64_t r0 = (int64_t)ti * 32, c0 = (int64_t)tj * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t i = r0 + r, j = c0 + threadIdx.x;
        if (i < n && j < n) t[r][threadIdx.x] = X[i * n + j];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t i = c0 + r, j = r0 + threadIdx.x;  // lower tile (tj, ti)
        if (i < n && j < n) X[i * n + j] = t[threadIdx.x][r];
    }
}

__global__ void trace_f64_kernel(const double* __restrict__ X, int64_t n, double* red) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        s += X[i * n + i];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) atomicAdd(red, s);
}

}  // namespace

int launch_step_f64(const double* A, const double* B, const double* E, double* C, int64_t n,
                    double cP, double cE, double cI, double dY, double dI, double* red,
                    cudaStream_t s) {
    if (n <= 0) return PURIFY_ERR_INVALID_ARG;
    const int64_t T = (n + BM - 1) / BM;
    const int64_t tiles = upper_tiles(T);
    if (tiles > 0x7fffffff) return PURIFY_ERR_INVALID_ARG;
    step_f64_kernel<<<(unsigned)tiles, NT, 0, s>>>(A, B, E, C, n, cP, cE, cI, dY, dI, red);
    PURIFY_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return PURIFY_OK;
}

int launch_affine_f64(const double* F, int64_t ldf, double* out, int64_t n, double a, double b,
                      cudaStream_t s) {
    if (n <= 0) return PURIFY_ERR_INVALID_ARG;
    const int64_t blocks = n < 152 * 16 ? n : 152 * 16;
    affine_f64_kernel<<<(unsigned)blocks, 256, 0, s>>>(F, ldf, out, n, a, b);
    PURIFY_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return PURIFY_OK;
}

int launch_mirror_upper_f64(double* X, int64_t n, cudaStream_t s) {
    if (n <= 0) return PURIFY_ERR_INVALID_ARG;
    const int64_t T = (n + 31) / 32;
    mirror_upper_kernel<<<(unsigned)upper_tiles(T), dim3(32, 8), 0, s>>>(X, n);
    PURIFY_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return PURIFY_OK;
}

int launch_trace_f64(const double* X, int64_t n, double* red, cudaStream_t s) {
    if (n <= 0) return PURIFY_ERR_INVALID_ARG;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152) blocks = 152;
    trace_f64_kernel<<<(unsigned)blocks, 256, 0, s>>>(X, n, red);
    PURIFY_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return PURIFY_OK;
}

}  // namespace purify
