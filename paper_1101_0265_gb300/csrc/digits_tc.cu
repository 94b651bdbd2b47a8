// Host side of the digit-plane products: the float64 -> digit-plane split
// kernel, tensor maps, kernel choice and launch.  The product kernel itself
// is in digits_kernel.cuh (instantiated in digits_k*.cu).
#include "digits_kernel.cuh"

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

namespace purify {

using namespace dk;

namespace {

// ---- float64 (with affine) -> digit planes ----------------------------------
// out = a F + b I for i, j < n, 0 in the padding; split into s planes with
// the scale 2^e.  GB300's float64 pipe runs at a small fraction of its
// float32 rate, so the per-element arithmetic is float32 and integer: each
// float64 F_ij is cut into two floats with integer operations (to 46 bits;
// the digits carry at most 43), the affine map runs in double-float with a
// and b as float pairs, and the digits come from the double-float value as in
// the product epilogue.

// x = h + l with |x - (h + l)| <= 2^-46 |x|, for 2^-74 <= |x| < 2^128 (both
// floats normal; the caller handles other magnitudes); integer operations
// only.
__device__ __forceinline__ df split_double_bits(unsigned int hi, unsigned int lo) {
    // 32-bit halves only: 64-bit integer operations would occupy the float64
    // pipe, which this pass otherwise leaves idle
    const unsigned int sign = hi & 0x80000000u;
    const int E = (int)((hi >> 20) & 0x7FFu) - 1023;                 // x = m 2^(E - 52)
    // the 24 leading mantissa bits (with the hidden one): m >> 29
    const unsigned int top = ((hi & 0xFFFFFu) | 0x100000u) << 3 | (lo >> 29);
    const float h = __uint_as_float(sign | (unsigned int)(E + 127) << 23 | (top & 0x7FFFFFu));
    // the 29 low mantissa bits times 2^(E - 52): the top 24 of them, normalised
    const unsigned int lo29 = lo & 0x1FFFFFFFu;
    unsigned int lbits = 0;
    if (lo29) {
        const int bits = 32 - __clz(lo29);
        const unsigned int mant = bits > 24 ? lo29 >> (bits - 24) : lo29 << (24 - bits);
        lbits = sign | (unsigned int)(E - 52 + bits - 1 + 127) << 23 | (mant & 0x7FFFFFu);
    }
    return {h, __uint_as_float(lbits)};
}

// Magnitudes outside [2^-74, 2^128), through the float64 conversions (out of
// line, so that the common path does not carry them).
__device__ __noinline__ df split_double_slow(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}

// One warp per strip of 32 rows x 128 columns, each lane on four consecutive
// columns: 32-byte pieces of F's rows per lane (two 16-byte loads when F's
// rows are 16-byte aligned), one 8-byte store per digit plane and row, and,
// when bnorm2 is not null, ||.||_F^2 of the strip's four 32 x 32 blocks
// (float, in a fixed order) for blocks I <= J.
__device__ __forceinline__ df split_entry(double x) {
    const unsigned int hi = (unsigned int)__double2hiint(x), lo = (unsigned int)__double2loint(x);
    const int E = (int)((hi >> 20) & 0x7FFu) - 1023;
    // zeros (most of a sparse F) and normal magnitudes stay off the float64 pipe
    if (((hi << 1) | lo) == 0u) return {0.f, 0.f};
    return (E >= -74 && E <= 127) ? split_double_bits(hi, lo) : split_double_slow(x);
}

// F's entries (i, j0 .. j0 + 3) of a strip row, from dense storage.
struct DenseRows {
    const double* F;
    int64_t ldf;
    int n;
    bool vec;
    __device__ __forceinline__ void operator()(int i, int j0, int, double (&x)[4]) const {
        x[0] = x[1] = x[2] = x[3] = 0.0;
        if (i >= n) return;
        const double* row = F + (int64_t)i * ldf + j0;
        if (vec && j0 + 3 < n) {
            const double2 u0 = __ldg((const double2*)row), u1 = __ldg((const double2*)row + 1);
            x[0] = u0.x;
            x[1] = u0.y;
            x[2] = u1.x;
            x[3] = u1.y;
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (j0 + c < n) x[c] = __ldg(row + c);
        }
    }
};

// The same entries from CSR storage (warp-collective: the warp gathers row
// i's entries in the strip's 128 columns into its shared-memory row buffer,
// then each lane reads its four).  Absent entries are zero.
struct CsrRows {
    const int64_t* ptr;
    const int* col;
    const double* val;
    int n;
    double* buf;  // 128 doubles per warp
    __device__ __forceinline__ void operator()(int i, int j0, int lane, double (&x)[4]) const {
        const int c0 = j0 - 4 * lane;
#pragma unroll
        for (int c = 0; c < 4; ++c) buf[4 * lane + c] = 0.0;
        __syncwarp();
        if (i < n) {
            const int64_t p1 = ptr[i + 1];
            for (int64_t k = ptr[i] + lane; k < p1; k += 32) {
                const int j = col[k];
                if (j >= c0 && j < c0 + 128) buf[j - c0] = val[k];
            }
        }
        __syncwarp();
#pragma unroll
        for (int c = 0; c < 4; ++c) x[c] = buf[4 * lane + c];
        __syncwarp();
    }
};

// One 32 x 128 strip of the split (see split_kernel); tr accumulates the
// diagonal's trace (float), the strip's block norms go to bnorm2 when set.
// POOLED: the planes go to the pool slots that pidx (nb x nb) gives the
// blocks (slot 0: not written); a null pidx writes nothing (norms only).
// `rows` reads F's entries (DenseRows or CsrRows).
template <bool POOLED, class Rows>
__device__ __forceinline__ void split_strip(const Rows& rows, int n, int n_pad, df a, df b, float digit_scale,
                                            float rscale, float rinv, int s, __nv_bfloat16* __restrict__ out,
                                            float* __restrict__ bnorm2, int strip, int lane, float& tr,
                                            const int* __restrict__ pidx = nullptr) {
    const int nb = n_pad / 32, ns = n_pad / 128;  // nb^2 < 2^27: 32-bit block indices
    const int64_t total = (int64_t)n_pad * n_pad;
    const int I = strip / ns, Jq = strip - I * ns;
    const int j0 = Jq * 128 + lane * 4;
    // the pool slot of this lane's block (I, j0 / 32); 0: not written
    const int slot = (POOLED && pidx) ? pidx[(size_t)I * nb + (j0 >> 5)] : 0;
    float bsum = 0.f;
#pragma unroll 2
    for (int r = 0; r < 32; ++r) {  // two rows' loads in flight per warp
        const int i = I * 32 + r;
        double x[4];
        rows(i, j0, lane, x);
        df z[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = j0 + c;
            z[c] = {0.f, 0.f};
            if (i < n && j < n) {
                z[c] = df_mul(a, split_entry(x[c]));
                if (i == j) {
                    z[c] = df_add(z[c], b);
                    tr += z[c].h + z[c].l;
                }
            }
            bsum += z[c].h * z[c].h;
            z[c] = df_scale(z[c], digit_scale);
        }
        if (POOLED && slot == 0) continue;  // (after rows(): every lane takes part in each row's read)
        // plane p at out + plane_index(p, i, j0, n_pad): pairs 2 total apart
        __nv_bfloat16* dst = out + (size_t)i * 2 * n_pad + ((j0 >> 5) << 6) + (j0 & 31);
        float plane_scale = 1.f;
        for (int p = 0; p < s; ++p) {
            __align__(8) __nv_bfloat16 dv[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float d = round_digit(z[c].h);
                // z.h - d is exact and either 0 or at least ulp(z.h) >= 2 |z.l|,
                // so the fast two-sum is exact (the same bits as two_sum)
                z[c] = fast_two_sum(__fsub_rn(z[c].h, d), z[c].l);
                dv[c] = digit_to_bf16(d * plane_scale);
                z[c] = df_scale(z[c], rscale);
            }
            if constexpr (POOLED)
                *(uint2*)(out + pool_index(slot, plane_pairs(s), p, r, j0 & 31)) = *(const uint2*)dv;
            else
                *(uint2*)(dst + (size_t)(p >> 1) * 2 * total + ((p & 1) << 5)) = *(const uint2*)dv;
            plane_scale *= rinv;
        }
    }
    if (bnorm2) {
        // lanes 8q .. 8q + 7 hold block column Jq * 4 + q
        bsum += __shfl_xor_sync(0xffffffffu, bsum, 4);
        bsum += __shfl_xor_sync(0xffffffffu, bsum, 2);
        bsum += __shfl_xor_sync(0xffffffffu, bsum, 1);
        const int J = Jq * 4 + (lane >> 3);
        if ((lane & 7) == 0 && I <= J) bnorm2[(size_t)I * nb + J] = bsum;
    }
}

__global__ void __launch_bounds__(256) split_kernel(const double* __restrict__ F, int64_t ldf, int n, int n_pad,
                                                    df a, df b, float digit_scale, float rscale, int s,
                                                    __nv_bfloat16* __restrict__ out, double* red,
                                                    float* __restrict__ bnorm2) {
    const int nb = n_pad / 32, ns = n_pad / 128;
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    const bool vec = (ldf & 1) == 0 && ((uintptr_t)F & 15) == 0;
    const float rinv = 1.f / rscale;
    float tr = 0.f;
    for (int strip = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); strip < nb * ns; strip += warps)
        split_strip<false>(DenseRows{F, ldf, n, vec}, n, n_pad, a, b, digit_scale, rscale, rinv, s, out, bnorm2, strip,
                           lane, tr);
    if (red) {
        tr = warp_sum_f(tr);
        if (lane == 0) atomicAdd(red, (double)tr);
    }
}

// The splits of many matrices in one launch (a batch's f_0 for every
// instance): strip u of the launch belongs to the job with the largest
// strip0 <= u; the warp that takes a job's first strip also clears its
// four-double reduction slot.
__global__ void __launch_bounds__(256) split_group_kernel(const SplitJob* __restrict__ jobs, int njobs,
                                                          int total_strips) {
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int u = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < total_strips; u += warps) {
        int lo = 0, hi = njobs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].strip0 <= u)
                lo = mid;
            else
                hi = mid - 1;
        }
        const SplitJob& J = jobs[lo];
        const int strip = u - J.strip0;
        if (strip == 0 && J.zero4 && lane < 4) J.zero4[lane] = 0.0;
        const bool vec = (J.ldf & 1) == 0 && ((uintptr_t)J.F & 15) == 0;
        float tr = 0.f;
        split_strip<false>(DenseRows{J.F, J.ldf, J.n, vec}, J.n, J.n_pad, df{J.a_h, J.a_l}, df{J.b_h, J.b_l},
                           J.digit_scale, J.rscale, 1.f / J.rscale, J.s, J.out, nullptr, strip, lane, tr);
    }
}

// The split into pooled planes (block-sparse runs); pidx null: block norms
// only.
__global__ void __launch_bounds__(256) split_pool_kernel(const double* __restrict__ F, int64_t ldf, int n, int n_pad,
                                                         df a, df b, float digit_scale, float rscale, int s,
                                                         __nv_bfloat16* __restrict__ pool, const int* __restrict__ pidx,
                                                         float* __restrict__ bnorm2) {
    const int nb = n_pad / 32, ns = n_pad / 128;
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    const bool vec = (ldf & 1) == 0 && ((uintptr_t)F & 15) == 0;
    const float rinv = 1.f / rscale;
    float tr = 0.f;
    for (int strip = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); strip < nb * ns; strip += warps)
        split_strip<true>(DenseRows{F, ldf, n, vec}, n, n_pad, a, b, digit_scale, rscale, rinv, s, pool, bnorm2, strip,
                          lane, tr, pidx);
}

// The pooled split from CSR storage, over a list of strips (I * (n_pad /
// 128) + 128-column segment): the strips that hold a block of the pattern.
__global__ void __launch_bounds__(256) split_csr_pool_kernel(const int64_t* __restrict__ ptr,
                                                             const int* __restrict__ col,
                                                             const double* __restrict__ val, int n, int n_pad, df a,
                                                             df b, float digit_scale, float rscale, int s,
                                                             __nv_bfloat16* __restrict__ pool,
                                                             const int* __restrict__ pidx, float* __restrict__ bnorm2,
                                                             const int* __restrict__ strips, int nstrips) {
    __shared__ double rowbuf[8][128];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int warps = gridDim.x * (blockDim.x >> 5);
    const float rinv = 1.f / rscale;
    const CsrRows rows{ptr, col, val, n, rowbuf[warp]};
    float tr = 0.f;
    for (int q = blockIdx.x * (blockDim.x >> 5) + warp; q < nstrips; q += warps)
        split_strip<true>(rows, n, n_pad, a, b, digit_scale, rscale, rinv, s, pool, bnorm2, strips[q], lane, tr,
                          pidx);
}

// ---- tensor maps --------------------------------------------------------------

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// 3D map over the plane pairs of an s-plane buffer (plane_index): dims
// {2 n_pad, n_pad, pairs}, box {64, 128, pairs}: one box row is 128 bytes, a
// 32-wide k-chunk of two planes; 128-byte swizzle.
int make_plane_map(CUtensorMap* map, const __nv_bfloat16* planes, int n_pad, int s, int kc) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return PURIFY_ERR_UNSUPPORTED;
    if (((uintptr_t)planes & 15) || n_pad % TILE || kc != 32) return PURIFY_ERR_INVALID_ARG;
    const int np = plane_pairs(s);
    cuuint64_t dims[3] = {(cuuint64_t)2 * n_pad, (cuuint64_t)n_pad, (cuuint64_t)np};
    cuuint64_t strides[2] = {(cuuint64_t)n_pad * 4, (cuuint64_t)n_pad * n_pad * 4};
    cuuint32_t box[3] = {64, (cuuint32_t)TILE, (cuuint32_t)np};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)planes, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? PURIFY_OK : PURIFY_ERR_CUDA;
}

// 3D map over a pool of 32 x 32 block slots of np plane pairs (pool_index):
// dims {64, 32, np slots}, box {64, 32, 1}: one block of one plane pair per
// box, 128-byte swizzle (the same shared-memory image as the rows of a dense
// panel).
int make_pool_map(CUtensorMap* map, const __nv_bfloat16* pool, int slots, int np) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return PURIFY_ERR_UNSUPPORTED;
    if (((uintptr_t)pool & 15) || slots < 1 || np < 1 || np > 3) return PURIFY_ERR_INVALID_ARG;
    cuuint64_t dims[3] = {64, 32, (cuuint64_t)slots * np};
    cuuint64_t strides[2] = {128, 32 * 128};
    cuuint32_t box[3] = {64, 32, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)pool, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? PURIFY_OK : PURIFY_ERR_CUDA;
}

df to_df(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}

}  // namespace

KernelFn kernel_for(int kc, int s);

// k-chunk width: 32 (the paired plane layout stores 32-wide chunks).
int digit_kc_for(int, bool) { return 32; }

int digit_step_kc(const DigitStep&) { return 32; }

int digit_kc_candidates(int s, int* kc) {
    if (!kernel_for(32, s)) return 0;
    kc[0] = 32;
    return 1;
}

int digit_kc(int) { return 32; }

int digit_stages(int s, int kc) {
    if (kc != 32) return 0;
    const int stage_bytes = 2 * plane_pairs(s) * PAIR_BYTES;
    int st = (200 * 1024) / stage_bytes;
    if (st > MAX_STAGES) st = MAX_STAGES;
    return st;
}

size_t digit_smem_bytes(int s, int kc) {
    // alignment slack, operand stages, barriers and flags, then phase 2's E
    // staging (one EW-column piece per epilogue warp, digit plane and lane)
    return 1024 + (size_t)digit_stages(s, kc) * 2 * plane_pairs(s) * PAIR_BYTES + BAR_AREA +
           (size_t)kEpiWarps * s * 32 * EW * 2;
}

KernelFn kernel_for(int kc, int s) {
    if (s < 1 || s > 6 || kc != 32) return nullptr;
    return s <= 3 ? kernel_k32_lo(s) : kernel_k32_hi(s);
}

// Opt every instantiation into the full 227 KB of shared memory (once).
int prepare_kernel(KernelFn fn) {
    static std::mutex mu;
    static std::vector<KernelFn> done;
    std::lock_guard<std::mutex> g(mu);
    for (KernelFn f : done)
        if (f == fn) return PURIFY_OK;
    PURIFY_CUDA_TRY(cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    done.push_back(fn);
    return PURIFY_OK;
}

// The queue-launch instantiation for a largest digit count s (uniform: every
// product has s digits).
static KernelFn queue_kernel(int s, bool uniform) {
    if (uniform) return s <= 3 ? kernel_queue_uniform_lo(s) : kernel_queue_uniform_hi(s);
    return s <= 3 ? kernel_queue_lo(s) : kernel_queue_hi(s);
}

int prepare_digit_kernels() {
    for (int s = 1; s <= kMaxDigitPlanes; ++s) {
        KernelFn fn = kernel_for(32, s);
        if (fn) PURIFY_TRY(prepare_kernel(fn));
    }
    for (int s = 1; s <= kMaxDigitPlanes; ++s) {
        PURIFY_TRY(prepare_kernel(queue_kernel(s, false)));
        PURIFY_TRY(prepare_kernel(queue_kernel(s, true)));
        PURIFY_TRY(prepare_kernel(s <= 3 ? kernel_pool_lo(s) : kernel_pool_hi(s)));
    }
    return PURIFY_OK;
}

int fill_digit_params(const DigitStep& st, DigitGemmParams* p, CUtensorMap* ma, CUtensorMap* mb) {
    if (st.s_in < 1 || st.s_in > kMaxDigitPlanes || st.s_out < 0 || st.s_out > kMaxDigitPlanes)
        return PURIFY_ERR_INVALID_ARG;
    if (st.n <= 0 || st.n_pad % TILE || st.n > st.n_pad) return PURIFY_ERR_INVALID_ARG;
    if (st.rbits < 4 || st.rbits > 8) return PURIFY_ERR_INVALID_ARG;
    const int kc = digit_step_kc(st);
    if (st.a_idx) {
        // (kc_mask: one block-column bitset per 128-row panel, see
        // pool_chunk_word; out64: a pool of 32 x 32 float64 blocks)
        if (!st.b_idx || ((st.out || st.out64) && !st.out_idx) || st.a_slots < 1 || st.b_slots < 1 || !st.kc_mask ||
            st.kc_cnt)
            return PURIFY_ERR_INVALID_ARG;
        PURIFY_TRY(make_pool_map(ma, st.A, st.a_slots, plane_pairs(st.s_in)));
        PURIFY_TRY(make_pool_map(mb, st.B, st.b_slots, plane_pairs(st.s_in)));
    } else {
        PURIFY_TRY(make_plane_map(ma, st.A, st.n_pad, st.s_in, kc));
        PURIFY_TRY(make_plane_map(mb, st.B, st.n_pad, st.s_in, kc));
    }
    std::memset(p, 0, sizeof(*p));
    p->n = st.n;
    p->n_pad = st.n_pad;
    p->s_in = st.s_in;
    p->s_out = st.out ? st.s_out : 0;
    p->tiles_per_row = st.n_pad / TILE;
    p->scale_in_h = ldexpf(1.f, st.eA + st.eB - 16);
    p->e_scale = ldexpf(1.f, st.eA - 8);
    p->out_digit_scale = ldexpf(1.f, 8 - st.e_out);
    p->out_rscale = ldexpf(1.f, st.rbits);
    p->cP = to_df(st.cP);
    p->cE = to_df(st.cE);
    p->cI = to_df(st.cI);
    p->dY = to_df(st.dY);
    p->dI = to_df(st.dI);
    p->use_E = st.use_E;
    p->affine_out = !(st.dY == 1.0 && st.dI == 0.0);
    p->A = st.A;
    p->out = st.out;
    p->out64 = st.out64;
    p->red = st.red;
    p->kc_cnt = st.kc_cnt;
    p->kc_mask = st.kc_mask;
    p->kc_words = (st.n_pad / 32 + 63) / 64;
    p->bnorm2 = st.bnorm2;
    p->nb = st.n_pad / 32;
    p->ctl = st.ctl;
    p->a_idx = st.a_idx;
    p->b_idx = st.b_idx;
    p->out_idx = st.out_idx;
    if (st.kc_cnt && !st.kc_mask) return PURIFY_ERR_INVALID_ARG;
    if ((st.kc_cnt || st.bnorm2) && kc != 32) return PURIFY_ERR_INVALID_ARG;
    return PURIFY_OK;
}

static KernelFn pool_kernel(int s) { return s <= 3 ? kernel_pool_lo(s) : kernel_pool_hi(s); }

static int launch_kernel(const DigitLaunch& L, int s, int kc, int grid, cudaStream_t stream, bool uniform = false) {
    KernelFn fn = L.qprm ? queue_kernel(s, uniform) : (L.prms[0].a_idx ? pool_kernel(s) : kernel_for(kc, s));
    if (!fn || grid < 1 || L.stages < 1) return PURIFY_ERR_INVALID_ARG;
    PURIFY_TRY(prepare_kernel(fn));
    fn<<<grid, NTHREADS, digit_smem_bytes(s, kc), stream>>>(L);
    PURIFY_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return PURIFY_OK;
}

// Whole waves of the persistent grid stay whole; the tiles of the last,
// partial wave are cut into up to 4 k-ranges (each at least 4 k-chunks) so
// that their parts fill the grid.
void digit_split_plan(int tiles, int ctas, int k_chunks, int* split_begin, int* ways) {
    *split_begin = tiles;
    *ways = 1;
    if (ctas < 2 || tiles <= 0) return;
    const int full = tiles / ctas * ctas;
    const int tail = tiles - full;
    if (tail == 0) return;
    int w = std::min(4, ctas / tail);
    while (w > 1 && k_chunks / w < 4) --w;
    if (w < 2) return;
    *split_begin = full;
    *ways = w;
}

int launch_digit_step(const DigitStep& st, cudaStream_t stream) {
    DigitLaunch L;
    std::memset(&L, 0, sizeof(L));
    PURIFY_TRY(fill_digit_params(st, &L.prms[0], &L.maps[0], &L.maps[1]));
    L.ngroups = 1;
    const int T = st.n_pad / TILE;
    const int tiles = T * (T + 1) / 2;
    const int kc = digit_step_kc(st);
    L.stages = digit_stages(st.s_in, kc);
    L.scratch = st.scratch;
    L.err = st.err;
    L.wait_cycles = st.wait_cycles;
    if (!st.scratch || !st.err) return PURIFY_ERR_INVALID_ARG;
    L.split_begin = tiles;
    L.split_ways = 1;
    if (st.partial && st.split_cnt && !st.kc_cnt && st.split_ways != 1) {
        digit_split_plan(tiles, st.max_ctas, st.n_pad / kc, &L.split_begin, &L.split_ways);
        if (st.split_ways > 1 && L.split_ways > 1) {
            // a chosen number of ranges: at most 4, each of at least 4
            // k-chunks, and at most max_ctas parts in all (the partial buffer
            // holds digit_partial_floats(max_ctas))
            const int tail = tiles - L.split_begin;
            int w = st.split_ways < 4 ? st.split_ways : 4;
            while (w > 1 && ((st.n_pad / kc) / w < 4 || tail * w > st.max_ctas)) --w;
            L.split_ways = w;
            if (w < 2) L.split_begin = tiles;
        }
    }
    if (L.split_ways < 2) {
        L.split_begin = tiles;
        L.split_ways = 1;
    }
    L.num_items = L.split_begin + (tiles - L.split_begin) * L.split_ways;
    if (L.split_ways > 1 && (tiles - L.split_begin) * L.split_ways > st.max_ctas) return PURIFY_ERR_INVALID_ARG;
    if (L.split_ways > 1) {
        // per-region arrival counters of the split tiles, then the claim
        // counter (tiles - split_begin < max_ctas, so both fit in
        // digit_split_counters(max_ctas))
        const size_t counters = (size_t)kEpiWarps * (size_t)(tiles - L.split_begin);
        L.partial = st.partial;
        L.split_cnt = st.split_cnt;
        L.claim = st.split_cnt + counters;
        PURIFY_CUDA_TRY(cudaMemsetAsync(st.split_cnt, 0, sizeof(int) * (counters + 1), stream));
    }
    const int grid = L.num_items < st.max_ctas ? L.num_items : st.max_ctas;
    return launch_kernel(L, st.s_in, kc, grid, stream);
}

int launch_digit_group(int s, const DigitStep* steps, int count, const int4* work, int num_items,
                       float2* scratch, int max_ctas, int* err, cudaStream_t stream, long long wait_cycles) {
    if (s < 1 || s > kMaxDigitPlanes || count < 1 || count > GMAX || !work || !scratch || !err)
        return PURIFY_ERR_INVALID_ARG;
    if (num_items <= 0) return PURIFY_OK;
    DigitLaunch L;
    std::memset(&L, 0, sizeof(L));
    const bool sparse = steps[0].kc_cnt || steps[0].bnorm2;
    for (int g = 0; g < count; ++g) {
        if (steps[g].s_in != s || (bool)(steps[g].kc_cnt || steps[g].bnorm2) != sparse)
            return PURIFY_ERR_INVALID_ARG;
        PURIFY_TRY(fill_digit_params(steps[g], &L.prms[g], &L.maps[2 * g], &L.maps[2 * g + 1]));
    }
    const int kc = digit_kc_for(s, sparse);
    L.ngroups = count;
    L.work = work;
    L.num_items = num_items;
    L.stages = digit_stages(s, kc);
    L.scratch = scratch;
    L.err = err;
    L.wait_cycles = wait_cycles;
    L.split_begin = num_items;  // grouped launches are not split
    L.split_ways = 1;
    const int grid = num_items < max_ctas ? num_items : max_ctas;
    return launch_kernel(L, s, kc, grid, stream);
}

int queue_kc(int) { return 32; }

int fill_queue_product(const DigitStep& st0, int smax, DigitGemmParams* p, CUtensorMap* maps) {
    if (st0.s_in > smax || st0.kc_cnt || st0.bnorm2) return PURIFY_ERR_INVALID_ARG;
    DigitStep st = st0;
    st.kc = queue_kc(smax);  // one k-chunk width for the whole launch
    CUtensorMap m[2];        // encoded at their own alignment, then copied to the staging area
    PURIFY_TRY(fill_digit_params(st, p, &m[0], &m[1]));
    std::memcpy(maps, m, sizeof(m));
    return PURIFY_OK;
}

int launch_digit_queue(int smax, bool uniform, const DigitGemmParams* prm, const CUtensorMap* maps, int* cnt,
                       int* ticket, const int4* work, int num_items, float2* scratch, int max_ctas, int* err,
                       cudaStream_t stream, long long wait_cycles) {
    if (smax < 1 || smax > kMaxDigitPlanes || !prm || !maps || !cnt || !ticket || !work || !scratch || !err)
        return PURIFY_ERR_INVALID_ARG;
    if (num_items <= 0) return PURIFY_OK;
    DigitLaunch L;
    std::memset(&L, 0, sizeof(L));
    L.qprm = prm;
    L.qmaps = maps;
    L.qcnt = cnt;
    L.work = work;
    L.num_items = num_items;
    L.stages = digit_stages(smax, queue_kc(smax));
    L.scratch = scratch;
    L.err = err;
    L.wait_cycles = wait_cycles;
    L.claim = ticket;  // every item claimed in ticket order
    L.split_begin = 0;             // (item_of reads the work list: no split parts)
    L.split_ways = 1;
    const int grid = num_items < max_ctas ? num_items : max_ctas;
    return launch_kernel(L, smax, queue_kc(smax), grid, stream, uniform);
}

int split_strips(int n_pad) { return (n_pad / 32) * (n_pad / 128); }

int make_split_job(const double* F, int64_t ldf, int n, int n_pad, double a, double b, int e, int s, int rbits,
                   __nv_bfloat16* out, double* zero4, int strip0, SplitJob* job) {
    if (s < 1 || s > kMaxDigitPlanes || n <= 0 || n_pad < n || n_pad % 128 || n_pad > (1 << 17) || rbits < 4 ||
        rbits > 8 || !F || !out || ldf < n || strip0 < 0)
        return PURIFY_ERR_INVALID_ARG;
    const df ad = to_df(a), bd = to_df(b);
    job->F = F;
    job->ldf = ldf;
    job->n = n;
    job->n_pad = n_pad;
    job->a_h = ad.h;
    job->a_l = ad.l;
    job->b_h = bd.h;
    job->b_l = bd.l;
    job->digit_scale = ldexpf(1.f, 8 - e);
    job->rscale = ldexpf(1.f, rbits);
    job->s = s;
    job->out = out;
    job->zero4 = zero4;
    job->strip0 = strip0;
    return PURIFY_OK;
}

int launch_split_group(const SplitJob* jobs, int njobs, int total_strips, cudaStream_t stream) {
    if (njobs <= 0 || total_strips <= 0) return PURIFY_OK;
    if (!jobs) return PURIFY_ERR_INVALID_ARG;
    int64_t blocks = ((int64_t)total_strips + 7) / 8;  // 8 warps per CTA, one strip each
    if (blocks > 152 * 8) blocks = 152 * 8;
    split_group_kernel<<<(unsigned)blocks, 256, 0, stream>>>(jobs, njobs, total_strips);
    PURIFY_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return PURIFY_OK;
}

int launch_split_pool(const double* F, int64_t ldf, int n, int n_pad, double a, double b, int e, int s, int rbits,
                      __nv_bfloat16* pool, const int* pidx, float* bnorm2, cudaStream_t stream) {
    if (s < 1 || s > kMaxDigitPlanes || n <= 0 || n_pad < n || n_pad % 128 || n_pad > (1 << 17) || rbits < 4 ||
        rbits > 8 || (pidx && !pool) || (!pidx && !bnorm2))
        return PURIFY_ERR_INVALID_ARG;
    const int64_t strips = (int64_t)(n_pad / 32) * (n_pad / 128);
    int64_t blocks = (strips + 7) / 8;
    if (blocks > 152 * 8) blocks = 152 * 8;
    split_pool_kernel<<<(unsigned)blocks, 256, 0, stream>>>(F, ldf, n, n_pad, to_df(a), to_df(b), ldexpf(1.f, 8 - e),
                                                             ldexpf(1.f, rbits), s, pool, pidx, bnorm2);
    PURIFY_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return PURIFY_OK;
}

int launch_split_csr_pool(const int64_t* ptr, const int* col, const double* val, int n, int n_pad, double a,
                          double b, int e, int s, int rbits, __nv_bfloat16* pool, const int* pidx, float* bnorm2,
                          const int* strips, int nstrips, cudaStream_t stream) {
    if (s < 1 || s > kMaxDigitPlanes || n <= 0 || n_pad < n || n_pad % 128 || n_pad > (1 << 18) || rbits < 4 ||
        rbits > 8 || (pidx && !pool) || (!pidx && !bnorm2) || !ptr || nstrips < 0 || (nstrips && !strips))
        return PURIFY_ERR_INVALID_ARG;
    if (nstrips == 0) return PURIFY_OK;
    int64_t blocks = ((int64_t)nstrips + 7) / 8;
    if (blocks > 152 * 8) blocks = 152 * 8;
    split_csr_pool_kernel<<<(unsigned)blocks, 256, 0, stream>>>(ptr, col, val, n, n_pad, to_df(a), to_df(b),
                                                                 ldexpf(1.f, 8 - e), ldexpf(1.f, rbits), s, pool,
                                                                 pidx, bnorm2, strips, nstrips);
    PURIFY_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return PURIFY_OK;
}

int launch_split(const double* F, int64_t ldf, int n, int n_pad, double a, double b, int e, int s,
                 int rbits, __nv_bfloat16* out, double* red, cudaStream_t stream, float* bnorm2) {
    if (s < 1 || s > kMaxDigitPlanes || n <= 0 || n_pad < n || n_pad % 128 || n_pad > (1 << 17) || rbits < 4 ||
        rbits > 8)
        return PURIFY_ERR_INVALID_ARG;
    const int64_t strips = (int64_t)(n_pad / 32) * (n_pad / 128);
    int64_t blocks = (strips + 7) / 8;  // 8 warps per CTA, one 32 x 128 strip each
    if (blocks > 152 * 8) blocks = 152 * 8;
    split_kernel<<<(unsigned)blocks, 256, 0, stream>>>(F, ldf, n, n_pad, to_df(a), to_df(b), ldexpf(1.f, 8 - e),
                                                        ldexpf(1.f, rbits), s, out, red, bnorm2);
    PURIFY_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return PURIFY_OK;
}

}  // namespace purify
