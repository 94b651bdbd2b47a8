// Digit-plane symmetric products on the tcgen05 tensor cores (sm_103a).
//
// A float64 matrix X with |X_ij| <= 2^e is held as s bf16 "digit planes"
//     X = 2^(e-8) * sum_p V_p,    V_p = d_p * 2^(-r p),  d_p integer,
// with a leading digit of 8 bits (|d_0| <= 256) and remainder digits of
// r = 7 bits (|d_p| <= 65; r = 6 above n = 4096), all round-to-nearest.
// bf16 stores every such value exactly.  The product of two such
// matrices is the sum over digit pairs (p, q) of V_p V_q^T.  Pairs with
// p + q = l form "level" l; levels 0, 1 and 2 each get their own fp32
// accumulator in tensor memory and are exact: by Cauchy-Schwarz a row of d_0
// has 2-norm <= 256 ||X_i||_2 / 2^e + sqrt(n)/2, so level 0 and level 1 stay
// below 2^24 in their own units for n <= 8192; level 2 holds the sum of
// squares of the remainder digits on the product's diagonal, about
// n 2^(2r) / 12, which the choice of r keeps below 2^24 for uniformly
// distributed remainders (8-bit remainders exceed it at n = 4096).  All levels
// >= 3 share a fourth accumulator whose rounding sits 2^-48 below the
// leading term.  Pairs with p + q >= s are dropped (their size is that of
// the digits' own truncation).  The four accumulators are recombined in
// double-float (pairs of fp32) arithmetic in the epilogue, which also
// applies the step's polynomial (Eq. 4 / Eq. 5 / Algorithm 1's 3S - 2S X_s),
// re-splits the result into the next step's digit planes, optionally writes
// float64, and reduces trace and Frobenius norms.
//
// Only output tiles on or above the diagonal are formed; each is written
// twice (itself and its mirror), so every product is exactly symmetric.
// Exact symmetry matters: antisymmetric rounding errors are not damped by
// the purification maps.
//
// Structure of one CTA (one 128 x 128 output tile at a time, 64 + 32 EPI_WARPS
// threads):
//   warp 0  TMA producer: per 32-wide k-chunk one 3D TMA load of the A row
//           panel's plane pairs (128-byte box rows: two planes' chunks side
//           by side, 128-byte swizzle) and one of the B row panel's
//   warp 1  TMEM allocator and MMA issuer (tcgen05.mma kind::f16, bf16 in,
//           fp32 accumulate, M = N = 128, K = 16)
//   warps 2.. epilogue (tcgen05.ld; warp w reads TMEM lane quarter w % 4 and
//           the (w - 2) / 4-th group of EPI_COLS columns).  Phase 1 drains
//           the accumulators into a double-float tile in global scratch and
//           releases TMEM; phase 2 (polynomial, re-split, stores) then
//           overlaps the next tile's MMAs, with the E digits of the next pass
//           copied into shared memory while the current pass computes.
// Tiles are numbered in bands of 12 tile columns so that the CTAs resident
// at one time share row panels in L2.  Whole waves of tiles go round-robin
// over the CTAs; the parts of a split last wave are claimed at run time.
// Every wait on an mbarrier is bounded; on time-out the CTA records an error
// flag, waits (bounded) for its own copies and MMAs, frees its tensor memory
// and exits.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "digits_tc.h"

namespace purify {
namespace dk {

constexpr int TILE = 128;        // output tile edge
constexpr int BAND = 12;         // tile columns per rasterisation band
constexpr int MAX_STAGES = 8;
constexpr int NUM_ACC = 4;       // tensor-memory accumulators (levels 0, 1, 2, >= 3)
constexpr int EPI_WARPS = kEpiWarps;      // 8 or 16
constexpr int NTHREADS = 64 + 32 * EPI_WARPS;
constexpr int EPI_COLS = TILE * 4 / EPI_WARPS;  // columns of one epilogue warp's region
// registers per thread: each of the SM's four sub-partitions holds 16384 and
// takes every fourth warp
constexpr int MAX_REGS = (16384 / (32 * ((NTHREADS / 32 + 3) / 4))) / 8 * 8;
constexpr int EW = 8;            // epilogue columns per pass (a multiple of 8)
constexpr int BAR_AREA = 512;    // bytes of barriers and flags after the operand stages
constexpr long long WAIT_CYCLES = 1ll << 31;  // one wait gives up after ~1 s at 2 GHz
// Bits of the device error flag (OR-ed into *L.err): which role's wait gave
// up, and the internal check that a tile's k-chunk count matches its bitmask.
constexpr int ERR_PRODUCER_WAIT = 1, ERR_MMA_WAIT = 2, ERR_EPI_WAIT = 4, ERR_PLAN = 8, ERR_CLAIM_WAIT = 16;

// ---- PTX wrappers ------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0,
                                            int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
        "l"((uint64_t)map), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

// 16-byte asynchronous copy global -> shared (L2 only), its group commit and wait.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

// 32 lanes x 32 bits, 16 consecutive columns per thread.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor for a K-major operand tile of 128-byte
// rows written by TMA with the 128-byte swizzle (a plane pair: two planes'
// 32-wide k-chunks side by side): 8-row groups 1024 bytes apart; one K = 16
// step advances 32 bytes, the pair's second plane starts 64 bytes in.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    constexpr uint64_t layout = 2;                   // 128-byte swizzle
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);          // start address
    d |= (uint64_t)1 << 16;                          // leading byte offset (unused here)
    d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset
    d |= (uint64_t)1 << 46;                          // descriptor version (tcgen05)
    d |= layout << 61;
    return d;
}

constexpr int PAIR_BYTES = TILE * 128;  // one plane pair of a 128-row panel, one 32-wide k-chunk

// Descriptor offset (16-byte units) of plane p's 16-wide k-step kk inside an
// operand's stage region.
__host__ __device__ constexpr int plane_desc_off(int p, int kk) {
    return ((p >> 1) * PAIR_BYTES + (p & 1) * 64 + kk * 32) >> 4;
}

// Instruction descriptor: kind::f16, bf16 A and B (K-major), fp32 D,
// M = 128, N = 128.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TILE >> 3) << 17) |
                           ((uint32_t)(TILE >> 4) << 24);

// ---- double-float arithmetic (pairs of fp32) ---------------------------------

struct df {
    float h, l;
};

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df df_add_f(df x, float y) {
    const df s = two_sum(x.h, y);
    return fast_two_sum(s.h, __fadd_rn(s.l, x.l));
}

__device__ __forceinline__ df df_add(df x, df y) {
    const df s = two_sum(x.h, y.h);
    const df t = two_sum(x.l, y.l);
    df u = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
    return fast_two_sum(u.h, __fadd_rn(u.l, t.l));
}

__device__ __forceinline__ df df_mul(df x, df y) {
    const float p = __fmul_rn(x.h, y.h);
    float e = __fmaf_rn(x.h, y.h, -p);
    e = __fmaf_rn(x.h, y.l, e);
    e = __fmaf_rn(x.l, y.h, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ df df_scale(df x, float pow2) { return {x.h * pow2, x.l * pow2}; }

// float64 -> double-float: the nearest float and the float of the remainder
__device__ __forceinline__ df dev_df(double x) {
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
}

// ---- digits: float32 additions and bit operations only ---------------------
// (both exact for digits, so no rounding or conversion instruction is needed)

// Nearest integer, ties to even, for |x| < 2^22: after adding 1.5 * 2^23 the
// sum has no fraction bits, and the subtraction is exact.
__device__ __forceinline__ float round_digit(float x) {
    constexpr float kMagic = 12582912.f;  // 1.5 * 2^23
    return __fsub_rn(__fadd_rn(x, kMagic), kMagic);
}

// bf16 of a float whose low 16 bits are zero (a digit: an integer of at most
// 8 significant bits times a power of two), exactly.
__device__ __forceinline__ __nv_bfloat16 digit_to_bf16(float v) {
    return __ushort_as_bfloat16((unsigned short)(__float_as_uint(v) >> 16));
}

__device__ __forceinline__ float bf16_to_float(__nv_bfloat16 v) {
    return __uint_as_float((unsigned int)__bfloat16_as_ushort(v) << 16);
}

// ---- kernel parameters ------------------------------------------------------

struct DigitGemmParams {
    int n, n_pad, s_in;      // matrix size, padded size (multiple of 128), digits of A and B
    int s_out;               // digits of the output (0 = none)
    int tiles_per_row;       // n_pad / 128
    float scale_in_h;        // 2^(eA + eB - 16): value of one unit of the accumulators
    float e_scale;           // 2^(eA - 8): value of one unit of A's planes (for E)
    float out_digit_scale;   // 2^(8 - e_out)
    float out_rscale;        // 2^r of the output's remainder digits
    df cP, cE, cI, dY, dI;   // Y = cP P + cE E + cI I;  out = dY Y + dI I
    int use_E;               // E = A (the matrix in the A operand)
    int affine_out;          // (dY, dI) != (1, 0)
    const __nv_bfloat16* A;  // A's s_in planes (for E), paired layout (plane_index)
    __nv_bfloat16* out;      // output's s_out planes, paired layout (may be null)
    double* out64;           // float64 output n x n (leading dimension n) or null
    double* red;             // [0] trace(Y), [1] ||E - P||_F^2, [2] ||Y||_F^2 (atomics) or null
    // block sparsity (null: dense): per upper tile t = tj (tj + 1) / 2 + ti,
    // kc_cnt[t] = number of 32-wide k-chunks that contribute (-1: all of
    // them) and kc_mask[t * kc_words ..] their bitmask (bit k of word k / 64);
    // bnorm2[I * nb + J] receives ||out block (I, J)||_F^2 for upper 32 x 32
    // blocks I <= J (k-chunk width must be 32)
    const int* kc_cnt;
    const unsigned long long* kc_mask;
    int kc_words;
    float* bnorm2;
    int nb;
    // device-side control of a single product (null: the fields above)
    const DevStep* ctl;
    // queue launches: the products whose outputs this one reads as A and as B
    // (-1: written before the launch; an item waits for the two row panels
    // it reads), up to two products whose every item must have finished
    // before this one starts (they read the buffer this one overwrites; -1:
    // none), and the offset of this product's counters in DigitLaunch::qcnt
    // (tiles_per_row row-panel counts, then the total).  Unused elsewhere.
    int q_depA, q_depB, q_war0, q_war1, q_cnt;
    // pooled planes (block-sparse runs, QM = 3): A, B and the output as pools
    // of 32 x 32 block slots (pool_index), found through nb x nb slot tables
    // (slot 0: the shared zero block; an output block with slot 0 is not
    // stored); maps[0] and maps[1] are then tensor maps over A's and B's
    // pools (make_pool_map).  Null elsewhere.
    const int* a_idx;
    const int* b_idx;
    const int* out_idx;
};

// Element offset of (plane p, row r, column c) of the 32 x 32 block in pool
// slot k of a pool with np plane pairs per slot: a slot holds its block's
// plane pairs, each 32 rows of 64 elements (the two planes' 32 columns side by
// side, as in the dense paired layout).
__host__ __device__ inline size_t pool_index(int k, int np, int p, int r, int c) {
    return ((size_t)(k * np + (p >> 1)) * 32 + r) * 64 + ((p & 1) << 5) + c;
}

// Pooled runs: kc_mask holds one bitset of kc_words words per 128-row panel
// (the block columns in which one of the panel's four block rows has a
// block); tile (ti, tj) walks the k-chunks set in both panels' bitsets.
__device__ __forceinline__ unsigned long long pool_chunk_word(const DigitGemmParams& P, int ti, int tj, int w) {
    return P.kc_mask[(size_t)ti * P.kc_words + w] & P.kc_mask[(size_t)tj * P.kc_words + w];
}
__device__ __forceinline__ int pool_chunk_count(const DigitGemmParams& P, int ti, int tj) {
    int c = 0;
    for (int w = 0; w < P.kc_words; ++w) c += __popcll(pool_chunk_word(P, ti, tj, w));
    return c;
}
// (warp-collective) whether tile (ti, tj) has any k-chunk
__device__ __forceinline__ bool pool_chunks_any(const DigitGemmParams& P, int ti, int tj, int lane) {
    unsigned long long a = 0ull;
    for (int w = lane; w < P.kc_words; w += 32) a |= pool_chunk_word(P, ti, tj, w);
    return __any_sync(0xffffffffu, a != 0ull);
}

// Products per grouped launch, whose tensor maps and parameters travel as
// kernel parameters (grid constants).  Queue launches read theirs from
// global memory instead, each CTA fencing a map through the tensor-map proxy
// before its copies use it (maps rewritten at the same address were seen
// stale by TMA without that fence).
constexpr int GMAX = 64;

// One launch: products g = 0 .. ngroups-1 (tensor maps and parameters by
// value) and the list of work items {g, ti, tj, -} in global memory, or, when
// `work` is null, all upper tiles of product 0 in banded order.
//
// Split tiles (single launches only): the tiles from `split_begin` on in
// banded order (the last, partial wave of the persistent grid) are each cut
// into `split_ways` ranges of k-chunks, one work item per range, so that the
// last wave fills the grid.  Each epilogue warp of a part stores its raw
// accumulators for its 32 x 64 region in `partial`, then counts itself in
// split_cnt[slot][region]; the warp that arrives last adds the parts in part
// order (a fixed order, so the result does not depend on which part finished
// last) and runs the epilogue for that region.  Nothing waits on another CTA.
struct DigitLaunch {
    CUtensorMap maps[2 * GMAX];      // A and B map of product g at [2g], [2g + 1]
    DigitGemmParams prms[GMAX];
    int ngroups;
    const int4* work;
    int num_items;                   // work items: tiles, tile parts (single) or list entries (group)
    int stages;                      // depth of the shared-memory ring
    float2* scratch;                 // per CTA 128 x 128 double-float tile
    int* err;                        // device error flag (ERR_* bits)
    long long wait_cycles;           // bound of one work wait (claim, stage, tensor-memory
                                     // hand-offs); the waits for copies and MMAs in flight at
                                     // teardown keep WAIT_CYCLES
    int split_begin;                 // single launches: first split tile (== tiles: none)
    int split_ways;                  // parts per split tile (1: none)
    float* partial;                  // [slot][part][region 8][acc 4][16-col group 4][row 32][16]
    int* split_cnt;                  // [slot][region 8], zero at launch
    int* claim;                      // split launches: counter of claimed split items, zero at launch
    // queue mode (many products in one launch; null: off): every product's
    // parameters and its A and B tensor maps in global memory (prms and maps
    // are unused), each product with its own digit count <= the kernel's S.
    // An item's operands are loaded once the row panels it reads are
    // complete (see DigitGemmParams::q_depA): each epilogue warp of a tile
    // (ti, tj) counts itself in the product's counters of panels ti and tj and
    // in its total after its stores.
    const DigitGemmParams* qprm;
    const CUtensorMap* qmaps;        // [2 * products]
    int* qcnt;                       // zero at launch
};

// Items of a split launch's last wave, and every item of a queue launch, are
// claimed at run time (an atomic counter): a CTA whose earlier items ran slow
// leaves the rest to CTAs that are free.  The producer claims and hands each
// claimed item to the MMA and epilogue warps through a ring of MAX_CLAIMS
// shared-memory slots.
constexpr int MAX_CLAIMS = 8;

constexpr int REGION_FLOATS = NUM_ACC * EPI_COLS * 32;  // one epilogue warp's accumulators

__device__ __forceinline__ void decode_banded(int t, int T, int& ti, int& tj);

// Work item t -> product g, tile (ti, tj), and for a part of a split tile
// its slot (index among the split tiles) and part; slot = -1 otherwise.
__device__ __forceinline__ void item_of(const DigitLaunch& L, int t, int& g, int& ti, int& tj, int& slot,
                                        int& part) {
    slot = -1;
    part = 0;
    if (L.work) {
        const int4 w = L.work[t];
        g = w.x;
        ti = w.y;
        tj = w.z;
    } else {
        g = 0;
        int tile = t;
        if (t >= L.split_begin) {
            const int u = t - L.split_begin;
            slot = u / L.split_ways;
            part = u - slot * L.split_ways;
            tile = L.split_begin + slot;
        }
        decode_banded(tile, L.prms[0].tiles_per_row, ti, tj);
    }
}

// The k-chunks of a dense item: all of them, or the part's range.
__device__ __forceinline__ void dense_k_range(const DigitLaunch& L, int nkt, int slot, int part, int& kb, int& nk) {
    if (slot < 0) {
        kb = 0;
        nk = nkt;
    } else {
        kb = part * nkt / L.split_ways;
        nk = (part + 1) * nkt / L.split_ways - kb;
    }
}

template <bool Q>
__device__ __forceinline__ const DigitGemmParams& params_of(const DigitLaunch& L, int g) {
    if constexpr (Q)
        return L.qprm[g];
    else
        return L.prms[g];
}

// Queue mode: wait (bounded) until a counter reaches `need` epilogue-warp
// completions; false when the wait gives up (at the bound, or at once when
// another CTA has failed: the count may then never be reached).  The acquire
// orders the counted warps' plane stores before this thread's later copies,
// and the proxy fence makes them visible to the tensor copies (async proxy).
__device__ __forceinline__ bool wait_count(const DigitLaunch& L, const int* c, int need, long long limit) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(c) : "memory");
    if (v < need) {
        const long long t0 = clock64();
        do {
            if (clock64() - t0 > limit || *(volatile int*)L.err) return false;
            __nanosleep(64);
            asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(c) : "memory");
        } while (v < need);
    }
    asm volatile("fence.proxy.async.global;" ::: "memory");
    return true;
}

// Row panel r of product d complete: every tile touching it (tiles_per_row
// of them) counted by all epilogue warps.
__device__ __forceinline__ bool wait_panel(const DigitLaunch& L, int d, int r, long long limit) {
    const DigitGemmParams& D = L.qprm[d];
    return wait_count(L, L.qcnt + D.q_cnt + r, EPI_WARPS * D.tiles_per_row, limit);
}

// Every item of product d finished.
__device__ __forceinline__ bool wait_all(const DigitLaunch& L, int d, long long limit) {
    const DigitGemmParams& D = L.qprm[d];
    const int T = D.tiles_per_row;
    return wait_count(L, L.qcnt + D.q_cnt + T, EPI_WARPS * (T * (T + 1) / 2), limit);
}

// A tensor map in global memory, written by the host before the launch, is
// read by the copy engine through the tensor-map proxy: acquire it first.
__device__ __forceinline__ void acquire_map(const CUtensorMap* m) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)m) : "memory");
}

template <int SS>
__device__ __forceinline__ void issue_chunk(uint32_t tmem, uint64_t da, uint64_t db, uint32_t later);

// issue_chunk for a digit count known at run time (<= SS)
template <int SS>
__device__ __forceinline__ void issue_chunk_runtime(int s, uint32_t tmem, uint64_t da, uint64_t db, uint32_t later) {
    if constexpr (SS >= 1) {
        if (s == SS) {
            issue_chunk<SS>(tmem, da, db, later);
            return;
        }
        issue_chunk_runtime<SS - 1>(s, tmem, da, db, later);
    }
}

// The unrolled MMA issue of one 32-wide k-chunk for SS digit planes (pairs
// p + q < SS; levels 0..2 in their own accumulators, >= 3 in the fourth),
// pair by pair with a pair's two 16-wide k-steps back to back (runs of MMAs
// into one accumulator).  A's plane pairs at da, B's at db.
template <int SS>
__device__ __forceinline__ void issue_chunk(uint32_t tmem, uint64_t da, uint64_t db, uint32_t later) {
#pragma unroll
    for (int p = 0; p < SS; ++p) {
#pragma unroll
        for (int q = 0; q < SS - p; ++q) {
            const int a = (p + q < NUM_ACC - 1) ? p + q : NUM_ACC - 1;
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
                // the first write of accumulator a in a tile is pair (0, a) at
                // k = 0; all later ones accumulate
                const uint32_t acc_in = (kk > 0 || p > 0 || q > NUM_ACC - 1) ? 1u : later;
                mma_bf16(tmem + (uint32_t)(a * TILE), da + (uint64_t)plane_desc_off(p, kk),
                         db + (uint64_t)plane_desc_off(q, kk), IDESC, acc_in);
            }
        }
    }
}

// Tile t of the upper triangle (ti <= tj) of a T x T tile grid, in bands of
// BAND tile columns; inside a band row by row.
__device__ __forceinline__ void decode_banded(int t, int T, int& ti, int& tj) {
    int b0 = 0;
    for (;;) {
        const int b1 = min(T, b0 + BAND);
        const int cnt = (b1 * (b1 + 1) - b0 * (b0 + 1)) / 2;
        if (t < cnt || b1 == T) {
            for (int r = 0;; ++r) {
                const int first = max(b0, r);
                const int c = b1 - first;
                if (t < c) {
                    ti = r;
                    tj = first + t;
                    return;
                }
                t -= c;
            }
        }
        t -= cnt;
        b0 = b1;
    }
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Bounded wait measured from its own start: false when it gives up.  A phase
// that has completed already returns at the first test, without reading the
// clock (the fast path of the pipeline's hand-offs).
__device__ __forceinline__ bool mbar_wait_for(uint32_t bar, uint32_t parity, long long limit = WAIT_CYCLES) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

// Persistent CTA: work items blockIdx.x, blockIdx.x + gridDim.x, ...  The
// four accumulators of a tile are drained into a double-float tile in the
// CTA's scratch (global, 128 x 128 x 8 bytes) so that tensor memory is
// released before the polynomial, the re-split and the stores; those overlap
// the next tile's MMAs.  All digit counts of a launch are S.
// QM: 0 = a single or grouped launch; 1 = a queue launch (per-product
// parameters and tensor maps in device memory, dependency waits and
// completion counts) whose products have digit counts up to S, read at run
// time; 2 = a queue launch whose products all have S digits.  Separate
// instantiations, so that launches with one digit count keep it a
// compile-time constant throughout (a run-time count in the epilogue costs
// about 4 % of a product).
template <int KC, int S, int QM>
__global__ void __maxnreg__(MAX_REGS) digit_gemm_kernel(const __grid_constant__ DigitLaunch L) {
    constexpr bool Q = QM == 1 || QM == 2;  // queue launch
    constexpr bool QRT = QM == 1;           // digit counts read at run time
    constexpr bool POOL = QM == 3;          // pooled planes (block-sparse runs)
    static_assert(KC == 32, "digit planes are stored for 32-wide k-chunks");
    constexpr int NP = plane_pairs(S);           // plane pairs of one operand per stage
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1024-byte aligned operand area: stages x (A planes | B planes)
    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr int stage_bytes = 2 * NP * PAIR_BYTES;
    const int stages = L.stages;
    uint64_t* bars = (uint64_t*)(base + (size_t)stages * stage_bytes);
    // bars: full[stages] | empty[stages] | tmem_full | tmem_empty | drain | claim[MAX_CLAIMS] |
    // claim_free[MAX_CLAIMS]
    uint64_t* full_bar = bars;
    uint64_t* empty_bar = bars + stages;
    uint64_t* tmem_full = bars + 2 * stages;
    uint64_t* tmem_empty = tmem_full + 1;
    uint64_t* drain = tmem_full + 2;
    uint64_t* claim_bar = drain + 1;                // [MAX_CLAIMS] ring: slot published
    uint64_t* claim_free = claim_bar + MAX_CLAIMS;  // [MAX_CLAIMS] ring: slot read by every consumer
    uint32_t* tmem_slot = (uint32_t*)(claim_free + MAX_CLAIMS);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    volatile int* claimed = abort_flag + 1;  // [MAX_CLAIMS] item (-1: none left)
    // phase 2's E digits, fetched one pass ahead: [epilogue warp][plane][lane] x EW / 8 uint4
    uint4* e_stage = (uint4*)((uint8_t*)bars + BAR_AREA);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int num_items = L.num_items;
    const long long wait = L.wait_cycles > 0 ? L.wait_cycles : WAIT_CYCLES;
    // a step controlled on the device: only the launch whose digit count the
    // schedule chose runs, and none once the run has stopped (uniform over
    // the grid: the control was written by an earlier kernel)
    if (L.prms[0].ctl) {
        const DevStep* c = L.prms[0].ctl;
        if (c->done || c->s_in != S) return;
    }

    if (threadIdx.x == 0) {
        for (int i = 0; i < 2 * stages; ++i) mbar_init(smem_u32(&bars[i]), 1);
        mbar_init(smem_u32(tmem_full), 1);
        mbar_init(smem_u32(tmem_empty), EPI_WARPS);
        mbar_init(smem_u32(drain), 1);
        for (int i = 0; i < MAX_CLAIMS; ++i) {
            mbar_init(smem_u32(&claim_bar[i]), 1);
            mbar_init(smem_u32(&claim_free[i]), 1 + EPI_WARPS);  // the MMA thread and each epilogue warp
        }
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1) tmem_alloc(smem_u32(tmem_slot), NUM_ACC * TILE);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    // Work items of this CTA, the same sequence in every role: whole waves
    // round-robin (blockIdx.x + k gridDim.x), then, in a launch with a claim
    // counter, items claimed in ticket order by the producer (-1 ends the
    // sequence) and handed to the MMA thread and the epilogue warps through a
    // ring of MAX_CLAIMS slots.  A queue launch claims every item: an item is
    // then only ever claimed after every item before it, so the items it
    // waits for are held by CTAs that are running.
    const bool claiming = L.claim != nullptr;
    const int static_end = claiming ? L.split_begin : num_items;
    int n_claims = 0;  // producer: claims published; consumers: claims taken
    bool ended = false;  // producer: a -1 has been published
    auto publish = [&](int t) -> bool {
        const int slot = n_claims % MAX_CLAIMS;
        const int round = n_claims / MAX_CLAIMS;
        if (round > 0 && !mbar_wait_for(smem_u32(&claim_free[slot]), (uint32_t)((round - 1) & 1), wait)) {
            atomicOr(L.err, ERR_CLAIM_WAIT);
            *abort_flag = 1;
            return false;
        }
        claimed[slot] = t;
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&claim_bar[slot])) : "memory");
        ++n_claims;
        if (t < 0) ended = true;
        return true;
    };
    auto producer_claim = [&]() -> int {
        if (*abort_flag) return -1;
        int t = L.split_begin + atomicAdd(L.claim, 1);
        if (t >= num_items) t = -1;
        return publish(t) ? t : -1;
    };
    auto consumer_take = [&]() -> int {  // one thread per role
        if (*abort_flag) return -1;
        const int slot = n_claims % MAX_CLAIMS;
        if (!mbar_wait_for(smem_u32(&claim_bar[slot]), (uint32_t)((n_claims / MAX_CLAIMS) & 1), wait)) {
            atomicOr(L.err, ERR_CLAIM_WAIT);
            *abort_flag = 1;
            return -1;
        }
        const int t = claimed[slot];
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&claim_free[slot])) : "memory");
        ++n_claims;
        return t;
    };
    auto first_item = [&](bool producer) -> int {
        if ((int)blockIdx.x < static_end) return blockIdx.x;
        if (!claiming) return -1;
        return producer ? producer_claim() : consumer_take();
    };
    auto next_item = [&](int t, bool producer) -> int {
        if (t + (int)gridDim.x < static_end) return t + gridDim.x;
        if (!claiming) return -1;
        return producer ? producer_claim() : consumer_take();
    };
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // producer: one continuous ring of k-chunks over all work items
            int it = 0;
            for (int t = first_item(true); t >= 0 && !*abort_flag; t = next_item(t, true)) {
                int g, ti, tj, slot, part;
                item_of(L, t, g, ti, tj, slot, part);
                const DigitGemmParams& Pg = params_of<Q>(L, g);
                const int tix = tj * (tj + 1) / 2 + ti;
                // -1: every k-chunk
                const int cnt = POOL ? pool_chunk_count(Pg, ti, tj) : (Pg.kc_cnt ? Pg.kc_cnt[tix] : -1);
                const unsigned long long* km =
                    (!POOL && cnt >= 0) ? Pg.kc_mask + (size_t)tix * Pg.kc_words : nullptr;
                const bool masked = POOL || km != nullptr;
                int kb, nk;
                dense_k_range(L, Pg.n_pad / KC, slot, part, kb, nk);
                if (cnt >= 0) nk = cnt;
                const CUtensorMap* mA = Q ? &L.qmaps[2 * g] : &L.maps[2 * g];
                const CUtensorMap* mB = Q ? &L.qmaps[2 * g + 1] : &L.maps[2 * g + 1];
                const int s_it = QRT ? Pg.s_in : S;  // this item's digit planes
                if constexpr (Q) {
                    acquire_map(mA);
                    acquire_map(mB);
                    const bool ready = (Pg.q_war0 < 0 || wait_all(L, Pg.q_war0, wait)) &&
                                       (Pg.q_war1 < 0 || wait_all(L, Pg.q_war1, wait)) &&
                                       (Pg.q_depA < 0 || wait_panel(L, Pg.q_depA, ti, wait)) &&
                                       (Pg.q_depB < 0 || wait_panel(L, Pg.q_depB, tj, wait));
                    if (!ready) {
                        atomicOr(L.err, ERR_PRODUCER_WAIT);
                        *abort_flag = 1;
                        break;
                    }
                }
                int w = 0;
                unsigned long long bits = POOL ? pool_chunk_word(Pg, ti, tj, 0) : (km ? km[0] : 0ull);
                // pooled: the next k-chunk and its eight slot-table entries are
                // read one chunk ahead, so that their latency overlaps the
                // current chunk's wait and copies
                int ka[4] = {0, 0, 0, 0}, kb2[4] = {0, 0, 0, 0};
                int na[4] = {0, 0, 0, 0}, nb2[4] = {0, 0, 0, 0};
                int kc_next = -1;
                auto pool_next = [&]() -> int {
                    while (bits == 0ull && w + 1 < Pg.kc_words) {
                        ++w;
                        bits = pool_chunk_word(Pg, ti, tj, w);
                    }
                    if (bits == 0ull) return -1;
                    const int k = w * 64 + __ffsll((long long)bits) - 1;
                    bits &= bits - 1;
                    return k;
                };
                auto pool_fetch = [&](int k) {
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        na[r] = Pg.a_idx[(size_t)(4 * ti + r) * Pg.nb + k];
                        nb2[r] = Pg.b_idx[(size_t)(4 * tj + r) * Pg.nb + k];
                    }
                };
                if constexpr (POOL) {
                    if (nk > 0) {
                        kc_next = pool_next();
                        if (kc_next >= 0) pool_fetch(kc_next);
                    }
                }
                for (int c = 0; c < nk; ++c, ++it) {
                    int kc = kb + c;
                    if constexpr (POOL) {
                        kc = kc_next;
                        if (kc < 0) {  // count and mask disagree
                            atomicOr(L.err, ERR_PLAN);
                            *abort_flag = 1;
                            break;
                        }
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            ka[r] = na[r];
                            kb2[r] = nb2[r];
                        }
                        kc_next = c + 1 < nk ? pool_next() : -1;
                        if (kc_next >= 0) pool_fetch(kc_next);
                    } else if (masked) {
                        while (bits == 0ull && w + 1 < Pg.kc_words) {
                            ++w;
                            bits = POOL ? pool_chunk_word(Pg, ti, tj, w) : km[w];
                        }
                        if (bits == 0ull) {  // count and mask disagree
                            atomicOr(L.err, ERR_PLAN);
                            *abort_flag = 1;
                            break;
                        }
                        kc = w * 64 + __ffsll((long long)bits) - 1;
                        bits &= bits - 1;
                    }
                    const int st = it % stages;
                    if (it >= stages &&
                        !mbar_wait_for(smem_u32(&empty_bar[st]), (uint32_t)(((it / stages) & 1) ^ 1), wait)) {
                        atomicOr(L.err, ERR_PRODUCER_WAIT);
                        *abort_flag = 1;
                        break;
                    }
                    if (*abort_flag) break;
                    const uint32_t fb = smem_u32(&full_bar[st]);
                    uint8_t* sa = base + (size_t)st * stage_bytes;
                    mbar_arrive_expect_tx(fb, (uint32_t)(2 * plane_pairs(s_it) * PAIR_BYTES));
                    if constexpr (POOL) {
                        // the panels' four 32-row blocks of k-block kc, one box per
                        // block and plane pair (absent blocks: the zero slot)
#pragma unroll
                        for (int r = 0; r < 4; ++r)
#pragma unroll
                            for (int m = 0; m < NP; ++m) {
                                tma_load_3d(smem_u32(sa + m * PAIR_BYTES + r * (PAIR_BYTES / 4)), mA, fb, 0, 0,
                                            ka[r] * NP + m);
                                tma_load_3d(smem_u32(sa + (NP + m) * PAIR_BYTES + r * (PAIR_BYTES / 4)), mB, fb,
                                            0, 0, kb2[r] * NP + m);
                            }
                    } else {
                        tma_load_3d(smem_u32(sa), mA, fb, kc * 64, ti * TILE, 0);
                        tma_load_3d(smem_u32(sa + NP * PAIR_BYTES), mB, fb, kc * 64, tj * TILE, 0);
                    }
                }
            }
            // a -1 ends the other roles' sequences (also after an abort; if
            // its slot does not come free in time they give up on their own)
            if (claiming && !ended) publish(-1);
            // wait (bounded) for the copies still in flight
            for (int k = (it > stages ? it - stages : 0); k < it; ++k)
                mbar_wait_for(smem_u32(&full_bar[k % stages]), (uint32_t)((k / stages) & 1));
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer.  Descriptors are one base plus compile-time offsets
            // (the start address sits in the low 14 bits and never carries).
            const uint64_t desc_base = smem_desc(smem_u32(base));
            int it = 0, lt = 0;
            bool ok = true;
            for (int t = first_item(false); t >= 0 && ok; t = next_item(t, false), ++lt) {
                int g, ti, tj, slot, part;
                item_of(L, t, g, ti, tj, slot, part);
                const DigitGemmParams& Pg = params_of<Q>(L, g);
                const int nl = POOL ? pool_chunk_count(Pg, ti, tj)
                                    : (Pg.kc_cnt ? Pg.kc_cnt[tj * (tj + 1) / 2 + ti] : -1);
                const int s_it = QRT ? Pg.s_in : S;
                int kb, nk;
                dense_k_range(L, Pg.n_pad / KC, slot, part, kb, nk);
                if (nl >= 0) nk = nl;
                if (lt > 0 && !mbar_wait_for(smem_u32(tmem_empty), (uint32_t)((lt - 1) & 1), wait)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int kc = 0; kc < nk; ++kc, ++it) {
                    const int st = it % stages;
                    // (an aborting role stops feeding this wait, so it runs out;
                    // the abort flag is not read on this path)
                    if (!mbar_wait_for(smem_u32(&full_bar[st]), (uint32_t)((it / stages) & 1), wait)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t da = desc_base + (uint64_t)((st * stage_bytes) >> 4);
                    const uint64_t db = da + (uint64_t)((NP * PAIR_BYTES) >> 4);
                    const uint32_t later = kc > 0 ? 1u : 0u;
                    if (!QRT || s_it == S)
                        issue_chunk<S>(tmem, da, db, later);
                    else if constexpr (QRT)
                        issue_chunk_runtime<S - 1>(s_it, tmem, da, db, later);
                    mma_commit(smem_u32(&empty_bar[st]));
                }
                if (!ok) break;
                mma_commit(smem_u32(tmem_full));
            }
            if (!ok) {
                atomicOr(L.err, ERR_MMA_WAIT);
                *abort_flag = 1;
            }
            // every MMA this thread issued has completed before teardown
            mma_commit(smem_u32(drain));
            mbar_wait_for(smem_u32(drain), 0);
        }
    } else {
        // epilogue warps: lane quarter warp % 4, column group (warp - 2) / 4
        const int quarter = warp & 3;
        const int col0 = ((warp - 2) >> 2) * EPI_COLS;
        const int row_in_tile = quarter * 32 + lane;
        // the CTA's double-float tile, laid out so that a warp's accesses are
        // contiguous: region (warp) x 8-column group x lane x 8 columns
        float2* scr = L.scratch + (size_t)blockIdx.x * TILE * TILE + (size_t)(warp - 2) * EPI_COLS * 32 + lane * 8;
        int lt = 0;
        const int region = warp - 2;
        // lane 0 follows the item sequence for the warp (tcgen05.ld is warp-collective)
        auto warp_item = [&](int t, bool first) -> int {
            int v = 0;
            if (lane == 0) v = first ? first_item(false) : next_item(t, false);
            return __shfl_sync(0xffffffffu, v, 0);
        };
        for (int t = warp_item(0, true); t >= 0; t = warp_item(t, false), ++lt) {
            int g, ti, tj, slot, part;
            item_of(L, t, g, ti, tj, slot, part);
            const DigitGemmParams& P = params_of<Q>(L, g);
            const int s = QRT ? P.s_in : S;  // this item's digit planes
            bool ready = mbar_wait_for(smem_u32(tmem_full), (uint32_t)(lt & 1), wait);
            if (!ready) {
                atomicOr(L.err, ERR_EPI_WAIT);
                *abort_flag = 1;
            }
            // tcgen05.ld is warp-collective: decide once per warp
            ready = __all_sync(0xffffffffu, ready && !*abort_flag);
            if (!ready) break;
            tc_fence_after();
            // phase 1: accumulators -> double-float P in scratch; release TMEM
            // (a tile with no k-chunk of either operand has P = 0)
            const bool empty = POOL ? !pool_chunks_any(P, ti, tj, lane)
                                    : (P.kc_cnt && P.kc_cnt[tj * (tj + 1) / 2 + ti] == 0);
            const int nacc = empty ? 0 : (s < NUM_ACC ? s : NUM_ACC);
            if (slot >= 0) {
                // a part of a split tile: publish this region's accumulators
                float* mine = L.partial + ((size_t)(slot * L.split_ways + part) * EPI_WARPS + region) * REGION_FLOATS;
#pragma unroll 1
                for (int c0 = col0, cg = 0; c0 < col0 + EPI_COLS; c0 += 8, ++cg) {
#pragma unroll
                    for (int a = 0; a < NUM_ACC; ++a) {
                        if (a < nacc) {
                            float v[8];
                            tmem_ld8(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(a * TILE + c0), v);
                            float4* d = (float4*)(mine + ((size_t)(a * (EPI_COLS / 8) + cg) * 32 + lane) * 8);
                            __stcg(d, make_float4(v[0], v[1], v[2], v[3]));
                            __stcg(d + 1, make_float4(v[4], v[5], v[6], v[7]));
                        }
                    }
                }
                __threadfence();
                __syncwarp();
                int last = 0;
                if (lane == 0) {
                    last = atomicAdd(&L.split_cnt[slot * EPI_WARPS + region], 1) == L.split_ways - 1;
                    if (last) __threadfence();
                }
                last = __shfl_sync(0xffffffffu, last, 0);
                if (!last) {
                    // another part finishes this region
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0)
                        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(tmem_empty)) : "memory");
                    continue;
                }
            }
            // a tile split in two: the other part's accumulators for the next
            // 8-column group are loaded while this group is summed (the loads
            // come from L2 and their latency would otherwise add up over the
            // groups); fp32 addition commutes, so acc + other is the part-order sum
            const bool two = slot >= 0 && L.split_ways == 2;
            const float4* oth = nullptr;
            float4 nx[NUM_ACC][2];
            if (two) {
                oth = (const float4*)(L.partial +
                      ((size_t)(slot * 2 + (1 - part)) * EPI_WARPS + region) * REGION_FLOATS) + lane * 2;
#pragma unroll
                for (int a = 0; a < NUM_ACC; ++a) {
                    if (a < nacc) {
                        nx[a][0] = __ldcg(oth + (size_t)a * (EPI_COLS / 8) * 64);
                        nx[a][1] = __ldcg(oth + (size_t)a * (EPI_COLS / 8) * 64 + 1);
                    }
                }
            }
#pragma unroll 1
            for (int c0 = col0, cg = 0; c0 < col0 + EPI_COLS; c0 += 8, ++cg) {
                float acc[NUM_ACC][8];
#pragma unroll
                for (int a = 0; a < NUM_ACC; ++a) {
                    if (a < nacc) {
                        tmem_ld8(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(a * TILE + c0), acc[a]);
                    } else {
#pragma unroll
                        for (int c = 0; c < 8; ++c) acc[a][c] = 0.f;
                    }
                }
                if (two) {
#pragma unroll
                    for (int a = 0; a < NUM_ACC; ++a) {
                        if (a < nacc) {
                            acc[a][0] += nx[a][0].x; acc[a][1] += nx[a][0].y;
                            acc[a][2] += nx[a][0].z; acc[a][3] += nx[a][0].w;
                            acc[a][4] += nx[a][1].x; acc[a][5] += nx[a][1].y;
                            acc[a][6] += nx[a][1].z; acc[a][7] += nx[a][1].w;
                            if (cg + 1 < EPI_COLS / 8) {
                                nx[a][0] = __ldcg(oth + (size_t)(a * (EPI_COLS / 8) + cg + 1) * 64);
                                nx[a][1] = __ldcg(oth + (size_t)(a * (EPI_COLS / 8) + cg + 1) * 64 + 1);
                            }
                        }
                    }
                } else if (slot >= 0) {
                    // the sum of all parts, in part order
#pragma unroll
                    for (int a = 0; a < NUM_ACC; ++a) {
                        if (a >= nacc) continue;
                        float sum[8];
                        for (int q = 0; q < L.split_ways; ++q) {
                            float v[8];
                            if (q == part) {
#pragma unroll
                                for (int c = 0; c < 8; ++c) v[c] = acc[a][c];
                            } else {
                                const float4* src = (const float4*)(L.partial +
                                    ((size_t)(slot * L.split_ways + q) * EPI_WARPS + region) * REGION_FLOATS +
                                    ((size_t)(a * (EPI_COLS / 8) + cg) * 32 + lane) * 8);
                                const float4 f0 = __ldcg(src), f1 = __ldcg(src + 1);
                                v[0] = f0.x; v[1] = f0.y; v[2] = f0.z; v[3] = f0.w;
                                v[4] = f1.x; v[5] = f1.y; v[6] = f1.z; v[7] = f1.w;
                            }
#pragma unroll
                            for (int c = 0; c < 8; ++c) sum[c] = (q == 0) ? v[c] : sum[c] + v[c];
                        }
#pragma unroll
                        for (int c = 0; c < 8; ++c) acc[a][c] = sum[c];
                    }
                }
                // one 8-column group: 32 lanes x 8 float2
                float4* dst = (float4*)(scr + ((c0 - col0) >> 3) * 256);
#pragma unroll
                for (int c = 0; c < 8; c += 2) {
                    df P0 = two_sum(acc[0][c], acc[1][c]);
                    P0 = df_add_f(P0, acc[2][c]);
                    P0 = df_add_f(P0, acc[3][c]);
                    df P1 = two_sum(acc[0][c + 1], acc[1][c + 1]);
                    P1 = df_add_f(P1, acc[2][c + 1]);
                    P1 = df_add_f(P1, acc[3][c + 1]);
                    dst[c / 2] = make_float4(P0.h, P0.l, P1.h, P1.l);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(tmem_empty)) : "memory");

            // phase 2: polynomial, outputs, reductions
            const int i = ti * TILE + row_in_tile;
            const bool diag_tile = (ti == tj);
            const int n = P.n, n_pad = P.n_pad;
            // the step's parameters in registers (as far as the compiler can
            // tell, the loop's stores might alias the parameter block)
            const bool use_E = P.use_E, affine = P.affine_out;
            const __nv_bfloat16* const Ain = P.A;
            const float scale_in_h = P.scale_in_h, e_scale = P.e_scale;
            df cP = P.cP, cE = P.cE, cI = P.cI;
            const df dY = P.dY, dI = P.dI;
            const bool want_bn = P.bnorm2 != nullptr, want_red = P.red != nullptr;
            double* out64 = P.out64;
            __nv_bfloat16* outp = P.out;
            const float out_digit_scale = P.out_digit_scale, out_rscale = P.out_rscale;
            int s_out = P.s_out;
            if (P.ctl) {  // this step's coefficients and outputs, chosen on the device
                cP = dev_df(P.ctl->cP);
                cE = dev_df(P.ctl->cE);
                cI = dev_df(P.ctl->cI);
                s_out = P.ctl->s_out;
                if (s_out == 0) outp = nullptr;
                if (!P.ctl->write64) out64 = nullptr;
            }
            double s_tr = 0.0;  // the trace decides the occupation check: float64
            float s_idem = 0.f, s_fro = 0.f;
            float bn2_0 = 0.f, bn2_1 = 0.f;  // this row's share of two 32 x 32 output blocks
            // E for a pass is copied to shared memory while the previous pass
            // computes (each lane copies and reads only its own 16-byte pieces)
            // (regions laid out for the kernel's S planes: in a queue launch the
            // epilogue warps may be on items with different digit counts)
            uint4* const e_mine = e_stage + (size_t)region * S * 32 * (EW / 8) + lane * (EW / 8);
            // Addresses: 64-bit products once per item (or per pass), 32-bit
            // offsets inside (64-bit integer operations run on the float64 pipe).
            const int two_np = 2 * n_pad;                    // one row of a plane pair
            const size_t pair_stride = (size_t)two_np * n_pad;  // one plane pair
            // row i of A's planes (paired layout, see plane_index)
            const __nv_bfloat16* const e_row = Ain + (size_t)i * two_np;
            auto fetch_E = [&](int c_first) {
                if constexpr (POOL) {
                    // the warp's block row i / 32 and the pass's block column
                    const int j0 = tj * TILE + c_first;
                    const int k = P.a_idx[(size_t)(i >> 5) * P.nb + (j0 >> 5)];
#pragma unroll
                    for (int p = 0; p < s; ++p)
#pragma unroll
                        for (int q = 0; q < EW / 8; ++q)
                            cp_async16(smem_u32(e_mine + p * 32 * (EW / 8) + q),
                                       Ain + pool_index(k, NP, p, i & 31, (j0 & 31) + 8 * q));
                } else {
                    const __nv_bfloat16* ep = e_row;
#pragma unroll
                    for (int p = 0; p < s; ++p) {
#pragma unroll
                        for (int q = 0; q < EW / 8; ++q) {
                            const int j = tj * TILE + c_first + 8 * q;
                            cp_async16(smem_u32(e_mine + p * 32 * (EW / 8) + q),
                                       ep + (((j >> 5) << 6) + ((p & 1) << 5) + (j & 31)));
                        }
                        if (p & 1) ep += pair_stride;
                    }
                }
                cp_async_commit();
            };
            // the warp's columns [c_lo, c_hi).  Pooled: leading and trailing
            // 32 x 32 blocks outside the output pattern are skipped; there X
            // and the product are exactly zero (every k-chunk product has a
            // zero operand block), so Y, its norms and its reductions are
            // zero too
            int c_lo = col0, c_hi = col0 + EPI_COLS;
            if constexpr (POOL) {
                const int* orow = P.out_idx + (size_t)(i >> 5) * P.nb + ((tj * TILE) >> 5);
                while (c_lo < c_hi && orow[c_lo >> 5] == 0) c_lo += 32;
                while (c_hi > c_lo && orow[(c_hi - 32) >> 5] == 0) c_hi -= 32;
            }
            if (use_E && c_lo < c_hi) fetch_E(c_lo);
            // the double-float P of the next pass is loaded while this pass
            // re-splits and stores
            float4 pv_next[EW / 2];
            if (c_lo < c_hi) {
                const float4* src = (const float4*)(scr + ((c_lo - col0) >> 3) * 256);
#pragma unroll
                for (int c = 0; c < EW / 2; ++c) pv_next[c] = src[(c >> 2) * 128 + (c & 3)];
            }
            // EW columns per pass: a short loop body keeps the epilogue's
            // instructions resident while the other warps run
#pragma unroll 1
            for (int c0 = c_lo; c0 < c_hi; c0 += EW) {
                const int jb = tj * TILE + c0;
                df Ov[EW];
                {
                    float4 pv[EW / 2];
#pragma unroll
                    for (int c = 0; c < EW / 2; ++c) pv[c] = pv_next[c];
                    // E = A at (i, jb .. jb + EW - 1): exact two-float sum of its digits
                    float eh[EW], el[EW];
#pragma unroll
                    for (int c = 0; c < EW; ++c) eh[c] = el[c] = 0.f;
                    if (use_E) {
                        cp_async_wait_all();
#pragma unroll
                        for (int p = 0; p < s; ++p) {
                            uint4 u[EW / 8];
#pragma unroll
                            for (int q = 0; q < EW / 8; ++q) u[q] = e_mine[p * 32 * (EW / 8) + q];
                            const __nv_bfloat16* hv = (const __nv_bfloat16*)u;
                            if (p < 3) {
#pragma unroll
                                for (int c = 0; c < EW; ++c) eh[c] += bf16_to_float(hv[c]);
                            } else {
#pragma unroll
                                for (int c = 0; c < EW; ++c) el[c] += bf16_to_float(hv[c]);
                            }
                        }
                        // this pass's pieces are in registers: fetch the next pass's
                        if (c0 + EW < c_hi) fetch_E(c0 + EW);
                    }
                    float bsum = 0.f;
#pragma unroll
                    for (int c = 0; c < EW; ++c) {
                        const int j = jb + c;
                        const float4 q4 = pv[c >> 1];
                        const df Pv = df_scale((c & 1) ? df{q4.z, q4.w} : df{q4.x, q4.y}, scale_in_h);
                        const df E = df_scale(fast_two_sum(eh[c], el[c]), e_scale);
                        df Y = df_mul(cP, Pv);
                        if (use_E) Y = df_add(Y, df_mul(cE, E));
                        if (i == j) Y = df_add(Y, cI);
                        df O = Y;
                        if (affine) {
                            O = df_mul(dY, Y);
                            if (i == j) O = df_add(O, dI);
                        }
                        const bool valid = i < n && j < n;
                        if (!valid) O = {0.f, 0.f};
                        Ov[c] = O;
                        if (want_bn && (!diag_tile || i <= j)) {
                            const float bw = (i == j || ((i >> 5) != (j >> 5))) ? 1.f : 2.f;
                            bsum += bw * O.h * O.h;
                        }
                        if (want_red && valid && (!diag_tile || i <= j)) {
                            const float w = (i == j) ? 1.f : 2.f;
                            if (i == j) s_tr += (double)Y.h + (double)Y.l;
                            const df dE = df_add(E, {-Pv.h, -Pv.l});
                            s_idem += w * dE.h * dE.h;
                            s_fro += w * Y.h * Y.h;
                        }
                    }
                    if (c0 - col0 < 32)
                        bn2_0 += bsum;
                    else
                        bn2_1 += bsum;
                }
                if (c0 + EW < c_hi) {
                    const float4* src = (const float4*)(scr + ((c0 + EW - col0) >> 3) * 256);
#pragma unroll
                    for (int c = 0; c < EW / 2; ++c) pv_next[c] = src[(c >> 2) * 128 + (c & 3)];
                }
                // float64 output (n x n): row segment and its mirror column
                if (POOL && out64 && i < n) {
                    // pooled: 32 x 32 float64 blocks (i / 32, jb / 32) and its
                    // mirror in the slots the output table gives (0: not stored)
                    const int kr = P.out_idx[(size_t)(i >> 5) * P.nb + (jb >> 5)];
                    const int kcl = P.out_idx[(size_t)(jb >> 5) * P.nb + (i >> 5)];
                    double* const o_row = out64 + (size_t)kr * 1024 + (i & 31) * 32 + (jb & 31);
                    double* const o_col = out64 + (size_t)kcl * 1024 + (jb & 31) * 32 + (i & 31);
#pragma unroll
                    for (int c = 0; c < EW; ++c) {
                        const int j = jb + c;
                        if (j < n && (!diag_tile || i <= j)) {
                            const double v = (double)Ov[c].h + (double)Ov[c].l;
                            if (kr) o_row[c] = v;
                            if (i != j && kcl) o_col[c * 32] = v;
                        }
                    }
                } else if (out64 && i < n) {
                    double* const o_row = out64 + (size_t)i * n;
                    double* const o_col = out64 + (size_t)jb * n + i;
#pragma unroll
                    for (int c = 0; c < EW; ++c) {
                        const int j = jb + c;
                        if (j < n && (!diag_tile || i <= j)) {
                            const double v = (double)Ov[c].h + (double)Ov[c].l;
                            o_row[j] = v;
                            if (i != j) o_col[c * n] = v;
                        }
                    }
                }
                // digit planes of the output (next step's operand)
                if (outp) {
                    df z[EW];
#pragma unroll
                    for (int c = 0; c < EW; ++c) z[c] = df_scale(Ov[c], out_digit_scale);
                    float plane_scale = 1.f;
                    const float rs = out_rscale, rinv = 1.f / out_rscale;
                    // plane pair 0's row segment (i, jb ..) and mirror column base
                    __nv_bfloat16* seg0 = nullptr;
                    __nv_bfloat16* col0p = nullptr;
                    int col_step = two_np;     // elements between rows of the mirror column
                    size_t pair_step = pair_stride;
                    bool store_row = true, store_col = true;
                    if constexpr (POOL) {
                        // blocks (i / 32, jb / 32) and (jb / 32, i / 32) in the output
                        // pool (slot 0: not stored; the product is zero there)
                        const int kr = P.out_idx[(size_t)(i >> 5) * P.nb + (jb >> 5)];
                        const int kcl = P.out_idx[(size_t)(jb >> 5) * P.nb + (i >> 5)];
                        store_row = kr != 0;
                        store_col = kcl != 0;
                        const int onp = plane_pairs(s_out);
                        seg0 = outp + pool_index(kr, onp, 0, i & 31, jb & 31);
                        col0p = outp + pool_index(kcl, onp, 0, jb & 31, i & 31);
                        col_step = 64;
                        pair_step = 32 * 64;
                    } else {
                        seg0 = outp + (size_t)i * two_np + (((jb >> 5) << 6) + (jb & 31));
                        col0p = outp + (size_t)jb * two_np + (((i >> 5) << 6) + (i & 31));
                    }
#pragma unroll 1
                    for (int p = 0; p < s_out; ++p) {
                        __align__(16) __nv_bfloat16 dv[EW];
#pragma unroll
                        for (int c = 0; c < EW; ++c) {
                            // z.h - d is exact; |z.l| <= ulp(z.h) / 2, so the
                            // fast two-sum renormalises exactly
                            const float d = round_digit(z[c].h);
                            z[c] = df_scale(fast_two_sum(__fsub_rn(z[c].h, d), z[c].l), rs);
                            dv[c] = digit_to_bf16(d * plane_scale);
                        }
                        plane_scale *= rinv;
                        // plane p in the paired layout (see plane_index): row r,
                        // column j at pair base + r 2 n_pad + (j / 32) 64 + (p % 2) 32 + j % 32.
                        // The row segment (i, jb ..) and its mirror column; in a
                        // diagonal tile only j >= i is written here (j < i is
                        // the mirror of another row's element)
                        __nv_bfloat16* const seg = seg0 + ((p & 1) << 5);
                        if (!store_row) {
                        } else if (!diag_tile || jb >= i) {
                            uint4* row = (uint4*)seg;
#pragma unroll
                            for (int q = 0; q < EW / 8; ++q) row[q] = ((const uint4*)dv)[q];
                        } else if (jb + EW > i) {
#pragma unroll
                            for (int c = 0; c < EW; ++c)
                                if (jb + c >= i) seg[c] = dv[c];
                        }
                        __nv_bfloat16* const col = col0p + ((p & 1) << 5);
                        if (!store_col) {
                        } else if (!diag_tile) {
#pragma unroll
                            for (int c = 0; c < EW; ++c) col[c * col_step] = dv[c];
                        } else if (jb + EW > i + 1) {
#pragma unroll
                            for (int c = 0; c < EW; ++c)
                                if (jb + c > i) col[c * col_step] = dv[c];
                        }
                        if (p & 1) {
                            seg0 += pair_step;
                            col0p += pair_step;
                        }
                    }
                }
            }
            if (P.bnorm2) {
                // lanes are the 32 rows of one block row: reduce each block
#pragma unroll
                for (int b = 0; b < EPI_COLS / 32; ++b) {
                    const float v = warp_sum_f(b ? bn2_1 : bn2_0);
                    const int I = (ti * TILE + quarter * 32) >> 5;
                    const int J = (tj * TILE + col0 + 32 * b) >> 5;
                    if (lane == 0 && I <= J) P.bnorm2[(size_t)I * P.nb + J] = v;
                }
            }
            if (P.red) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s_tr += __shfl_xor_sync(0xffffffffu, s_tr, o);
                s_idem = warp_sum_f(s_idem);
                s_fro = warp_sum_f(s_fro);
                if (lane == 0) {
                    atomicAdd(&P.red[0], s_tr);
                    atomicAdd(&P.red[1], (double)s_idem);
                    atomicAdd(&P.red[2], (double)s_fro);
                }
            }
            if constexpr (Q) {
                // this warp's share of the item is stored: count it, so that
                // the instance's next product may load the planes (tensor
                // copies read through the async proxy)
                asm volatile("fence.proxy.async.global;" ::: "memory");
                __threadfence();
                __syncwarp();
                if (lane == 0) {
                    int* c = L.qcnt + P.q_cnt;
                    atomicAdd(c + ti, 1);
                    if (tj != ti) atomicAdd(c + tj, 1);
                    atomicAdd(c + P.tiles_per_row, 1);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, NUM_ACC * TILE);
    }
}

typedef void (*KernelFn)(const DigitLaunch);

// Kernel pointers of the instantiations in digits_k32_<lo|hi>.cu (1..3 and
// 4..6 digits) and, for queue launches, digits_queue_<lo|hi>.cu.
KernelFn kernel_k32_lo(int s);
KernelFn kernel_k32_hi(int s);
KernelFn kernel_queue_hi(int s);
KernelFn kernel_queue_lo(int s);
KernelFn kernel_queue_uniform_hi(int s);  // digits_queue_uniform_<lo|hi>.cu (QM = 2)
KernelFn kernel_queue_uniform_lo(int s);
KernelFn kernel_pool_lo(int s);           // digits_pool_<lo|hi>.cu (QM = 3)
KernelFn kernel_pool_hi(int s);

}  // namespace dk
}  // namespace purify
