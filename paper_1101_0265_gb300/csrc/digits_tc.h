// Digit-plane tensor-core products (see digits_tc.cu for the representation).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "internal.h"

namespace purify {

constexpr int kMaxDigitPlanes = 6;

// Control of one product written on the device by the trace-rule schedule
// kernel (trace_sched.cu), so that a whole run can be replayed from a CUDA
// graph with no host decision between steps.  A launch that carries it runs
// only when s_in is its digit count and done is 0 (every other launch of the
// step exits at once); it takes its coefficients, output digit count and
// float64-output switch from here instead of its parameters.
struct DevStep {
    double cP, cE, cI;  // Y = cP P + cE E + cI I
    int s_in;           // digit planes of the operands
    int s_out;          // digit planes of the output (0: none)
    int write64;        // 1: write the float64 result
    int done;           // 1: the run has stopped
};

// Digit planes in HBM are stored in pairs (2m, 2m + 1).  A pair is an
// n_pad x 2 n_pad bf16 matrix whose 128-byte row pieces hold the two planes'
// 32-wide k-chunks side by side, so that one tensor-map box row (128 bytes)
// carries two planes: element (p, i, j) sits at
//   (p / 2) 2 n_pad^2 + i 2 n_pad + (j / 32) 64 + (p % 2) 32 + j % 32.
// A buffer for s planes holds plane_pairs(s) pairs (an odd count leaves the
// last pair's second half unused and unread).
__host__ __device__ constexpr int plane_pairs(int s) { return (s + 1) >> 1; }
__host__ __device__ inline size_t plane_index(int p, int i, int j, int n_pad) {
    return (size_t)(p >> 1) * 2 * n_pad * n_pad + (size_t)i * 2 * n_pad + ((j >> 5) << 6) + ((p & 1) << 5) + (j & 31);
}
// Bytes of a buffer of s digit planes at size n_pad.
inline size_t plane_buffer_bytes(int s, int n_pad) { return (size_t)plane_pairs(s) * 2 * n_pad * n_pad * 2; }

// One fused step: P = A B (A, B symmetric, held as s_in digit planes each,
// scale exponents eA, eB), Y = cP P + cE E + cI I with E = A when use_E,
// out = dY Y + dI I written as s_out digit planes with exponent e_out and
// remainder digits of rbits bits (when `out` is not null) and/or as float64
// n x n (when `out64` is not null).  red (3 doubles, atomics): trace(Y),
// ||E - P||_F^2, ||Y||_F^2.
struct DigitStep {
    int n = 0, n_pad = 0;
    const __nv_bfloat16* A = nullptr;
    const __nv_bfloat16* B = nullptr;
    int s_in = 0, eA = 0, eB = 0;
    double cP = 1.0, cE = 0.0, cI = 0.0, dY = 1.0, dI = 0.0;
    int use_E = 0;
    __nv_bfloat16* out = nullptr;
    int s_out = 0, e_out = 0;
    int rbits = 7;  // bits of the output's remainder digits
    double* out64 = nullptr;
    double* red = nullptr;
    int* err = nullptr;
    float2* scratch = nullptr;  // max_ctas x 128 x 128 float2 (digit_scratch_bytes)
    int max_ctas = 0;           // persistent grid size (the SM count)
    // block sparsity (device arrays, see DigitGemmParams); null = dense
    const int* kc_cnt = nullptr;
    const unsigned long long* kc_mask = nullptr;
    float* bnorm2 = nullptr;
    // split of the persistent grid's last wave along K (dense single
    // products): partial holds digit_partial_floats(max_ctas) floats and
    // split_cnt digit_split_counters(max_ctas) ints; null = no split
    float* partial = nullptr;
    int* split_cnt = nullptr;
    // launch shape (dense products): k-chunk width 16, 32 or 64 and the
    // number of k-ranges of the last wave's tiles (1 = whole tiles); 0 = the
    // rule (digit_kc, digit_split_plan)
    int kc = 0;
    int split_ways = 0;
    // bound of the kernel's work waits in SM cycles (0: about one second)
    long long wait_cycles = 0;
    // pooled planes (block-sparse runs): A, B and out are pools of 32 x 32
    // block slots (slot 0 the zero block) with nb x nb slot tables in device
    // memory; a_slots and b_slots are the pools' capacities in slots of
    // pool_slot_bytes(s_in), the output pool's slots hold s_out planes, and
    // out64 (when set) is a pool of 32 x 32 row-major float64 blocks under
    // out_idx.  kc_mask then holds one block-column bitset per 128-row panel
    // and kc_cnt is null.  Null: dense paired planes.
    const int* a_idx = nullptr;
    const int* b_idx = nullptr;
    const int* out_idx = nullptr;
    int a_slots = 0, b_slots = 0;
    // device-side control (null: the fields above decide)
    const DevStep* ctl = nullptr;
};

// Epilogue warps of the product kernel (each owns a 32-row x (512 / kEpiWarps)
// column region of the 128 x 128 tile).
constexpr int kEpiWarps = 8;

inline size_t digit_partial_floats(int ctas) { return (size_t)ctas * 4 * 128 * 128; }
inline size_t digit_split_counters(int ctas) { return (size_t)ctas * kEpiWarps; }

// Split plan of a single dense product: tiles [split_begin, tiles) are cut
// into `ways` ranges of k-chunks (ways = 1: no split).
void digit_split_plan(int tiles, int ctas, int k_chunks, int* split_begin, int* ways);

// Device scratch of the persistent product kernel for a grid of `ctas`.
inline size_t digit_scratch_bytes(int ctas) { return (size_t)ctas * 128 * 128 * sizeof(float2); }

int launch_digit_step(const DigitStep& st, cudaStream_t stream);

// Opt every product-kernel instantiation into the full shared memory (once
// per process; call before capturing launches into a graph).
int prepare_digit_kernels();

// One launch over `num_items` work items {g, ti, tj, -} (device memory) of
// `count` <= 64 products that all have s digits; their tensor maps and
// parameters are passed by value.
int launch_digit_group(int s, const DigitStep* steps, int count, const int4* work, int num_items,
                       float2* scratch, int max_ctas, int* err, cudaStream_t stream,
                       long long wait_cycles = 0);

// Products per grouped launch.
constexpr int kGroupMax = 64;

}  // namespace purify
namespace purify {
namespace dk {
struct DigitGemmParams;
}
// Queue launches (many products in one persistent launch, see DigitLaunch):
// the k-chunk width of such a launch; one product's parameters (without the
// q_* dependency fields, which the caller sets) and its A and B tensor maps
// (maps[0], maps[1]); and the launch itself over `num_items` work items
// {product, ti, tj, -} in device memory, claimed in order from *ticket
// (uniform: every product has smax digits, the kernel then holds the count
// as a compile-time constant).  cnt holds every product's counters
// (DigitGemmParams::q_cnt); cnt and *ticket are zero at launch.  All arrays
// are in device memory.
int queue_kc(int smax);
int fill_queue_product(const DigitStep& st, int smax, dk::DigitGemmParams* p, CUtensorMap* maps);
int launch_digit_queue(int smax, bool uniform, const dk::DigitGemmParams* prm, const CUtensorMap* maps, int* cnt,
                       int* ticket, const int4* work, int num_items, float2* scratch, int max_ctas, int* err,
                       cudaStream_t stream, long long wait_cycles);

// Bytes of one pool slot: the s digit planes (plane_pairs(s) pairs) of a
// 32 x 32 block.
inline size_t pool_slot_bytes(int s) { return (size_t)plane_pairs(s) * 32 * 64 * 2; }

// The split into pooled planes (block-sparse runs): block (I, J) of the s
// planes of a F + b I goes to pool slot pidx[I nb + J] (pool_index; slot 0:
// not written); bnorm2 (may be null) receives the blocks' ||.||_F^2 for
// I <= J.  pidx null: the norms only.
int launch_split_pool(const double* F, int64_t ldf, int n, int n_pad, double a, double b, int e, int s, int rbits,
                      __nv_bfloat16* pool, const int* pidx, float* bnorm2, cudaStream_t stream);

// The same from F in CSR storage (row pointers ptr[n + 1], column indices
// sorted within each row), over `nstrips` strips (I * (n_pad / 128) + the
// 128-column segment; device array) that hold every block to be written or
// measured; bnorm2 entries of other blocks are left as they are.  The digits
// and norms are those launch_split_pool computes from the dense F.
int launch_split_csr_pool(const int64_t* ptr, const int* col, const double* val, int n, int n_pad, double a,
                          double b, int e, int s, int rbits, __nv_bfloat16* pool, const int* pidx, float* bnorm2,
                          const int* strips, int nstrips, cudaStream_t stream);

// Many splits in one launch (see launch_split): a job per matrix, its strips
// (32 x 128 pieces of the padded matrix, split_strips of them) numbered from
// strip0 in the launch; zero4 (4 doubles, may be null) is cleared.  The jobs
// array is in device memory; jobs are in increasing strip0.
struct SplitJob {
    const double* F;
    long long ldf;
    int n, n_pad;
    float a_h, a_l, b_h, b_l;  // a and b as float pairs
    float digit_scale, rscale;
    int s;
    __nv_bfloat16* out;
    double* zero4;
    int strip0;
};
int split_strips(int n_pad);
int make_split_job(const double* F, int64_t ldf, int n, int n_pad, double a, double b, int e, int s, int rbits,
                   __nv_bfloat16* out, double* zero4, int strip0, SplitJob* job);
int launch_split_group(const SplitJob* jobs, int njobs, int total_strips, cudaStream_t stream);

// out planes of a F + b I (i, j < n; zero padding up to n_pad), exponent e,
// s digits.  red[0] += trace (float accuracy) when red is not null;
// bnorm2[I * (n_pad / 32) + J] = ||block (I, J)||_F^2 (float) for I <= J when
// bnorm2 is not null.
int launch_split(const double* F, int64_t ldf, int n, int n_pad, double a, double b, int e, int s,
                 int rbits, __nv_bfloat16* out, double* red, cudaStream_t stream, float* bnorm2 = nullptr);

// Bits of the remainder digits for a padded size: 7 up to 4096 (level-2
// sums of squares stay below 2^24), 6 above.
inline int remainder_bits(int n_pad) { return n_pad <= 4096 ? 7 : 6; }

// Bits carried by s digits (8 leading + r per remainder digit).
inline int digit_bits(int s, int rbits) { return 8 + rbits * (s - 1); }

int digit_kc(int s);
// The k-chunk width a step launches with (its own, or the rule's).
int digit_step_kc(const DigitStep& st);
// k-chunk widths worth timing for s digits (dense products; at least one
// stage pair must fit): writes up to 3 and returns the count.
int digit_kc_candidates(int s, int* kc);
int digit_stages(int s, int kc);
size_t digit_smem_bytes(int s, int kc);

inline int pad128(int64_t n) { return (int)((n + 127) / 128 * 128); }

}  // namespace purify
