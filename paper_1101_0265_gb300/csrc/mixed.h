// Mixed-precision (digit-plane tensor-core) path of the iteration driver.
#pragma once

#include <cuda_bf16.h>

#include <vector>

#include "digits_tc.h"
#include "internal.h"

namespace purify {

// State of a trace-rule run whose scalar schedule lives on the device
// (trace_sched.cu): constants of the run, the evolving schedule, the next
// product's control and a pointer to the per-iteration history
// (kHistCount arrays of max_iter doubles).
enum { kHistAlpha = 0, kHistBranch, kHistBeta, kHistBetabar, kHistDigits, kHistTrace, kHistIdem, kHistCount };
struct TraceSchedDev {
    double nocc, tol;
    int have_gap, scaled, max_iter, fixed_digits;
    double floor_bits, gap_bits;
    int rbits, pad0;
    double c0n, c1;          // trace(X_0) = c0n + c1 trace(F)
    double b, bb, tr;        // beta, beta_bar, trace of the current iterate
    int it, consumed, done, converged, s_cur, prev_last;
    DevStep step;
    double* hist;
};
size_t trace_sched_bytes(int max_iter);

constexpr int kMaxDigits = 6;  // equals kMaxDigitPlanes (digits_tc.h)

// Device buffers of the mixed path, owned by a handle.
struct MixedState {
    int n_pad_cap = 0;
    __nv_bfloat16* Xd[2] = {nullptr, nullptr};
    __nv_bfloat16* Sd = nullptr;
    int* err = nullptr;
    float2* scratch = nullptr;  // persistent product kernel, one tile per CTA
    int ctas = 0;
    __nv_bfloat16* Pd[2] = {nullptr, nullptr};  // P_{3,3} intermediates (V then T, and Q)
    int pd_cap = 0;
    float* partial = nullptr;   // split last-wave tiles: per-part accumulators
    int* split_cnt = nullptr;   // and per-region arrival counters
    // block-sparse runs: per-tile k-chunk counts, then (8-byte aligned) the
    // per-tile k-chunk bitmasks, in one array of 8-byte words
    unsigned long long* kc_buf = nullptr;
    size_t kc_buf_cap = 0;
    float* bnorm2 = nullptr;
    size_t bnorm2_cap = 0;
    int2* drops = nullptr;
    size_t drops_cap = 0;
    unsigned long long* pat_dev = nullptr;  // a step's block pattern (device truncation selection)
    size_t pat_dev_cap = 0;
    void* tsel = nullptr;                   // selection state: histograms and the selected key
    std::vector<int> nnzb_history;  // upper blocks kept: X_0, then after every step
    // trace rule with the schedule on the device: its state and the captured
    // block of steps, with what the capture depends on
    void* tsched = nullptr;
    size_t tsched_cap = 0;
    cudaGraphExec_t tgraph = nullptr;
    int tg_n = 0, tg_smin = 0, tg_smax = 0, tg_wait = 0, tg_split = 0;
    const void* tg_state = nullptr;
    const double* tg_red = nullptr;
    const double* tg_D = nullptr;
    const void* tg_X0 = nullptr;
    // a whole run as queue launches: staging (host and device copies)
    std::vector<uint8_t> qhost;
    void* qdev = nullptr;
    size_t qdev_cap = 0;
    // block-sparse runs: the iterates' digit planes as pools of 32 x 32 block
    // slots (slot 0 the zero block), their nb x nb slot tables, and the work
    // list of a product's tiles
    __nv_bfloat16* pool[2] = {nullptr, nullptr};
    size_t pool_cap[2] = {0, 0};  // bytes
    int* pidx[2] = {nullptr, nullptr};
    size_t pidx_cap = 0;
    int4* pwork = nullptr;
    size_t pwork_cap = 0;
    double pool_bytes_peak = 0.0;  // most pool bytes in use at once in the last run
    // slot tables made on the device from a pattern's bits and row bases
    unsigned long long* spat = nullptr;
    size_t spat_cap = 0;
    int* rowbase = nullptr;
    size_t rowbase_cap = 0;
    int* strips = nullptr;  // the split's strip list (CSR input)
    size_t strips_cap = 0;
    // the density of a block-sparse run: 32 x 32 float64 blocks in dpool
    // under the slot table pidx[1]; d_blocks lists its upper blocks (I <= J)
    // in row-major order
    double* dpool = nullptr;
    size_t dpool_cap = 0;  // bytes
    bool d_pooled = false;
    std::vector<int2> d_blocks;
};

// Allocate (or grow) the handle's mixed-path buffers for a padded size
// (planes = false: the state without the dense digit planes).
int ensure_mixed(purify_ctx* h, int n_pad, bool planes = true);
// Default per-step digit rule: a step's operands carry at least kBitsFloor
// bits and kBitsGap bits beyond log2(1 / mapped gap).
constexpr double kBitsFloor = 30.0;
constexpr double kBitsGap = 26.0;
int digits_for_gap(double g, const purify_options& o, int rbits);
// F[key[k]] = v[k] for distinct keys row * n + col (device arrays).
int launch_scatter_coo(const int64_t* key, const double* v, int64_t nnz, double* F, cudaStream_t s);
// F (n x n, zeroed beforehand) from CSR storage.
int launch_scatter_csr(const CsrF& F, int64_t n, double* out, cudaStream_t s);
// The pooled density of the last block-sparse run (MixedState::d_pooled)
// into D (host or device, leading dimension ld), and its kept upper blocks:
// *count = their number, at most cap of them written as (I, J) pairs into ij
// and 1024 row-major doubles each into values (either may be null; host or
// device memory).
int density_pooled(purify_ctx* h, double* D, int64_t ld);
int density_blocks(purify_ctx* h, int32_t* ij, double* values, int64_t cap, int64_t* count);
// Block-sparse Algorithm 2 run (sparse.cu).
int run_block_sparse(purify_ctx* h, int scheme, const Schedule& S, int* cur, std::vector<double>& red);

// Run the scheme's coefficient schedule with every matrix product on the
// tcgen05 tensor cores (see mixed.cu).  Sets *cur (index into h->X of the
// float64 density), fills `red` with the per-step reductions and the
// mixed-path fields of h->st.
// Algorithm 2 with Niklasson's trace rule on the mixed path: the branch of
// each step from trace(X_{i-1}) (reduced in float64 by the previous step's
// epilogue; for X_0 from trace(F)); one host round trip per step.  With gap
// bounds beta and beta_bar follow the branches taken; without them the run
// stops when ||X - X^2||_F <= tol.  Fills S with the steps taken.
int run_mixed_trace(purify_ctx* h, int scheme, double tol, int max_iter, Schedule& S, int* cur, int* iters);
// The same rule with the scalar schedule on the device (trace_sched.cu): the
// steps replay from a CUDA graph in blocks, with one host read per block.
int run_mixed_trace_graph(purify_ctx* h, int scheme, double tol, int max_iter, Schedule& S, int* cur, int* iters);
// The launch shape measured for st's kind in this process, if any (no
// measurement is made: usable while a stream is being captured).
void tuned_shape_if_known(int device, DigitStep* st);
// The fixed-mu schemes with P_{3,3}, P_{1,3} and P_{3,1} on the digit planes
// (product plans in mixed.cu; see purify.h).
int run_mixed_poly(purify_ctx* h, int scheme, double mu, const Schedule& S, int* cur, std::vector<double>& red);
int run_mixed(purify_ctx* h, int scheme, double mu, const Schedule& S, int* cur,
              std::vector<double>& red);
void mixed_free(MixedState* ms);

}  // namespace purify
