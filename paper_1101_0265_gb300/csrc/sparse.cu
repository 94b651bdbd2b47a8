// Block-sparse purification with truncation (Algorithm 2, mixed path).
//
// The paper's closing discussion counts on sparsity in the linear-scaling
// regime and leaves the truncation scheme open, asking only that the forward
// error stay controlled.  Here every iterate X_i is kept as a pattern of
// 32 x 32 blocks:
//   - the product X_{i-1}^2 is formed only over 32-wide k-chunks in which
//     both row panels of an output tile hold a nonzero block (per-tile k-chunk
//     bitmasks fed to the same tensor-core kernel), and tiles with no such
//     chunk run the epilogue alone;
//   - the epilogue reports ||B||_F^2 of every 32 x 32 output block;
//   - truncation drops the blocks of smallest norm while the dropped mass
//     (off-diagonal blocks twice, for B and B^T) stays <= tau^2, so each step
//     moves X by at most tau in the Frobenius norm; dropped blocks are zeroed
//     in the digit planes and leave the pattern.
// The digit planes of an iterate are a pool of 32 x 32 block slots (all
// planes of a block in one 12 KB slot, pool_index) found through an nb x nb
// slot table; absent blocks map to slot 0, which holds zeros.  Memory and
// work both follow the pattern.  Patterns are bitsets on the host: the
// pattern of X^2 is the union over K in row I of the rows K.
#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstring>
#include <functional>
#include <thread>
#include <vector>

#include "digits_kernel.cuh"
#include "digits_tc.h"
#include "mixed.h"
#include "queue_plan.h"

namespace purify {

namespace {

// Blocks (I, J) and (J, I) leave the pattern's bits (words per row) and,
// when idx is set, a pool's slot table: from then on they read as slot 0,
// the zero block.
__global__ void drop_blocks_kernel(unsigned long long* pat, int words, int* idx, int nb, const int2* blocks,
                                   int count) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
        const int2 b = blocks[k];
        atomicAnd(&pat[(size_t)b.x * words + (b.y >> 6)], ~(1ull << (b.y & 63)));
        atomicAnd(&pat[(size_t)b.y * words + (b.x >> 6)], ~(1ull << (b.x & 63)));
        if (idx) {
            idx[(size_t)b.x * nb + b.y] = 0;
            idx[(size_t)b.y * nb + b.x] = 0;
        }
    }
}

// ---- truncation selection on the device -------------------------------------
// The greedy reading of the truncation (blocks in ascending norm, ties by
// row then column, dropped while the dropped mass stays within tau^2) picks a
// prefix of that order.  Its end is found by a two-pass radix select on the
// float bits of the norms: masses are summed as fixed-point integers (the
// budget is 2^40 units), so every sum is exact and independent of the order
// in which the device adds them.  Candidates are the upper blocks of the
// step's pattern whose weighted mass (off-diagonal blocks twice) is within the
// budget; lighter ones than the selected key are dropped, and blocks of
// exactly that key are handed to the host, which walks them in (row, column)
// order.
constexpr int kHistBins = 1 << 16;
constexpr double kBudgetUnits = 1099511627776.0;  // 2^40

struct TruncSel {
    unsigned long long hist_fx[kHistBins];
    unsigned int hist_cnt[kHistBins];
    unsigned long long cum_before;  // mass of the keys below the found bin
    int found, bin;                 // bin of the crossing (found = 0: none)
    int hi;                         // pass 0's bin: the key's high 16 bits
    unsigned key;                   // the selected key (after pass 1)
    int ndrop, ntie;
};

__device__ __forceinline__ bool trunc_candidate(const float* bn2, const unsigned long long* pat, int words, int nb,
                                                int idx, double budget, unsigned* key, unsigned long long* fx, int* I,
                                                int* J) {
    *I = idx / nb;
    *J = idx - *I * nb;
    if (*J < *I) return false;
    if (!((pat[(size_t)*I * words + (*J >> 6)] >> (*J & 63)) & 1ull)) return false;
    const float m = bn2[idx];
    const double mass = (*I == *J ? 1.0 : 2.0) * (double)m;
    if (!(mass <= budget)) return false;
    *key = __float_as_uint(m);
    *fx = budget > 0.0 ? (unsigned long long)(mass / budget * kBudgetUnits) : 0ull;
    return true;
}

// pass 0: histogram of the high 16 key bits; pass 1: of the low 16 bits of
// the keys whose high bits are sel->bin
__global__ void trunc_hist_kernel(const float* __restrict__ bn2, const unsigned long long* __restrict__ pat, int words,
                                  int nb, double budget, int pass, TruncSel* sel) {
    if (pass && !sel->found) return;
    const int hi = pass ? sel->hi : 0;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nb * nb; idx += gridDim.x * blockDim.x) {
        unsigned key;
        unsigned long long fx;
        int I, J;
        if (!trunc_candidate(bn2, pat, words, nb, idx, budget, &key, &fx, &I, &J)) continue;
        if (pass && (int)(key >> 16) != hi) continue;
        const int bin = pass ? (int)(key & 0xFFFFu) : (int)(key >> 16);
        if (fx) atomicAdd(&sel->hist_fx[bin], fx);
        atomicAdd(&sel->hist_cnt[bin], 1u);
    }
}

__device__ __forceinline__ unsigned long long sat_add(unsigned long long a, unsigned long long b) {
    const unsigned long long c = a + b;
    return c < a ? ~0ull : c;
}

// One CTA of 1024 threads: the first bin whose cumulative mass (added to
// `base`) exceeds the budget; clears the histogram for the next pass.  Warp
// w owns bins [2048 w, 2048 w + 2048) and reads them 32 at a time
// (coalesced): first its total, then, after an exclusive prefix of the 32
// warp totals, its bins in order with a warp scan per 32 until the crossing.
// Sums saturate (only sums up to the crossing matter, and those stay within
// the budget plus one bin).
__global__ void __launch_bounds__(1024) trunc_scan_kernel(TruncSel* sel, int pass) {
    constexpr int kWarps = 32, kPerWarp = kHistBins / kWarps;
    __shared__ unsigned long long wsum[kWarps];
    __shared__ int first;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned long long base = pass ? sel->cum_before : 0ull;
    const unsigned long long budget = (unsigned long long)kBudgetUnits;
    const unsigned long long* fx = sel->hist_fx + warp * kPerWarp;
    const unsigned int* cnt = sel->hist_cnt + warp * kPerWarp;
    unsigned long long s = 0;
#pragma unroll 8
    for (int c = lane; c < kPerWarp; c += 32) s = sat_add(s, fx[c]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = sat_add(s, __shfl_xor_sync(0xffffffffu, s, o));
    if (lane == 0) wsum[warp] = s;
    if (threadIdx.x == 0) first = kHistBins;
    __syncthreads();
    unsigned long long cum = base;  // base + the bins of the warps before this one
    for (int q = 0; q < warp; ++q) cum = sat_add(cum, wsum[q]);
    int mine = kHistBins;
    unsigned long long before = 0;
    for (int c0 = 0; c0 < kPerWarp; c0 += 32) {
        const unsigned long long v = fx[c0 + lane];
        const bool has = cnt[c0 + lane] != 0;
        unsigned long long incl = v;  // this chunk's bins up to this lane
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl = sat_add(incl, u);
        }
        unsigned long long excl = __shfl_up_sync(0xffffffffu, incl, 1);
        if (lane == 0) excl = 0ull;
        const unsigned m = __ballot_sync(0xffffffffu, has && sat_add(cum, incl) > budget);
        if (m) {
            if (lane == __ffs(m) - 1) {
                mine = warp * kPerWarp + c0 + lane;
                before = cum + excl;
            }
            break;
        }
        cum = sat_add(cum, __shfl_sync(0xffffffffu, incl, 31));
    }
    if (mine < kHistBins) atomicMin(&first, mine);
    __syncthreads();
    if (mine < kHistBins && mine == first) {
        sel->found = 1;
        sel->bin = mine;
        sel->cum_before = before;
        if (pass == 0)
            sel->hi = mine;
        else
            sel->key = ((unsigned)sel->hi << 16) | (unsigned)mine;
    }
    __syncthreads();
    if (threadIdx.x == 0 && first == kHistBins) sel->found = 0;
    for (int b = threadIdx.x; b < kHistBins; b += 1024) {
        sel->hist_fx[b] = 0;
        sel->hist_cnt[b] = 0;
    }
}

// Candidates below the selected key are dropped; those of exactly that key
// are listed for the host.  Without a crossing every candidate is dropped.
__global__ void trunc_collect_kernel(const float* __restrict__ bn2, const unsigned long long* __restrict__ pat,
                                     int words, int nb, double budget, TruncSel* sel, int2* drop, int drop_cap, int2* tie,
                                     int tie_cap) {
    const bool all = sel->found == 0;
    const unsigned sel_key = sel->key;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nb * nb; idx += gridDim.x * blockDim.x) {
        unsigned key;
        unsigned long long fx;
        int I, J;
        if (!trunc_candidate(bn2, pat, words, nb, idx, budget, &key, &fx, &I, &J)) continue;
        if (all || key < sel_key) {
            const int k = atomicAdd(&sel->ndrop, 1);
            if (k < drop_cap) drop[k] = make_int2(I, J);
        } else if (key == sel_key) {
            const int k = atomicAdd(&sel->ntie, 1);
            if (k < tie_cap) tie[k] = make_int2(I, J);
        }
    }
}

// Block pattern: bit (I, J) of an nb x nb symmetric pattern.
struct Pattern {
    int nb = 0, words = 0;
    std::vector<uint64_t> bits;
    void init(int nb_) {
        nb = nb_;
        words = (nb + 63) / 64;
        bits.assign((size_t)nb * words, 0);
    }
    bool get(int I, int J) const { return (bits[(size_t)I * words + (J >> 6)] >> (J & 63)) & 1u; }
    void set(int I, int J) { bits[(size_t)I * words + (J >> 6)] |= (uint64_t)1 << (J & 63); }
    void clear(int I, int J) { bits[(size_t)I * words + (J >> 6)] &= ~((uint64_t)1 << (J & 63)); }
    const uint64_t* row(int I) const { return &bits[(size_t)I * words]; }
    uint64_t* row(int I) { return &bits[(size_t)I * words]; }
    int count_upper() const {  // blocks with J >= I
        int c = 0;
        for (int I = 0; I < nb; ++I) {
            const uint64_t* r = row(I);
            c += __builtin_popcountll(r[I >> 6] & (~0ull << (I & 63)));
            for (int w = (I >> 6) + 1; w < words; ++w) c += __builtin_popcountll(r[w]);
        }
        return c;
    }
};

// Pattern of X^2, of X and of the diagonal together (the blocks that Eq. 4
// and Eq. 5 can make nonzero).  Rows are independent: large patterns are
// split over host threads.
void output_pattern(const Pattern& X, Pattern& out) {
    out.init(X.nb);
    auto rows = [&](int I0, int I1) {
        for (int I = I0; I < I1; ++I) {
            uint64_t* o = out.row(I);
            const uint64_t* xi = X.row(I);
            for (int w = 0; w < X.words; ++w) {
                o[w] |= xi[w];
                uint64_t m = xi[w];
                while (m) {
                    const int K = w * 64 + __builtin_ctzll(m);
                    m &= m - 1;
                    const uint64_t* xk = X.row(K);
                    for (int v = 0; v < X.words; ++v) o[v] |= xk[v];
                }
            }
            out.set(I, I);
        }
    };
    const int hw = (int)std::thread::hardware_concurrency();
    const int nt = X.nb >= 512 ? std::max(1, std::min(hw, 16)) : 1;
    if (nt == 1) {
        rows(0, X.nb);
        return;
    }
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t) pool.emplace_back(rows, (int)((int64_t)X.nb * t / nt), (int)((int64_t)X.nb * (t + 1) / nt));
    for (std::thread& th : pool) th.join();
}

// Error-controlled truncation of the upper blocks of `pat` by their squared
// norms bn2 (row-major nb x nb, upper part): ascending norm, ties by row then
// column; drop while the dropped mass stays <= tau^2.  Dropped blocks leave
// `pat` and are listed in `drop`.
void select_drops(Pattern& pat, const float* bn2, double tau, std::vector<int2>& drop) {
    struct Cand {
        double m;
        int I, J;
    };
    // a block whose weighted mass alone exceeds the budget is never dropped,
    // and every block after it in the order is at least as heavy: only the
    // lighter ones need sorting
    const double budget = tau * tau;
    std::vector<Cand> c;
    for (int I = 0; I < pat.nb; ++I)
        for (int J = I; J < pat.nb; ++J) {
            if (!pat.get(I, J)) continue;
            const double m = (double)bn2[(size_t)I * pat.nb + J];
            if ((I == J ? 1.0 : 2.0) * m <= budget) c.push_back({m, I, J});
        }
    std::sort(c.begin(), c.end(), [](const Cand& a, const Cand& b) {
        if (a.m != b.m) return a.m < b.m;
        if (a.I != b.I) return a.I < b.I;
        return a.J < b.J;
    });
    drop.clear();
    double acc = 0.0;
    for (const Cand& x : c) {
        const double m = (x.I == x.J ? 1.0 : 2.0) * x.m;
        if (m > 0.0 && acc + m > budget) break;
        acc += m;
        drop.push_back(make_int2(x.I, x.J));
        pat.clear(x.I, x.J);
        pat.clear(x.J, x.I);
    }
}

template <typename T>
int grow(T** p, size_t* cap, size_t n) {
    if (n <= *cap) return PURIFY_OK;
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    const size_t c = std::max(n, (size_t)1024) * 2;
    PURIFY_CUDA_TRY(cudaMalloc(p, sizeof(T) * c));
    *cap = c;
    return PURIFY_OK;
}

// Remove the chosen blocks (ms->drops[0 .. count)) from the device pattern
// (words per row) and from the output pool's slot table.
int apply_drops(purify_ctx* h, size_t count, int words, int* idx, int nb) {
    MixedState* ms = h->mixed;
    if (count == 0) return PURIFY_OK;
    const unsigned grid = (unsigned)std::min<size_t>((count + 255) / 256, 152 * 4);
    drop_blocks_kernel<<<grid, 256, 0, h->stream>>>(ms->pat_dev, words, idx, nb, ms->drops, (int)count);
    PURIFY_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return PURIFY_OK;
}

// Choose the drops of one step on the device (see trunc_hist_kernel) and
// remove them; the host walks the blocks tied at the selected norm in (row,
// column) order and receives the pattern that remains.
int truncate_step(purify_ctx* h, Pattern& pat, double tau, int* idx) {
    MixedState* ms = h->mixed;
    const int nb = pat.nb, words = pat.words;
    const double budget = tau * tau;
    const size_t upper = (size_t)nb * (nb + 1) / 2;
    constexpr int kTieCap = 1 << 16;
    PURIFY_TRY(grow(&ms->drops, &ms->drops_cap, upper + kTieCap));
    PURIFY_TRY(grow(&ms->pat_dev, &ms->pat_dev_cap, pat.bits.size()));
    if (!ms->tsel) PURIFY_CUDA_TRY(cudaMalloc(&ms->tsel, sizeof(TruncSel)));
    TruncSel* sel = (TruncSel*)ms->tsel;
    PURIFY_CUDA_TRY(cudaMemcpyAsync(ms->pat_dev, pat.bits.data(), sizeof(uint64_t) * pat.bits.size(),
                                    cudaMemcpyHostToDevice, h->stream));
    PURIFY_CUDA_TRY(cudaMemsetAsync(sel, 0, sizeof(TruncSel), h->stream));
    int64_t grid = ((int64_t)nb * nb + 255) / 256;
    if (grid > 152 * 8) grid = 152 * 8;
    int2* tie_dev = ms->drops + upper;
    for (int pass = 0; pass < 2; ++pass) {
        trunc_hist_kernel<<<(unsigned)grid, 256, 0, h->stream>>>(ms->bnorm2, ms->pat_dev, words, nb, budget, pass, sel);
        trunc_scan_kernel<<<1, 1024, 0, h->stream>>>(sel, pass);
    }
    trunc_collect_kernel<<<(unsigned)grid, 256, 0, h->stream>>>(ms->bnorm2, ms->pat_dev, words, nb, budget, sel,
                                                                ms->drops, (int)upper, tie_dev, kTieCap);
    PURIFY_CUDA_TRY(cudaGetLastError());
    count_launches(6);
    struct {
        unsigned long long cum_before;
        int found, bin, hi;
        unsigned key;
        int ndrop, ntie;
    } head;
    static_assert(sizeof(head) == sizeof(TruncSel) - offsetof(TruncSel, cum_before), "TruncSel tail layout");
    PURIFY_CUDA_TRY(cudaMemcpyAsync(&head, &sel->cum_before, sizeof(head), cudaMemcpyDeviceToHost, h->stream));
    PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (head.ntie > kTieCap) return PURIFY_ERR_INTERNAL;
    size_t nd = (size_t)head.ndrop;
    std::vector<int2> tie((size_t)head.ntie);
    if (head.ntie)
        PURIFY_CUDA_TRY(cudaMemcpyAsync(tie.data(), tie_dev, sizeof(int2) * tie.size(), cudaMemcpyDeviceToHost,
                                        h->stream));
    PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (head.found && !tie.empty()) {
        // the tied blocks in (row, column) order, each with its fixed-point
        // mass, while the budget holds
        std::sort(tie.begin(), tie.end(), [](int2 a, int2 b) { return a.x != b.x ? a.x < b.x : a.y < b.y; });
        float mk;
        std::memcpy(&mk, &head.key, sizeof(mk));
        unsigned long long acc = head.cum_before;
        const unsigned long long cap = (unsigned long long)kBudgetUnits;
        size_t k = 0;
        for (; k < tie.size(); ++k) {
            const double mass = (tie[k].x == tie[k].y ? 1.0 : 2.0) * (double)mk;
            const unsigned long long fx = budget > 0.0 ? (unsigned long long)(mass / budget * kBudgetUnits) : 0ull;
            if (mass > 0.0 && acc + fx > cap) break;
            acc += fx;
        }
        if (k) {
            PURIFY_CUDA_TRY(cudaMemcpyAsync(ms->drops + nd, tie.data(), sizeof(int2) * k, cudaMemcpyHostToDevice,
                                            h->stream));
            nd += k;
        }
    }
    PURIFY_TRY(apply_drops(h, nd, words, idx, nb));
    if (nd)
        PURIFY_CUDA_TRY(cudaMemcpyAsync(pat.bits.data(), ms->pat_dev, sizeof(uint64_t) * pat.bits.size(),
                                        cudaMemcpyDeviceToHost, h->stream));
    PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return PURIFY_OK;
}

void tc_coeffs(int branch, double a, double* cP, double* cE, double* cI) {
    if (branch) {
        *cP = sq1p(a);
        *cE = -2.0 * a * (1.0 + a);
        *cI = a * a;
    } else {
        *cP = -sq1p(a);
        *cE = 2.0 * (1.0 + a);
        *cI = 0.0;
    }
}

// Distinct keys (row * n + col): plain stores.
__global__ void scatter_coo_kernel(const int64_t* __restrict__ key, const double* __restrict__ v, int64_t nnz,
                                   double* F) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x)
        F[key[k]] = v[k];
}

}  // namespace

// F[key[k]] = v[k] for distinct keys (device arrays); F zeroed beforehand.
int launch_scatter_coo(const int64_t* key, const double* v, int64_t nnz, double* F, cudaStream_t s) {
    if (nnz <= 0) return PURIFY_OK;
    int64_t blocks = (nnz + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    scatter_coo_kernel<<<(unsigned)blocks, 256, 0, s>>>(key, v, nnz, F);
    PURIFY_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return PURIFY_OK;
}

namespace {

// Pool k holds at least `bytes` bytes (capacity grows by a quarter beyond the
// request, up to `max_bytes`).  The pool being resized is the one about to be
// filled: nothing in it is kept.
template <typename T>
int ensure_bytes(purify_ctx* h, T** buf, size_t* cap, size_t bytes, size_t max_bytes) {
    if (bytes <= *cap) return PURIFY_OK;
    PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
    cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    const size_t c = std::max(bytes, std::min(bytes + bytes / 4 + (64 << 10), max_bytes));
    PURIFY_CUDA_TRY(cudaMalloc(buf, c));
    *cap = c;
    return PURIFY_OK;
}

// Copy the kept blocks of a pool into a compact one: block (I, J) with slot
// d = didx[I nb + J] != 0 receives slot sidx[I nb + J] of src (np plane
// pairs per slot).  One warp per table entry.
__global__ void compact_slots_kernel(const __nv_bfloat16* __restrict__ src, const int* __restrict__ sidx,
                                     __nv_bfloat16* __restrict__ dst, const int* __restrict__ didx, int nb, int np) {
    const int lane = threadIdx.x & 31;
    const int total = nb * nb;  // nb <= 8192
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < total; e += warps) {
        const int d = didx[e];
        if (d == 0) continue;
        const uint4* from = (const uint4*)(src + (size_t)sidx[e] * np * 2048);
        uint4* to = (uint4*)(dst + (size_t)d * np * 2048);
        for (int q = lane; q < np * 256; q += 32) to[q] = from[q];
    }
}

constexpr int kMaxPatternWords = 128;  // nb <= 8192

// Slot table of a block pattern (nb rows of `words` 64-bit words): block
// (I, J) set gets row_base[I] + (the set blocks before it in row I), unset
// blocks 0.  One warp per block row; the per-word prefix counts go through
// shared memory.
__global__ void __launch_bounds__(256) slot_table_kernel(const unsigned long long* __restrict__ pat, int nb,
                                                         int words, const int* __restrict__ row_base,
                                                         int* __restrict__ idx) {
    __shared__ int pre[8][kMaxPatternWords];
    __shared__ unsigned long long wv[8][kMaxPatternWords];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int I = blockIdx.x * 8 + warp; I < nb; I += gridDim.x * 8) {
        const unsigned long long* row = pat + (size_t)I * words;
        int carry = 0;
        for (int w0 = 0; w0 < words; w0 += 32) {
            const int w = w0 + lane;
            const unsigned long long v = w < words ? row[w] : 0ull;
            const int own = __popcll(v);
            int c = own;  // inclusive prefix over the 32 words
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, c, o);
                if (lane >= o) c += t;
            }
            if (w < words) {
                pre[warp][w] = carry + c - own;
                wv[warp][w] = v;
            }
            carry += __shfl_sync(0xffffffffu, c, 31);
        }
        __syncwarp();
        const int base = row_base[I];
        int* out = idx + (size_t)I * nb;
        for (int J0 = 0; J0 < nb; J0 += 32) {
            const int J = J0 + lane;
            if (J < nb) {
                const int w = J >> 6, b = J & 63;
                const unsigned long long v = wv[warp][w];
                const bool set = (v >> b) & 1ull;
                out[J] = set ? base + pre[warp][w] + __popcll(v & ((1ull << b) - 1ull)) : 0;
            }
        }
        __syncwarp();
    }
}

// F[i n + col] = val over CSR rows (F zeroed beforehand); one warp per row.
__global__ void scatter_csr_kernel(const int64_t* __restrict__ ptr, const int* __restrict__ col,
                                   const double* __restrict__ val, int n, double* F) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        const int64_t p1 = ptr[i + 1];
        for (int64_t k = ptr[i] + lane; k < p1; k += 32) F[(size_t)i * n + col[k]] = val[k];
    }
}

// Rows [I0 * 32, I1 * 32) of the pooled density into dst (leading dimension
// ld, rows from I0 * 32; zeroed beforehand): one warp per table entry of
// those block rows, rows and columns >= n left out.
__global__ void scatter_dpool_kernel(const double* __restrict__ dpool, const int* __restrict__ tbl, int nb, int n,
                                     int I0, int I1, double* __restrict__ dst, int64_t ld) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int entries = (I1 - I0) * nb;
    for (int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < entries; e += warps) {
        const int I = I0 + e / nb, J = e % nb;
        const int k = tbl[(size_t)I * nb + J];
        if (k == 0) continue;
        const double* blk = dpool + (size_t)k * 1024;
        const int j = J * 32 + lane;
        if (j >= n) continue;
        for (int r = 0; r < 32 && I * 32 + r < n; ++r)
            dst[(size_t)((I - I0) * 32 + r) * ld + j] = blk[r * 32 + lane];
    }
}

// Blocks list[b0 .. b0 + count) of the pooled density, 1024 doubles each, into dst.
__global__ void gather_dpool_kernel(const double* __restrict__ dpool, const int* __restrict__ tbl, int nb,
                                    const int2* __restrict__ list, int64_t count, double* __restrict__ dst) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < count; b += warps) {
        const int2 ij = list[b];
        const int k = tbl[(size_t)ij.x * nb + ij.y];
        const double* blk = dpool + (size_t)k * 1024;
        for (int q = lane; q < 1024; q += 32) dst[b * 1024 + q] = blk[q];
    }
}

// Row bases of a pattern's slot table (slot 0 reserved) and the slots used
// (slot 0 included).
size_t row_bases(const Pattern& P, std::vector<int>& base) {
    base.resize(P.nb);
    size_t k = 1;
    for (int I = 0; I < P.nb; ++I) {
        base[I] = (int)k;
        const uint64_t* r = P.row(I);
        for (int w = 0; w < P.words; ++w) k += (size_t)__builtin_popcountll(r[w]);
    }
    return k;
}

// Slot table k from pattern P on the device; returns the slots used.
int upload_table(purify_ctx* h, const Pattern& P, int* table, size_t* used) {
    MixedState* ms = h->mixed;
    if (P.words > kMaxPatternWords) return PURIFY_ERR_INVALID_ARG;
    std::vector<int> base;
    *used = row_bases(P, base);
    PURIFY_TRY(grow(&ms->spat, &ms->spat_cap, P.bits.size()));
    PURIFY_TRY(grow(&ms->rowbase, &ms->rowbase_cap, base.size()));
    PURIFY_CUDA_TRY(cudaMemcpyAsync(ms->spat, P.bits.data(), sizeof(uint64_t) * P.bits.size(),
                                    cudaMemcpyHostToDevice, h->stream));
    PURIFY_CUDA_TRY(cudaMemcpyAsync(ms->rowbase, base.data(), sizeof(int) * base.size(), cudaMemcpyHostToDevice,
                                    h->stream));
    const unsigned grid = (unsigned)std::min(152 * 8, (P.nb + 7) / 8);
    slot_table_kernel<<<grid, 256, 0, h->stream>>>(ms->spat, P.nb, P.words, ms->rowbase, table);
    PURIFY_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return PURIFY_OK;
}

// Per 128-row panel t of X: the block columns where one of its four block
// rows has a block (X.words words per panel).
void panel_bits(const Pattern& X, int T, std::vector<uint64_t>& pan) {
    pan.assign((size_t)T * X.words, 0);
    for (int t = 0; t < T; ++t)
        for (int r = 4 * t; r < 4 * t + 4 && r < X.nb; ++r)
            for (int w = 0; w < X.words; ++w) pan[(size_t)t * X.words + w] |= X.row(r)[w];
}

// The upper 128 x 128 tiles holding a block of `out`, in banded order (see
// banded_tiles): the product's work items {0, ti, tj, 0}; chunks receives
// the k-chunk products they run (the popcount of the two panels' bits of X).
// Bands are independent: large patterns are split over host threads.
void pattern_tiles(const Pattern& out, const std::vector<uint64_t>& xpan, int words, int T,
                   std::vector<int4>& work, double* chunks) {
    std::vector<uint64_t> opan;
    panel_bits(out, T, opan);
    const int bands = (T + dk::BAND - 1) / dk::BAND;
    auto run = [&](int b_lo, int b_hi, std::vector<int4>& w_out, double& c_out) {
        double c = 0.0;
        for (int band = b_lo; band < b_hi; ++band) {
            const int b0 = band * dk::BAND, b1 = std::min(T, b0 + dk::BAND);
            for (int r = 0; r < b1; ++r)
                for (int t = std::max(b0, r); t < b1; ++t) {
                    const int J0 = 4 * t;
                    if (!((opan[(size_t)r * words + (J0 >> 6)] >> (J0 & 63)) & 0xFull)) continue;
                    w_out.push_back(make_int4(0, r, t, 0));
                    const uint64_t* a = &xpan[(size_t)r * words];
                    const uint64_t* b = &xpan[(size_t)t * words];
                    for (int w = 0; w < words; ++w) c += (double)__builtin_popcountll(a[w] & b[w]);
                }
        }
        c_out = c;
    };
    const int hw = (int)std::thread::hardware_concurrency();
    const int nt = T >= 256 ? std::max(1, std::min({hw, 16, bands})) : 1;
    std::vector<std::vector<int4>> parts(nt);
    std::vector<double> csum(nt, 0.0);
    if (nt == 1) {
        run(0, bands, parts[0], csum[0]);
    } else {
        std::vector<std::thread> pool;
        for (int t = 0; t < nt; ++t)
            pool.emplace_back(run, (int)((int64_t)bands * t / nt), (int)((int64_t)bands * (t + 1) / nt),
                              std::ref(parts[t]), std::ref(csum[t]));
        for (std::thread& th : pool) th.join();
    }
    work.clear();
    double c = 0.0;
    for (int t = 0; t < nt; ++t) {
        work.insert(work.end(), parts[t].begin(), parts[t].end());
        c += csum[t];
    }
    *chunks = c;
}

// X_0's strips (block row I, 128-column segment) that hold a block of P.
void pattern_strips(const Pattern& P, int ns, std::vector<int>& strips) {
    strips.clear();
    for (int I = 0; I < P.nb; ++I)
        for (int q = 0; q < ns; ++q) {
            const int J0 = 4 * q;
            if ((P.row(I)[J0 >> 6] >> (J0 & 63)) & 0xFull) strips.push_back(I * ns + q);
        }
}

}  // namespace

int launch_scatter_csr(const CsrF& F, int64_t n, double* out, cudaStream_t s) {
    const unsigned grid = (unsigned)std::min<int64_t>(152 * 8, (n + 7) / 8);
    scatter_csr_kernel<<<grid, 256, 0, s>>>(F.ptr, F.col, F.val, (int)n, out);
    PURIFY_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return PURIFY_OK;
}

int density_pooled(purify_ctx* h, double* D, int64_t ld) {
    MixedState* ms = h->mixed;
    const int n = (int)h->n, nb = pad128(n) / 32;
    cudaPointerAttributes attr;
    PURIFY_CUDA_TRY(cudaPointerGetAttributes(&attr, D));
    const bool dev = attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
    // block rows per pass: all of them into device memory, else through a
    // staging panel of at most 256 MB
    int rows = nb;
    double* stage = D;
    int64_t sld = ld;
    if (!dev) {
        rows = (int)std::max<int64_t>(1, std::min<int64_t>(nb, (256ll << 20) / (32ll * 8 * n)));
        PURIFY_TRY(ensure_scratch(h, (int64_t)rows * 32 * n));
        stage = h->scratch;
        sld = n;
    }
    for (int I0 = 0; I0 < nb; I0 += rows) {
        const int I1 = std::min(nb, I0 + rows);
        const int r0 = I0 * 32, r1 = std::min(n, I1 * 32);
        if (r1 <= r0) break;
        double* dst = dev ? D + (size_t)r0 * ld : stage;
        PURIFY_CUDA_TRY(cudaMemset2DAsync(dst, sizeof(double) * sld, 0, sizeof(double) * n, r1 - r0, h->stream));
        const int64_t entries = (int64_t)(I1 - I0) * nb;
        const unsigned grid = (unsigned)std::min<int64_t>(152 * 8, (entries + 7) / 8);
        scatter_dpool_kernel<<<grid, 256, 0, h->stream>>>(ms->dpool, ms->pidx[1], nb, n, I0, I1, dst, sld);
        PURIFY_CUDA_TRY(cudaGetLastError());
        count_launches(1);
        if (!dev)
            PURIFY_CUDA_TRY(cudaMemcpy2DAsync(D + (size_t)r0 * ld, sizeof(double) * ld, stage, sizeof(double) * n,
                                              sizeof(double) * n, r1 - r0, cudaMemcpyDeviceToHost, h->stream));
    }
    PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return PURIFY_OK;
}

int density_blocks(purify_ctx* h, int32_t* ij, double* values, int64_t cap, int64_t* count) {
    MixedState* ms = h->mixed;
    const int nb = pad128(h->n) / 32;
    const int64_t total = (int64_t)ms->d_blocks.size();
    *count = total;
    const int64_t m = std::min(cap, total);
    if (m <= 0) return PURIFY_OK;
    if (ij) {
        std::vector<int32_t> flat(2 * (size_t)m);
        for (int64_t b = 0; b < m; ++b) {
            flat[2 * b] = ms->d_blocks[b].x;
            flat[2 * b + 1] = ms->d_blocks[b].y;
        }
        PURIFY_CUDA_TRY(cudaMemcpyAsync(ij, flat.data(), sizeof(int32_t) * flat.size(), cudaMemcpyDefault, h->stream));
        PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
    }
    if (!values) return PURIFY_OK;
    cudaPointerAttributes attr;
    PURIFY_CUDA_TRY(cudaPointerGetAttributes(&attr, values));
    const bool dev = attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
    // the block list on the device (in the drop-list buffer, free after a run)
    PURIFY_TRY(grow(&ms->drops, &ms->drops_cap, (size_t)m));
    PURIFY_CUDA_TRY(cudaMemcpyAsync(ms->drops, ms->d_blocks.data(), sizeof(int2) * m, cudaMemcpyHostToDevice,
                                    h->stream));
    const int64_t per = dev ? m : std::max<int64_t>(1, (256ll << 20) / (1024 * 8));
    if (!dev) PURIFY_TRY(ensure_scratch(h, std::min(per, m) * 1024));
    for (int64_t b0 = 0; b0 < m; b0 += per) {
        const int64_t c = std::min(per, m - b0);
        double* dst = dev ? values + b0 * 1024 : h->scratch;
        const unsigned grid = (unsigned)std::min<int64_t>(152 * 8, (c + 7) / 8);
        gather_dpool_kernel<<<grid, 256, 0, h->stream>>>(ms->dpool, ms->pidx[1], nb, ms->drops + b0, c, dst);
        PURIFY_CUDA_TRY(cudaGetLastError());
        count_launches(1);
        if (!dev)
            PURIFY_CUDA_TRY(cudaMemcpyAsync(values + b0 * 1024, h->scratch, sizeof(double) * 1024 * c,
                                            cudaMemcpyDeviceToHost, h->stream));
        PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
    }
    return PURIFY_OK;
}

int run_block_sparse(purify_ctx* h, int scheme, const Schedule& S, int* cur, std::vector<double>& red) {
    if (scheme != PURIFY_TC_SF && scheme != PURIFY_TC_MONO) return PURIFY_ERR_UNSUPPORTED;
    const int m_sched = (int)S.alpha.size();
    // a total budget spreads over X_0 and the m scheduled steps
    const double tau = h->opt.trunc_budget > 0.0 ? h->opt.trunc_budget / (m_sched + 1) : h->opt.trunc_tau;
    if (!(tau >= 0.0)) return PURIFY_ERR_INVALID_ARG;
    const int n = (int)h->n;
    const int n_pad = pad128(n);
    PURIFY_TRY(ensure_mixed(h, n_pad, false));
    MixedState* ms = h->mixed;
    ms->d_pooled = false;
    ms->d_blocks.clear();
    const int nb = n_pad / 32, T = n_pad / 128, ns = n_pad / 128;
    if ((nb + 63) / 64 > kMaxPatternWords) return PURIFY_ERR_INVALID_ARG;
    const int rb = remainder_bits(n_pad);
    const int m = (int)S.alpha.size();
    std::vector<int> sd(m + 1);
    for (int i = 0; i < m; ++i) {
        const double b = i ? S.beta[i - 1] : S.beta0;
        const double bb = i ? S.betabar[i - 1] : S.betabar0;
        sd[i] = digits_for_gap(bb - b, h->opt, rb);
    }
    sd[m] = sd[m ? m - 1 : 0];
    int dmax = 0;
    for (int i = 0; i < m; ++i) dmax = std::max(dmax, sd[i]);
    h->st.digit_max = dmax;
    const bool csr = h->csr_valid;
    if (!csr && !h->F_dense) return PURIFY_ERR_STATE;
    PURIFY_TRY(grow(&ms->bnorm2, &ms->bnorm2_cap, (size_t)nb * nb));
    if (ms->pidx_cap < (size_t)nb * nb) {
        for (int k = 0; k < 2; ++k) {
            cudaFree(ms->pidx[k]);
            ms->pidx[k] = nullptr;
        }
        ms->pidx_cap = 0;
        for (int k = 0; k < 2; ++k) PURIFY_CUDA_TRY(cudaMalloc(&ms->pidx[k], sizeof(int) * (size_t)nb * nb));
        ms->pidx_cap = (size_t)nb * nb;
    }
    const int slots = 2 * m + 2;
    PURIFY_TRY(ensure_red(h, 4 * (int64_t)slots));
    PURIFY_CUDA_TRY(cudaMemsetAsync(h->red, 0, sizeof(double) * 4 * slots, h->stream));
    PURIFY_CUDA_TRY(cudaMemsetAsync(ms->err, 0, sizeof(int), h->stream));
    PURIFY_CUDA_TRY(cudaEventRecord(h->e0, h->stream));

    const double lmin = h->b.lmin, lmax = h->b.lmax;
    const double c0 = lmax / (lmax - lmin), c1 = -1.0 / (lmax - lmin);
    std::vector<float> bn2((size_t)nb * nb, 0.f);
    ms->nnzb_history.clear();
    ms->pool_bytes_peak = 0.0;
    // X_0 = c0 I + c1 F: its block norms first (the split without planes),
    // then its pattern, truncated like every iterate, and its planes in the
    // pool slots of the kept blocks.  From CSR the split visits only the
    // strips that hold a block of F's pattern (blocks outside it are zero).
    const int s0 = std::max(sd[0], 1);
    std::vector<int> strips;
    if (csr) {
        Pattern P0;
        P0.nb = nb;
        P0.words = h->f_pattern_words;
        P0.bits = h->f_pattern;
        pattern_strips(P0, ns, strips);
        PURIFY_TRY(grow(&ms->strips, &ms->strips_cap, strips.size()));
        PURIFY_CUDA_TRY(cudaMemcpyAsync(ms->strips, strips.data(), sizeof(int) * strips.size(),
                                        cudaMemcpyHostToDevice, h->stream));
        PURIFY_CUDA_TRY(cudaMemsetAsync(ms->bnorm2, 0, sizeof(float) * (size_t)nb * nb, h->stream));
        PURIFY_TRY(launch_split_csr_pool(h->csr_ptr, h->csr_col, h->csr_val, n, n_pad, c1, c0, 0, s0, rb, nullptr,
                                         nullptr, ms->bnorm2, ms->strips, (int)strips.size(), h->stream));
    } else {
        PURIFY_TRY(launch_split_pool(h->F, n, n, n_pad, c1, c0, 0, s0, rb, nullptr, nullptr, ms->bnorm2,
                                     h->stream));
    }
    PURIFY_CUDA_TRY(cudaMemcpyAsync(bn2.data(), ms->bnorm2, sizeof(float) * (size_t)nb * nb,
                                    cudaMemcpyDeviceToHost, h->stream));
    PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
    Pattern X;
    X.init(nb);
    for (int I = 0; I < nb; ++I)
        for (int J = I; J < nb; ++J)
            if (bn2[(size_t)I * nb + J] > 0.f || I == J) {
                X.set(I, J);
                X.set(J, I);
            }
    {
        std::vector<int2> drop;
        select_drops(X, bn2.data(), tau, drop);
    }
    ms->nnzb_history.push_back(X.count_upper());
    // pool 0 holds the current iterate compactly (its kept blocks), pool 1
    // the product's output pattern before truncation; after each truncation
    // the kept blocks move from pool 1 into pool 0
    const size_t max_bytes = ((size_t)nb * nb + 1) * pool_slot_bytes(kMaxDigitPlanes);
    size_t used0 = 0;
    PURIFY_TRY(upload_table(h, X, ms->pidx[0], &used0));
    PURIFY_TRY(ensure_bytes(h, &ms->pool[0], &ms->pool_cap[0], used0 * pool_slot_bytes(s0), max_bytes));
    PURIFY_CUDA_TRY(cudaMemsetAsync(ms->pool[0], 0, pool_slot_bytes(s0), h->stream));
    if (csr)
        PURIFY_TRY(launch_split_csr_pool(h->csr_ptr, h->csr_col, h->csr_val, n, n_pad, c1, c0, 0, s0, rb,
                                         ms->pool[0], ms->pidx[0], nullptr, ms->strips, (int)strips.size(),
                                         h->stream));
    else
        PURIFY_TRY(launch_split_pool(h->F, n, n, n_pad, c1, c0, 0, s0, rb, ms->pool[0], ms->pidx[0], nullptr,
                                     h->stream));
    ms->pool_bytes_peak = (double)(used0 * pool_slot_bytes(s0));

    *cur = 0;
    std::vector<uint64_t> xpan;
    std::vector<int4> work;
    const double pairs_tile = 2.0 * 128.0 * 128.0 * 32.0;  // one pair, one 32-wide k-chunk
    for (int i = 0; i < m; ++i) {
        const int s = sd[i], so = sd[i + 1];
        const bool last = (i + 1 == m);
        Pattern out;
        output_pattern(X, out);
        panel_bits(X, T, xpan);
        double chunks = 0.0;
        pattern_tiles(out, xpan, X.words, T, work, &chunks);
        PURIFY_TRY(grow(&ms->kc_buf, &ms->kc_buf_cap, xpan.size()));
        PURIFY_TRY(grow(&ms->pwork, &ms->pwork_cap, work.size()));
        PURIFY_CUDA_TRY(cudaMemcpyAsync(ms->kc_buf, xpan.data(), sizeof(uint64_t) * xpan.size(),
                                        cudaMemcpyHostToDevice, h->stream));
        PURIFY_CUDA_TRY(cudaMemcpyAsync(ms->pwork, work.data(), sizeof(int4) * work.size(), cudaMemcpyHostToDevice,
                                        h->stream));
        size_t used1 = 0;
        PURIFY_TRY(upload_table(h, out, ms->pidx[1], &used1));
        if (!last) {
            PURIFY_TRY(ensure_bytes(h, &ms->pool[1], &ms->pool_cap[1], used1 * pool_slot_bytes(so), max_bytes));
            PURIFY_CUDA_TRY(cudaMemsetAsync(ms->pool[1], 0, pool_slot_bytes(so), h->stream));
        } else {
            // the density: 32 x 32 float64 blocks, zeroed (rows and columns
            // >= n are not written).  When the device lacks room for it, the
            // planes pool this step does not write is given back first.
            const size_t need = used1 * 8192;
            if (need > ms->dpool_cap && ms->pool[1]) {
                size_t fr = 0, tot = 0;
                PURIFY_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
                if (fr + ms->dpool_cap < need + need / 4 + ((size_t)1 << 30)) {
                    PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
                    cudaFree(ms->pool[1]);
                    ms->pool[1] = nullptr;
                    ms->pool_cap[1] = 0;
                }
            }
            PURIFY_TRY(ensure_bytes(h, &ms->dpool, &ms->dpool_cap, need, ((size_t)nb * nb + 1) * 8192));
            PURIFY_CUDA_TRY(cudaMemsetAsync(ms->dpool, 0, used1 * 8192, h->stream));
        }
        ms->pool_bytes_peak = std::max(ms->pool_bytes_peak,
                                       (double)(used0 * pool_slot_bytes(s) + used1 * pool_slot_bytes(so)));
        DigitStep st;
        st.n = n;
        st.n_pad = n_pad;
        st.rbits = rb;
        st.A = st.B = ms->pool[0];
        st.a_idx = st.b_idx = ms->pidx[0];
        st.a_slots = st.b_slots = (int)(ms->pool_cap[0] / pool_slot_bytes(s));
        st.s_in = s;
        st.eA = st.eB = 0;
        st.use_E = 1;
        tc_coeffs(S.branch[i], S.alpha[i], &st.cP, &st.cE, &st.cI);
        st.red = h->red + 4 * (2 * i + 1);
        st.err = ms->err;
        st.scratch = ms->scratch;
        st.max_ctas = ms->ctas;
        st.kc_mask = ms->kc_buf;
        st.bnorm2 = ms->bnorm2;
        st.wait_cycles = 1000ll * h->opt.wait_kcycles;
        st.out_idx = ms->pidx[1];
        if (last) {
            st.out64 = ms->dpool;
        } else {
            st.out = ms->pool[1];
            st.s_out = so;
            st.e_out = 0;
        }
        PURIFY_TRY(product_begin(h));
        PURIFY_TRY(launch_digit_group(s, &st, 1, ms->pwork, (int)work.size(), ms->scratch, ms->ctas, ms->err,
                                      h->stream, st.wait_cycles));
        ++h->st.product_launches;
        h->st.tensor_flops += 0.5 * s * (s + 1) * pairs_tile * chunks;
        PURIFY_TRY(product_end(h));
        PURIFY_TRY(truncate_step(h, out, tau, ms->pidx[1]));
        X = out;
        ms->nnzb_history.push_back(X.count_upper());
        if (!last) {
            // the kept blocks into pool 0 (the step that read it is complete:
            // truncate_step waited for the stream)
            PURIFY_TRY(upload_table(h, X, ms->pidx[0], &used0));
            PURIFY_TRY(ensure_bytes(h, &ms->pool[0], &ms->pool_cap[0], used0 * pool_slot_bytes(so), max_bytes));
            PURIFY_CUDA_TRY(cudaMemsetAsync(ms->pool[0], 0, pool_slot_bytes(so), h->stream));
            const unsigned grid = (unsigned)std::min<int64_t>(152 * 8, ((int64_t)nb * nb + 7) / 8);
            compact_slots_kernel<<<grid, 256, 0, h->stream>>>(ms->pool[1], ms->pidx[1], ms->pool[0], ms->pidx[0], nb,
                                                               plane_pairs(so));
            PURIFY_CUDA_TRY(cudaGetLastError());
            count_launches(1);
            ms->pool_bytes_peak = std::max(ms->pool_bytes_peak,
                                           (double)((used0 + used1) * pool_slot_bytes(so)));
        } else {
            ms->pool_bytes_peak = std::max(ms->pool_bytes_peak, (double)(used0 * pool_slot_bytes(s) + used1 * 8192));
            for (int I = 0; I < nb; ++I) {
                const uint64_t* r = X.row(I);
                for (int w = I >> 6; w < X.words; ++w) {
                    uint64_t bits = r[w];
                    if (w == (I >> 6)) bits &= ~0ull << (I & 63);  // J >= I
                    for (; bits; bits &= bits - 1)
                        ms->d_blocks.push_back(make_int2(I, w * 64 + __builtin_ctzll(bits)));
                }
            }
            ms->d_pooled = true;
        }
    }
    if (m == 0) {
        PURIFY_TRY(ensure_dense_F(h));
        PURIFY_TRY(launch_affine_f64(h->F, n, h->X[0], n, c1, c0, h->stream));
    }
    PURIFY_CUDA_TRY(cudaEventRecord(h->e1, h->stream));
    red.assign(4 * (size_t)slots, 0.0);
    int err = 0;
    PURIFY_CUDA_TRY(cudaMemcpyAsync(red.data(), h->red, sizeof(double) * red.size(), cudaMemcpyDeviceToHost,
                                    h->stream));
    PURIFY_CUDA_TRY(cudaMemcpyAsync(&err, ms->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->st.device_flag = err;
    h->st.plane_pool_mib = (int)std::ceil(ms->pool_bytes_peak / (1024.0 * 1024.0));
    if (err) return device_flag_status(err);
    if (m > 0) {
        h->st.trace = red[4 * (size_t)(2 * (m - 1) + 1)];
        h->st.idem_err_fro = std::sqrt(std::max(red[4 * (size_t)(2 * (m - 1) + 1) + 1], 0.0));
    } else {
        h->st.trace = NAN;
        h->st.idem_err_fro = NAN;
    }
    return PURIFY_OK;
}

}  // namespace purify
