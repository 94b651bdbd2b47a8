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
#include <vector>

#include "digits_tc.h"
#include "mixed.h"
#include "queue_plan.h"

namespace purify {

namespace {

// Blocks (I, J) and (J, I) leave a pool's slot table: from then on they
// read as slot 0, the zero block.
__global__ void drop_slots_kernel(int* idx, int nb, const int2* blocks, int count) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
        const int2 b = blocks[k];
        idx[(size_t)b.x * nb + b.y] = 0;
        idx[(size_t)b.y * nb + b.x] = 0;
    }
}

// Zero blocks (I, J) and (J, I) of an n x n float64 matrix.
__global__ void mask_f64_kernel(double* D, int n, const int2* blocks) {
    const int2 b = blocks[blockIdx.x];
    for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
        const int r = e >> 5, c = e & 31;
        const int i0 = b.x * 32 + r, j0 = b.y * 32 + c;
        if (i0 < n && j0 < n) D[(size_t)i0 * n + j0] = 0.0;
        const int i1 = b.y * 32 + r, j1 = b.x * 32 + c;
        if (i1 < n && j1 < n) D[(size_t)i1 * n + j1] = 0.0;
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

// One CTA of 1024 threads: the first bin whose cumulative mass (added to
// `base`) exceeds the budget; clears the histogram for the next pass.
__global__ void __launch_bounds__(1024) trunc_scan_kernel(TruncSel* sel, int pass) {
    __shared__ unsigned long long part[1024];
    __shared__ int first;
    const int t = threadIdx.x;
    constexpr int per = kHistBins / 1024;
    const unsigned long long base = pass ? sel->cum_before : 0ull;
    unsigned long long sum = 0;
    for (int b = t * per; b < (t + 1) * per; ++b) sum += sel->hist_fx[b];
    part[t] = sum;
    if (t == 0) first = kHistBins;
    __syncthreads();
    // exclusive prefix of the 1024 partial sums (fixed order)
    for (int o = 1; o < 1024; o <<= 1) {
        const unsigned long long v = t >= o ? part[t - o] : 0ull;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    unsigned long long cum = base + (t ? part[t - 1] : 0ull);
    const unsigned long long budget = (unsigned long long)kBudgetUnits;
    int mine = kHistBins;
    unsigned long long before = 0;
    for (int b = t * per; b < (t + 1) * per; ++b) {
        const unsigned long long v = sel->hist_fx[b];
        if (sel->hist_cnt[b] && cum + v > budget) {
            mine = b;
            before = cum;
            break;
        }
        cum += v;
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
    if (t == 0 && first == kHistBins) sel->found = 0;
    for (int b = t; b < kHistBins; b += 1024) {
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
    int count_upper() const {
        int c = 0;
        for (int I = 0; I < nb; ++I)
            for (int J = I; J < nb; ++J) c += get(I, J);
        return c;
    }
};

// Pattern of X^2, of X and of the diagonal together (the blocks that Eq. 4
// and Eq. 5 can make nonzero).
void output_pattern(const Pattern& X, Pattern& out) {
    out.init(X.nb);
    for (int I = 0; I < X.nb; ++I) {
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
}

// Per upper 128 x 128 tile t = tj (tj + 1) / 2 + ti: the 32-wide k-chunks
// where both row panels hold a nonzero block, as a bitmask (X.words words per
// tile) and a count (-1 when that is every chunk).
void chunk_masks(const Pattern& X, int T, std::vector<int>& cnt, std::vector<uint64_t>& mask) {
    const int words = X.words, nb = X.nb;
    std::vector<uint64_t> panel((size_t)T * words, 0);
    for (int t = 0; t < T; ++t)
        for (int r = 4 * t; r < 4 * t + 4 && r < nb; ++r)
            for (int w = 0; w < words; ++w) panel[(size_t)t * words + w] |= X.row(r)[w];
    const size_t tiles = (size_t)T * (T + 1) / 2;
    cnt.assign(tiles, 0);
    mask.assign(tiles * words, 0);
    for (int tj = 0; tj < T; ++tj)
        for (int ti = 0; ti <= tj; ++ti) {
            const size_t t = (size_t)tj * (tj + 1) / 2 + ti;
            int c = 0;
            for (int w = 0; w < words; ++w) {
                const uint64_t m = panel[(size_t)ti * words + w] & panel[(size_t)tj * words + w];
                mask[t * words + w] = m;
                c += __builtin_popcountll(m);
            }
            cnt[t] = (c == nb) ? -1 : c;
        }
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

// Remove the chosen blocks from a pool's slot table and / or zero them in
// the float64 result.
int apply_drops(purify_ctx* h, size_t count, int* idx, int nb, double* out64, int n) {
    MixedState* ms = h->mixed;
    if (count == 0) return PURIFY_OK;
    if (idx) {
        const unsigned grid = (unsigned)std::min<size_t>((count + 255) / 256, 152 * 4);
        drop_slots_kernel<<<grid, 256, 0, h->stream>>>(idx, nb, ms->drops, (int)count);
        PURIFY_CUDA_TRY(cudaGetLastError());
        count_launches(1);
    }
    if (out64) {
        mask_f64_kernel<<<(unsigned)count, 256, 0, h->stream>>>(out64, n, ms->drops);
        PURIFY_CUDA_TRY(cudaGetLastError());
        count_launches(1);
    }
    return PURIFY_OK;
}

// Choose the drops of one step on the device (see trunc_hist_kernel) and
// zero them; the host receives the dropped blocks for its pattern and walks
// the blocks tied at the selected norm in (row, column) order.
int truncate_step(purify_ctx* h, Pattern& pat, double tau, int* idx, double* out64, int n) {
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
    std::vector<int2> drop(nd);
    if (nd)
        PURIFY_CUDA_TRY(cudaMemcpyAsync(drop.data(), ms->drops, sizeof(int2) * nd, cudaMemcpyDeviceToHost, h->stream));
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
            drop.insert(drop.end(), tie.begin(), tie.begin() + (ptrdiff_t)k);
            nd += k;
        }
    }
    for (const int2& b : drop) {
        pat.clear(b.x, b.y);
        pat.clear(b.y, b.x);
    }
    return apply_drops(h, nd, idx, nb, out64, n);
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
int ensure_pool(purify_ctx* h, int k, size_t bytes, size_t max_bytes) {
    MixedState* ms = h->mixed;
    if (bytes <= ms->pool_cap[k]) return PURIFY_OK;
    PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
    cudaFree(ms->pool[k]);
    ms->pool[k] = nullptr;
    ms->pool_cap[k] = 0;
    const size_t c = std::max(bytes, std::min(bytes + bytes / 4 + (64 << 10), max_bytes));
    PURIFY_CUDA_TRY(cudaMalloc(&ms->pool[k], c));
    ms->pool_cap[k] = c;
    return PURIFY_OK;
}

// Copy the kept blocks of a pool into a compact one: block (I, J) with slot
// d = didx[I nb + J] != 0 receives slot sidx[I nb + J] of src (np plane
// pairs per slot).  One warp per table entry.
__global__ void compact_slots_kernel(const __nv_bfloat16* __restrict__ src, const int* __restrict__ sidx,
                                     __nv_bfloat16* __restrict__ dst, const int* __restrict__ didx, int nb, int np) {
    const int lane = threadIdx.x & 31;
    const int total = nb * nb;  // nb <= 4096
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < total; e += warps) {
        const int d = didx[e];
        if (d == 0) continue;
        const uint4* from = (const uint4*)(src + (size_t)sidx[e] * np * 2048);
        uint4* to = (uint4*)(dst + (size_t)d * np * 2048);
        for (int q = lane; q < np * 256; q += 32) to[q] = from[q];
    }
}

// Slot table of a pattern (every block of it, both triangles): slots 1, 2,
// .. in row-major block order.  Returns the slots used, slot 0 included.
size_t assign_slots(const Pattern& P, std::vector<int>& idx) {
    idx.assign((size_t)P.nb * P.nb, 0);
    int k = 1;
    for (int I = 0; I < P.nb; ++I)
        for (int J = 0; J < P.nb; ++J)
            if (P.get(I, J)) idx[(size_t)I * P.nb + J] = k++;
    return (size_t)k;
}

// The upper 128 x 128 tiles holding a block of `out`, in banded order: the
// product's work items {0, ti, tj, 0}.
void pattern_tiles(const Pattern& out, int T, std::vector<int4>& work) {
    std::vector<int2> band;
    banded_tiles(T, band);
    work.clear();
    for (const int2& t : band) {
        bool any = false;
        for (int r = 4 * t.x; r < 4 * t.x + 4 && !any; ++r)
            any = ((out.row(r)[(4 * t.y) >> 6] >> ((4 * t.y) & 63)) & 0xFull) != 0;
        if (any) work.push_back(make_int4(0, t.x, t.y, 0));
    }
}

// Table k and a zero slot 0 for a pool whose slots hold s planes (slot 0
// is cleared each time: slots of another size may have overlapped it).
int upload_slots(purify_ctx* h, int k, const std::vector<int>& idx, int s) {
    MixedState* ms = h->mixed;
    PURIFY_CUDA_TRY(cudaMemcpyAsync(ms->pidx[k], idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice,
                                    h->stream));
    PURIFY_CUDA_TRY(cudaMemsetAsync(ms->pool[k], 0, pool_slot_bytes(s), h->stream));
    return PURIFY_OK;
}

}  // namespace

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
    const int nb = n_pad / 32, T = n_pad / 128;
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
    // pool slots of the kept blocks
    const int s0 = std::max(sd[0], 1);
    PURIFY_TRY(launch_split_pool(h->F, n, n, n_pad, c1, c0, 0, s0, rb, nullptr, nullptr, ms->bnorm2, h->stream));
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
    std::vector<int> idx;
    size_t used0 = assign_slots(X, idx);
    PURIFY_TRY(ensure_pool(h, 0, used0 * pool_slot_bytes(s0), max_bytes));
    PURIFY_TRY(upload_slots(h, 0, idx, s0));
    PURIFY_TRY(launch_split_pool(h->F, n, n, n_pad, c1, c0, 0, s0, rb, ms->pool[0], ms->pidx[0], nullptr,
                                 h->stream));
    ms->pool_bytes_peak = (double)(used0 * pool_slot_bytes(s0));

    double* D = h->X[0];
    *cur = 0;
    std::vector<int> cnt;
    std::vector<uint64_t> mask;
    std::vector<int4> work;
    const size_t tiles = (size_t)T * (T + 1) / 2;
    const size_t cnt_words = (tiles + 1) / 2;  // the counts, two ints per word
    const double pairs_tile = 2.0 * 128.0 * 128.0 * 32.0;  // one pair, one 32-wide k-chunk
    for (int i = 0; i < m; ++i) {
        const int s = sd[i], so = sd[i + 1];
        const bool last = (i + 1 == m);
        Pattern out;
        output_pattern(X, out);
        chunk_masks(X, T, cnt, mask);
        pattern_tiles(out, T, work);
        PURIFY_TRY(grow(&ms->kc_buf, &ms->kc_buf_cap, cnt_words + mask.size()));
        PURIFY_TRY(grow(&ms->pwork, &ms->pwork_cap, work.size()));
        int* kc_cnt = (int*)ms->kc_buf;
        unsigned long long* kc_mask = ms->kc_buf + cnt_words;
        PURIFY_CUDA_TRY(cudaMemcpyAsync(kc_cnt, cnt.data(), sizeof(int) * tiles, cudaMemcpyHostToDevice, h->stream));
        PURIFY_CUDA_TRY(cudaMemcpyAsync(kc_mask, mask.data(), sizeof(uint64_t) * mask.size(), cudaMemcpyHostToDevice,
                                        h->stream));
        PURIFY_CUDA_TRY(cudaMemcpyAsync(ms->pwork, work.data(), sizeof(int4) * work.size(), cudaMemcpyHostToDevice,
                                        h->stream));
        double chunks = 0.0;
        for (const int4& w : work) {
            const int c = cnt[(size_t)w.z * (w.z + 1) / 2 + w.y];
            chunks += c < 0 ? (double)nb : (double)c;
        }
        size_t used1 = 0;
        if (!last) {
            used1 = assign_slots(out, idx);
            PURIFY_TRY(ensure_pool(h, 1, used1 * pool_slot_bytes(so), max_bytes));
            PURIFY_TRY(upload_slots(h, 1, idx, so));
        } else if (work.size() < tiles) {
            // tiles outside the work list are not written
            PURIFY_CUDA_TRY(cudaMemsetAsync(D, 0, sizeof(double) * (size_t)n * n, h->stream));
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
        st.kc_cnt = kc_cnt;
        st.kc_mask = kc_mask;
        st.bnorm2 = ms->bnorm2;
        st.wait_cycles = 1000ll * h->opt.wait_kcycles;
        if (last) {
            st.out64 = D;
        } else {
            st.out = ms->pool[1];
            st.out_idx = ms->pidx[1];
            st.s_out = so;
            st.e_out = 0;
        }
        PURIFY_TRY(product_begin(h));
        PURIFY_TRY(launch_digit_group(s, &st, 1, ms->pwork, (int)work.size(), ms->scratch, ms->ctas, ms->err,
                                      h->stream, st.wait_cycles));
        ++h->st.product_launches;
        h->st.tensor_flops += 0.5 * s * (s + 1) * pairs_tile * chunks;
        PURIFY_TRY(product_end(h));
        PURIFY_TRY(truncate_step(h, out, tau, last ? nullptr : ms->pidx[1], last ? D : nullptr, n));
        X = out;
        ms->nnzb_history.push_back(X.count_upper());
        if (!last) {
            // the kept blocks into pool 0 (the step that read it is complete:
            // truncate_step waited for the stream)
            used0 = assign_slots(X, idx);
            PURIFY_TRY(ensure_pool(h, 0, used0 * pool_slot_bytes(so), max_bytes));
            PURIFY_TRY(upload_slots(h, 0, idx, so));
            const int total_warps = nb * nb;
            const unsigned grid = (unsigned)std::min(152 * 8, (total_warps + 7) / 8);
            compact_slots_kernel<<<grid, 256, 0, h->stream>>>(ms->pool[1], ms->pidx[1], ms->pool[0], ms->pidx[0], nb,
                                                               plane_pairs(so));
            PURIFY_CUDA_TRY(cudaGetLastError());
            count_launches(1);
            ms->pool_bytes_peak = std::max(ms->pool_bytes_peak,
                                           (double)((used0 + used1) * pool_slot_bytes(so)));
        }
    }
    if (m == 0) PURIFY_TRY(launch_affine_f64(h->F, n, D, n, c1, c0, h->stream));
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
