// Many purifications of uneven size on one device: the grouped step engine
// behind purify_batch_* (batch runs captured in a CUDA graph, and the
// continuous-batching serving loop).
//
// Every instance's product steps (Algorithm 1: two per iteration; Algorithm 2:
// one) are planned when it is added: digit counts from its own mapped gaps,
// coefficients from its own scalar schedule, buffers of its own.  A round
// advances every active instance by one product.  The tiles of all instances
// that share a digit count go to one persistent launch of the digit-plane
// product kernel, largest products first; instances finish at their own
// iteration counts and drop out of later rounds.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <queue>
#include <vector>

#include "digits_kernel.cuh"
#include "mixed.h"
#include "queue_plan.h"

using namespace purify;

namespace purify {
int digits_for_gap(double g, const purify_options& o, int rbits);
int build_schedule_public(int scheme, double lmin, double lmax, double mu, double homo, double lumo,
                          double tol, int max_iter, Schedule& S);
}  // namespace purify

namespace {

struct Instance {
    int id = -1;
    int n = 0, n_pad = 0, scheme = 0, rbits = 7;
    int64_t nocc = -1;
    double mu = NAN, tol = 0.0;
    purify_bounds b{};
    Schedule S;
    bool converged = false;
    int state = 0;        // 0 pending (split not queued), 1 active, 2 done, <0 error
    int k = 0;            // next product step
    std::vector<DigitStep> steps;
    double split_a = 0.0, split_b = 0.0;
    int split_e = 0, split_s = 0;
    double* F = nullptr;
    double* D = nullptr;
    double* red = nullptr;  // 4 doubles: last step's reductions
    __nv_bfloat16* Xd[2] = {nullptr, nullptr};
    __nv_bfloat16* Sd = nullptr;
    size_t bytes = 0;
    int digit_max = 0;
    double tensor_flops = 0.0;
    double useful_flops = 0.0;
    int mult = 0;
};

void free_instance(Instance& in) {
    cudaFree(in.F);
    cudaFree(in.D);
    cudaFree(in.red);
    cudaFree(in.Xd[0]);
    cudaFree(in.Xd[1]);
    cudaFree(in.Sd);
    in.F = in.D = in.red = nullptr;
    in.Xd[0] = in.Xd[1] = in.Sd = nullptr;
}


}  // namespace

struct purify_batch {
    int device = 0;
    cudaStream_t stream = nullptr;       // private, non-blocking (capturable)
    cudaStream_t user_stream = nullptr;  // the caller's stream (null = legacy default)
    cudaEvent_t join_ev = nullptr;
    bool own_stream = false;
    purify_options opt{};
    int ctas = 0;
    float2* scratch = nullptr;
    int* err = nullptr;
    std::vector<Instance*> inst;  // index = id
    size_t bytes_in_use = 0;
    // staging for grouped launches
    void* dev_buf = nullptr;
    size_t dev_cap = 0;
    std::vector<uint8_t> host_buf;
    // staging of the last whole-batch queue (own buffer: a captured graph
    // reads it on every replay)
    void* qdev_buf = nullptr;
    size_t qdev_cap = 0;
    QueueStaging last_queue;
    size_t split_jobs_off = 0;  // the queue's f_0 splits, staged after it
    int split_jobs = 0, split_strips = 0;
    int last_mode = -1;
    // graph of the last full run
    cudaGraphExec_t graph = nullptr;
    std::vector<int> graph_ids;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double last_seconds = 0.0;
};

namespace {

int64_t footprint(int64_t n, int digits) {
    const int64_t n_pad = (n + 127) / 128 * 128;
    return 2 * 8 * n * n + 3 * 2 * (int64_t)digits * n_pad * n_pad + 64;
}

// Algorithm 2 coefficients: Y = cP X^2 + cE X + cI I.
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

bool fixed_mu_scheme(int scheme) { return scheme == PURIFY_FIXED_MU_SF || scheme == PURIFY_FIXED_MU_MONO; }

// The product steps of one instance (same arithmetic as the single-matrix
// mixed path).
void plan_steps(purify_batch* B, Instance& in) {
    const int m = (int)in.S.alpha.size();
    const bool fixed = fixed_mu_scheme(in.scheme);
    std::vector<int> sd(m + 1);
    for (int i = 0; i < m; ++i) {
        const double b = i ? in.S.beta[i - 1] : in.S.beta0;
        const double bb = i ? in.S.betabar[i - 1] : in.S.betabar0;
        sd[i] = digits_for_gap(bb - b, B->opt, in.rbits);
    }
    sd[m] = sd[m ? m - 1 : 0];
    in.digit_max = 0;
    for (int i = 0; i < m; ++i) in.digit_max = std::max(in.digit_max, sd[i]);
    const double lmin = in.b.lmin, lmax = in.b.lmax;
    double c0, c1;
    if (fixed) {
        const double gamma = 2.0 * std::max(lmax - in.mu, in.mu - lmin);
        c0 = in.mu / gamma + 0.5;
        c1 = -1.0 / gamma;
        const double a1 = m ? in.S.alpha[0] : 1.0;
        in.split_a = a1 * c1;
        in.split_b = a1 * (c0 - 0.5) + 0.5;
        in.split_e = 1;
    } else {
        c0 = lmax / (lmax - lmin);
        c1 = -1.0 / (lmax - lmin);
        in.split_a = c1;
        in.split_b = c0;
        in.split_e = 0;
    }
    in.split_s = sd[0];
    const int T = in.n_pad / 128;
    const double tile_flops = 2.0 * 128.0 * 128.0 * (double)in.n_pad * (double)(T * (T + 1) / 2);
    in.steps.clear();
    in.tensor_flops = 0.0;
    int x = 0;
    for (int i = 0; i < m; ++i) {
        const int s = sd[i];
        const bool last = (i + 1 == m);
        DigitStep st;
        st.n = in.n;
        st.n_pad = in.n_pad;
        st.rbits = in.rbits;
        st.s_in = s;
        if (fixed) {
            st.A = st.B = in.Xd[x];
            st.eA = st.eB = 1;
            st.out = in.Sd;
            st.s_out = s;
            st.e_out = 1;
            in.steps.push_back(st);
            DigitStep p2 = st;
            p2.A = in.Sd;
            p2.B = in.Xd[x];
            p2.use_E = 1;
            p2.cP = -2.0;
            p2.cE = 3.0;
            if (last) {
                p2.out = nullptr;
                p2.s_out = 0;
                p2.out64 = in.D;
                p2.red = in.red;
            } else {
                const double an = in.S.alpha[i + 1];
                p2.dY = an;
                p2.dI = 0.5 * (1.0 - an);
                p2.out = in.Xd[x ^ 1];
                p2.s_out = sd[i + 1];
            }
            in.steps.push_back(p2);
            in.tensor_flops += 2.0 * 0.5 * s * (s + 1) * tile_flops;
        } else {
            st.A = st.B = in.Xd[x];
            st.eA = st.eB = 0;
            st.use_E = 1;
            tc_coeffs(in.S.branch[i], in.S.alpha[i], &st.cP, &st.cE, &st.cI);
            if (last) {
                st.out64 = in.D;
                st.red = in.red;
            } else {
                st.out = in.Xd[x ^ 1];
                st.s_out = sd[i + 1];
                st.e_out = 0;
            }
            in.steps.push_back(st);
            in.tensor_flops += 0.5 * s * (s + 1) * tile_flops;
        }
        x ^= 1;
    }
    in.mult = (int)in.steps.size();
    const double nn = (double)in.n;
    in.useful_flops = in.mult * nn * nn * (nn + 1.0);
}

int ensure_dev(purify_batch* B, size_t bytes) {
    if (bytes <= B->dev_cap) return PURIFY_OK;
    if (B->graph) {  // the cached graph points into the old buffer
        cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
        B->graph_ids.clear();
    }
    PURIFY_CUDA_TRY(cudaStreamSynchronize(B->stream));
    cudaFree(B->dev_buf);
    B->dev_buf = nullptr;
    B->dev_cap = 0;
    const size_t cap = std::max(bytes, (size_t)1 << 20) * 2;
    PURIFY_CUDA_TRY(cudaMalloc(&B->dev_buf, cap));
    B->dev_cap = cap;
    return PURIFY_OK;
}

// One grouped launch of one round: up to kGroupMax products with a common
// digit count; their work list is staged at work_off.
struct GroupPlan {
    int s = 0;
    std::vector<DigitStep> steps;
    size_t work_off = 0;
    int items = 0;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Stage the grouped launches of one round (the next product of every listed
// instance): work lists into host_buf from `off`; append the group plans.
int stage_round(purify_batch* B, const std::vector<Instance*>& act, size_t& off, std::vector<GroupPlan>& groups) {
    for (int s = 1; s <= kMaxDigitPlanes; ++s) {
        std::vector<Instance*> all_s;
        for (Instance* in : act)
            if (in->steps[in->k].s_in == s) all_s.push_back(in);
        if (all_s.empty()) continue;
        // largest products first: long work items are handed out before short ones
        std::stable_sort(all_s.begin(), all_s.end(), [](Instance* a, Instance* b) { return a->n_pad > b->n_pad; });
        for (size_t c0 = 0; c0 < all_s.size(); c0 += kGroupMax) {
            const size_t c1 = std::min(all_s.size(), c0 + (size_t)kGroupMax);
            GroupPlan g;
            g.s = s;
            std::vector<std::vector<int4>> per;
            size_t items = 0;
            for (size_t k = c0; k < c1; ++k) {
                Instance* in = all_s[k];
                const int gi = (int)(k - c0);
                g.steps.push_back(in->steps[in->k]);
                const int T = in->n_pad / 128;
                per.emplace_back();
                for (int tj = 0; tj < T; ++tj)
                    for (int ti = 0; ti <= tj; ++ti) per.back().push_back(make_int4(gi, ti, tj, 0));
                items += per.back().size();
            }
            g.work_off = align_up(off, 128);
            const size_t end = g.work_off + sizeof(int4) * items;
            if (B->host_buf.size() < end) B->host_buf.resize(end * 2);
            int4* work = (int4*)(B->host_buf.data() + g.work_off);
            // interleaved by tile rank so the persistent CTAs start on large products
            size_t w = 0;
            for (size_t r = 0;; ++r) {
                bool any = false;
                for (size_t gi = 0; gi < per.size(); ++gi)
                    if (r < per[gi].size()) {
                        work[w++] = per[gi][r];
                        any = true;
                    }
                if (!any) break;
            }
            g.items = (int)items;
            off = end;
            groups.push_back(std::move(g));
        }
    }
    return PURIFY_OK;
}

int launch_groups(purify_batch* B, const std::vector<GroupPlan>& groups) {
    const uint8_t* dev = (const uint8_t*)B->dev_buf;
    for (const GroupPlan& g : groups)
        PURIFY_TRY(launch_digit_group(g.s, g.steps.data(), (int)g.steps.size(), (const int4*)(dev + g.work_off),
                                      g.items, B->scratch, B->ctas, B->err, B->stream,
                                      1000ll * B->opt.wait_kcycles));
    return PURIFY_OK;
}

// The whole batch as one persistent launch (queue mode of the product
// kernel): every product of every instance in one work list, claimed in list
// order by the persistent CTAs; on the device an item of product k of an
// instance waits until product k-1 of that instance has completed, so each
// instance advances on its own.  The list order comes from a list-scheduling
// simulation of the launch on the host: CTAs take the next item when they
// come free, an instance's next product becomes available once its previous
// one has finished, and among available products the one with the longest
// items goes first.  stage_queue_products checks that no item precedes one
// it waits for.
// Steps [k0, k1) of one instance, for a queue launch.
struct StepRange {
    Instance* in;
    int k0, k1;
};

int stage_queue(purify_batch* B, const std::vector<StepRange>& ranges, QueueStaging& q) {
    // products: instance-major; an instance's product waits for every item
    // of its previous one (which reads the buffer it overwrites, and wrote
    // what it reads)
    struct Prod {
        Instance* in;
        int k;         // step index
        int T;         // tile rows
        int items;     // upper tiles
        double cost;   // modelled cycles of one item
        int dep;       // product index it waits for, -1: none
        int next = -1; // the instance's following product
    };
    std::vector<Prod> prods;
    std::vector<QueueProduct> qp;
    for (const StepRange& rg : ranges) {
        Instance* in = rg.in;
        const int T = in->n_pad / 128;
        for (int k = rg.k0; k < rg.k1; ++k) {
            const int s = in->steps[k].s_in;
            // MMA cycles: s(s+1)/2 digit pairs of a 128 x 128 x n_pad product
            // at 8192 flop per clock
            const double cost = 0.5 * s * (s + 1) * 4.0 * in->n_pad;
            Prod p{in, k, T, T * (T + 1) / 2, cost, k > rg.k0 ? (int)prods.size() - 1 : -1};
            if (k > rg.k0) prods.back().next = (int)prods.size();
            prods.push_back(p);
            QueueProduct x;
            x.st = in->steps[k];
            x.war0 = p.dep;
            qp.push_back(x);
        }
    }
    const int products = (int)prods.size();
    size_t items = 0;
    for (const Prod& p : prods) items += (size_t)p.items;
    std::vector<int4> work;
    work.reserve(items);
    // List scheduling over B->ctas simulated CTAs.  A CTA has two resources:
    // its MMA pipe, free again once an item's accumulators are drained
    // (phase 1), and its epilogue warps, busy until phase 2 ends; it claims
    // its next item when its current MMAs end.  An instance's next product
    // becomes ready when the last phase 2 of its current one ends.  Epilogue
    // costs in SM cycles, measured on a stamped copy of the kernel (~5 and
    // ~40 us at 1.9 GHz).
    constexpr double kPhase1 = 10000.0, kPhase2 = 76000.0;
    struct Cta {
        double claim, mma_free, epi_free;
    };
    auto later = [](const std::pair<double, int>& x, const std::pair<double, int>& y) { return x.first > y.first; };
    std::vector<Cta> ctas(std::max(1, B->ctas), Cta{0.0, 0.0, 0.0});
    std::priority_queue<std::pair<double, int>, std::vector<std::pair<double, int>>, decltype(later)> next_cta(later);
    for (int c = 0; c < (int)ctas.size(); ++c) next_cta.push({0.0, c});
    using TP = std::pair<double, int>;
    std::priority_queue<TP, std::vector<TP>, std::greater<TP>> future;  // (ready time, product)
    std::priority_queue<TP> ready;                                      // (item cost, -product)
    std::vector<int> placed(products, 0);
    std::vector<double> finish(products, 0.0);
    for (int pi = 0; pi < products; ++pi)
        if (prods[pi].dep < 0) future.push({0.0, pi});
    while (work.size() < items) {
        const int c = next_cta.top().second;
        next_cta.pop();
        Cta& C = ctas[c];
        double f = C.claim;
        while (!future.empty() && future.top().first <= f) {
            ready.push({prods[future.top().second].cost, -future.top().second});
            future.pop();
        }
        if (ready.empty()) {  // this CTA waits until the next product is ready
            f = future.top().first;
            ready.push({prods[future.top().second].cost, -future.top().second});
            future.pop();
        }
        const int pi = -ready.top().second;
        Prod& p = prods[pi];
        const int r = placed[pi]++;
        // items of a product in order: tile column tj, rows ti <= tj
        int tj = 0;
        while ((tj + 1) * (tj + 2) / 2 <= r) ++tj;
        const int ti = r - tj * (tj + 1) / 2;
        work.push_back(make_int4(pi, ti, tj, 0));
        const double mma_start = std::max(f, C.mma_free);
        const double mma_end = mma_start + p.cost;
        const double p1_end = std::max(mma_end, C.epi_free) + kPhase1;
        const double p2_end = p1_end + kPhase2;
        C.claim = mma_end;
        C.mma_free = p1_end;
        C.epi_free = p2_end;
        next_cta.push({C.claim, c});
        finish[pi] = std::max(finish[pi], p2_end);
        if (placed[pi] == p.items) {
            ready.pop();
            if (p.next >= 0) future.push({finish[pi], p.next});
        }
    }
    return stage_queue_products(qp, work, B->host_buf, q);
}

int launch_batch_splits(purify_batch* B) {
    return launch_split_group((const SplitJob*)((uint8_t*)B->qdev_buf + B->split_jobs_off), B->split_jobs,
                              B->split_strips, B->stream);
}

int launch_queue(purify_batch* B, const QueueStaging& q) {
    return launch_staged_queue(q, B->qdev_buf, B->scratch, B->ctas, B->err, B->stream, 1000ll * B->opt.wait_kcycles);
}

int queue_split(purify_batch* B, Instance& in) {
    PURIFY_CUDA_TRY(cudaMemsetAsync(in.red, 0, 4 * sizeof(double), B->stream));
    return launch_split(in.F, in.n, in.n, in.n_pad, in.split_a, in.split_b, in.split_e, in.split_s, in.rbits,
                        in.Xd[0], nullptr, B->stream);
}

void finish_instance(Instance& in) { in.state = 2; }

int check_err(purify_batch* B) {
    int e = 0;
    PURIFY_CUDA_TRY(cudaMemcpyAsync(&e, B->err, sizeof(int), cudaMemcpyDeviceToHost, B->stream));
    PURIFY_CUDA_TRY(cudaStreamSynchronize(B->stream));
    return device_flag_status(e);
}

}  // namespace

extern "C" {

int64_t purify_batch_footprint(int64_t n) {
    if (n <= 0) return 0;
    return footprint(n, kMaxDigitPlanes);
}

int purify_batch_create(purify_batch_t* out, int device, void* cuda_stream, const purify_options* opt) {
    if (!out) return PURIFY_ERR_INVALID_ARG;
    *out = nullptr;
    purify_options o;
    purify_options_default(&o);
    if (opt) o = *opt;
    if (o.digits != 0 && (o.digits < 2 || o.digits > kMaxDigitPlanes)) return PURIFY_ERR_INVALID_ARG;
    if (o.bits_floor != 0 && (o.bits_floor < 16 || o.bits_floor > 43)) return PURIFY_ERR_INVALID_ARG;
    if (o.bits_gap != 0 && (o.bits_gap < 16 || o.bits_gap > 43)) return PURIFY_ERR_INVALID_ARG;
    int ndev = 0;
    PURIFY_CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return PURIFY_ERR_INVALID_ARG;
    cudaDeviceProp prop;
    PURIFY_CUDA_TRY(cudaGetDeviceProperties(&prop, device));
    if (!(prop.major == 10 && prop.minor == 3)) return PURIFY_ERR_UNSUPPORTED;
    PURIFY_CUDA_TRY(cudaSetDevice(device));
    purify_batch* B = new (std::nothrow) purify_batch();
    if (!B) return PURIFY_ERR_OOM;
    B->device = device;
    B->opt = o;
    B->ctas = prop.multiProcessorCount;
    if (const char* e = getenv("PURIFY_BATCH_MAX_CTAS")) {  // share the device: cap the persistent grid
        const int cap = atoi(e);
        if (cap > 0 && cap < B->ctas) B->ctas = cap;
    }
    int r = PURIFY_OK;
    B->user_stream = (cudaStream_t)cuda_stream;
    if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess) r = PURIFY_ERR_CUDA;
    B->own_stream = (r == PURIFY_OK);
    if (r == PURIFY_OK && cudaEventCreateWithFlags(&B->join_ev, cudaEventDisableTiming) != cudaSuccess)
        r = PURIFY_ERR_CUDA;
    if (r == PURIFY_OK && (cudaMalloc(&B->scratch, digit_scratch_bytes(B->ctas)) != cudaSuccess ||
                           cudaMalloc(&B->err, sizeof(int)) != cudaSuccess))
        r = PURIFY_ERR_OOM;
    if (r == PURIFY_OK && (cudaEventCreate(&B->e0) != cudaSuccess || cudaEventCreate(&B->e1) != cudaSuccess))
        r = PURIFY_ERR_CUDA;
    if (r == PURIFY_OK && cudaMemsetAsync(B->err, 0, sizeof(int), B->stream) != cudaSuccess) r = PURIFY_ERR_CUDA;
    if (r == PURIFY_OK) r = prepare_digit_kernels();  // before any stream capture
    if (r != PURIFY_OK) {
        purify_batch_destroy(B);
        return r;
    }
    *out = B;
    return PURIFY_OK;
}

int purify_batch_destroy(purify_batch_t B) {
    if (!B) return PURIFY_OK;
    cudaSetDevice(B->device);
    if (B->stream) cudaStreamSynchronize(B->stream);
    for (Instance* in : B->inst)
        if (in) {
            free_instance(*in);
            delete in;
        }
    if (B->graph) cudaGraphExecDestroy(B->graph);
    cudaFree(B->scratch);
    cudaFree(B->err);
    cudaFree(B->dev_buf);
    cudaFree(B->qdev_buf);
    if (B->e0) cudaEventDestroy(B->e0);
    if (B->e1) cudaEventDestroy(B->e1);
    if (B->join_ev) cudaEventDestroy(B->join_ev);
    if (B->own_stream && B->stream) cudaStreamDestroy(B->stream);
    delete B;
    return PURIFY_OK;
}

int purify_batch_add(purify_batch_t B, const double* F, int64_t n, int64_t ld, int64_t nocc, double mu,
                     const purify_bounds* b, int scheme, double tol, int max_iter, int* id) {
    if (!B || !F || !b || !id || n <= 0 || ld < n || n > 16384) return PURIFY_ERR_INVALID_ARG;
    if (scheme < PURIFY_FIXED_MU_SF || scheme > PURIFY_TC_MONO) return PURIFY_ERR_INVALID_ARG;
    if (!(tol >= 0.0) || max_iter < 0 || max_iter > 10000) return PURIFY_ERR_INVALID_ARG;
    if (std::isnan(b->lmin) || std::isnan(b->lmax) || std::isnan(b->homo) || std::isnan(b->lumo))
        return PURIFY_ERR_BOUNDS;
    if (!(b->lmax > b->lmin) || !(b->homo < b->lumo) || b->homo < b->lmin || b->lumo > b->lmax)
        return PURIFY_ERR_BOUNDS;
    if (nocc > n) return PURIFY_ERR_INVALID_ARG;
    PURIFY_CUDA_TRY(cudaSetDevice(B->device));
    PURIFY_TRY(join_streams(B->stream, B->user_stream, B->join_ev));
    Instance* in = new (std::nothrow) Instance();
    if (!in) return PURIFY_ERR_OOM;
    in->n = (int)n;
    in->n_pad = pad128(n);
    in->rbits = remainder_bits(in->n_pad);
    in->scheme = scheme;
    in->nocc = nocc;
    in->b = *b;
    in->tol = tol;
    in->mu = mu;
    if (fixed_mu_scheme(scheme)) {
        if (std::isnan(in->mu)) in->mu = 0.5 * (b->homo + b->lumo);
        if (!(std::min(in->mu - b->homo, b->lumo - in->mu) > 0.0) || in->mu <= b->lmin || in->mu >= b->lmax) {
            delete in;
            return PURIFY_ERR_BOUNDS;
        }
    }
    int r = build_schedule_public(scheme, b->lmin, b->lmax, in->mu, b->homo, b->lumo, tol, max_iter, in->S);
    if (r != PURIFY_OK) {
        delete in;
        return r;
    }
    in->converged = in->S.converged;
    if (in->S.alpha.empty()) {  // nothing to do: still run one unscaled step so D is defined
        delete in;
        return PURIFY_ERR_INVALID_ARG;
    }
    // buffers sized for this instance's largest digit count
    int smax = 0;
    {
        const int m = (int)in->S.alpha.size();
        for (int i = 0; i < m; ++i) {
            const double bb0 = i ? in->S.betabar[i - 1] : in->S.betabar0;
            const double b0 = i ? in->S.beta[i - 1] : in->S.beta0;
            smax = std::max(smax, digits_for_gap(bb0 - b0, B->opt, in->rbits));
        }
    }
    const size_t plane_bytes = plane_buffer_bytes(smax, in->n_pad);
    const size_t nb = sizeof(double) * (size_t)n * n;
    bool ok = cudaMalloc(&in->F, nb) == cudaSuccess && cudaMalloc(&in->D, nb) == cudaSuccess &&
              cudaMalloc(&in->red, 4 * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&in->Xd[0], plane_bytes) == cudaSuccess && cudaMalloc(&in->Xd[1], plane_bytes) == cudaSuccess &&
              cudaMalloc(&in->Sd, fixed_mu_scheme(scheme) ? plane_bytes : 16) == cudaSuccess;
    if (!ok) {
        free_instance(*in);
        delete in;
        return PURIFY_ERR_OOM;
    }
    in->bytes = 2 * nb + (fixed_mu_scheme(scheme) ? 3 : 2) * plane_bytes;
    r = copy_in_matrix(in->F, F, n, ld, B->stream);
    if (r == PURIFY_OK) r = launch_mirror_upper_f64(in->F, n, B->stream);
    if (r != PURIFY_OK) {
        free_instance(*in);
        delete in;
        return r;
    }
    plan_steps(B, *in);
    in->id = (int)B->inst.size();
    B->inst.push_back(in);
    B->bytes_in_use += in->bytes;
    *id = in->id;
    return join_streams(B->user_stream, B->stream, B->join_ev);
}

// One round: queue the f_0 split of pending instances, then one product of
// every active instance.  Synchronises the stream at the end.
int purify_batch_step(purify_batch_t B, int* active_out, int* finished_out) {
    if (!B) return PURIFY_ERR_INVALID_ARG;
    PURIFY_CUDA_TRY(cudaSetDevice(B->device));
    PURIFY_TRY(join_streams(B->stream, B->user_stream, B->join_ev));
    std::vector<Instance*> act;
    for (Instance* in : B->inst) {
        if (!in || in->state >= 2 || in->state < 0) continue;
        if (in->state == 0) {
            in->k = 0;
            PURIFY_TRY(queue_split(B, *in));
            in->state = 1;
        }
        act.push_back(in);
    }
    int finished = 0;
    if (!act.empty()) {
        size_t off = 0;
        std::vector<GroupPlan> groups;
        PURIFY_TRY(stage_round(B, act, off, groups));
        PURIFY_TRY(ensure_dev(B, off));
        PURIFY_CUDA_TRY(cudaMemcpyAsync(B->dev_buf, B->host_buf.data(), off, cudaMemcpyHostToDevice, B->stream));
        PURIFY_TRY(launch_groups(B, groups));
        PURIFY_TRY(check_err(B));
        for (Instance* in : act) {
            ++in->k;
            if (in->k == (int)in->steps.size()) {
                finish_instance(*in);
                ++finished;
            }
        }
    }
    if (active_out) *active_out = (int)act.size() - finished;
    if (finished_out) *finished_out = finished;
    return join_streams(B->user_stream, B->stream, B->join_ev);
}

int ensure_qdev(purify_batch* B, size_t bytes);

// Continuous batching with fewer host round trips: one queue launch advances
// every active instance by up to max_products products (an instance's
// products chained on the device, instances independent), then
// synchronises.  Instances added since the last call get their f_0 split
// first.
int purify_batch_advance(purify_batch_t B, int max_products, int* active_out, int* finished_out) {
    if (!B || max_products < 1) return PURIFY_ERR_INVALID_ARG;
    PURIFY_CUDA_TRY(cudaSetDevice(B->device));
    PURIFY_TRY(join_streams(B->stream, B->user_stream, B->join_ev));
    std::vector<StepRange> ranges;
    for (Instance* in : B->inst) {
        if (!in || in->state >= 2 || in->state < 0) continue;
        if (in->state == 0) {
            in->k = 0;
            PURIFY_TRY(queue_split(B, *in));
            in->state = 1;
        }
        ranges.push_back({in, in->k, std::min((int)in->steps.size(), in->k + max_products)});
    }
    int finished = 0;
    if (!ranges.empty()) {
        if (B->graph) {  // the staging buffer a captured run reads is about to change
            PURIFY_CUDA_TRY(cudaStreamSynchronize(B->stream));
            cudaGraphExecDestroy(B->graph);
            B->graph = nullptr;
            B->graph_ids.clear();
        }
        QueueStaging q;
        PURIFY_TRY(stage_queue(B, ranges, q));
        PURIFY_TRY(ensure_qdev(B, q.end));
        PURIFY_CUDA_TRY(cudaMemcpyAsync(B->qdev_buf, B->host_buf.data(), q.end, cudaMemcpyHostToDevice, B->stream));
        PURIFY_TRY(launch_staged_queue(q, B->qdev_buf, B->scratch, B->ctas, B->err, B->stream,
                                       1000ll * B->opt.wait_kcycles));
        PURIFY_TRY(check_err(B));
        for (const StepRange& rg : ranges) {
            rg.in->k = rg.k1;
            if (rg.in->k == (int)rg.in->steps.size()) {
                finish_instance(*rg.in);
                ++finished;
            }
        }
    }
    if (active_out) *active_out = (int)ranges.size() - finished;
    if (finished_out) *finished_out = finished;
    return join_streams(B->user_stream, B->stream, B->join_ev);
}

int ensure_qdev(purify_batch* B, size_t bytes) {
    if (bytes <= B->qdev_cap) return PURIFY_OK;
    PURIFY_CUDA_TRY(cudaStreamSynchronize(B->stream));
    cudaFree(B->qdev_buf);
    B->qdev_buf = nullptr;
    B->qdev_cap = 0;
    const size_t cap = std::max(bytes, (size_t)1 << 16) * 2;
    PURIFY_CUDA_TRY(cudaMalloc(&B->qdev_buf, cap));
    B->qdev_cap = cap;
    return PURIFY_OK;
}

// Run every added instance from its start to completion.  mode bit 0: the
// whole run is captured once into a CUDA graph and replayed while the set of
// instances is unchanged.  mode bit 1: one grouped launch per round (the
// products of all instances at the same step, host-ordered) instead of the
// single queue launch in which every instance advances on its own.
int purify_batch_run(purify_batch_t B, int mode) {
    if (!B || mode < 0 || mode > 3) return PURIFY_ERR_INVALID_ARG;
    const bool use_graph = mode & 1;
    const bool rounds_mode = mode & 2;
    PURIFY_CUDA_TRY(cudaSetDevice(B->device));
    PURIFY_TRY(join_streams(B->stream, B->user_stream, B->join_ev));
    std::vector<Instance*> all;
    std::vector<int> ids;
    for (Instance* in : B->inst)
        if (in) {
            all.push_back(in);
            ids.push_back(in->id);
        }
    if (all.empty()) return PURIFY_OK;
    const bool reuse = use_graph && B->graph && ids == B->graph_ids && B->last_mode == mode;
    std::vector<std::vector<GroupPlan>> rounds;
    if (!reuse) {
        // stage the whole batch up front (host arithmetic, untimed)
        if (B->graph) {
            cudaGraphExecDestroy(B->graph);
            B->graph = nullptr;
            B->graph_ids.clear();
        }
        if (rounds_mode) {
            size_t off = 0;
            for (Instance* in : all) in->k = 0;
            for (;;) {
                std::vector<Instance*> act;
                for (Instance* in : all)
                    if (in->k < (int)in->steps.size()) act.push_back(in);
                if (act.empty()) break;
                std::vector<GroupPlan> groups;
                PURIFY_TRY(stage_round(B, act, off, groups));
                rounds.push_back(groups);
                for (Instance* in : act) ++in->k;
            }
            PURIFY_TRY(ensure_dev(B, off));
            PURIFY_CUDA_TRY(cudaMemcpyAsync(B->dev_buf, B->host_buf.data(), off, cudaMemcpyHostToDevice, B->stream));
        } else {
            QueueStaging q;
            std::vector<StepRange> ranges;
            for (Instance* in : all) ranges.push_back({in, 0, (int)in->steps.size()});
            PURIFY_TRY(stage_queue(B, ranges, q));
            // every instance's f_0 split as one launch: its jobs after the queue
            const size_t jobs_off = (q.end + 255) / 256 * 256;
            std::vector<SplitJob> jobs(all.size());
            int strips = 0;
            for (size_t k = 0; k < all.size(); ++k) {
                Instance& in = *all[k];
                PURIFY_TRY(make_split_job(in.F, in.n, in.n, in.n_pad, in.split_a, in.split_b, in.split_e, in.split_s,
                                          in.rbits, in.Xd[0], in.red, strips, &jobs[k]));
                strips += split_strips(in.n_pad);
            }
            const size_t end = jobs_off + sizeof(SplitJob) * jobs.size();
            if (B->host_buf.size() < end) B->host_buf.resize(end);
            std::memcpy(B->host_buf.data() + jobs_off, jobs.data(), sizeof(SplitJob) * jobs.size());
            PURIFY_TRY(ensure_qdev(B, end));
            PURIFY_CUDA_TRY(cudaMemcpyAsync(B->qdev_buf, B->host_buf.data(), end, cudaMemcpyHostToDevice, B->stream));
            B->last_queue = q;
            B->split_jobs_off = jobs_off;
            B->split_jobs = (int)jobs.size();
            B->split_strips = strips;
        }
        PURIFY_CUDA_TRY(cudaStreamSynchronize(B->stream));
        B->last_mode = mode;
        if (use_graph) {
            PURIFY_TRY(prepare_digit_kernels());
            cudaGraph_t g = nullptr;
            PURIFY_CUDA_TRY(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
            int r = PURIFY_OK;
            if (rounds_mode) {
                for (Instance* in : all)
                    if (r == PURIFY_OK) r = queue_split(B, *in);
                for (auto& groups : rounds)
                    if (r == PURIFY_OK) r = launch_groups(B, groups);
            } else {
                r = launch_batch_splits(B);
                if (r == PURIFY_OK) r = launch_queue(B, B->last_queue);
            }
            cudaError_t e = cudaStreamEndCapture(B->stream, &g);
            if (r == PURIFY_OK && e != cudaSuccess) r = cuda_status(e, "cudaStreamEndCapture");
            if (r == PURIFY_OK) {
                e = cudaGraphInstantiate(&B->graph, g, 0);
                if (e != cudaSuccess) r = cuda_status(e, "cudaGraphInstantiate");
            }
            if (g) cudaGraphDestroy(g);
            if (r != PURIFY_OK) return r;
            B->graph_ids = ids;
        }
    }
    PURIFY_CUDA_TRY(cudaEventRecord(B->e0, B->stream));
    if (use_graph) {
        PURIFY_CUDA_TRY(cudaGraphLaunch(B->graph, B->stream));
    } else {
        if (rounds_mode) {
            for (Instance* in : all) PURIFY_TRY(queue_split(B, *in));
            for (auto& groups : rounds) PURIFY_TRY(launch_groups(B, groups));
        } else {
            PURIFY_TRY(launch_batch_splits(B));
            PURIFY_TRY(launch_queue(B, B->last_queue));
        }
    }
    PURIFY_CUDA_TRY(cudaEventRecord(B->e1, B->stream));
    PURIFY_TRY(check_err(B));
    float ms = 0.f;
    PURIFY_CUDA_TRY(cudaEventElapsedTime(&ms, B->e0, B->e1));
    B->last_seconds = 1e-3 * ms;
    for (Instance* in : all) {
        in->k = (int)in->steps.size();
        finish_instance(*in);
    }
    return join_streams(B->user_stream, B->stream, B->join_ev);
}

int purify_batch_status(purify_batch_t B, int id) {
    if (!B || id < 0 || id >= (int)B->inst.size() || !B->inst[id]) return PURIFY_ERR_INVALID_ARG;
    return B->inst[id]->state == 2 ? 1 : 0;
}

int purify_batch_get_density(purify_batch_t B, int id, double* D, int64_t ld) {
    if (!B || !D || id < 0 || id >= (int)B->inst.size() || !B->inst[id]) return PURIFY_ERR_INVALID_ARG;
    Instance* in = B->inst[id];
    if (ld < in->n) return PURIFY_ERR_INVALID_ARG;
    if (in->state != 2) return PURIFY_ERR_STATE;
    PURIFY_CUDA_TRY(cudaSetDevice(B->device));
    PURIFY_TRY(join_streams(B->stream, B->user_stream, B->join_ev));
    PURIFY_CUDA_TRY(cudaMemcpy2DAsync(D, sizeof(double) * ld, in->D, sizeof(double) * in->n,
                                      sizeof(double) * in->n, in->n, cudaMemcpyDefault, B->stream));
    PURIFY_CUDA_TRY(cudaStreamSynchronize(B->stream));
    return join_streams(B->user_stream, B->stream, B->join_ev);
}

int purify_batch_stats(purify_batch_t B, int id, purify_stats_t* st) {
    if (!B || !st || id < 0 || id >= (int)B->inst.size() || !B->inst[id]) return PURIFY_ERR_INVALID_ARG;
    Instance* in = B->inst[id];
    std::memset(st, 0, sizeof(*st));
    const int m = (int)in->S.alpha.size();
    st->iterations = m;
    st->multiplications = in->mult;
    st->err_bound = m ? std::max(in->S.beta[m - 1], 1.0 - in->S.betabar[m - 1]) : NAN;
    st->lmin = in->b.lmin;
    st->lmax = in->b.lmax;
    st->homo = in->b.homo;
    st->lumo = in->b.lumo;
    st->mu = in->mu;
    st->digit_max = in->digit_max;
    st->tensor_flops = in->tensor_flops;
    st->useful_flops = in->useful_flops;
    st->seconds = B->last_seconds;
    st->product_seconds = NAN;
    st->trace = NAN;
    st->idem_err_fro = NAN;
    st->trace_err = NAN;
    if (in->state == 2) {
        double red[4];
        PURIFY_CUDA_TRY(cudaSetDevice(B->device));
        PURIFY_CUDA_TRY(cudaMemcpyAsync(red, in->red, sizeof(red), cudaMemcpyDeviceToHost, B->stream));
        PURIFY_CUDA_TRY(cudaStreamSynchronize(B->stream));
        st->trace = red[0];
        if (!fixed_mu_scheme(in->scheme)) st->idem_err_fro = std::sqrt(std::max(red[1], 0.0));
        st->trace_err = in->nocc >= 0 ? std::fabs(red[0] - (double)in->nocc) : NAN;
    }
    int status = in->converged ? PURIFY_OK : PURIFY_ERR_NOT_CONVERGED;
    if (in->state == 2 && status == PURIFY_OK && in->nocc >= 0 && !(st->trace_err <= 0.5)) status = PURIFY_ERR_BOUNDS;
    st->status = in->state == 2 ? status : PURIFY_ERR_STATE;
    return PURIFY_OK;
}

int purify_batch_release(purify_batch_t B, int id) {
    if (!B || id < 0 || id >= (int)B->inst.size() || !B->inst[id]) return PURIFY_ERR_INVALID_ARG;
    PURIFY_CUDA_TRY(cudaSetDevice(B->device));
    PURIFY_CUDA_TRY(cudaStreamSynchronize(B->stream));
    Instance* in = B->inst[id];
    B->bytes_in_use -= in->bytes;
    free_instance(*in);
    delete in;
    B->inst[id] = nullptr;
    if (B->graph) {
        cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
        B->graph_ids.clear();
    }
    return PURIFY_OK;
}

int64_t purify_batch_bytes_in_use(purify_batch_t B) { return B ? (int64_t)B->bytes_in_use : 0; }

}  // extern "C"
