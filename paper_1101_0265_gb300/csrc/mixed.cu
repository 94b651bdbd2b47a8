// Driver of the mixed path: every matrix product of the scheme runs as a
// digit-plane product on the tcgen05 tensor cores (digits_tc.cu).
//
// Precision per step.  Rounding added at step i in the block that couples
// occupied and unoccupied states is not damped by later steps: it reaches
// the result multiplied by about 1 / (beta_bar - beta), the gap between the
// mapped gap edges at step i (the scalar bounds of Algorithm 1 and
// Algorithm 2).  The digit count of step i is therefore chosen from that
// mapped gap g_i: the smallest s in [3, 6] whose digits carry
// max(30, 26 + log2(1 / g_i)) bits (8 + 7 (s - 1) bits up to n = 4096), so
// early steps (small g) carry 43 bits and late ones 36.
#include "mixed.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>

#include "digits_tc.h"
#include "queue_plan.h"

namespace purify {

void mixed_free(MixedState* ms) {
    if (!ms) return;
    cudaFree(ms->Xd[0]);
    cudaFree(ms->Xd[1]);
    cudaFree(ms->Sd);
    cudaFree(ms->Pd[0]);
    cudaFree(ms->Pd[1]);
    cudaFree(ms->err);
    cudaFree(ms->scratch);
    cudaFree(ms->partial);
    cudaFree(ms->split_cnt);
    cudaFree(ms->kc_buf);
    cudaFree(ms->bnorm2);
    cudaFree(ms->drops);
    cudaFree(ms->pat_dev);
    cudaFree(ms->tsel);
    cudaFree(ms->tsched);
    cudaFree(ms->qdev);
    for (int k = 0; k < 2; ++k) {
        cudaFree(ms->pool[k]);
        cudaFree(ms->pidx[k]);
    }
    cudaFree(ms->pwork);
    cudaFree(ms->spat);
    cudaFree(ms->rowbase);
    cudaFree(ms->strips);
    cudaFree(ms->dpool);
    if (ms->tgraph) cudaGraphExecDestroy(ms->tgraph);
    delete ms;
}

int ensure_mixed(purify_ctx* h, int n_pad, bool planes) {
    if (!h->mixed) {
        h->mixed = new (std::nothrow) MixedState();
        if (!h->mixed) return PURIFY_ERR_OOM;
        PURIFY_CUDA_TRY(cudaMalloc(&h->mixed->err, sizeof(int)));
        int sms = 0;
        PURIFY_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
        h->mixed->ctas = sms;
        PURIFY_CUDA_TRY(cudaMalloc(&h->mixed->scratch, digit_scratch_bytes(sms)));
        PURIFY_CUDA_TRY(cudaMalloc(&h->mixed->partial, sizeof(float) * digit_partial_floats(sms)));
        PURIFY_CUDA_TRY(cudaMalloc(&h->mixed->split_cnt, sizeof(int) * digit_split_counters(sms)));
    }
    MixedState* ms = h->mixed;
    if (!planes || n_pad <= ms->n_pad_cap) return PURIFY_OK;
    cudaFree(ms->Xd[0]);
    cudaFree(ms->Xd[1]);
    cudaFree(ms->Sd);
    ms->Xd[0] = ms->Xd[1] = ms->Sd = nullptr;
    ms->n_pad_cap = 0;
    const size_t bytes = plane_buffer_bytes(kMaxDigitPlanes, n_pad);
    PURIFY_CUDA_TRY(cudaMalloc(&ms->Xd[0], bytes));
    PURIFY_CUDA_TRY(cudaMalloc(&ms->Xd[1], bytes));
    PURIFY_CUDA_TRY(cudaMalloc(&ms->Sd, bytes));
    ms->n_pad_cap = n_pad;
    return PURIFY_OK;
}

// Digits for a step whose mapped gap (distance between the images of the
// gap edges) is g: options.digits when fixed, else the fewest digits whose
// bits cover max(bits_floor, bits_gap + log2(1 / g)).
int digits_for_gap(double g, const purify_options& o, int rbits) {
    if (o.digits > 0) return o.digits;
    if (!(g > 0.0)) return kMaxDigitPlanes;
    const double floor_bits = o.bits_floor > 0 ? o.bits_floor : kBitsFloor;
    const double gap_bits = o.bits_gap > 0 ? o.bits_gap : kBitsGap;
    const double need = std::max(floor_bits, gap_bits + std::log2(1.0 / g));
    for (int s = 3; s < kMaxDigitPlanes; ++s)
        if (digit_bits(s, rbits) >= need) return s;
    return kMaxDigitPlanes;
}

static double pairs_of(int s) { return 0.5 * s * (s + 1); }

// The two further plane buffers (P_{3,3} intermediates; the queue run's
// third X and second S buffer), at the handle's capacity.
static int ensure_pd(MixedState* ms) {
    if (ms->pd_cap >= ms->n_pad_cap) return PURIFY_OK;
    cudaFree(ms->Pd[0]);
    cudaFree(ms->Pd[1]);
    ms->Pd[0] = ms->Pd[1] = nullptr;
    ms->pd_cap = 0;
    const size_t bytes = plane_buffer_bytes(kMaxDigitPlanes, ms->n_pad_cap);
    PURIFY_CUDA_TRY(cudaMalloc(&ms->Pd[0], bytes));
    PURIFY_CUDA_TRY(cudaMalloc(&ms->Pd[1], bytes));
    ms->pd_cap = ms->n_pad_cap;
    return PURIFY_OK;
}

// Algorithm 2 step coefficients: Y = cP X^2 + cE X + cI I.
static void tc_coeffs(int branch, double a, double* cP, double* cE, double* cI) {
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

// ---- launch-shape autotuning ----------------------------------------------
// Shapes measured in this process, per (device, digits, padded size): the
// first product of a kind times every candidate and all later products of
// that kind use the fastest.  The mutex also serialises the measurement, so
// every handle of the process gets the same shape for a kind.
namespace {
struct TunedShape {
    int kc, ways;
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, TunedShape> g_tuned;

// Device time of one launch of `st` (the smaller of two, after one warm-up).
int time_launch(const DigitStep& st, cudaStream_t stream, cudaEvent_t a, cudaEvent_t b, float* ms) {
    PURIFY_TRY(launch_digit_step(st, stream));
    *ms = INFINITY;
    for (int r = 0; r < 2; ++r) {
        PURIFY_CUDA_TRY(cudaEventRecord(a, stream));
        PURIFY_TRY(launch_digit_step(st, stream));
        PURIFY_CUDA_TRY(cudaEventRecord(b, stream));
        PURIFY_CUDA_TRY(cudaEventSynchronize(b));
        float t = 0.f;
        PURIFY_CUDA_TRY(cudaEventElapsedTime(&t, a, b));
        *ms = std::min(*ms, t);
    }
    return PURIFY_OK;
}

// Times the candidates on the step itself (its inputs are read, its output
// planes written; reductions, float64 output and block norms are left out,
// so the real launch that follows is unaffected).
int tune_shape(const DigitStep& st, cudaStream_t stream, TunedShape* best) {
    int kcs[3];
    const int nk = digit_kc_candidates(st.s_in, kcs);
    cudaEvent_t a = nullptr, b = nullptr;
    PURIFY_CUDA_TRY(cudaEventCreate(&a));
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return PURIFY_ERR_CUDA;
    }
    float best_ms = INFINITY;
    *best = {0, 0};
    int rc = PURIFY_OK;
    for (int i = 0; i < nk && rc == PURIFY_OK; ++i) {
        for (int ways : {0, 1}) {
            if (ways != 0 && !st.partial) continue;
            DigitStep c = st;
            c.kc = kcs[i];
            c.split_ways = ways;
            c.red = nullptr;
            c.out64 = nullptr;
            c.bnorm2 = nullptr;
            float ms = INFINITY;
            rc = time_launch(c, stream, a, b, &ms);
            if (rc != PURIFY_OK) break;
            if (ms < best_ms) {
                best_ms = ms;
                *best = {kcs[i], ways};
            }
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return rc;
}
}  // namespace

void tuned_shape_if_known(int device, DigitStep* st) {
    if (st->kc_cnt || st->bnorm2 || st->kc != 0) return;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    const auto f = g_tuned.find(std::make_tuple(device, st->s_in, st->n_pad));
    if (f == g_tuned.end()) return;
    st->kc = f->second.kc;
    st->split_ways = f->second.ways;
}

static int product(purify_ctx* h, const DigitStep& st0, double flops) {
    DigitStep st = st0;
    if (h->opt.split_k) {
        st.partial = h->mixed->partial;
        st.split_cnt = h->mixed->split_cnt;
    }
    st.wait_cycles = 1000ll * h->opt.wait_kcycles;
    if (h->opt.autotune && h->opt.wait_kcycles == 0 && !st.kc_cnt && !st.bnorm2 && st.kc == 0) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        const auto key = std::make_tuple(h->device, st.s_in, st.n_pad);
        auto f = g_tuned.find(key);
        if (f == g_tuned.end()) {
            TunedShape t;
            PURIFY_TRY(tune_shape(st, h->stream, &t));
            f = g_tuned.emplace(key, t).first;
        }
        st.kc = f->second.kc;
        st.split_ways = f->second.ways;
    }
    h->st.digit_kc = digit_step_kc(st);
    PURIFY_TRY(product_begin(h));
    PURIFY_TRY(launch_digit_step(st, h->stream));
    ++h->st.product_launches;
    h->st.tensor_flops += flops;
    return product_end(h);
}

int run_mixed_trace(purify_ctx* h, int scheme, double tol, int max_iter, Schedule& S, int* cur, int* iters) {
    if (scheme != PURIFY_TC_SF && scheme != PURIFY_TC_MONO) return PURIFY_ERR_UNSUPPORTED;
    if (h->nocc < 0) return PURIFY_ERR_INVALID_ARG;
    const int n = (int)h->n;
    const int n_pad = pad128(n);
    PURIFY_TRY(ensure_mixed(h, n_pad));
    MixedState* ms = h->mixed;
    const int T = n_pad / 128;
    const int rb = remainder_bits(n_pad);
    const double tile_flops = 2.0 * 128.0 * 128.0 * (double)n_pad * (double)(T * (T + 1) / 2);
    const bool have_gap = !std::isnan(h->b.homo) && !std::isnan(h->b.lumo);
    const bool scaled = scheme == PURIFY_TC_SF;
    const int fixed = h->opt.digits;
    const double lmin = h->b.lmin, lmax = h->b.lmax;
    const double c0 = lmax / (lmax - lmin), c1 = -1.0 / (lmax - lmin);
    double b = S.beta0, bb = S.betabar0;
    auto digits = [&](double beta, double betabar) {
        return have_gap ? digits_for_gap(betabar - beta, h->opt, rb) : (fixed > 0 ? fixed : kMaxDigitPlanes);
    };
    S.alpha.clear();
    S.branch.clear();
    S.beta.clear();
    S.betabar.clear();
    // slots 0 .. max_iter - 1: the steps; slot max_iter: trace(F)
    PURIFY_TRY(ensure_red(h, 4 * (int64_t)(max_iter + 1)));
    PURIFY_CUDA_TRY(cudaMemsetAsync(h->red, 0, sizeof(double) * 4 * (max_iter + 1), h->stream));
    PURIFY_CUDA_TRY(cudaMemsetAsync(ms->err, 0, sizeof(int), h->stream));
    PURIFY_CUDA_TRY(cudaEventRecord(h->e0, h->stream));
    double* trF = h->red + 4 * (int64_t)max_iter;
    PURIFY_TRY(launch_trace_f64(h->F, n, trF, h->stream));
    int s = digits(b, bb);
    PURIFY_TRY(launch_split(h->F, n, n, n_pad, c1, c0, 0, s, rb, ms->Xd[0], nullptr, h->stream));
    double tf = 0.0;
    PURIFY_CUDA_TRY(cudaMemcpyAsync(&tf, trF, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
    double tr_prev = c0 * (double)n + c1 * tf;  // trace(X_0)
    double* D = h->X[0];
    *cur = 0;
    int x = 0, it = 0, dmax = 0;
    bool done = have_gap && std::max(b, 1.0 - bb) <= tol;
    if (done) PURIFY_TRY(launch_affine_f64(h->F, n, D, n, c1, c0, h->stream));
    while (!done && it < max_iter) {
        const int br = tr_prev > (double)h->nocc ? 1 : 0;
        const double a = scaled ? tc_alpha(br, b, bb) : 0.0;
        double nb = b, nbb = bb;
        if (have_gap) {
            nb = tc_map(br, a, b);
            nbb = tc_map(br, a, bb);
        }
        // with gap bounds the last step is known before it runs; without,
        // every step also writes the float64 density
        const bool last_known = have_gap && std::max(nb, 1.0 - nbb) <= tol;
        DigitStep st;
        st.n = n;
        st.n_pad = n_pad;
        st.rbits = rb;
        st.A = st.B = ms->Xd[x];
        st.s_in = s;
        st.eA = st.eB = 0;
        st.use_E = 1;
        tc_coeffs(br, a, &st.cP, &st.cE, &st.cI);
        st.red = h->red + 4 * (int64_t)it;
        st.err = ms->err;
        st.scratch = ms->scratch;
        st.max_ctas = ms->ctas;
        const int s_next = digits(nb, nbb);
        if (!have_gap || last_known) st.out64 = D;
        if (!last_known) {
            st.out = ms->Xd[x ^ 1];
            st.s_out = s_next;
            st.e_out = 0;
        }
        PURIFY_TRY(product(h, st, 0.5 * s * (s + 1) * tile_flops));
        dmax = std::max(dmax, s);
        double r[4];
        PURIFY_CUDA_TRY(cudaMemcpyAsync(r, st.red, sizeof(r), cudaMemcpyDeviceToHost, h->stream));
        PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
        tr_prev = r[0];
        h->st.trace = r[0];
        h->st.idem_err_fro = std::sqrt(std::max(r[1], 0.0));
        h->hist_trace.push_back(r[0]);
        h->hist_idem.push_back(h->st.idem_err_fro);
        b = nb;
        bb = nbb;
        S.alpha.push_back(a);
        S.branch.push_back(br);
        S.beta.push_back(b);
        S.betabar.push_back(bb);
        ++it;
        x ^= 1;
        s = s_next;
        if (have_gap) done = last_known;
        else done = h->st.idem_err_fro <= tol;
    }
    S.converged = done;
    h->st.digit_max = dmax;
    PURIFY_CUDA_TRY(cudaEventRecord(h->e1, h->stream));
    int err = 0;
    PURIFY_CUDA_TRY(cudaMemcpyAsync(&err, ms->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->st.device_flag = err;
    if (err) return device_flag_status(err);
    if (it == 0) {
        h->st.trace = tr_prev;
        h->st.idem_err_fro = NAN;
    }
    *iters = it;
    return PURIFY_OK;
}

// Smallest e with 2^e >= 1.01 max |p(x)| over x in [lo, hi] (sampled; the
// polynomials' slopes keep the sampling error far below the 1 % margin).
template <typename Fn>
static int bound_exponent(Fn p, double lo, double hi) {
    double mx = 0.0;
    for (int k = 0; k <= 4096; ++k) mx = std::max(mx, std::fabs(p(lo + (hi - lo) * k / 4096.0)));
    int e = 0;
    while (std::ldexp(1.0, e) < 1.01 * mx) ++e;
    return e;
}

// One product of a polynomial's plan: operands and output name buffers
// (kX: X_s, kB0 / kB1: the two intermediates, kS: X_s^2, kOut: the
// iteration's result), Y = cP A B + cE A + cI I; `val` is the buffer's value
// as a function of x (an eigenvalue of X_s), which bounds its exponent.
enum { kX = 0, kB0 = 1, kB1 = 2, kS = 3, kOut = 4 };
struct PlanStep {
    int a, b, out;
    int use_E;
    double cP, cE, cI;
    double (*val)(double);
};

static double v_x2(double x) { return x * x; }
static double v_x4(double x) { return x * x * x * x; }
static double v_p33_v(double x) { return 70.0 * x - 20.0 * x * x; }
static double v_p33_q(double x) { return 35.0 - 84.0 * x + 70.0 * x * x - 20.0 * x * x * x; }
static double v_p13_v(double x) { return 15.0 * x - 4.0 * x * x; }
static double v_p13_q(double x) { return 10.0 - 20.0 * x + 15.0 * x * x - 4.0 * x * x * x; }

// P_{3,3} = x^4 (35 - 84x + 70x^2 - 20x^3)
static const PlanStep kPlan33[] = {{kX, kX, kB0, 1, -20.0, 70.0, 0.0, v_p33_v},
                                   {kX, kB0, kB1, 1, 1.0, -84.0, 35.0, v_p33_q},
                                   {kX, kX, kS, 0, 1.0, 0.0, 0.0, v_x2},
                                   {kS, kS, kB0, 0, 1.0, 0.0, 0.0, v_x4},
                                   {kB0, kB1, kOut, 0, 1.0, 0.0, 0.0, nullptr}};
// P_{3,1} = x^4 (5 - 4x)
static const PlanStep kPlan31[] = {{kX, kX, kS, 0, 1.0, 0.0, 0.0, v_x2},
                                   {kS, kS, kB0, 0, 1.0, 0.0, 0.0, v_x4},
                                   {kB0, kX, kOut, 1, -4.0, 5.0, 0.0, nullptr}};
// P_{1,3} = x^2 (10 - 20x + 15x^2 - 4x^3)
static const PlanStep kPlan13[] = {{kX, kX, kB0, 1, -4.0, 15.0, 0.0, v_p13_v},
                                   {kX, kB0, kB1, 1, 1.0, -20.0, 10.0, v_p13_q},
                                   {kX, kX, kS, 0, 1.0, 0.0, 0.0, v_x2},
                                   {kS, kB1, kOut, 0, 1.0, 0.0, 0.0, nullptr}};

int run_mixed_poly(purify_ctx* h, int scheme, double mu, const Schedule& S, int* cur, std::vector<double>& red) {
    if (h->opt.refine_squares) return PURIFY_ERR_UNSUPPORTED;
    int pi, pj;
    pij_orders(scheme, &pi, &pj);
    const PlanStep* plan = pi == 3 && pj == 3 ? kPlan33 : (pi == 3 ? kPlan31 : kPlan13);
    const int np = products_per_iteration(scheme);
    const double c = pi == pj ? 0.5 : pij_fixed_point(pi, pj);
    const int n = (int)h->n;
    const int n_pad = pad128(n);
    PURIFY_TRY(ensure_mixed(h, n_pad));
    MixedState* ms = h->mixed;
    PURIFY_TRY(ensure_pd(ms));
    const int m = (int)S.alpha.size();
    const int fixed = h->opt.digits;
    const int T = n_pad / 128;
    const int rb = remainder_bits(n_pad);
    const double tile_flops = 2.0 * 128.0 * 128.0 * (double)n_pad * (double)(T * (T + 1) / 2);
    // exponents: the eigenvalues of X_s lie in [c (1 - alpha), c + alpha (1 - c)]
    double amax = 1.0;
    for (double a : S.alpha) amax = std::max(amax, a);
    if (amax > 3.0) return PURIFY_ERR_UNSUPPORTED;
    const double lo = c * (1.0 - amax) - 1e-3, hi = c + amax * (1.0 - c) + 1e-3;
    // a buffer's exponent is that of its latest content (V and T share one),
    // so each step's operand and output exponents come from walking the plan
    const int eX = bound_exponent([](double x) { return x; }, lo, hi);
    int ecur[4] = {eX, 0, 0, 0};
    int e_a[8], e_b[8], e_o[8];
    for (int k = 0; k < np; ++k) {
        e_a[k] = ecur[plan[k].a];
        e_b[k] = ecur[plan[k].b];
        e_o[k] = plan[k].out == kOut ? eX : bound_exponent(plan[k].val, lo, hi);
        if (plan[k].out != kOut) ecur[plan[k].out] = e_o[k];
    }
    // digits per iteration: the mapped-gap rule plus one (intermediates sit
    // several bits above X_s)
    std::vector<int> sd(m + 1);
    for (int i = 0; i < m; ++i) {
        const double b = i ? S.beta[i - 1] : S.beta0;
        const double bb = i ? S.betabar[i - 1] : S.betabar0;
        sd[i] = std::min(kMaxDigitPlanes, digits_for_gap(bb - b, h->opt, rb) + (fixed > 0 ? 0 : 1));
    }
    sd[m] = sd[m ? m - 1 : 0];
    int dmax = 0;
    for (int i = 0; i < m; ++i) dmax = std::max(dmax, sd[i]);
    h->st.digit_max = dmax;
    const int slots = 2 * m + 2;
    PURIFY_TRY(ensure_red(h, 4 * (int64_t)slots));
    PURIFY_CUDA_TRY(cudaMemsetAsync(h->red, 0, sizeof(double) * 4 * slots, h->stream));
    PURIFY_CUDA_TRY(cudaMemsetAsync(ms->err, 0, sizeof(int), h->stream));
    PURIFY_CUDA_TRY(cudaEventRecord(h->e0, h->stream));
    const double gamma = std::max((mu - h->b.lmin) / (1.0 - c), (h->b.lmax - mu) / c);
    double* D = h->X[0];
    *cur = 0;
    if (m == 0) {  // X_0 = c I + (mu I - F) / gamma
        PURIFY_TRY(launch_affine_f64(h->F, n, D, n, -1.0 / gamma, c + mu / gamma, h->stream));
    } else {
        // X_s = c I + alpha_1 (X_0 - c I)
        const double a1 = S.alpha[0];
        PURIFY_TRY(launch_split(h->F, n, n, n_pad, -a1 / gamma, c + a1 * mu / gamma, eX, sd[0], rb, ms->Xd[0],
                                nullptr, h->stream));
        int x = 0;
        for (int i = 0; i < m; ++i) {
            const int s = sd[i];
            const double fl = pairs_of(s) * tile_flops;
            __nv_bfloat16* buf[4] = {ms->Xd[x], ms->Pd[0], ms->Pd[1], ms->Sd};
            for (int k = 0; k < np; ++k) {
                const PlanStep& ps = plan[k];
                DigitStep st;
                st.n = n;
                st.n_pad = n_pad;
                st.rbits = rb;
                st.s_in = s;
                st.err = ms->err;
                st.scratch = ms->scratch;
                st.max_ctas = ms->ctas;
                st.A = buf[ps.a];
                st.eA = e_a[k];
                st.B = buf[ps.b];
                st.eB = e_b[k];
                st.use_E = ps.use_E;
                st.cP = ps.cP;
                st.cE = ps.cE;
                st.cI = ps.cI;
                if (ps.out != kOut) {
                    st.out = buf[ps.out];
                    st.s_out = s;
                    st.e_out = e_o[k];
                } else if (i + 1 == m) {
                    st.red = h->red + 4 * (2 * i + 1);
                    st.out64 = D;
                } else {  // the next iteration's X_s = alpha (X - c I) + c I
                    st.red = h->red + 4 * (2 * i + 1);
                    const double an = S.alpha[i + 1];
                    st.dY = an;
                    st.dI = c * (1.0 - an);
                    st.out = ms->Xd[x ^ 1];
                    st.s_out = sd[i + 1];
                    st.e_out = eX;
                }
                PURIFY_TRY(product(h, st, fl));
            }
            x ^= 1;
        }
    }
    PURIFY_CUDA_TRY(cudaEventRecord(h->e1, h->stream));
    red.assign(4 * (size_t)slots, 0.0);
    int err = 0;
    PURIFY_CUDA_TRY(cudaMemcpyAsync(red.data(), h->red, sizeof(double) * red.size(), cudaMemcpyDeviceToHost,
                                    h->stream));
    PURIFY_CUDA_TRY(cudaMemcpyAsync(&err, ms->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->st.device_flag = err;
    if (err) return device_flag_status(err);
    h->st.trace = m > 0 ? red[4 * (size_t)(2 * (m - 1) + 1)] : NAN;
    h->st.idem_err_fro = NAN;
    return PURIFY_OK;
}

// A dense run (Algorithm 1 or 2 with the beta-based schedule, optional
// refinement squares) as queue launches of the product kernel after the f_0
// split: one per run of consecutive products with the same digit count
// (usually two: the first steps at 6 digits, the rest at 5).  The products
// are the same as the per-product path's; they differ in two ways:
//  - plane buffers rotate so that no product overwrites planes a running
//    product may still read: X over three buffers, Algorithm 1's S (and the
//    refinement's square) over two;
//  - every product's tiles run in chain_tile_order, and an item waits on the
//    device only for the two row panels of the products it reads (plus the
//    completion of the products that read the buffer it overwrites), so a
//    product's first items start while the previous product's last wave is
//    still running.
// The arithmetic of every tile is the per-product path's (whole tiles, no
// split of the last wave).
static int run_mixed_queue(purify_ctx* h, int scheme, double mu, const Schedule& S, int* cur,
                           std::vector<double>& red) {
    const int n = (int)h->n;
    const int n_pad = pad128(n);
    MixedState* ms = h->mixed;
    PURIFY_TRY(ensure_pd(ms));
    const bool fixed_mu = scheme == PURIFY_FIXED_MU_SF || scheme == PURIFY_FIXED_MU_MONO;
    const int m = (int)S.alpha.size();
    const int R = h->opt.refine_squares;
    const int fixed = h->opt.digits;
    const int T = n_pad / 128;
    const int rb = remainder_bits(n_pad);
    const double tile_flops = 2.0 * 128.0 * 128.0 * (double)n_pad * (double)(T * (T + 1) / 2);

    std::vector<int> sd(m + R + 1);
    for (int i = 0; i < m; ++i) {
        const double b = i ? S.beta[i - 1] : S.beta0;
        const double bb = i ? S.betabar[i - 1] : S.betabar0;
        sd[i] = digits_for_gap(bb - b, h->opt, rb);
    }
    for (int i = m; i <= m + R; ++i) sd[i] = fixed > 0 ? fixed : kMaxDigitPlanes;
    int dmax = 0;
    for (int i = 0; i < m + R; ++i) dmax = sd[i] > dmax ? sd[i] : dmax;
    h->st.digit_max = dmax;
    h->st.digit_kc = 32;

    const int slots = 2 * (m + R) + 2;
    PURIFY_TRY(ensure_red(h, 4 * (int64_t)slots));

    // buffers 0..2 hold X values, 3..4 S values; the writer and the readers
    // of each buffer's current content give the dependencies
    __nv_bfloat16* buf[5] = {ms->Xd[0], ms->Xd[1], ms->Pd[0], ms->Sd, ms->Pd[1]};
    int writer[5] = {-1, -1, -1, -1, -1};
    std::vector<int> readers[5];
    std::vector<QueueProduct> prods;
    double flops = 0.0;
    auto add = [&](DigitStep st, int a, int b, int out) -> int {
        QueueProduct q;
        st.n = n;
        st.n_pad = n_pad;
        st.rbits = rb;
        st.A = buf[a];
        st.B = buf[b];
        st.err = ms->err;
        st.scratch = ms->scratch;
        st.max_ctas = ms->ctas;
        if (out >= 0) st.out = buf[out];
        q.st = st;
        q.depA = writer[a];
        q.depB = writer[b];
        if (out >= 0) {
            if (readers[out].size() > 2) return PURIFY_ERR_INTERNAL;
            if (readers[out].size() > 0) q.war0 = readers[out][0];
            if (readers[out].size() > 1) q.war1 = readers[out][1];
        }
        const int g = (int)prods.size();
        readers[a].push_back(g);
        if (b != a) readers[b].push_back(g);
        if (out >= 0) {
            writer[out] = g;
            readers[out].clear();
        }
        prods.push_back(q);
        flops += pairs_of(st.s_in) * tile_flops;
        return PURIFY_OK;
    };

    const double lmin = h->b.lmin, lmax = h->b.lmax;
    double c0, c1;  // X_0 = c0 I + c1 F
    if (fixed_mu) {
        const double gamma = 2.0 * std::max(lmax - mu, mu - lmin);
        c0 = mu / gamma + 0.5;
        c1 = -1.0 / gamma;
    } else {
        c0 = lmax / (lmax - lmin);
        c1 = -1.0 / (lmax - lmin);
    }
    double* D = h->X[0];
    *cur = 0;
    int x = 0;  // X buffer of the current iterate
    if (fixed_mu) {
        for (int i = 0; i < m + R; ++i) {
            const int s = sd[i];
            const int sb = 3 + (i & 1), xn = (x + 1) % 3;
            DigitStep p1;
            p1.s_in = s;
            p1.eA = p1.eB = 1;
            p1.s_out = s;
            p1.e_out = 1;
            PURIFY_TRY(add(p1, x, x, sb));
            // X_i = 3 S - 2 S X_s, emitted as the next X_s (or as D)
            DigitStep p2;
            p2.s_in = s;
            p2.eA = p2.eB = 1;
            p2.e_out = 1;
            p2.use_E = 1;
            p2.cP = -2.0;
            p2.cE = 3.0;
            p2.red = h->red + 4 * (2 * i + 1);
            if (i + 1 == m + R) {
                p2.out64 = D;
                PURIFY_TRY(add(p2, sb, x, -1));
            } else {
                const double an = (i + 1 < m) ? S.alpha[i + 1] : 1.0;
                p2.dY = an;
                p2.dI = 0.5 * (1.0 - an);
                p2.s_out = sd[i + 1];
                PURIFY_TRY(add(p2, sb, x, xn));
            }
            x = xn;
        }
    } else {
        for (int i = 0; i < m; ++i) {
            const int s = sd[i];
            const int xn = (x + 1) % 3;
            DigitStep st;
            st.s_in = s;
            st.eA = st.eB = 0;
            st.use_E = 1;
            tc_coeffs(S.branch[i], S.alpha[i], &st.cP, &st.cE, &st.cI);
            st.red = h->red + 4 * (2 * i + 1);
            if ((i + 1 == m) && R == 0) {
                st.out64 = D;
                PURIFY_TRY(add(st, x, x, -1));
            } else {
                st.s_out = sd[i + 1];
                st.e_out = 0;
                PURIFY_TRY(add(st, x, x, xn));
            }
            x = xn;
        }
        // refinement: unscaled McWeeny X <- 3 X^2 - 2 X^3 at the finest digits
        for (int r = 0; r < R; ++r) {
            const int i = m + r;
            const int s = sd[i];
            const int sb = 3 + (r & 1), xn = (x + 1) % 3;
            DigitStep p1;
            p1.s_in = s;
            p1.eA = p1.eB = 0;
            p1.s_out = s;
            p1.e_out = 0;
            p1.use_E = 1;  // ||X - X^2|| of the iterate
            p1.cP = 1.0;
            p1.cE = 0.0;
            p1.red = (r + 1 == R) ? h->red + 4 * (2 * i) : nullptr;
            PURIFY_TRY(add(p1, x, x, sb));
            DigitStep p2;
            p2.s_in = s;
            p2.eA = p2.eB = 0;
            p2.e_out = 0;
            p2.use_E = 1;
            p2.cP = -2.0;
            p2.cE = 3.0;
            p2.red = (r + 1 == R) ? h->red + 4 * (2 * i + 1) : nullptr;
            if (r + 1 == R) {
                p2.out64 = D;
                PURIFY_TRY(add(p2, sb, x, -1));
            } else {
                p2.s_out = sd[i + 1];
                PURIFY_TRY(add(p2, sb, x, xn));
            }
            x = xn;
        }
    }
    // one queue launch per run of products with the same digit count (the
    // kernel then holds the count as a compile-time constant); a dependency
    // on a product of an earlier launch is met by stream order
    std::vector<int2> order;
    chain_tile_order(T, ms->ctas, order);
    struct Segment {
        QueueStaging q;
        size_t off;
    };
    std::vector<Segment> segs;
    std::vector<uint8_t> seg_host;
    size_t total = 0;
    ms->qhost.clear();
    for (int a = 0; a < (int)prods.size();) {
        int b = a + 1;
        while (b < (int)prods.size() && prods[b].st.s_in == prods[a].st.s_in) ++b;
        std::vector<QueueProduct> part(prods.begin() + a, prods.begin() + b);
        for (QueueProduct& p : part)
            for (int* d : {&p.depA, &p.depB, &p.war0, &p.war1}) *d = *d >= a ? *d - a : -1;
        std::vector<int4> work;
        work.reserve(order.size() * part.size());
        for (int g = 0; g < (int)part.size(); ++g)
            for (const int2& t : order) work.push_back(make_int4(g, t.x, t.y, 0));
        Segment sg;
        PURIFY_TRY(stage_queue_products(part, work, seg_host, sg.q));
        sg.off = total;
        total += (sg.q.end + 255) / 256 * 256;
        ms->qhost.resize(total);
        std::memcpy(ms->qhost.data() + sg.off, seg_host.data(), sg.q.end);
        segs.push_back(sg);
        a = b;
    }
    if (total > ms->qdev_cap) {
        PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
        cudaFree(ms->qdev);
        ms->qdev = nullptr;
        ms->qdev_cap = 0;
        const size_t cap = std::max(total, (size_t)1 << 20) * 2;
        PURIFY_CUDA_TRY(cudaMalloc(&ms->qdev, cap));
        ms->qdev_cap = cap;
    }

    PURIFY_CUDA_TRY(cudaMemsetAsync(h->red, 0, sizeof(double) * 4 * slots, h->stream));
    PURIFY_CUDA_TRY(cudaMemsetAsync(ms->err, 0, sizeof(int), h->stream));
    PURIFY_CUDA_TRY(cudaEventRecord(h->e0, h->stream));
    if (fixed_mu) {
        // X_s of the first iteration, e = 1 (eigenvalues in [(1-a)/2, (1+a)/2])
        const double a1 = m ? S.alpha[0] : 1.0;
        PURIFY_TRY(launch_split(h->F, n, n, n_pad, a1 * c1, a1 * (c0 - 0.5) + 0.5, 1, sd[0], rb, buf[0], nullptr,
                                h->stream));
    } else {
        PURIFY_TRY(launch_split(h->F, n, n, n_pad, c1, c0, 0, sd[0], rb, buf[0], nullptr, h->stream));
    }
    PURIFY_CUDA_TRY(cudaMemcpyAsync(ms->qdev, ms->qhost.data(), total, cudaMemcpyHostToDevice, h->stream));
    // with time_products, one interval covers the queue launches (the
    // products overlap, so they have no times of their own)
    PURIFY_TRY(product_begin(h));
    for (const Segment& sg : segs)
        PURIFY_TRY(launch_staged_queue(sg.q, (uint8_t*)ms->qdev + sg.off, ms->scratch, ms->ctas, ms->err, h->stream,
                                       1000ll * h->opt.wait_kcycles));
    PURIFY_TRY(product_end(h));
    h->st.product_launches += (int)prods.size();
    h->st.tensor_flops += flops;
    PURIFY_CUDA_TRY(cudaEventRecord(h->e1, h->stream));
    red.assign(4 * (size_t)slots, 0.0);
    int err = 0;
    PURIFY_CUDA_TRY(cudaMemcpyAsync(red.data(), h->red, sizeof(double) * red.size(),
                                    cudaMemcpyDeviceToHost, h->stream));
    PURIFY_CUDA_TRY(cudaMemcpyAsync(&err, ms->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->st.device_flag = err;
    if (err) return device_flag_status(err);
    h->st.refine_multiplications = 2 * R;
    const int last = m + R - 1;
    if (last >= 0) {
        h->st.trace = red[4 * (size_t)(2 * last + 1)];
        if (!fixed_mu && R == 0) {
            h->st.idem_err_fro = std::sqrt(std::max(red[4 * (size_t)(2 * last + 1) + 1], 0.0));
        } else if (R > 0) {
            h->st.idem_err_fro = std::sqrt(std::max(red[4 * (size_t)(2 * last) + 1], 0.0));
        } else {
            h->st.idem_err_fro = NAN;
        }
    } else {
        h->st.trace = NAN;
        h->st.idem_err_fro = NAN;
    }
    return PURIFY_OK;
}

int run_mixed(purify_ctx* h, int scheme, double mu, const Schedule& S, int* cur,
              std::vector<double>& red) {
    const int n = (int)h->n;
    const int n_pad = pad128(n);
    PURIFY_TRY(ensure_mixed(h, n_pad));
    MixedState* ms = h->mixed;
    {
        // queue launches for the whole run when a product has at least two
        // waves of tiles (below that the split of the last wave pays more)
        const int Tq = n_pad / 128;
        if (!h->opt.launch_per_product && S.alpha.size() + h->opt.refine_squares > 0 &&
            Tq * (Tq + 1) / 2 >= 2 * ms->ctas)
            return run_mixed_queue(h, scheme, mu, S, cur, red);
    }
    const bool fixed_mu = scheme == PURIFY_FIXED_MU_SF || scheme == PURIFY_FIXED_MU_MONO;
    const int m = (int)S.alpha.size();
    const int R = h->opt.refine_squares;
    const int fixed = h->opt.digits;
    const int T = n_pad / 128;
    const int rb = remainder_bits(n_pad);
    const double tile_flops = 2.0 * 128.0 * 128.0 * (double)n_pad * (double)(T * (T + 1) / 2);

    // digit count of every product step (index m.. are refinement steps)
    std::vector<int> sd(m + R + 1);
    for (int i = 0; i < m; ++i) {
        const double b = i ? S.beta[i - 1] : S.beta0;
        const double bb = i ? S.betabar[i - 1] : S.betabar0;
        sd[i] = digits_for_gap(bb - b, h->opt, rb);
    }
    for (int i = m; i <= m + R; ++i) sd[i] = fixed > 0 ? fixed : kMaxDigitPlanes;
    int dmax = 0;
    for (int i = 0; i < m + R; ++i) dmax = sd[i] > dmax ? sd[i] : dmax;
    h->st.digit_max = dmax;

    const int slots = 2 * (m + R) + 2;
    PURIFY_TRY(ensure_red(h, 4 * (int64_t)slots));
    PURIFY_CUDA_TRY(cudaMemsetAsync(h->red, 0, sizeof(double) * 4 * slots, h->stream));
    PURIFY_CUDA_TRY(cudaMemsetAsync(ms->err, 0, sizeof(int), h->stream));
    PURIFY_CUDA_TRY(cudaEventRecord(h->e0, h->stream));

    const double lmin = h->b.lmin, lmax = h->b.lmax;
    double c0, c1;  // X_0 = c0 I + c1 F
    if (fixed_mu) {
        const double gamma = 2.0 * std::max(lmax - mu, mu - lmin);
        c0 = mu / gamma + 0.5;
        c1 = -1.0 / gamma;
    } else {
        c0 = lmax / (lmax - lmin);
        c1 = -1.0 / (lmax - lmin);
    }
    double* D = h->X[0];
    *cur = 0;
    if (m + R == 0) {
        PURIFY_TRY(launch_affine_f64(h->F, n, D, n, c1, c0, h->stream));
    } else if (fixed_mu) {
        // X_s of the first iteration, e = 1 (eigenvalues in [(1-a)/2, (1+a)/2])
        const double a1 = m ? S.alpha[0] : 1.0;
        PURIFY_TRY(launch_split(h->F, n, n, n_pad, a1 * c1, a1 * (c0 - 0.5) + 0.5, 1, sd[0], rb,
                                ms->Xd[0], nullptr, h->stream));
        int x = 0;
        for (int i = 0; i < m + R; ++i) {
            const int s = sd[i];
            DigitStep p1;
            p1.n = n;
            p1.n_pad = n_pad;
            p1.rbits = rb;
            p1.A = p1.B = ms->Xd[x];
            p1.s_in = s;
            p1.eA = p1.eB = 1;
            p1.out = ms->Sd;
            p1.s_out = s;
            p1.e_out = 1;
            p1.red = nullptr;
            p1.err = ms->err;
            p1.scratch = ms->scratch;
            p1.max_ctas = ms->ctas;
            PURIFY_TRY(product(h, p1, pairs_of(s) * tile_flops));
            // X_i = 3 S - 2 S X_s, emitted as the next X_s (or as D)
            DigitStep p2 = p1;
            p2.A = ms->Sd;
            p2.B = ms->Xd[x];
            p2.use_E = 1;
            p2.cP = -2.0;
            p2.cE = 3.0;
            // every iteration reduces trace(X_i) (slot 2 i + 1)
            const bool last = (i + 1 == m + R);
            p2.red = h->red + 4 * (2 * i + 1);
            if (last) {
                p2.out = nullptr;
                p2.s_out = 0;
                p2.out64 = D;
            } else {
                const double an = (i + 1 < m) ? S.alpha[i + 1] : 1.0;
                p2.dY = an;
                p2.dI = 0.5 * (1.0 - an);
                p2.out = ms->Xd[x ^ 1];
                p2.s_out = sd[i + 1];
            }
            PURIFY_TRY(product(h, p2, pairs_of(s) * tile_flops));
            x ^= 1;
        }
    } else {
        PURIFY_TRY(launch_split(h->F, n, n, n_pad, c1, c0, 0, sd[0], rb, ms->Xd[0], nullptr, h->stream));
        int x = 0;
        for (int i = 0; i < m; ++i) {
            const int s = sd[i];
            DigitStep st;
            st.n = n;
            st.n_pad = n_pad;
            st.rbits = rb;
            st.A = st.B = ms->Xd[x];
            st.s_in = s;
            st.eA = st.eB = 0;
            st.use_E = 1;
            tc_coeffs(S.branch[i], S.alpha[i], &st.cP, &st.cE, &st.cI);
            // every step reduces trace(X_i) and ||X_{i-1} - X_{i-1}^2||_F (slot 2 i + 1)
            st.red = h->red + 4 * (2 * i + 1);
            st.err = ms->err;
            st.scratch = ms->scratch;
            st.max_ctas = ms->ctas;
            const bool last = (i + 1 == m) && R == 0;
            if (last) {
                st.out64 = D;
            } else {
                st.out = ms->Xd[x ^ 1];
                st.s_out = sd[i + 1];
                st.e_out = 0;
            }
            PURIFY_TRY(product(h, st, pairs_of(s) * tile_flops));
            x ^= 1;
        }
        // refinement: unscaled McWeeny X <- 3 X^2 - 2 X^3 at the finest digits
        for (int r = 0; r < R; ++r) {
            const int i = m + r;
            const int s = sd[i];
            DigitStep p1;
            p1.n = n;
            p1.n_pad = n_pad;
            p1.rbits = rb;
            p1.A = p1.B = ms->Xd[x];
            p1.s_in = s;
            p1.eA = p1.eB = 0;
            p1.out = ms->Sd;
            p1.s_out = s;
            p1.e_out = 0;
            p1.use_E = 1;  // ||X - X^2|| of the iterate
            p1.cP = 1.0;
            p1.cE = 0.0;
            p1.red = (r + 1 == R) ? h->red + 4 * (2 * i) : nullptr;
            p1.err = ms->err;
            p1.scratch = ms->scratch;
            p1.max_ctas = ms->ctas;
            PURIFY_TRY(product(h, p1, pairs_of(s) * tile_flops));
            DigitStep p2 = p1;
            p2.A = ms->Sd;
            p2.B = ms->Xd[x];
            p2.cP = -2.0;
            p2.cE = 3.0;
            p2.red = (r + 1 == R) ? h->red + 4 * (2 * i + 1) : nullptr;
            if (r + 1 == R) {
                p2.out = nullptr;
                p2.s_out = 0;
                p2.out64 = D;
            } else {
                p2.out = ms->Xd[x ^ 1];
                p2.s_out = sd[i + 1];
            }
            PURIFY_TRY(product(h, p2, pairs_of(s) * tile_flops));
            x ^= 1;
        }
    }
    PURIFY_CUDA_TRY(cudaEventRecord(h->e1, h->stream));
    red.assign(4 * (size_t)slots, 0.0);
    int err = 0;
    PURIFY_CUDA_TRY(cudaMemcpyAsync(red.data(), h->red, sizeof(double) * red.size(),
                                    cudaMemcpyDeviceToHost, h->stream));
    PURIFY_CUDA_TRY(cudaMemcpyAsync(&err, ms->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->st.device_flag = err;
    if (err) return device_flag_status(err);
    h->st.refine_multiplications = 2 * R;
    // statistics: trace of the result; idempotency of the last squared iterate
    const int last = m + R - 1;
    if (last >= 0) {
        h->st.trace = red[4 * (size_t)(2 * last + 1)];
        if (!fixed_mu && R == 0) {
            h->st.idem_err_fro = std::sqrt(std::max(red[4 * (size_t)(2 * last + 1) + 1], 0.0));
        } else if (R > 0) {
            h->st.idem_err_fro = std::sqrt(std::max(red[4 * (size_t)(2 * last) + 1], 0.0));
        } else {
            h->st.idem_err_fro = NAN;
        }
    } else {
        h->st.trace = NAN;
        h->st.idem_err_fro = NAN;
    }
    return PURIFY_OK;
}

}  // namespace purify

using namespace purify;

extern "C" int purify_k_digit_product_f64(const double* A, const double* B, double* C, int64_t n,
                                          int digits, int eA, int eB, void* stream) {
    if (!A || !B || !C || n <= 0 || n > (int64_t)1 << 15) return PURIFY_ERR_INVALID_ARG;
    if (digits < 1 || digits > kMaxDigitPlanes || eA < -8 || eA > 8 || eB < -8 || eB > 8)
        return PURIFY_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int n_pad = pad128(n);
    const size_t plane_bytes = plane_buffer_bytes(digits, n_pad);
    __nv_bfloat16 *pa = nullptr, *pb = nullptr;
    int* err = nullptr;
    float2* scratch = nullptr;
    float* partial = nullptr;
    int* split_cnt = nullptr;
    int r = PURIFY_OK;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PURIFY_ERR_CUDA;
    if (cudaMalloc(&pa, plane_bytes) != cudaSuccess || cudaMalloc(&pb, plane_bytes) != cudaSuccess ||
        cudaMalloc(&err, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&scratch, digit_scratch_bytes(sms)) != cudaSuccess ||
        cudaMalloc(&partial, sizeof(float) * digit_partial_floats(sms)) != cudaSuccess ||
        cudaMalloc(&split_cnt, sizeof(int) * digit_split_counters(sms)) != cudaSuccess)
        r = PURIFY_ERR_OOM;
    if (r == PURIFY_OK && cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) r = PURIFY_ERR_CUDA;
    const int rb = remainder_bits(n_pad);
    if (r == PURIFY_OK) r = launch_split(A, n, (int)n, n_pad, 1.0, 0.0, eA, digits, rb, pa, nullptr, s);
    if (r == PURIFY_OK) r = launch_split(B, n, (int)n, n_pad, 1.0, 0.0, eB, digits, rb, pb, nullptr, s);
    if (r == PURIFY_OK) {
        DigitStep st;
        st.n = (int)n;
        st.n_pad = n_pad;
        st.A = pa;
        st.B = pb;
        st.s_in = digits;
        st.eA = eA;
        st.eB = eB;
        st.out64 = C;
        st.err = err;
        st.scratch = scratch;
        st.max_ctas = sms;
        st.partial = partial;
        st.split_cnt = split_cnt;
        r = launch_digit_step(st, s);
    }
    int herr = 0;
    if (r == PURIFY_OK) {
        cudaError_t e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) r = cuda_status(e, "digit product");
    } else {
        cudaStreamSynchronize(s);
    }
    cudaFree(pa);
    cudaFree(pb);
    cudaFree(err);
    cudaFree(scratch);
    cudaFree(partial);
    cudaFree(split_cnt);
    if (r == PURIFY_OK && herr) r = device_flag_status(herr);
    return r;
}

int purify_tuned_shape(int device, int digits, int64_t n, int* kc, int* split_ways) {
    using namespace purify;
    if (!kc || !split_ways || n <= 0 || digits < 1 || digits > kMaxDigitPlanes) return PURIFY_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    const auto f = g_tuned.find(std::make_tuple(device, digits, pad128(n)));
    if (f == g_tuned.end()) return PURIFY_ERR_STATE;
    *kc = f->second.kc;
    *split_ways = f->second.ways;
    return PURIFY_OK;
}

extern "C" int purify_k_split_plan(int tiles, int ctas, int k_chunks, int* split_begin, int* ways) {
    if (tiles <= 0 || ctas <= 0 || k_chunks <= 0 || !split_begin || !ways) return PURIFY_ERR_INVALID_ARG;
    purify::digit_split_plan(tiles, ctas, k_chunks, split_begin, ways);
    return PURIFY_OK;
}
