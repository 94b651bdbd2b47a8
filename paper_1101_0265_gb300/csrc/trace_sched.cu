// Niklasson's trace rule for the trace-correcting schemes (Algorithm 2 with
// the branch taken from trace(X_{i-1}) against nocc) with its scalar
// schedule on the device, so that a whole run replays from a CUDA graph.
//
// Per step a one-thread schedule kernel reads the float64 reductions that the
// previous product's fused epilogue left (trace(X_{i-1}) and ||X_{i-2} -
// X_{i-2}^2||_F), applies the stop test, chooses the branch, alpha (Algorithm
// 2's scaling, or 0 for the alpha = 0 scheme), the coefficients of Eq. 4 /
// Eq. 5 and the next digit count, and writes them into a DevStep record.
// The step's product is launched once per digit count the run can reach;
// the launch whose count the schedule chose runs, the others exit at once.
// After the run has stopped every later kernel of the graph exits at once.
// The host launches the captured steps in blocks and reads the schedule's
// state once per block instead of once per step.
#include <cmath>
#include <cstring>
#include <mutex>

#include "digits_tc.h"
#include "mixed.h"

namespace purify {

namespace {

// Digit rule on the device (the host rule of digits_for_gap): the fewest
// digits whose bits cover max(floor, gap_bits + log2(1 / g)).
__device__ int dev_digits(const TraceSchedDev& c, double g) {
    if (c.fixed_digits > 0) return c.fixed_digits;
    if (!(g > 0.0)) return kMaxDigitPlanes;
    const double need = fmax(c.floor_bits, __dadd_rn(c.gap_bits, log2(__ddiv_rn(1.0, g))));
    for (int s = 3; s < kMaxDigitPlanes; ++s)
        if (8 + c.rbits * (s - 1) >= need) return s;
    return kMaxDigitPlanes;
}

// The stop test of the step whose product wrote `slot`: records its trace
// and idempotency and returns true when the run is over.
__device__ bool consume(TraceSchedDev* c, const double* slot) {
    const int i = c->it - 1;
    const double tr = slot[0];
    const double idem = sqrt(fmax(slot[1], 0.0));
    c->hist[kHistTrace * c->max_iter + i] = tr;
    c->hist[kHistIdem * c->max_iter + i] = idem;
    c->tr = tr;
    const bool stop = c->have_gap ? c->prev_last != 0 : idem <= c->tol;
    if (stop) c->converged = 1;
    return stop || c->it >= c->max_iter;
}

// Schedule of graph position j (of K): consume the previous product's
// reductions, then (unless the run is over or consume_only) set the next
// product's control and clear its reduction slot.
__global__ void trace_sched_kernel(TraceSchedDev* c, double* red, const double* trF, int j, int K, int consume_only) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (c->done) {
        c->step.done = 1;
        return;
    }
    if (c->it > 0 && c->consumed < c->it) {
        c->consumed = c->it;
        if (consume(c, red + 4 * ((j + K - 1) % K))) {
            c->done = 1;
            c->step.done = 1;
            return;
        }
    }
    if (consume_only) return;
    if (c->it == 0) c->tr = __dadd_rn(c->c0n, __dmul_rn(c->c1, trF[0]));  // trace(X_0) = c0 n + c1 trace(F)
    // the host schedule's float64 arithmetic operation by operation (no
    // contraction into fused multiply-adds), so both take the same values;
    // only (1 + alpha)^2 is a product here and the C library's pow there
    const int br = c->tr > c->nocc ? 1 : 0;
    const double b = c->b, bb = c->bb;
    const double a = c->scaled ? (br ? __ddiv_rn(b, __dsub_rn(2.0, b)) : __ddiv_rn(__dsub_rn(1.0, bb), __dadd_rn(1.0, bb)))
                               : 0.0;
    const double a1 = __dadd_rn(1.0, a);
    const double q = __dmul_rn(a1, a1);
    double nb = b, nbb = bb;
    if (c->have_gap) {
        if (br) {  // ((1 + a) x - a)^2
            const double y = __dsub_rn(__dmul_rn(a1, b), a), yy = __dsub_rn(__dmul_rn(a1, bb), a);
            nb = __dmul_rn(y, y);
            nbb = __dmul_rn(yy, yy);
        } else {   // 2 (1 + a) x - (1 + a)^2 x x
            nb = __dsub_rn(__dmul_rn(__dmul_rn(2.0, a1), b), __dmul_rn(__dmul_rn(q, b), b));
            nbb = __dsub_rn(__dmul_rn(__dmul_rn(2.0, a1), bb), __dmul_rn(__dmul_rn(q, bb), bb));
        }
    }
    const bool last = c->have_gap && fmax(nb, __dsub_rn(1.0, nbb)) <= c->tol;
    const int s_next = c->have_gap ? dev_digits(*c, __dsub_rn(nbb, nb)) : c->s_cur;
    DevStep& st = c->step;
    if (br) {
        st.cP = q;
        st.cE = __dmul_rn(__dmul_rn(-2.0, a), a1);
        st.cI = __dmul_rn(a, a);
    } else {
        st.cP = -q;
        st.cE = __dmul_rn(2.0, a1);
        st.cI = 0.0;
    }
    st.s_in = c->s_cur;
    st.s_out = last ? 0 : s_next;
    st.write64 = (!c->have_gap || last) ? 1 : 0;
    st.done = 0;
    const int i = c->it;
    c->hist[kHistAlpha * c->max_iter + i] = a;
    c->hist[kHistBranch * c->max_iter + i] = br;
    c->hist[kHistBeta * c->max_iter + i] = nb;
    c->hist[kHistBetabar * c->max_iter + i] = nbb;
    c->hist[kHistDigits * c->max_iter + i] = c->s_cur;
    c->b = nb;
    c->bb = nbb;
    c->s_cur = s_next;
    c->prev_last = last ? 1 : 0;
    c->it = i + 1;
    double* slot = red + 4 * j;
    slot[0] = slot[1] = slot[2] = slot[3] = 0.0;
}

constexpr int kBlock = 16;  // steps per captured graph (even: the digit buffers alternate)

}  // namespace

size_t trace_sched_bytes(int max_iter) { return sizeof(TraceSchedDev) + sizeof(double) * kHistCount * max_iter; }

int run_mixed_trace_graph(purify_ctx* h, int scheme, double tol, int max_iter, Schedule& S, int* cur, int* iters) {
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
    const double lmin = h->b.lmin, lmax = h->b.lmax;
    const double c0 = lmax / (lmax - lmin), c1 = -1.0 / (lmax - lmin);
    // digit counts the run can reach: from the floor's count to the most
    const purify_options& o = h->opt;
    int smin = kMaxDigitPlanes, smax = kMaxDigitPlanes;
    if (o.digits > 0) {
        smin = smax = o.digits;
    } else if (have_gap) {
        smin = digits_for_gap(1.0, o, rb);
    }
    int s0 = have_gap ? digits_for_gap(S.betabar0 - S.beta0, o, rb) : smax;
    if (s0 < smin) s0 = smin;
    // device state and history
    const size_t bytes = trace_sched_bytes(max_iter);
    if (ms->tsched_cap < bytes) {
        cudaFree(ms->tsched);
        ms->tsched = nullptr;
        ms->tsched_cap = 0;
        PURIFY_CUDA_TRY(cudaMalloc(&ms->tsched, bytes));
        ms->tsched_cap = bytes;
    }
    TraceSchedDev init;
    std::memset(&init, 0, sizeof(init));
    init.nocc = (double)h->nocc;
    init.tol = tol;
    init.have_gap = have_gap ? 1 : 0;
    init.scaled = scheme == PURIFY_TC_SF ? 1 : 0;
    init.max_iter = max_iter;
    init.fixed_digits = o.digits;
    init.floor_bits = o.bits_floor > 0 ? o.bits_floor : kBitsFloor;
    init.gap_bits = o.bits_gap > 0 ? o.bits_gap : kBitsGap;
    init.rbits = rb;
    init.c0n = c0 * (double)n;
    init.c1 = c1;
    init.b = S.beta0;
    init.bb = S.betabar0;
    init.s_cur = s0;
    init.step.done = 1;
    TraceSchedDev* dev = (TraceSchedDev*)ms->tsched;
    init.hist = (double*)((char*)ms->tsched + sizeof(TraceSchedDev));
    PURIFY_TRY(ensure_red(h, 4 * (int64_t)(kBlock + 1)));
    double* red = h->red;
    double* trF = h->red + 4 * kBlock;
    // captured steps: one block of kBlock steps and a final consume
    const bool key_ok = ms->tgraph && ms->tg_n == n && ms->tg_smin == smin && ms->tg_smax == smax &&
                        ms->tg_state == ms->tsched && ms->tg_red == red && ms->tg_D == h->X[0] &&
                        ms->tg_X0 == ms->Xd[0] && ms->tg_wait == o.wait_kcycles && ms->tg_split == o.split_k;
    if (!key_ok) {
        if (ms->tgraph) cudaGraphExecDestroy(ms->tgraph);
        ms->tgraph = nullptr;
        PURIFY_TRY(prepare_digit_kernels());
        cudaGraph_t g = nullptr;
        PURIFY_CUDA_TRY(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        int rc = PURIFY_OK;
        for (int j = 0; j < kBlock && rc == PURIFY_OK; ++j) {
            trace_sched_kernel<<<1, 32, 0, h->stream>>>(dev, red, trF, j, kBlock, 0);
            for (int s = smin; s <= smax && rc == PURIFY_OK; ++s) {
                DigitStep st;
                st.n = n;
                st.n_pad = n_pad;
                st.rbits = rb;
                st.A = st.B = ms->Xd[j & 1];
                st.s_in = s;
                st.eA = st.eB = 0;
                st.use_E = 1;
                st.red = red + 4 * j;
                st.err = ms->err;
                st.scratch = ms->scratch;
                st.max_ctas = ms->ctas;
                st.out = ms->Xd[(j + 1) & 1];
                st.s_out = kMaxDigitPlanes;
                st.e_out = 0;
                st.out64 = h->X[0];
                st.ctl = &dev->step;
                st.wait_cycles = 1000ll * o.wait_kcycles;
                if (o.split_k) {
                    st.partial = ms->partial;
                    st.split_cnt = ms->split_cnt;
                }
                tuned_shape_if_known(h->device, &st);
                rc = launch_digit_step(st, h->stream);
            }
        }
        if (rc == PURIFY_OK) trace_sched_kernel<<<1, 32, 0, h->stream>>>(dev, red, trF, kBlock, kBlock, 1);
        const cudaError_t ce = cudaStreamEndCapture(h->stream, &g);
        if (rc != PURIFY_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        PURIFY_CUDA_TRY(ce);
        const cudaError_t ie = cudaGraphInstantiate(&ms->tgraph, g, 0);
        cudaGraphDestroy(g);
        PURIFY_CUDA_TRY(ie);
        ms->tg_n = n;
        ms->tg_smin = smin;
        ms->tg_smax = smax;
        ms->tg_state = ms->tsched;
        ms->tg_red = red;
        ms->tg_D = h->X[0];
        ms->tg_X0 = ms->Xd[0];
        ms->tg_wait = o.wait_kcycles;
        ms->tg_split = o.split_k;
    }
    PURIFY_CUDA_TRY(cudaMemsetAsync(ms->err, 0, sizeof(int), h->stream));
    PURIFY_CUDA_TRY(cudaEventRecord(h->e0, h->stream));
    PURIFY_CUDA_TRY(cudaMemcpyAsync(dev, &init, sizeof(init), cudaMemcpyHostToDevice, h->stream));
    PURIFY_CUDA_TRY(cudaMemsetAsync(trF, 0, sizeof(double), h->stream));
    PURIFY_TRY(launch_trace_f64(h->F, n, trF, h->stream));
    PURIFY_TRY(launch_split(h->F, n, n, n_pad, c1, c0, 0, s0, rb, ms->Xd[0], nullptr, h->stream));
    *cur = 0;
    TraceSchedDev now;
    int blocks = 0;
    for (;;) {
        PURIFY_CUDA_TRY(cudaGraphLaunch(ms->tgraph, h->stream));
        ++blocks;
        PURIFY_CUDA_TRY(cudaMemcpyAsync(&now, dev, sizeof(now), cudaMemcpyDeviceToHost, h->stream));
        PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
        if (now.done || now.it >= max_iter) break;
    }
    PURIFY_CUDA_TRY(cudaEventRecord(h->e1, h->stream));
    const int m = now.it;
    std::vector<double> hist((size_t)kHistCount * max_iter);
    int err = 0;
    PURIFY_CUDA_TRY(cudaMemcpyAsync(hist.data(), init.hist, sizeof(double) * hist.size(), cudaMemcpyDeviceToHost,
                                    h->stream));
    PURIFY_CUDA_TRY(cudaMemcpyAsync(&err, ms->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    PURIFY_CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->st.device_flag = err;
    if (err) return device_flag_status(err);
    S.alpha.clear();
    S.branch.clear();
    S.beta.clear();
    S.betabar.clear();
    int dmax = 0;
    double tflops = 0.0;
    for (int i = 0; i < m; ++i) {
        S.alpha.push_back(hist[(size_t)kHistAlpha * max_iter + i]);
        S.branch.push_back((int)hist[(size_t)kHistBranch * max_iter + i]);
        S.beta.push_back(have_gap ? hist[(size_t)kHistBeta * max_iter + i] : NAN);
        S.betabar.push_back(have_gap ? hist[(size_t)kHistBetabar * max_iter + i] : NAN);
        const int s = (int)hist[(size_t)kHistDigits * max_iter + i];
        dmax = std::max(dmax, s);
        tflops += 0.5 * s * (s + 1) * tile_flops;
        h->hist_trace.push_back(hist[(size_t)kHistTrace * max_iter + i]);
        h->hist_idem.push_back(hist[(size_t)kHistIdem * max_iter + i]);
    }
    S.converged = now.converged != 0;
    h->st.digit_max = dmax;
    h->st.tensor_flops = tflops;
    h->st.product_launches = m;
    count_launches(blocks * (kBlock * (1 + smax - smin + 1) + 1) + 2);
    h->st.trace = m > 0 ? h->hist_trace.back() : NAN;
    h->st.idem_err_fro = m > 0 ? h->hist_idem.back() : NAN;
    *iters = m;
    return PURIFY_OK;
}

}  // namespace purify
