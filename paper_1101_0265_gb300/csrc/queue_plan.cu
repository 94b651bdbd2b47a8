// Staging and launch of queue launches (see queue_plan.h).
#include "queue_plan.h"

#include <algorithm>
#include <cstring>

#include "digits_kernel.cuh"

namespace purify {

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

void banded_tiles(int T, std::vector<int2>& tiles) {
    tiles.clear();
    for (int b0 = 0; b0 < T; b0 += dk::BAND) {
        const int b1 = std::min(T, b0 + dk::BAND);
        for (int r = 0; r < b1; ++r)
            for (int c = std::max(b0, r); c < b1; ++c) tiles.push_back(make_int2(r, c));
    }
}

void chain_tile_order(int T, int ctas, std::vector<int2>& tiles) {
    int L = 1;  // the first L panels: their upper triangle is at least one wave
    while (L < T && L * (L + 1) / 2 < ctas) ++L;
    std::vector<int2> band;
    banded_tiles(T, band);
    tiles.clear();
    for (const int2& t : band)
        if (t.y < L) tiles.push_back(t);
    for (int r = 0; r < L; ++r)  // row by row: panel r is complete after its row
        for (int c = L; c < T; ++c) tiles.push_back(make_int2(r, c));
    for (int r = L; r < T; ++r)
        for (int c = r; c < T; ++c) tiles.push_back(make_int2(r, c));
}

int stage_queue_products(const std::vector<QueueProduct>& prods, const std::vector<int4>& work,
                         std::vector<uint8_t>& host, QueueStaging& q) {
    q = QueueStaging();
    q.products = (int)prods.size();
    q.items = (int)work.size();
    if (q.products == 0) return PURIFY_OK;
    std::vector<int> T(q.products), cnt0(q.products);
    int cnt_ints = 0;
    int smin = kMaxDigitPlanes + 1;
    for (int g = 0; g < q.products; ++g) {
        const QueueProduct& p = prods[g];
        q.smax = std::max(q.smax, p.st.s_in);
        smin = std::min(smin, p.st.s_in);
        T[g] = p.st.n_pad / 128;
        cnt0[g] = cnt_ints;
        cnt_ints += T[g] + 1;  // row panels, then the total
        for (int d : {p.depA, p.depB, p.war0, p.war1})
            if (d >= g || d < -1) return PURIFY_ERR_INTERNAL;  // only earlier products
        if (p.depA >= 0 && T[p.depA] != T[g]) return PURIFY_ERR_INTERNAL;
        if (p.depB >= 0 && T[p.depB] != T[g]) return PURIFY_ERR_INTERNAL;
    }
    q.uniform = smin == q.smax;
    // the deadlock-freedom property of the list (see the header)
    std::vector<std::vector<int>> panel_seen(q.products);
    std::vector<int> seen(q.products, 0);
    std::vector<std::vector<char>> tile_seen(q.products);
    for (int g = 0; g < q.products; ++g) {
        panel_seen[g].assign(T[g], 0);
        tile_seen[g].assign((size_t)T[g] * T[g], 0);
    }
    for (const int4& w : work) {
        const int g = w.x, ti = w.y, tj = w.z;
        if (g < 0 || g >= q.products || ti < 0 || ti > tj || tj >= T[g]) return PURIFY_ERR_INTERNAL;
        char& ts = tile_seen[g][(size_t)ti * T[g] + tj];
        if (ts) return PURIFY_ERR_INTERNAL;
        ts = 1;
        const QueueProduct& p = prods[g];
        if (p.depA >= 0 && panel_seen[p.depA][ti] != T[g]) return PURIFY_ERR_INTERNAL;
        if (p.depB >= 0 && panel_seen[p.depB][tj] != T[g]) return PURIFY_ERR_INTERNAL;
        for (int d : {p.war0, p.war1})
            if (d >= 0 && seen[d] != T[d] * (T[d] + 1) / 2) return PURIFY_ERR_INTERNAL;
        ++panel_seen[g][ti];
        if (tj != ti) ++panel_seen[g][tj];
        ++seen[g];
    }
    for (int g = 0; g < q.products; ++g)
        if (seen[g] != T[g] * (T[g] + 1) / 2) return PURIFY_ERR_INTERNAL;

    q.maps_off = 0;
    q.prm_off = align_up(q.maps_off + sizeof(CUtensorMap) * 2 * (size_t)q.products, 128);
    q.cnt_off = align_up(q.prm_off + sizeof(dk::DigitGemmParams) * (size_t)q.products, 128);
    q.cnt_bytes = sizeof(int) * ((size_t)cnt_ints + 1);  // + the claim ticket
    q.work_off = align_up(q.cnt_off + q.cnt_bytes, 128);
    q.end = q.work_off + sizeof(int4) * work.size();
    if (host.size() < q.end) host.resize(q.end);
    uint8_t* hb = host.data();
    CUtensorMap* maps = (CUtensorMap*)(hb + q.maps_off);
    dk::DigitGemmParams* prm = (dk::DigitGemmParams*)(hb + q.prm_off);
    for (int g = 0; g < q.products; ++g) {
        const QueueProduct& p = prods[g];
        PURIFY_TRY(fill_queue_product(p.st, q.smax, &prm[g], &maps[2 * g]));
        prm[g].q_depA = p.depA;
        prm[g].q_depB = p.depB;
        prm[g].q_war0 = p.war0;
        prm[g].q_war1 = p.war1;
        prm[g].q_cnt = cnt0[g];
    }
    std::memset(hb + q.cnt_off, 0, q.cnt_bytes);
    if (!work.empty()) std::memcpy(hb + q.work_off, work.data(), sizeof(int4) * work.size());
    return PURIFY_OK;
}

int launch_staged_queue(const QueueStaging& q, void* dev, float2* scratch, int max_ctas, int* err,
                        cudaStream_t stream, long long wait_cycles) {
    if (q.items == 0) return PURIFY_OK;
    uint8_t* d = (uint8_t*)dev;
    PURIFY_CUDA_TRY(cudaMemsetAsync(d + q.cnt_off, 0, q.cnt_bytes, stream));
    int* cnt = (int*)(d + q.cnt_off);
    int* ticket = cnt + (q.cnt_bytes / sizeof(int) - 1);
    return launch_digit_queue(q.smax, q.uniform, (const dk::DigitGemmParams*)(d + q.prm_off),
                              (const CUtensorMap*)(d + q.maps_off), cnt, ticket, (const int4*)(d + q.work_off),
                              q.items, scratch, max_ctas, err, stream, wait_cycles);
}

}  // namespace purify
