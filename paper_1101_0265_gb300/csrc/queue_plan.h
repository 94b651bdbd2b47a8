// Host side of queue launches: many digit-plane products in one persistent
// launch of the product kernel (queue mode, see DigitLaunch).  Callers
// describe the products, their dependencies and the order of the work items;
// this module stages parameters, tensor maps, counters and the work list in
// one buffer, checks that the order cannot deadlock, and launches.
#pragma once

#include <vector>

#include "digits_tc.h"

namespace purify {

struct QueueProduct {
    DigitStep st;        // the product (A, B, outputs, reductions)
    int depA = -1;       // product that writes A's planes (-1: written before the launch)
    int depB = -1;       // product that writes B's planes
    int war0 = -1;       // products that must have finished every item first
    int war1 = -1;       // (they read the buffer this product overwrites)
};

struct QueueStaging {
    int smax = 0;          // largest digit count (the kernel instantiation)
    bool uniform = false;  // every product has smax digits
    int products = 0;
    int items = 0;
    size_t maps_off = 0, prm_off = 0, cnt_off = 0, cnt_bytes = 0, work_off = 0, end = 0;
};

// Stage `prods` and the work list (items {product, ti, tj, 0}, in claim
// order) into `host` (resized to fit; the layout is recorded in q).  Checks
// that every product's items appear exactly once and that each item comes
// after every item it waits for (the items of depA / depB touching its row
// panels, and all items of war0 / war1): tickets are taken in list order,
// so the items an item waits for are then always held by running CTAs.
// PURIFY_ERR_INTERNAL when the list breaks this.
int stage_queue_products(const std::vector<QueueProduct>& prods, const std::vector<int4>& work,
                         std::vector<uint8_t>& host, QueueStaging& q);

// Zero the counters of a staged queue in `dev` (a device copy of the host
// buffer) and launch it on `stream`.
int launch_staged_queue(const QueueStaging& q, void* dev, float2* scratch, int max_ctas, int* err,
                        cudaStream_t stream, long long wait_cycles);

// The tiles of a T x T upper triangle in the product kernel's banded order
// (bands of 12 tile columns, inside a band row by row).
void banded_tiles(int T, std::vector<int2>& tiles);

// Work order for a chain of products of one size (each reading the previous
// one's output).  With L the fewest leading row panels whose upper triangle
// holds a wave of tiles (L (L + 1) / 2 >= ctas, at most T): first the tiles
// inside the first L panels (banded order), then the tiles that join them to
// the others, row by row (so panel r is complete after row r), then the
// remaining corner row by row.  A product's last wave is then mostly the
// corner, and the next product's first wave (inside the first L panels)
// waits little for it.
void chain_tile_order(int T, int ctas, std::vector<int2>& tiles);

}  // namespace purify
