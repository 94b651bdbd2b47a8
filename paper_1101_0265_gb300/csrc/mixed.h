// Mixed-precision (digit-plane tensor-core) path of the iteration driver.
#pragma once

#include <vector>

#include "internal.h"

namespace purify {

struct MixedState;
constexpr int kMaxDigits = 6;  // equals kMaxDigitPlanes (digits_tc.h)

// Run the scheme's coefficient schedule with every matrix product on the
// tcgen05 tensor cores (see mixed.cu).  Sets *cur (index into h->X of the
// float64 density), fills `red` with the per-step reductions and the
// mixed-path fields of h->st.
int run_mixed(purify_ctx* h, int scheme, double mu, const Schedule& S, int* cur,
              std::vector<double>& red);
void mixed_free(MixedState* ms);

}  // namespace purify
