#include "mixed.h"

namespace purify {

struct MixedState {
    int dummy;
};

int run_mixed(purify_ctx*, int, double, const Schedule&, int*, std::vector<double>&) {
    return PURIFY_ERR_UNSUPPORTED;
}

void mixed_free(MixedState* ms) { delete ms; }

}  // namespace purify
