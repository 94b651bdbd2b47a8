// Instantiations of the product kernel with pooled digit planes (block-sparse
// runs: 32 x 32 blocks in pool slots found through slot tables), 1..3 digits.
#include "digits_kernel.cuh"

namespace purify {
namespace dk {

KernelFn kernel_pool_lo(int s) {
    switch (s) {
        case 1: return digit_gemm_kernel<32, 1, 3>;
        case 2: return digit_gemm_kernel<32, 2, 3>;
        case 3: return digit_gemm_kernel<32, 3, 3>;
        default: return nullptr;
    }
}

}  // namespace dk
}  // namespace purify
