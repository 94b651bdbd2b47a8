// Instantiations of the product kernel with pooled digit planes (block-sparse
// runs: 32 x 32 blocks in pool slots found through slot tables), 4..6 digits.
#include "digits_kernel.cuh"

namespace purify {
namespace dk {

KernelFn kernel_pool_hi(int s) {
    switch (s) {
        case 4: return digit_gemm_kernel<32, 4, 3>;
        case 5: return digit_gemm_kernel<32, 5, 3>;
        case 6: return digit_gemm_kernel<32, 6, 3>;
        default: return nullptr;
    }
}

}  // namespace dk
}  // namespace purify
