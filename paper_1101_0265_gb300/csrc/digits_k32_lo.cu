// Instantiations of the digit-plane product kernel: k-chunk 32, digit
// counts 1..3 (one translation unit each, compiled in parallel).
#include "digits_kernel.cuh"

namespace purify {
namespace dk {

KernelFn kernel_k32_lo(int s) {
    switch (s) {
        case 1: return digit_gemm_kernel<32, 1, 0>;
        case 2: return digit_gemm_kernel<32, 2, 0>;
        case 3: return digit_gemm_kernel<32, 3, 0>;
        default: return nullptr;
    }
}

}  // namespace dk
}  // namespace purify
