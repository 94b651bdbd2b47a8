// Instantiations of the digit-plane product kernel: k-chunk 32, digit
// counts 4..6 (one translation unit each, compiled in parallel).
#include "digits_kernel.cuh"

namespace purify {
namespace dk {

KernelFn kernel_k32_hi(int s) {
    switch (s) {
        case 4: return digit_gemm_kernel<32, 4, 0>;
        case 5: return digit_gemm_kernel<32, 5, 0>;
        case 6: return digit_gemm_kernel<32, 6, 0>;
        default: return nullptr;
    }
}

}  // namespace dk
}  // namespace purify
