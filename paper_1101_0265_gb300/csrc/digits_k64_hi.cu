// Instantiations of the digit-plane product kernel: k-chunk 64, digit
// counts 4..6 (one translation unit each, compiled in parallel).
#include "digits_kernel.cuh"

namespace purify {
namespace dk {

KernelFn kernel_k64_hi(int s) {
    switch (s) {
        case 4: return digit_gemm_kernel<64, 4, false>;
        case 5: return digit_gemm_kernel<64, 5, false>;
        case 6: return digit_gemm_kernel<64, 6, false>;
        default: return nullptr;
    }
}

}  // namespace dk
}  // namespace purify
