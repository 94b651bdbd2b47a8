// Instantiations of the digit-plane product kernel: k-chunk 16 (32-byte
// swizzle, twice the pipeline depth of k-chunk 32), digit counts 4..6.
#include "digits_kernel.cuh"

namespace purify {
namespace dk {

KernelFn kernel_k16_hi(int s) {
    switch (s) {
        case 4: return digit_gemm_kernel<16, 4, false>;
        case 5: return digit_gemm_kernel<16, 5, false>;
        case 6: return digit_gemm_kernel<16, 6, false>;
        default: return nullptr;
    }
}

}  // namespace dk
}  // namespace purify
