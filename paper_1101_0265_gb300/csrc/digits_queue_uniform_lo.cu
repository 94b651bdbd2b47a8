// Instantiations of the product kernel for queue launches whose products all
// have the kernel's digit count (1..3).
#include "digits_kernel.cuh"

namespace purify {
namespace dk {

KernelFn kernel_queue_uniform_lo(int s) {
    switch (s) {
        case 1: return digit_gemm_kernel<32, 1, 2>;
        case 2: return digit_gemm_kernel<32, 2, 2>;
        case 3: return digit_gemm_kernel<32, 3, 2>;
        default: return nullptr;
    }
}

}  // namespace dk
}  // namespace purify
