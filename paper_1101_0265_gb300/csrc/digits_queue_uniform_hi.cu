// Instantiations of the product kernel for queue launches whose products all
// have the kernel's digit count (4..6).
#include "digits_kernel.cuh"

namespace purify {
namespace dk {

KernelFn kernel_queue_uniform_hi(int s) {
    switch (s) {
        case 4: return digit_gemm_kernel<32, 4, 2>;
        case 5: return digit_gemm_kernel<32, 5, 2>;
        case 6: return digit_gemm_kernel<32, 6, 2>;
        default: return nullptr;
    }
}

}  // namespace dk
}  // namespace purify
