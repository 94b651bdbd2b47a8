// Instantiations of the product kernel for queue launches (a whole batch in
// one launch): largest digit count 1..3.
#include "digits_kernel.cuh"

namespace purify {
namespace dk {

KernelFn kernel_queue_lo(int s) {
    switch (s) {
        case 1: return digit_gemm_kernel<32, 1, 1>;
        case 2: return digit_gemm_kernel<32, 2, 1>;
        case 3: return digit_gemm_kernel<32, 3, 1>;
        default: return nullptr;
    }
}

}  // namespace dk
}  // namespace purify
