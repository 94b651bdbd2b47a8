// Instantiations of the product kernel for queue launches (a whole batch in
// one launch): largest digit count 4..6.
#include "digits_kernel.cuh"

namespace purify {
namespace dk {

KernelFn kernel_queue_hi(int s) {
    switch (s) {
        case 4: return digit_gemm_kernel<32, 4, 1>;
        case 5: return digit_gemm_kernel<32, 5, 1>;
        case 6: return digit_gemm_kernel<32, 6, 1>;
        default: return nullptr;
    }
}

}  // namespace dk
}  // namespace purify
