// Thread-tiled solver instantiations for the square family (n = 1..8).
#include "nls_thread_kernels.cuh"

namespace nls {
KernelInfo thread_kernel_square(int n, bool mixed, bool analytic)
{
    return thread_info_family<FAM_SQUARE>(n, mixed, analytic);
}
} // namespace nls
