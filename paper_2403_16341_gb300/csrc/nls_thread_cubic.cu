// Thread-tiled solver instantiations for the cubic family (n = 1..8).
#include "nls_thread_kernels.cuh"

namespace nls {
KernelInfo thread_kernel_cubic(int n, bool mixed, bool analytic)
{
    return thread_info_family<FAM_CUBIC>(n, mixed, analytic);
}
} // namespace nls
