// Thread-tiled solver instantiations for the bratu family (n = 1..8).
#include "nls_thread_kernels.cuh"

namespace nls {
KernelInfo thread_kernel_bratu(int n, bool mixed, bool analytic)
{
    return thread_info_family<FAM_BRATU>(n, mixed, analytic);
}
} // namespace nls
