// Thread-tiled solver instantiations for the rosenbrock family (n = 1..8).
#include "nls_thread_kernels.cuh"

namespace nls {
KernelInfo thread_kernel_rosenbrock(int n, bool mixed, bool analytic)
{
    return thread_info_family<FAM_ROSENBROCK>(n, mixed, analytic);
}
} // namespace nls
