// Thread-tiled Broyden and modified Broyden solver instantiations for the rosenbrock family (n = 1..8).
#include "nls_thread_ext.cuh"

namespace nls {
KernelInfo thread_broyden_rosenbrock(int n, bool mixed)
{
    return thread_ext_info_family<FAM_ROSENBROCK, ALG_BROYDEN>(n, mixed);
}
} // namespace nls
