// Thread-tiled Broyden and modified Broyden solver instantiations for the cubic family (n = 1..8).
#include "nls_thread_ext.cuh"

namespace nls {
KernelInfo thread_broyden_cubic(int n, bool mixed)
{
    return thread_ext_info_family<FAM_CUBIC, ALG_BROYDEN>(n, mixed);
}
} // namespace nls
