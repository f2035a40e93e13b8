// Thread-tiled Broyden and modified Broyden solver instantiations for the square family (n = 1..8).
#include "nls_thread_ext.cuh"

namespace nls {
KernelInfo thread_broyden_square(int n, bool mixed)
{
    return thread_ext_info_family<FAM_SQUARE, ALG_BROYDEN>(n, mixed);
}
} // namespace nls
