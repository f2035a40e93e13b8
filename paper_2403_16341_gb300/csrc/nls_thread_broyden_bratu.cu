// Thread-tiled Broyden and modified Broyden solver instantiations for the bratu family (n = 1..8).
#include "nls_thread_ext.cuh"

namespace nls {
KernelInfo thread_broyden_bratu(int n, bool mixed)
{
    return thread_ext_info_family<FAM_BRATU, ALG_BROYDEN>(n, mixed);
}
} // namespace nls
