// Thread-tiled Halley solver instantiations for the bratu family (n = 1..8).
#include "nls_thread_ext.cuh"

namespace nls {
KernelInfo thread_halley_bratu(int n, bool mixed)
{
    return thread_ext_info_family<FAM_BRATU, ALG_HALLEY>(n, mixed);
}
} // namespace nls
