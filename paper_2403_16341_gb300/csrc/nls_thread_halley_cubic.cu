// Thread-tiled Halley solver instantiations for the cubic family (n = 1..8).
#include "nls_thread_ext.cuh"

namespace nls {
KernelInfo thread_halley_cubic(int n, bool mixed)
{
    return thread_ext_info_family<FAM_CUBIC, ALG_HALLEY>(n, mixed);
}
} // namespace nls
