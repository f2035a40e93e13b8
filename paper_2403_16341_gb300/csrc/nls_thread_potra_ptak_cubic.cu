// Thread-tiled Potra-Ptak solver instantiations for the cubic family (n = 1..8).
#include "nls_thread_ext.cuh"

namespace nls {
KernelInfo thread_potra_ptak_cubic(int n, bool mixed)
{
    return thread_ext_info_family<FAM_CUBIC, ALG_POTRA_PTAK>(n, mixed);
}
} // namespace nls
