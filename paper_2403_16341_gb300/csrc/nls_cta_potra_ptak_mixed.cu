// CTA-tiled Potra-Ptak solver instantiations (mixed), register tiles R = 4 (n <= 64) and 8 (n <= 128).
#include "nls_cta_ext.cuh"

namespace nls {
KernelInfo cta_potra_ptak_mixed(int family, int n)
{
    return cta_ext_info_for<ALG_POTRA_PTAK, true>(family, n);
}
} // namespace nls
