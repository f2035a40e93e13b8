// CTA-tiled Halley solver instantiations (mixed), register tiles R = 4 (n <= 64) and 8 (n <= 128).
#include "nls_cta_ext.cuh"

namespace nls {
KernelInfo cta_halley_mixed(int family, int n)
{
    return cta_ext_info_for<ALG_HALLEY, true>(family, n);
}
} // namespace nls
