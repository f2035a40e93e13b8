// Warp-tiled Halley solver instantiations (mixed), L = 16 and 32 lanes per instance.
#include "nls_warp_ext.cuh"

namespace nls {
KernelInfo warp_halley_mixed(int family, int L)
{
    return warp_ext_info_for<ALG_HALLEY, true>(family, L);
}
} // namespace nls
