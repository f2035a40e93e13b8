// Warp-tiled Halley solver instantiations (fp64), L = 16 and 32 lanes per instance.
#include "nls_warp_ext.cuh"

namespace nls {
KernelInfo warp_halley_fp64(int family, int L)
{
    return warp_ext_info_for<ALG_HALLEY, false>(family, L);
}
} // namespace nls
