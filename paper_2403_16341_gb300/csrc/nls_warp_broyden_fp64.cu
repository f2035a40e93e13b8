// Warp-tiled Broyden and modified Broyden solver instantiations (fp64), L = 16 and 32 lanes per instance.
#include "nls_warp_ext.cuh"

namespace nls {
KernelInfo warp_broyden_fp64(int family, int L)
{
    return warp_ext_info_for<ALG_BROYDEN, false>(family, L);
}
} // namespace nls
