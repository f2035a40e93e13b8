// Warp-tiled solver instantiations (mixed), L = 8, 16, 32 lanes per instance.
#include "nls_internal.h"
#include "nls_warp.cuh"

namespace nls {

template <int L, int FAM>
static cudaError_t launch_warp_mixed(const SolveArgs &a, int grid, cudaStream_t st)
{
    k_solve_warp<L, FAM, true><<<grid, WARP_TPB, warp_smem_bytes<L, true>(), st>>>(a);
    return cudaGetLastError();
}

template <int L, int FAM>
static KernelInfo info_mixed()
{
    KernelInfo k;
    k.launch = &launch_warp_mixed<L, FAM>;
    k.func = reinterpret_cast<const void *>(&k_solve_warp<L, FAM, true>);
    k.block = WARP_TPB;
    k.smem = warp_smem_bytes<L, true>();
    k.per_cta = (WARP_TPB / 32) * (32 / L);
    return k;
}

template <int L>
static KernelInfo by_family_mixed(int family)
{
    switch (family) {
    case FAM_CUBIC: return info_mixed<L, FAM_CUBIC>();
    case FAM_BRATU: return info_mixed<L, FAM_BRATU>();
    case FAM_SQUARE: return info_mixed<L, FAM_SQUARE>();
    case FAM_ROSENBROCK: return info_mixed<L, FAM_ROSENBROCK>();
    default: return KernelInfo{};
    }
}

KernelInfo warp_kernel_mixed(int family, int L)
{
    switch (L) {
    case 8: return by_family_mixed<8>(family);
    case 16: return by_family_mixed<16>(family);
    case 32: return by_family_mixed<32>(family);
    default: return KernelInfo{};
    }
}

} // namespace nls
