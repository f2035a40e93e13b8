// CTA-tiled solver instantiations (fp64), register tiles R = 4 (n <= 64) and 8 (n <= 128).
#include "nls_cta.cuh"
#include "nls_internal.h"

namespace nls {

template <int R, int FAM>
static cudaError_t launch_cta_fp64(const SolveArgs &a, int grid, cudaStream_t st)
{
    k_solve_cta<R, FAM, false><<<grid, CTA_TPB, cta_smem_bytes<false, R>(), st>>>(a);
    return cudaGetLastError();
}

template <int R, int FAM>
static KernelInfo info_cta_fp64()
{
    // more than 48 KB of dynamic shared memory needs an opt-in, once per kernel
    static const cudaError_t attr = cudaFuncSetAttribute(
        reinterpret_cast<const void *>(&k_solve_cta<R, FAM, false>),
        cudaFuncAttributeMaxDynamicSharedMemorySize, cta_smem_bytes<false, R>());
    (void)attr;
    KernelInfo k;
    k.launch = &launch_cta_fp64<R, FAM>;
    k.func = reinterpret_cast<const void *>(&k_solve_cta<R, FAM, false>);
    k.block = CTA_TPB;
    k.smem = cta_smem_bytes<false, R>();
    k.per_cta = 1;
    return k;
}

template <int R>
static KernelInfo cta_by_family_fp64(int family)
{
    switch (family) {
    case FAM_CUBIC: return info_cta_fp64<R, FAM_CUBIC>();
    case FAM_BRATU: return info_cta_fp64<R, FAM_BRATU>();
    case FAM_SQUARE: return info_cta_fp64<R, FAM_SQUARE>();
    case FAM_ROSENBROCK: return info_cta_fp64<R, FAM_ROSENBROCK>();
    default: return KernelInfo{};
    }
}

KernelInfo cta_kernel_fp64(int family, int n)
{
    if (n <= 64) return cta_by_family_fp64<4>(family);
    if (n <= 128) return cta_by_family_fp64<8>(family);
    return KernelInfo{};
}

} // namespace nls
