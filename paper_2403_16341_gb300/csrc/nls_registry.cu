// nls_registry.cu -- which kernel serves a request: the KernelInfo factories
// of every tiling, algorithm family and precision, by (family, n, alg).
// The instantiation units (nls_thread_*.cu, nls_warp_*.cu, nls_cta_*.cu)
// define the per-family factories declared here.
#include "nls_internal.h"

namespace nls {
KernelInfo thread_kernel_cubic(int n, bool mixed, bool analytic);
KernelInfo thread_kernel_bratu(int n, bool mixed, bool analytic);
KernelInfo thread_kernel_square(int n, bool mixed, bool analytic);
KernelInfo thread_kernel_rosenbrock(int n, bool mixed, bool analytic);

KernelInfo thread_kernel(int family, int n, bool mixed, bool analytic)
{
    switch (family) {
    case FAM_CUBIC: return thread_kernel_cubic(n, mixed, analytic);
    case FAM_BRATU: return thread_kernel_bratu(n, mixed, analytic);
    case FAM_SQUARE: return thread_kernel_square(n, mixed, analytic);
    case FAM_ROSENBROCK: return thread_kernel_rosenbrock(n, mixed, analytic);
    default: return KernelInfo{};
    }
}
#define NLS_EXT_DECL(alg)                                  \
    KernelInfo thread_##alg##_cubic(int n, bool mixed);    \
    KernelInfo thread_##alg##_bratu(int n, bool mixed);    \
    KernelInfo thread_##alg##_square(int n, bool mixed);   \
    KernelInfo thread_##alg##_rosenbrock(int n, bool mixed);
NLS_EXT_DECL(potra_ptak)
NLS_EXT_DECL(halley)
NLS_EXT_DECL(broyden)
#undef NLS_EXT_DECL

// Potra-Ptak, Halley, Broyden and modified Broyden: one instance per thread.
KernelInfo thread_ext_kernel(int family, int n, int alg, bool mixed)
{
    using Fn = KernelInfo (*)(int, bool);
    static const Fn table[3][4] = {
        {thread_potra_ptak_cubic, thread_potra_ptak_bratu, thread_potra_ptak_square, thread_potra_ptak_rosenbrock},
        {thread_halley_cubic, thread_halley_bratu, thread_halley_square, thread_halley_rosenbrock},
        {thread_broyden_cubic, thread_broyden_bratu, thread_broyden_square, thread_broyden_rosenbrock}};
    const int row = alg == ALG_POTRA_PTAK ? 0 : alg == ALG_HALLEY ? 1
                    : (alg == ALG_BROYDEN || alg == ALG_MOD_BROYDEN) ? 2 : -1;
    if (row < 0 || family < FAM_CUBIC || family > FAM_ROSENBROCK) return KernelInfo{};
    return table[row][family](n, mixed);
}

KernelInfo warp_potra_ptak_fp64(int family, int L);
KernelInfo warp_potra_ptak_mixed(int family, int L);
KernelInfo warp_halley_fp64(int family, int L);
KernelInfo warp_halley_mixed(int family, int L);
KernelInfo warp_broyden_fp64(int family, int L);
KernelInfo warp_broyden_mixed(int family, int L);

// Potra-Ptak, Halley, Broyden and modified Broyden, one instance per warp
// segment of L = 16 or 32 lanes.
KernelInfo warp_ext_kernel(int family, int L, int alg, bool mixed)
{
    switch (alg) {
    case ALG_POTRA_PTAK: return mixed ? warp_potra_ptak_mixed(family, L) : warp_potra_ptak_fp64(family, L);
    case ALG_HALLEY: return mixed ? warp_halley_mixed(family, L) : warp_halley_fp64(family, L);
    case ALG_BROYDEN:
    case ALG_MOD_BROYDEN: return mixed ? warp_broyden_mixed(family, L) : warp_broyden_fp64(family, L);
    default: return KernelInfo{};
    }
}

KernelInfo cta_potra_ptak_fp64(int family, int n);
KernelInfo cta_potra_ptak_mixed(int family, int n);
KernelInfo cta_halley_fp64(int family, int n);
KernelInfo cta_halley_mixed(int family, int n);
KernelInfo cta_broyden_fp64(int family, int n);
KernelInfo cta_broyden_mixed(int family, int n);

// ... and one instance per CTA (n <= 128).
KernelInfo cta_ext_kernel(int family, int n, int alg, bool mixed)
{
    switch (alg) {
    case ALG_POTRA_PTAK: return mixed ? cta_potra_ptak_mixed(family, n) : cta_potra_ptak_fp64(family, n);
    case ALG_HALLEY: return mixed ? cta_halley_mixed(family, n) : cta_halley_fp64(family, n);
    case ALG_BROYDEN:
    case ALG_MOD_BROYDEN: return mixed ? cta_broyden_mixed(family, n) : cta_broyden_fp64(family, n);
    default: return KernelInfo{};
    }
}

KernelInfo warp_kernel_fp64(int family, int L);
KernelInfo warp_kernel_mixed(int family, int L);

KernelInfo cta_kernel_fp64(int family, int n);
KernelInfo cta_kernel_mixed(int family, int n);

KernelInfo cta_kernel(int family, int n, bool mixed)
{
    return mixed ? cta_kernel_mixed(family, n) : cta_kernel_fp64(family, n);
}

KernelInfo warp_kernel(int family, int n, bool mixed, int lanes)
{
    int L = lanes ? lanes : (n <= 8 ? 8 : n <= 16 ? 16 : 32);
    if (n > L || n > 32) return KernelInfo{};
    return mixed ? warp_kernel_mixed(family, L) : warp_kernel_fp64(family, L);
}
} // namespace nls
