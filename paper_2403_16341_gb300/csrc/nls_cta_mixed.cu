// CTA tiling (one instance per CTA, n <= 128) of Newton, backtracking and the
// dogleg trust region, mixed precision (FP32 Jacobian and LU): the column-panel solver of nls_panel.cuh,
// one instantiation unit per family (nls_panel_mixed_*.cu).
#include "nls_internal.h"

namespace nls {

KernelInfo panel_kernel_mixed_cubic(int n);
KernelInfo panel_kernel_mixed_bratu(int n);
KernelInfo panel_kernel_mixed_square(int n);
KernelInfo panel_kernel_mixed_rosenbrock(int n);

KernelInfo cta_kernel_mixed(int family, int n)
{
    switch (family) {
    case FAM_CUBIC: return panel_kernel_mixed_cubic(n);
    case FAM_BRATU: return panel_kernel_mixed_bratu(n);
    case FAM_SQUARE: return panel_kernel_mixed_square(n);
    case FAM_ROSENBROCK: return panel_kernel_mixed_rosenbrock(n);
    default: return KernelInfo{};
    }
}

} // namespace nls
