// Column-panel CTA solver instantiations: mixed, cubic family, n <= 32, 64, 96, 128.
#include "nls_panel_kernels.cuh"

namespace nls {

KernelInfo panel_kernel_mixed_cubic(int n) { return panel_info_for<FAM_CUBIC, true>(n); }

} // namespace nls
