// nls_panel_kernels.cuh -- launch helpers and registry entries of the
// column-panel CTA solver (nls_panel.cuh, mixed precision): one instance per
// CTA, n <= 32 S for S = 1 .. 4, 16 columns of J per warp.
#pragma once

#include "nls_internal.h"
#include "nls_panel.cuh"

namespace nls {

template <int S, int FAM, bool MIXED>
static cudaError_t launch_panel(const SolveArgs &a, int grid, cudaStream_t st)
{
    constexpr int C = panel_cols<MIXED>();
    k_solve_panel<S, C, FAM, MIXED>
        <<<grid, PanelSolver<S, C, FAM, MIXED>::TPB, panel_smem_bytes<S, C, MIXED>(), st>>>(a);
    return cudaGetLastError();
}

template <int S, int FAM, bool MIXED>
static KernelInfo panel_info()
{
    constexpr int C = panel_cols<MIXED>();
    constexpr int smem = panel_smem_bytes<S, C, MIXED>();
    const void *f = reinterpret_cast<const void *>(&k_solve_panel<S, C, FAM, MIXED>);
    if constexpr (smem > 48 * 1024) {
        // more than 48 KB of dynamic shared memory needs an opt-in, once per kernel
        static const cudaError_t attr = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        (void)attr;
    }
    KernelInfo k;
    k.launch = &launch_panel<S, FAM, MIXED>;
    k.func = f;
    k.block = PanelSolver<S, C, FAM, MIXED>::TPB;
    k.smem = smem;
    k.per_cta = 1;
    return k;
}

template <int FAM, bool MIXED>
static KernelInfo panel_info_for(int n)
{
    if (n <= 32) return panel_info<1, FAM, MIXED>();
    if (n <= 64) return panel_info<2, FAM, MIXED>();
    if (n <= 96) return panel_info<3, FAM, MIXED>();
    if (n <= 128) return panel_info<4, FAM, MIXED>();
    return KernelInfo{};
}

} // namespace nls
