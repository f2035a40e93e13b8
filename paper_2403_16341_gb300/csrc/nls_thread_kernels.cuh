// nls_thread_kernels.cuh -- KernelInfo factories for the thread tiling.
#pragma once

#include "nls_internal.h"
#include "nls_thread.cuh"

namespace nls {

template <int N, int FAM, bool MIXED, bool ANALYTIC>
cudaError_t launch_thread(const SolveArgs &a, int grid, cudaStream_t st)
{
    k_solve_thread<N, FAM, MIXED, ANALYTIC>
        <<<grid, THREAD_TPB, thread_newton_smem_bytes<N, FAM, MIXED>(), st>>>(a);
    return cudaGetLastError();
}

template <int N, int FAM, bool MIXED, bool ANALYTIC>
KernelInfo thread_info()
{
    KernelInfo k;
    k.launch = &launch_thread<N, FAM, MIXED, ANALYTIC>;
    k.func = reinterpret_cast<const void *>(&k_solve_thread<N, FAM, MIXED, ANALYTIC>);
    k.block = THREAD_TPB;
    k.smem = thread_newton_smem_bytes<N, FAM, MIXED>();
    k.per_cta = THREAD_TPB;
    return k;
}

template <int N, int FAM>
KernelInfo thread_info_n(bool mixed, bool analytic)
{
    if (mixed) return analytic ? thread_info<N, FAM, true, true>() : thread_info<N, FAM, true, false>();
    return analytic ? thread_info<N, FAM, false, true>() : thread_info<N, FAM, false, false>();
}

template <int FAM>
KernelInfo thread_info_family(int n, bool mixed, bool analytic)
{
    switch (n) {
    case 1: return thread_info_n<1, FAM>(mixed, analytic);
    case 2: return thread_info_n<2, FAM>(mixed, analytic);
    case 3: return thread_info_n<3, FAM>(mixed, analytic);
    case 4: return thread_info_n<4, FAM>(mixed, analytic);
    case 5: return thread_info_n<5, FAM>(mixed, analytic);
    case 6: return thread_info_n<6, FAM>(mixed, analytic);
    case 7: return thread_info_n<7, FAM>(mixed, analytic);
    case 8: return thread_info_n<8, FAM>(mixed, analytic);
    default: return KernelInfo{};
    }
}

} // namespace nls
