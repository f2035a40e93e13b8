// nls_poly.cu -- device side of the batched poly-algorithm (Sec. 3.2, Fig. 4):
// after a stage, the instances that did not converge are gathered (with
// their original u0) into compact arrays, solved by the next, more robust
// algorithm, and scattered back.  Counts stay on the device: the next
// stage's kernels read them (SolveArgs::dyn_batch).
#include <cuda_runtime.h>

#include "nls_internal.h"

namespace nls {

__global__ void k_poly_gather(PolyGatherArgs g)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.batch || g.status[k] == ST_SUCCESS) return;
    const int64_t pos = (int64_t)atomicAdd(g.count, 1ull);
    g.idx[pos] = k;
    for (int e = 0; e < g.E; ++e) g.cparams[(int64_t)e * g.batch + pos] = g.params[(int64_t)e * g.batch + k];
    for (int i = 0; i < g.n; ++i) g.cu[(int64_t)i * g.batch + pos] = g.u0[(int64_t)i * g.batch + k];
}

__global__ void k_poly_scatter(PolyScatterArgs s)
{
    const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= (int64_t)*s.count) return;
    const int64_t k = s.idx[pos];
    for (int i = 0; i < s.n; ++i) s.u[(int64_t)i * s.batch + k] = s.cu[(int64_t)i * s.batch + pos];
    s.status[k] = s.cstatus[pos];
    s.iters[k] = s.citers[pos];
    s.resid[k] = s.cresid[pos];
    s.nfev[k] += s.cnfev[pos]; // residual evaluations of every stage
}

// solved += the solved counts of the gathered stages (counter triples:
// gathered, solved, work)
__global__ void k_poly_total(unsigned long long *solved, const unsigned long long *ctr, int stages)
{
    unsigned long long t = 0;
    for (int s = 0; s < stages; ++s) t += ctr[3 * s + 1];
    *solved += t;
}

cudaError_t launch_poly_gather(const PolyGatherArgs &g, cudaStream_t st)
{
    const int64_t blocks = (g.batch + 255) / 256;
    k_poly_gather<<<(unsigned)blocks, 256, 0, st>>>(g);
    return cudaGetLastError();
}

cudaError_t launch_poly_scatter(const PolyScatterArgs &s, cudaStream_t st)
{
    const int64_t blocks = (s.batch + 255) / 256;
    k_poly_scatter<<<(unsigned)blocks, 256, 0, st>>>(s);
    return cudaGetLastError();
}

cudaError_t launch_poly_total(unsigned long long *solved, const unsigned long long *ctr, int stages,
                              cudaStream_t st)
{
    k_poly_total<<<1, 1, 0, st>>>(solved, ctr, stages);
    return cudaGetLastError();
}

} // namespace nls
