// nls_probe.cu -- diagnostic entry point exposing the device reciprocal used
// for the FP64 LU pivots, so that tests can bound its error against the
// correctly rounded quotient.
#include <cuda_runtime.h>

#include "../../include/nls.h"
#include "nls_common.cuh"

namespace {
__global__ void k_probe_rcp(const double *x, double *y, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = nls::rcp(x[i]);
}
} // namespace

extern "C" int nls_probe_rcp(const double *x, double *y, int64_t n, void *cuda_stream)
{
    if (n < 0 || (n > 0 && (!x || !y))) return NLS_E_INVALID;
    if (n == 0) return NLS_OK;
    const int64_t blocks = (n + 255) / 256;
    if (blocks > 0x7fffffff) return NLS_E_INVALID;
    k_probe_rcp<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(x, y, n);
    return cudaGetLastError() == cudaSuccess ? NLS_OK : NLS_E_CUDA;
}
