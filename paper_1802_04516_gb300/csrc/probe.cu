// Arithmetic-peak probe: the FP64 and FP32 FMA rates this GPU actually sustains, measured with
// the library's own kernel, as the denominators of the ALU-bound rooflines (the FP64 operator
// kernels of the FP64 path).  No counterpart in the paper.
//
// Each thread runs 8 independent FMA chains (enough instruction-level parallelism to cover the
// FMA latency), the grid fills every SM several times over, and the chains' results are
// folded into one store per thread so the compiler cannot drop them.
#include <algorithm>

#include "stdg.h"
#include "stdg_internal.h"

namespace stdg {
namespace {

template <typename R>
__global__ void __launch_bounds__(256) fma_chain_kernel(int iters, R a, R b, R* __restrict__ out) {
    R x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (R)(threadIdx.x + k) * (R)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    R s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

template <typename R>
int run_probe(int iters, double* tflops) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return STDG_ECUDA;
    const int threads = 256, blocks = nsm * 8;
    R* out = nullptr;
    if (cudaMalloc(&out, sizeof(R) * (size_t)threads * blocks) != cudaSuccess) return STDG_ENOMEM;
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { cudaFree(out); return STDG_ECUDA; }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // a, b with |a| < 1 keep every chain finite; the values do not matter for the rate
    fma_chain_kernel<R><<<blocks, threads, 0, st>>>(iters / 10 + 1, (R)0.999, (R)1e-4, out);   // warm-up
    cudaEventRecord(e0, st);
    fma_chain_kernel<R><<<blocks, threads, 0, st>>>(iters, (R)0.999, (R)1e-4, out);
    cudaEventRecord(e1, st);
    const cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    cudaFree(out);
    if (err != cudaSuccess || !(ms > 0)) return STDG_ECUDA;
    const double flops = 2.0 * 16.0 * 8.0 * (double)iters * threads * blocks;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return STDG_OK;
}

}  // namespace
}  // namespace stdg

extern "C" int stdg_measure_fma_peak(int fp64, double* tflops) {
    if (!tflops) return STDG_EINVAL;
    return fp64 ? stdg::run_probe<double>(2000, tflops) : stdg::run_probe<float>(20000, tflops);
}
