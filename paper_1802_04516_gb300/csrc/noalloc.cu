// An entry point that allocates no memory: the residual r = b - A x of the velocity
// system and its relative norm, for callers that cannot call cudaMalloc.
//
// Who cannot allocate: code that runs while a CUDA stream is being captured into a
// graph (cudaMalloc/cudaFree are not stream operations and break or serialise the
// capture), pipelines that must not take the device-wide synchronisation that cudaFree
// implies while other streams are busy, and hosts whose memory is entirely reserved by
// another allocator (for instance a framework's caching pool that owns nearly all of
// HBM).  They hand in every input and output buffer; the only other memory this call
// touches is a fixed scratch array compiled into the library.
//
// The scratch array holds one FP64 partial sum of ||b - A x||^2 and one of ||b||^2 per
// block of kChunk vector entries, so velocity vectors of up to kParts * kChunk values
// (2^28) are accepted; longer ones are rejected.  Every partial sum is written before it
// is read, so nothing has to be cleared between calls.  Each GPU that loads the library
// holds the array (1 MiB) until the process exits.  All calls share it: two calls whose
// work overlaps on the GPU (different streams, or different contexts on one device) race
// on it and must be ordered by the caller.
#include <mutex>

#include "stdg_internal.h"

namespace stdg {
namespace {

constexpr int kParts = 65536;          // partial sums per quantity
constexpr int kChunk = 4096;           // vector entries per partial sum (one block)
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_residual_scratch[2 * kParts];

std::mutex g_mutex;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of g_residual_scratch on the current device, looked up once per device.
int scratch_address(stdg_ctx* c, double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        c->err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return STDG_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        c->err = "device ordinal out of range for the residual scratch table";
        return STDG_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_residual_scratch);
        if (e != cudaSuccess || !p) {
            c->err = std::string("cudaGetSymbolAddress(residual scratch): ") + cudaGetErrorString(e);
            return STDG_ECUDA;
        }
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return STDG_OK;
}

__device__ __forceinline__ double block_total(double v) {
    __shared__ double red[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kThreads / 32; ++i) s += red[i];
    return s;
}

// r holds A x on entry and b - A x on exit; block k owns entries [k*kChunk, (k+1)*kChunk).
__global__ void __launch_bounds__(kThreads) residual_parts_kernel(int64_t n, const double* __restrict__ b,
                                                                  double* __restrict__ r, double* __restrict__ parts) {
    const int64_t lo = (int64_t)blockIdx.x * kChunk;
    const int64_t hi = lo + kChunk < n ? lo + kChunk : n;
    double rr = 0, bb = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kThreads) {
        const double ri = b[i] - r[i];
        r[i] = ri;
        rr += ri * ri;
        bb += b[i] * b[i];
    }
    const double s1 = block_total(rr);
    const double s2 = block_total(bb);
    if (threadIdx.x == 0) {
        parts[blockIdx.x] = s1;
        parts[kParts + blockIdx.x] = s2;
    }
}

// out[0] = ||b - A x|| / ||b|| (or ||b - A x|| when b = 0), out[1] = ||b - A x||
__global__ void __launch_bounds__(kThreads) residual_total_kernel(int nparts, const double* __restrict__ parts,
                                                                  double* __restrict__ out) {
    double rr = 0, bb = 0;
    for (int i = threadIdx.x; i < nparts; i += kThreads) {
        rr += parts[i];
        bb += parts[kParts + i];
    }
    const double s1 = block_total(rr);
    const double s2 = block_total(bb);
    if (threadIdx.x == 0) {
        const double rn = sqrt(s1), bn = sqrt(s2);
        out[0] = bn > 0.0 ? rn / bn : rn;
        out[1] = rn;
    }
}

}  // namespace
}  // namespace stdg

using namespace stdg;

extern "C" int stdg_residual_noalloc(stdg_ctx* c, double dt, const double* x_dev, const double* b_dev, double* r_dev,
                                     double* out_dev) {
    if (!c) return STDG_EINVAL;
    if (!c->have_mesh || !c->have_material) STDG_FAIL(c, STDG_ESTATE, "call stdg_set_mesh and stdg_set_material first");
    if (!x_dev || !b_dev || !r_dev || !out_dev || !(dt > 0)) STDG_FAIL(c, STDG_EINVAL, "bad residual arguments");
    // A x is written into r while the operator still reads x, and the kernels take b and r
    // as non-aliasing pointers
    if (r_dev == x_dev || r_dev == b_dev) STDG_FAIL(c, STDG_EINVAL, "r_dev must differ from x_dev and b_dev");
    const int64_t n = c->nvel;
    if (n > (int64_t)kParts * kChunk)
        STDG_FAIL(c, STDG_EINVAL, "velocity vector of " + std::to_string(n) + " values exceeds the residual scratch limit of " +
                                      std::to_string((int64_t)kParts * kChunk));
    double* parts = nullptr;
    int rc = scratch_address(c, &parts);
    if (rc != STDG_OK) return rc;
    STDG_CUDA(c, launch_apply(c, dt, x_dev, r_dev, 1.0));
    const int nparts = (int)((n + kChunk - 1) / kChunk);
    residual_parts_kernel<<<nparts, kThreads, 0, c->stream>>>(n, b_dev, r_dev, parts);
    residual_total_kernel<<<1, kThreads, 0, c->stream>>>(nparts, parts, out_dev);
    STDG_CUDA(c, cudaGetLastError());
    return STDG_OK;
}
