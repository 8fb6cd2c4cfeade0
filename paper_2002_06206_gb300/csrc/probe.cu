// probe.cu -- measured arithmetic rates of the GPU for the roofline reports: a kernel of independent
// fused multiply-add chains (no memory traffic) timed with CUDA events on the caller's stream.
#include "solver.cuh"

namespace {

#define PR_CHAINS 8          // independent chains per thread (hides the FMA latency)
#define PR_ITERS 4096        // FMAs per chain

template <class T>
__global__ void __launch_bounds__(256) k_fma_chains(T* out, T a, T b) {
    T x[PR_CHAINS];
#pragma unroll
    for (int c = 0; c < PR_CHAINS; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int it = 0; it < PR_ITERS; ++it) {
#pragma unroll
        for (int c = 0; c < PR_CHAINS; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < PR_CHAINS; ++c) s += x[c];
    if (s == (T)12345.678) out[0] = s;       // keeps the chains live; never true for these inputs
}

}  // namespace

extern "C" int ibm_probe_fma_rate(int32_t precision, double* tflops, void* stream) {
    if (!tflops || (precision != IBM_FP64 && precision != IBM_FP32_REFINE64))
        return ibm_fail(IBM_E_INVALID, "ibm_probe_fma_rate: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    IBM_CUDA(cudaGetDevice(&dev));
    IBM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const unsigned blocks = (unsigned)nsm * 8;
    void* out = nullptr;
    IBM_CUDA(cudaMallocAsync(&out, 16, s));
    cudaEvent_t e0, e1;
    IBM_CUDA(cudaEventCreate(&e0));
    IBM_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {           // the first launch warms up
        cudaEventRecord(e0, s);
        if (precision == IBM_FP64) k_fma_chains<double><<<blocks, 256, 0, s>>>((double*)out, 0.999999, 1e-7);
        else k_fma_chains<float><<<blocks, 256, 0, s>>>((float*)out, 0.999999f, 1e-7f);
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            cudaFreeAsync(out, s);
            return ibm_cuda_check(e, "ibm_probe_fma_rate");
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    IBM_CUDA(cudaFreeAsync(out, s));
    const double flops = 2.0 * (double)blocks * 256 * PR_CHAINS * PR_ITERS;
    *tflops = flops / (best * 1e-3) / 1e12;
    return IBM_OK;
}
