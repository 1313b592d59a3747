// exx_probe.cu -- measured roofline denominator of the FP64 path.
//
// The plain FP64 CG is bound by the FP64 pipe, not by HBM: every point and
// iteration of the 19-point stencil and the CG updates issues about two dozen
// FP64 instructions against 48 bytes of algorithmic traffic, and the GB300
// issues FP64 at a small fraction of its FP32 rate. Its roofline therefore
// needs the device's FP64 FMA rate, which no data sheet gives for this part;
// this probe measures it. Every thread runs eight independent chains of
// dependent FMAs (enough chains to cover the pipe's latency), the grid fills
// every SM several times over, and the rate is 2 flops per FMA over the
// best of a few launches timed with CUDA events.
#include <cuda_runtime.h>

#include <string>

#include "../../include/exx.h"

namespace exx {
void set_global_error(const std::string& msg);  // exx_api.cu
}

namespace {

constexpr int kChains = 8;

__global__ void fp64_fma_probe_kernel(double* __restrict__ sink, int iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    // never true for the arguments the host passes; keeps the chains live
    if (s == -1.0) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

exx_status probe_fail(cudaError_t e, const char* where) {
    exx::set_global_error(std::string("exx_probe_fp64_rate: ") + where + ": " + cudaGetErrorString(e));
    return EXX_ECUDA;
}

}  // namespace

extern "C" exx_status exx_probe_fp64_rate(double* tflops, void* stream) {
    if (!tflops) {
        exx::set_global_error("exx_probe_fp64_rate: tflops is NULL");
        return EXX_EINVAL;
    }
    int dev = 0, n_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return probe_fail(e, "device query");
    cudaStream_t st = (cudaStream_t)stream;
    const int threads = 256, blocks = 8 * n_sm, iters = 2048;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return probe_fail(e, "cudaEventCreate");
    }
    double best_ms = 1e30;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch also loads the kernel
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) {
            fp64_fma_probe_kernel<<<blocks, threads, 0, st>>>(nullptr, iters, 0.9999999, 1e-7);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && ms < best_ms) best_ms = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return probe_fail(e, "probe launch");
    const double fmas = (double)blocks * threads * iters * kChains;
    *tflops = 2.0 * fmas / (best_ms * 1e-3) / 1e12;
    return EXX_OK;
}
