// exx_static.cu -- the pair list without any device allocation.
//
// Some callers cannot call cudaMalloc: applications that hand all device
// memory to their own pool or arena (a framework's caching allocator, a
// service with a fixed per-process budget), where an allocation outside the
// pool breaks the budget or fails near the memory limit; and latency-bound
// loops that cannot afford cudaMalloc's implicit device synchronisation. For
// them, exx_pair_list_static builds the pair list of exx_compute with the very
// same count / scan / ordered-fill kernels (launch_pair_list_packed in
// exx_pairs.cu), its scratch in a file-scope __device__ array: the per-orbital
// pair counts, their prefix sums and the pair count. The caller passes the
// centres and the output buffer.
//
// The array is sized for kStaticMaxOrbitals orbitals. Every GPU that loads the
// library holds it (about 128 KiB) until the process exits. Every call uses the
// same array, and it keeps the previous call's contents. Each call writes every
// scratch word it reads before reading it, so nothing needs clearing. Calls that
// overlap on the GPU (two streams, or two host threads) race on the array and
// must be serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/exx.h"

namespace exx {
void set_global_error(const std::string& msg);  // defined in exx_api.cu
cudaError_t launch_pair_list_packed(int n, const double* centers, const double L[3], const double delta[3],
                                    const int N[3], double r_pair, int* scratch, int* out, int cap,
                                    cudaStream_t st);  // exx_pairs.cu
}

namespace {

constexpr int kStaticMaxOrbitals = 16384;
constexpr int kStaticMaxDevices = 64;

// counts [0, n), prefix sums [n, 2n + 1), pair count at 2n + 1, one spare word
static __device__ __align__(256) int g_static_scratch[2 * kStaticMaxOrbitals + 8];

std::mutex g_mu;
int* g_scratch_ptr[kStaticMaxDevices] = {nullptr};

exx_status static_fail(exx_status s, const std::string& msg) {
    exx::set_global_error(msg);
    return s;
}

exx_status static_cuda_fail(cudaError_t e, const char* where) {
    return static_fail(EXX_ECUDA, std::string("exx_pair_list_static: ") + where + ": " + cudaGetErrorString(e));
}

}  // namespace

extern "C" exx_status exx_pair_list_static(const double* centers, int n, const double cell[3], const int grid[3],
                                           double r_pair, int* pairs, int cap, int* n_pair, void* stream) {
    if (!centers || !cell || !grid || !pairs || !n_pair)
        return static_fail(EXX_EINVAL, "exx_pair_list_static: NULL argument");
    if (n < 1 || n > kStaticMaxOrbitals)
        return static_fail(EXX_EINVAL, "exx_pair_list_static: n must be in [1, 16384] (size of the static scratch)");
    if (cap < 0) return static_fail(EXX_EINVAL, "exx_pair_list_static: cap must be >= 0");
    if (!(r_pair > 0.0)) return static_fail(EXX_EINVAL, "exx_pair_list_static: r_pair must be > 0");
    double L[3], delta[3];
    int N[3];
    for (int a = 0; a < 3; ++a) {
        if (!(cell[a] > 0.0) || !std::isfinite(cell[a]) || grid[a] < 1)
            return static_fail(EXX_EINVAL, "exx_pair_list_static: invalid cell or grid");
        L[a] = cell[a];
        delta[a] = cell[a] / (double)grid[a];
        N[a] = grid[a];
    }

    // Set-up, once per device with that device current: the device address of
    // the scratch array (its name in host code is only a stand-in). The first
    // call on a device does this, so make that call before any stream capture.
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return static_cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kStaticMaxDevices) return static_fail(EXX_EINVAL, "exx_pair_list_static: device index too large");
    int* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess) return static_cuda_fail(e, "cudaGetSymbolAddress");
            g_scratch_ptr[dev] = static_cast<int*>(p);
        }
        scratch = g_scratch_ptr[dev];
    }

    cudaStream_t st = (cudaStream_t)stream;
    e = exx::launch_pair_list_packed(n, centers, L, delta, N, r_pair, scratch, pairs, cap, st);
    if (e != cudaSuccess) return static_cuda_fail(e, "kernel launch");
    int total = 0;
    e = cudaMemcpyAsync(&total, scratch + 2 * n + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return static_cuda_fail(e, "reading the pair count");
    *n_pair = total;
    if (total > cap)
        return static_fail(EXX_EINVAL, "exx_pair_list_static: more pairs than cap; only the first cap were written");
    return EXX_OK;
}
