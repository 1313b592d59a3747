// exx_static.cu -- the pair list without any device allocation.
//
// Some callers cannot call cudaMalloc. Examples: code that runs while a stream is
// being captured into a CUDA graph, where allocation is not permitted; hosts with
// a fixed device-memory budget or their own pool that forbids allocations
// outside it; and real-time loops that must not block in the allocator. For
// them, exx_pair_list_static builds the same pair list as exx_compute (the
// same count / scan / ordered-fill kernels and rounding) with its scratch in a
// file-scope __device__ array. The scratch is the per-orbital pair counts and
// their prefix sums. The caller passes the centres and the output buffer.
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
}

namespace {

constexpr int kStaticMaxOrbitals = 16384;
constexpr int kStaticMaxDevices = 64;

// [0, n): pair counts per orbital; [kStaticMaxOrbitals, +n+1): exclusive prefix sums.
static __device__ __align__(256) int g_static_scratch[2 * kStaticMaxOrbitals + 8];

std::mutex g_mu;
int* g_scratch_ptr[kStaticMaxDevices] = {nullptr};

struct StaticGeom {
    double L[3];
    double delta[3];
    int N[3];
    double r2cut;
};

__device__ __forceinline__ double minimg_s(double x, double L) {
    double t = __dadd_rn(__ddiv_rn(x, L), 0.5);
    return __dsub_rn(x, __dmul_rn(L, floor(t)));
}

__device__ __forceinline__ bool within_s(const double* __restrict__ C, int i, int j, const StaticGeom& G, double d[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = minimg_s(__dsub_rn(C[3 * j + a], C[3 * i + a]), G.L[a]);
    double d2 = __dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1]));
    d2 = __dadd_rn(d2, __dmul_rn(d[2], d[2]));
    return d2 < G.r2cut;
}

__global__ void static_count_kernel(int n, const double* __restrict__ C, StaticGeom G, int* __restrict__ scratch) {
    const int i = blockIdx.x;
    int cnt = 0;
    for (int j = i + threadIdx.x; j < n; j += blockDim.x) {
        double d[3];
        cnt += within_s(C, i, j, G, d) ? 1 : 0;
    }
    __shared__ int s[32];
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x < 32) {
        int t = threadIdx.x < (blockDim.x >> 5) ? s[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) scratch[i] = t;
    }
}

__global__ void static_scan_kernel(int n, int* __restrict__ scratch) {
    const int* counts = scratch;
    int* offsets = scratch + kStaticMaxOrbitals;
    __shared__ int s[1024];
    const int t = threadIdx.x;
    const int seg = (n + 1023) / 1024;
    const int b = t * seg, e = min(n, b + seg);
    int sum = 0;
    for (int k = b; k < e; ++k) sum += counts[k];
    s[t] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int v = t >= o ? s[t - o] : 0;
        __syncthreads();
        s[t] += v;
        __syncthreads();
    }
    int run = s[t] - sum;
    for (int k = b; k < e; ++k) {
        offsets[k] = run;
        run += counts[k];
    }
    if (t == 1023) offsets[n] = s[1023];
}

// Writes (i, j, g0, g1, g2) per pair at its list position; positions >= cap are skipped.
__global__ void static_fill_kernel(int n, const double* __restrict__ C, StaticGeom G, const int* __restrict__ scratch,
                                   int cap, int* __restrict__ out) {
    const int* offsets = scratch + kStaticMaxOrbitals;
    const int i = blockIdx.x;
    __shared__ int s_w[33];
    int base = offsets[i];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j0 = i; j0 < n; j0 += blockDim.x) {
        const int j = j0 + threadIdx.x;
        double d[3] = {0.0, 0.0, 0.0};
        const bool keep = j < n && within_s(C, i, j, G, d);
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) s_w[w] = __popc(m);
        __syncthreads();
        if (threadIdx.x == 0) {
            int run = 0;
            for (int k = 0; k < nw; ++k) {
                const int c = s_w[k];
                s_w[k] = run;
                run += c;
            }
            s_w[32] = run;
        }
        __syncthreads();
        if (keep) {
            const int pos = base + s_w[w] + __popc(m & ((1u << lane) - 1u));
            if (pos < cap) {
                int* rec = out + 5 * (long long)pos;
                rec[0] = i;
                rec[1] = j;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const double c = __dadd_rn(C[3 * i + a], __dmul_rn(0.5, d[a]));
                    const long long g = llround(__ddiv_rn(c, G.delta[a]));
                    const long long mm = g % G.N[a];
                    rec[2 + a] = (int)(mm < 0 ? mm + G.N[a] : mm);
                }
            }
        }
        base += s_w[32];
        __syncthreads();
    }
}

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
    StaticGeom G;
    for (int a = 0; a < 3; ++a) {
        if (!(cell[a] > 0.0) || !std::isfinite(cell[a]) || grid[a] < 1)
            return static_fail(EXX_EINVAL, "exx_pair_list_static: invalid cell or grid");
        G.L[a] = cell[a];
        G.delta[a] = cell[a] / (double)grid[a];
        G.N[a] = grid[a];
    }
    G.r2cut = r_pair * r_pair;

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
    static_count_kernel<<<n, 256, 0, st>>>(n, centers, G, scratch);
    static_scan_kernel<<<1, 1024, 0, st>>>(n, scratch);
    static_fill_kernel<<<n, 256, 0, st>>>(n, centers, G, scratch, cap, pairs);
    e = cudaGetLastError();
    if (e != cudaSuccess) return static_cuda_fail(e, "kernel launch");
    int total = 0;
    e = cudaMemcpyAsync(&total, scratch + kStaticMaxOrbitals + n, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return static_cuda_fail(e, "reading the pair count");
    *n_pair = total;
    if (total > cap)
        return static_fail(EXX_EINVAL, "exx_pair_list_static: more pairs than cap; only the first cap were written");
    return EXX_OK;
}
