// exx_kernels.cuh -- device building blocks shared by the pair kernels.
#pragma once

#include "exx_internal.h"

namespace exx {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int warp_sum_int(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum (fixed butterfly order). red is a [2][33] shared
// buffer used alternately, so consecutive reductions need no trailing barrier.
template <int NT, typename T>
__device__ __forceinline__ T block_sum(T v, T (*red)[33], int& flip) {
    v = warp_sum(v);
    T* buf = red[flip];
    flip ^= 1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) buf[w] = v;
    __syncthreads();
    if (w == 0) {
        T t = lane < NT / 32 ? buf[lane] : T(0);
        t = warp_sum(t);
        if (lane == 0) buf[32] = t;
    }
    __syncthreads();
    return buf[32];
}

// lap f at cube index c: c0 f + sum_q c_q (f(+q) + f(-q)) along each axis (Eq. d2_1).
template <typename T>
__device__ __forceinline__ T lap19(const T* __restrict__ f, long long c, int S, long long S2,
                                   const Stencil<T>& st) {
    T acc = st.c0 * f[c];
#pragma unroll
    for (int q = 1; q <= 3; ++q) {
        acc = fma(st.cx[q - 1], f[c + q * S2] + f[c - q * S2], acc);
        acc = fma(st.cy[q - 1], f[c + (long long)q * S] + f[c - (long long)q * S], acc);
        acc = fma(st.cz[q - 1], f[c + q] + f[c - q], acc);
    }
    return acc;
}

__device__ __forceinline__ int off_x(int packed) { return (packed & 0xff) - 128; }
__device__ __forceinline__ int off_y(int packed) { return ((packed >> 8) & 0xff) - 128; }
__device__ __forceinline__ int off_z(int packed) { return ((packed >> 16) & 0xff) - 128; }

__device__ __forceinline__ int wrap(int g, int n) {
    g += (g < 0) ? n : 0;
    g -= (g >= n) ? n : 0;
    return g;
}

__device__ __forceinline__ long long grid_index(const int* N, const int* g, int packed) {
    int x = wrap(g[0] + off_x(packed), N[0]);
    int y = wrap(g[1] + off_y(packed), N[1]);
    int z = wrap(g[2] + off_z(packed), N[2]);
    return ((long long)x * N[1] + y) * N[2] + z;
}

// Where orbital orb keeps grid point g + o (o packed as in pt_off): the
// full-grid index, or with compact boxes its index in the orbital's box, or
// -1 when the point lies outside the box (the orbital is zero there).
__device__ __forceinline__ long long orb_index(const int* N, const int* g, int packed, const int* box_org,
                                              const int* bdim, int orb) {
    const int x = wrap(g[0] + off_x(packed), N[0]);
    const int y = wrap(g[1] + off_y(packed), N[1]);
    const int z = wrap(g[2] + off_z(packed), N[2]);
    if (!box_org) return ((long long)x * N[1] + y) * N[2] + z;
    const int bx = wrap(x - box_org[3 * orb], N[0]), by = wrap(y - box_org[3 * orb + 1], N[1]),
              bz = wrap(z - box_org[3 * orb + 2], N[2]);
    if (bx >= bdim[0] || by >= bdim[1] || bz >= bdim[2]) return -1;
    return ((long long)bx * bdim[1] + by) * bdim[2] + bz;
}

}  // namespace exx
