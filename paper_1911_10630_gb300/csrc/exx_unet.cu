// exx_unet.cu -- the learned CG warm start: a 3D U-Net that maps the pair
// density rho_ij on a cube around the pair centre to a guess of v_ij.
//
// The paper starts each CG from a guess and names better guesses as the way to
// fewer iterations (Sec. III.C Step IV and the conclusions); the network is
// this library's own addition. Four levels (widths 16/32/64/128), two 3x3x3
// convolutions per level with ReLU, 2x2x2 average pooling down, nearest
// up-sampling and concatenation with the skip tensor up, a 1x1x1 head.
// Activations and weights are BF16 in channels-last layout, accumulation FP32.
//
// The 3x3x3 convolutions (all but the 2-channel input layer) are implicit GEMMs
// on the tcgen05 tensor cores: one CTA computes a 16 (H) x 8 (W) x DT (D)
// output tile for all output channels, the input halo tile and the weights of
// one 16-channel chunk are staged in shared memory as 8-row core matrices, and
// each of the 27 taps is one MMA (M = 128 voxels, N = cout, K = 16) whose A
// operand is the same staged tile seen through a shifted descriptor. The
// accumulators live in tensor memory and are read back with tcgen05.ld for
// the bias / ReLU / mask epilogue.
#include "exx_unet.cuh"
#include "exx_unet_tc.cuh"
#include "exx_phases.cuh"  // the multipole constants (this unit's copy of c_mp)

#include <algorithm>
#include <cmath>
#include <cstring>

namespace exx {
namespace unet {

namespace {

constexpr int kTH = 16, kTW = 8, kHH = kTH + 2, kWW = kTW + 2;
constexpr int kWaitLimit = 1 << 22;

__device__ __forceinline__ float bf2f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ __nv_bfloat16 f2bf(float v) { return __float2bfloat16_rn(v); }

struct ConvArgs {
    const __nv_bfloat16* x;
    const __nv_bfloat16* wp;
    const float* bias;
    const __nv_bfloat16* mask;
    __nv_bfloat16* y;
    int B, D, H, W, cin, cout;
    int epi, DT, ncols, nbuf;
    int fold;  // the three depth taps of a (dh, dw) in one MMA of N = 3 cout (depth-shifted TMEM slices)
    int tiles_d, tiles_h, tiles_w;
    uint32_t itile, wtile, stage;
    int* err;
};

__global__ void __launch_bounds__(128) conv3_tc_kernel(const ConvArgs a) {
    extern __shared__ unsigned char smem_dyn[];
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t s_tmem;
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_dyn) + 127) & ~uintptr_t(127));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int t = blockIdx.x;
    const int tw = t % a.tiles_w;
    t /= a.tiles_w;
    const int th = t % a.tiles_h;
    t /= a.tiles_h;
    const int td = t % a.tiles_d;
    const int b = t / a.tiles_d;
    const int DT = a.DT;
    const int d0 = td * DT, h0 = th * kTH, w0 = tw * kTW;

    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        tc::mbar_init_fence();
    }
    if (warp == 0) tc::tmem_alloc(&s_tmem, (uint32_t)a.ncols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = s_tmem;
    if (a.fold) {  // every slice accumulates from several MMAs: start from zero
        for (int c0 = 0; c0 < a.ncols; c0 += 16) tc::tmem_st16_zero(tbase + ((uint32_t)(warp * 32) << 16) + c0);
        tc::tmem_wait_st();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }

    const int nch = a.cin / 16;
    const uint32_t idesc = tc::idesc_bf16_f32(128, a.fold ? 3 * a.cout : a.cout);
    const int nvox = (DT + 2) * kHH * kWW;
    bool ok = true;
    for (int c = 0; c < nch; ++c) {
        const int s = a.nbuf == 2 ? (c & 1) : 0;
        unsigned char* st = base + (size_t)s * a.stage;
        if (c >= a.nbuf) {  // the MMAs of chunk c - nbuf read this buffer
            const int prev = c - a.nbuf;
            if (!tc::mbar_wait(&mbar[s], (uint32_t)((prev / a.nbuf) & 1), kWaitLimit)) ok = false;
        }
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        // input halo tile: two channel octets, [DT+2][18][10] voxels x 16 B each
        for (int u = tid; u < 2 * nvox; u += 128) {
            const int o = u >= nvox ? 1 : 0;
            const int vx = u - o * nvox;
            const int wx = vx % kWW, r2 = vx / kWW, hy = r2 % kHH, dz = r2 / kHH;
            const int d = d0 - 1 + dz, h = h0 - 1 + hy, w = w0 - 1 + wx;
            const bool in = d >= 0 && d < a.D && h >= 0 && h < a.H && w >= 0 && w < a.W;
            const __nv_bfloat16* src =
                in ? a.x + ((((size_t)b * a.D + d) * a.H + h) * a.W + w) * a.cin + c * 16 + o * 8 : a.x;
            tc::cp_async16(st + (size_t)o * a.itile + (size_t)vx * 16, src, in ? 16u : 0u);
        }
        // weights of chunk c: [27][cout/8][2][8][8] BF16, contiguous
        const unsigned char* wsrc = reinterpret_cast<const unsigned char*>(a.wp) + (size_t)c * a.wtile;
        unsigned char* wdst = st + 2 * (size_t)a.itile;
        for (uint32_t u = tid; u < a.wtile / 16; u += 128) tc::cp_async16(wdst + u * 16, wsrc + u * 16, 16u);
        tc::cp_async_wait_all();
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t sa = tc::smem_addr(st), sw = tc::smem_addr(wdst);
            if (a.fold) {
                // input slice u (depth d0 - 1 + u) feeds the outputs tt = u - dz,
                // dz = 2, 1, 0: TMEM slices u .. u + 2 (slice = tt + 2), with the
                // weights of (dh, dw) packed as three N-blocks in that order
                for (int u = 0; u < DT + 2; ++u) {
#pragma unroll 1
                    for (int hw = 0; hw < 9; ++hw) {
                        const int dh = hw / 3, dw = hw % 3;
                        const uint32_t aoff = (uint32_t)(((u * kHH + dh) * kWW + dw) * 16);
                        const uint64_t ad = tc::sdesc(sa + aoff, a.itile, kWW * 16);
                        const uint64_t bd = tc::sdesc(sw + (uint32_t)(hw * 3 * a.cout * 32), 128, 256);
                        tc::mma_bf16(tbase + (uint32_t)(u * a.cout), ad, bd, idesc, 1u);
                    }
                }
            } else {
                for (int tt = 0; tt < DT; ++tt) {
#pragma unroll 1
                    for (int tap = 0; tap < 27; ++tap) {
                        const int dd = tap / 9, dh = (tap / 3) % 3, dw = tap % 3;
                        const uint32_t aoff = (uint32_t)((((tt + dd) * kHH + dh) * kWW + dw) * 16);
                        const uint64_t ad = tc::sdesc(sa + aoff, a.itile, kWW * 16);
                        const uint64_t bd = tc::sdesc(sw + (uint32_t)(tap * a.cout * 32), 128, 256);
                        tc::mma_bf16(tbase + (uint32_t)(tt * a.cout), ad, bd, idesc, (c > 0 || tap > 0) ? 1u : 0u);
                    }
                }
            }
            tc::commit(&mbar[s]);
        }
    }
    if (ok) {
        const int last = nch - 1, s = a.nbuf == 2 ? (last & 1) : 0;
        if (!tc::mbar_wait(&mbar[s], (uint32_t)((last / a.nbuf) & 1), kWaitLimit)) ok = false;
    }
    ok = __syncthreads_and(ok);
    tc::fence_after_sync();
    if (ok) {
        const int m = warp * 32 + lane;  // accumulator row = TMEM lane
        const int h = h0 + (m >> 3), w = w0 + (m & 7);
        for (int tt = 0; tt < DT; ++tt) {
            const int d = d0 + tt;
            const bool live = d < a.D && h < a.H && w < a.W;
            const size_t vox = (((size_t)b * a.D + d) * a.H + h) * a.W + w;
            for (int c0 = 0; c0 < a.cout; c0 += 16) {
                float v[16];
                tc::tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)((tt + (a.fold ? 2 : 0)) * a.cout + c0),
                              v);
                if (!live) continue;
                if (a.bias) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) v[k] += a.bias[c0 + k];
                }
                if (a.epi == 1) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) v[k] = fmaxf(v[k], 0.0f);
                } else if (a.epi == 2) {
                    const uint4* mp = reinterpret_cast<const uint4*>(a.mask + vox * a.cout + c0);
                    uint4 mm[2] = {mp[0], mp[1]};
                    const __nv_bfloat16* mb = reinterpret_cast<const __nv_bfloat16*>(mm);
#pragma unroll
                    for (int k = 0; k < 16; ++k) v[k] = bf2f(mb[k]) > 0.0f ? v[k] : 0.0f;
                }
                uint4 o[2];
                __nv_bfloat16* ob = reinterpret_cast<__nv_bfloat16*>(o);
#pragma unroll
                for (int k = 0; k < 16; ++k) ob[k] = f2bf(v[k]);
                uint4* yp = reinterpret_cast<uint4*>(a.y + vox * a.cout + c0);
                yp[0] = o[0];
                yp[1] = o[1];
            }
        }
    } else if (tid == 0) {
        atomicExch(a.err, 1);
        // let MMAs still in flight finish before the tensor memory goes back
        tc::mbar_wait(&mbar[0], 0, 1024);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tbase, (uint32_t)a.ncols);
}

// ---- packing ---------------------------------------------------------------

// Packed operand: [K/16][27][N/8][2][8 n][8 k], k = 16 chunk + 8 half + e.
// Forward: K = cin, N = cout, value W[tap][k][n]. Data gradient (flip): the
// convolution maps cout -> cin channels, K = cout, N = cin, value
// W[26 - tap][n][k]. Depth-folded (fold): the 27 slots of a chunk are taken
// as [9 (dh, dw)][3], slot 3 hw + b holding the tap of depth offset dz = 2 - b.
__global__ void pack_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ wp, int cin, int cout,
                            int flip, int fold) {
    const int K = flip ? cout : cin, N = flip ? cin : cout;
    const long long total = 27LL * K * N;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        long long r = idx;
        const int e = (int)(r % 8);
        r /= 8;
        const int nl = (int)(r % 8);
        r /= 8;
        const int half = (int)(r % 2);
        r /= 2;
        const int ng = (int)(r % (N / 8));
        r /= (N / 8);
        const int slot = (int)(r % 27);
        const int tap = fold ? (2 - slot % 3) * 9 + slot / 3 : slot;
        const int chunk = (int)(r / 27);
        const int k = chunk * 16 + half * 8 + e, n = ng * 8 + nl;
        const float v = flip ? w[((size_t)(26 - tap) * cin + n) * cout + k] : w[((size_t)tap * cin + k) * cout + n];
        wp[idx] = f2bf(v);
    }
}

// ---- CUDA-core layers ------------------------------------------------------

// Input layer: kIn FP32 channels -> 16, ReLU. One thread per output voxel.
__global__ void conv_first_kernel(const float* __restrict__ in, const float* __restrict__ w,
                                  const float* __restrict__ bias, __nv_bfloat16* __restrict__ y, int B, int S) {
    constexpr int CI = kCin[0];
    __shared__ float ws[27 * CI * 16 + 16];
    for (int i = threadIdx.x; i < 27 * CI * 16; i += blockDim.x) ws[i] = w[i];
    if (threadIdx.x < 16) ws[27 * CI * 16 + threadIdx.x] = bias[threadIdx.x];
    __syncthreads();
    const long long nv = (long long)B * S * S * S;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv;
         v += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(v % S), yy = (int)((v / S) % S), z = (int)((v / ((long long)S * S)) % S);
        const long long bb = v / ((long long)S * S * S);
        float acc[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[c] = ws[27 * CI * 16 + c];
        for (int tap = 0; tap < 27; ++tap) {
            const int zz = z + tap / 9 - 1, y2 = yy + (tap / 3) % 3 - 1, x2 = x + tap % 3 - 1;
            if (zz < 0 || zz >= S || y2 < 0 || y2 >= S || x2 < 0 || x2 >= S) continue;
            const float* iv = in + (((bb * S + zz) * S + y2) * S + x2) * CI;
#pragma unroll
            for (int ci = 0; ci < CI; ++ci) {
                const float a = iv[ci];
#pragma unroll
                for (int c = 0; c < 16; ++c) acc[c] = fmaf(a, ws[(tap * CI + ci) * 16 + c], acc[c]);
            }
        }
        uint4 o[2];
        __nv_bfloat16* ob = reinterpret_cast<__nv_bfloat16*>(o);
#pragma unroll
        for (int c = 0; c < 16; ++c) ob[c] = f2bf(fmaxf(acc[c], 0.0f));
        uint4* yp = reinterpret_cast<uint4*>(y + v * 16);
        yp[0] = o[0];
        yp[1] = o[1];
    }
}

// 1x1x1 head: out = b + sum_c y0[c] w[c] (FP32).
__global__ void head_kernel(const __nv_bfloat16* __restrict__ y0, const float* __restrict__ hw, float* __restrict__ out,
                            long long nv) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv;
         v += (long long)gridDim.x * blockDim.x) {
        const uint4* p = reinterpret_cast<const uint4*>(y0 + v * 16);
        uint4 q[2] = {p[0], p[1]};
        const __nv_bfloat16* qb = reinterpret_cast<const __nv_bfloat16*>(q);
        float acc = hw[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) acc = fmaf(bf2f(qb[c]), hw[c], acc);
        out[v] = acc;
    }
}

// Loss L = sum_v m_v (out_v - t_v)^2 / (B S^3), m_v = input mask channel; the
// head's gradients, and the gradient at y0 masked by ReLU (y0 > 0). Each block
// writes its partial sums (16 weights, bias, loss) to part[block][18]; they are
// added in block order by reduce_parts_kernel, so the result does not depend
// on the order in which blocks run.
__global__ void head_backward_kernel(const float* __restrict__ in, const float* __restrict__ target,
                                     const float* __restrict__ out, const __nv_bfloat16* __restrict__ y0,
                                     const float* __restrict__ hw, __nv_bfloat16* __restrict__ g_y0,
                                     float* __restrict__ part, long long nv, float inv_n) {
    __shared__ float red[17][8];
    float lsum = 0.0f, gw[17];
#pragma unroll
    for (int c = 0; c < 17; ++c) gw[c] = 0.0f;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv;
         v += (long long)gridDim.x * blockDim.x) {
        const float m = in[kIn * v + kMaskChannel] > 0.5f ? 1.0f : 0.0f;
        const float diff = out[v] - target[v];
        lsum += m * diff * diff;
        const float g = 2.0f * m * diff * inv_n;
        const uint4* p = reinterpret_cast<const uint4*>(y0 + v * 16);
        uint4 q[2] = {p[0], p[1]};
        const __nv_bfloat16* qb = reinterpret_cast<const __nv_bfloat16*>(q);
        uint4 o[2];
        __nv_bfloat16* ob = reinterpret_cast<__nv_bfloat16*>(o);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const float yv = bf2f(qb[c]);
            gw[c] = fmaf(g, yv, gw[c]);
            ob[c] = f2bf(yv > 0.0f ? g * hw[c] : 0.0f);
        }
        gw[16] += g;
        uint4* gp = reinterpret_cast<uint4*>(g_y0 + v * 16);
        gp[0] = o[0];
        gp[1] = o[1];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 17; ++c) {
        float s = gw[c];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[c][wid] = s;
    }
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    __shared__ float lred[8];
    if (lane == 0) lred[wid] = lsum;
    __syncthreads();
    float* mine = part + (size_t)blockIdx.x * 18;
    if (threadIdx.x < 17) {
        float s = 0.0f;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[threadIdx.x][k];
        mine[threadIdx.x] = s;
    }
    if (threadIdx.x == 32) {
        float s = 0.0f;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += lred[k];
        mine[17] = s * inv_n;
    }
}

// out[i] = sum over s = 0 .. n_parts - 1 of part[s * stride + i], in that order
// (the fixed-order second stage of every gradient and loss reduction).
__global__ void reduce_parts_kernel(const float* __restrict__ part, int n_parts, long long stride, int count,
                                    float* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int k = 0; k < n_parts; ++k) s += part[(size_t)k * stride + i];
        out[i] = s;
    }
}

// 2x2x2 average pooling, channels last; one thread per (coarse voxel, 8 channels).
__global__ void pool_kernel(const __nv_bfloat16* __restrict__ x, __nv_bfloat16* __restrict__ y, int B, int S, int C) {
    const int s = S / 2, g8 = C / 8;
    const long long total = (long long)B * s * s * s * g8;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(i % g8);
        long long p = i / g8;
        const int px = (int)(p % s), py = (int)((p / s) % s), pz = (int)((p / ((long long)s * s)) % s);
        const long long bb = p / ((long long)s * s * s);
        float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int k = 0; k < 8; ++k) {
            const long long v = ((bb * S + 2 * pz + (k >> 2)) * S + 2 * py + ((k >> 1) & 1)) * S + 2 * px + (k & 1);
            const uint4 q = *reinterpret_cast<const uint4*>(x + v * C + g * 8);
            const __nv_bfloat16* qb = reinterpret_cast<const __nv_bfloat16*>(&q);
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] += bf2f(qb[c]);
        }
        uint4 o;
        __nv_bfloat16* ob = reinterpret_cast<__nv_bfloat16*>(&o);
#pragma unroll
        for (int c = 0; c < 8; ++c) ob[c] = f2bf(0.125f * acc[c]);
        *reinterpret_cast<uint4*>(y + p * C + g * 8) = o;
    }
}

// cat[v] = (low[parent(v)], skip[v]); fine side S, low has Cl channels, skip Cs.
__global__ void upcat_kernel(const __nv_bfloat16* __restrict__ low, const __nv_bfloat16* __restrict__ skip,
                             __nv_bfloat16* __restrict__ cat, int B, int S, int Cl, int Cs) {
    const int C = Cl + Cs, g8 = C / 8, s = S / 2;
    const long long total = (long long)B * S * S * S * g8;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(i % g8);
        const long long v = i / g8;
        const int x = (int)(v % S), y = (int)((v / S) % S), z = (int)((v / ((long long)S * S)) % S);
        const long long bb = v / ((long long)S * S * S);
        uint4 q;
        if (g * 8 < Cl) {
            const long long p = ((bb * s + z / 2) * s + y / 2) * s + x / 2;
            q = *reinterpret_cast<const uint4*>(low + p * Cl + g * 8);
        } else {
            q = *reinterpret_cast<const uint4*>(skip + v * Cs + g * 8 - Cl);
        }
        *reinterpret_cast<uint4*>(cat + v * C + g * 8) = q;
    }
}

// Gradient at the up-sampled input: dlow[p] = sum over the 8 children of
// dcat[child][0:Cl], masked by ReLU (low > 0).
__global__ void upcat_back_low_kernel(const __nv_bfloat16* __restrict__ dcat, const __nv_bfloat16* __restrict__ low,
                                      __nv_bfloat16* __restrict__ dlow, int B, int S, int Cl, int Cs) {
    const int C = Cl + Cs, s = S / 2, g8 = Cl / 8;
    const long long total = (long long)B * s * s * s * g8;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(i % g8);
        const long long p = i / g8;
        const int px = (int)(p % s), py = (int)((p / s) % s), pz = (int)((p / ((long long)s * s)) % s);
        const long long bb = p / ((long long)s * s * s);
        float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int k = 0; k < 8; ++k) {
            const long long v = ((bb * S + 2 * pz + (k >> 2)) * S + 2 * py + ((k >> 1) & 1)) * S + 2 * px + (k & 1);
            const uint4 q = *reinterpret_cast<const uint4*>(dcat + v * C + g * 8);
            const __nv_bfloat16* qb = reinterpret_cast<const __nv_bfloat16*>(&q);
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] += bf2f(qb[c]);
        }
        const uint4 lq = *reinterpret_cast<const uint4*>(low + p * Cl + g * 8);
        const __nv_bfloat16* lb = reinterpret_cast<const __nv_bfloat16*>(&lq);
        uint4 o;
        __nv_bfloat16* ob = reinterpret_cast<__nv_bfloat16*>(&o);
#pragma unroll
        for (int c = 0; c < 8; ++c) ob[c] = f2bf(bf2f(lb[c]) > 0.0f ? acc[c] : 0.0f);
        *reinterpret_cast<uint4*>(dlow + p * Cl + g * 8) = o;
    }
}

// Gradient at a skip tensor: from the pooling (dpool[parent] / 8) and from the
// concatenation (dcat[v][Cl:]), masked by ReLU (skip > 0).
__global__ void skip_back_kernel(const __nv_bfloat16* __restrict__ dpool, const __nv_bfloat16* __restrict__ dcat,
                                 const __nv_bfloat16* __restrict__ skip, __nv_bfloat16* __restrict__ dskip, int B,
                                 int S, int Cl, int Cs) {
    const int C = Cl + Cs, s = S / 2, g8 = Cs / 8;
    const long long total = (long long)B * S * S * S * g8;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(i % g8);
        const long long v = i / g8;
        const int x = (int)(v % S), y = (int)((v / S) % S), z = (int)((v / ((long long)S * S)) % S);
        const long long bb = v / ((long long)S * S * S);
        const long long p = ((bb * s + z / 2) * s + y / 2) * s + x / 2;
        const uint4 a = *reinterpret_cast<const uint4*>(dpool + p * Cs + g * 8);
        const uint4 c = *reinterpret_cast<const uint4*>(dcat + v * C + Cl + g * 8);
        const uint4 k = *reinterpret_cast<const uint4*>(skip + v * Cs + g * 8);
        const __nv_bfloat16 *ab = reinterpret_cast<const __nv_bfloat16*>(&a),
                            *cb = reinterpret_cast<const __nv_bfloat16*>(&c),
                            *kb = reinterpret_cast<const __nv_bfloat16*>(&k);
        uint4 o;
        __nv_bfloat16* ob = reinterpret_cast<__nv_bfloat16*>(&o);
#pragma unroll
        for (int e = 0; e < 8; ++e) ob[e] = f2bf(bf2f(kb[e]) > 0.0f ? 0.125f * bf2f(ab[e]) + bf2f(cb[e]) : 0.0f);
        *reinterpret_cast<uint4*>(dskip + v * Cs + g * 8) = o;
    }
}

// Weight gradient of a 3x3x3 layer, dW[tap][ci][co] = sum over samples and
// voxels of x[v + tap - 1][ci] g[v][co], all 27 taps in one block: the block
// stages a voxel tile of one sample (4 x 4 x 8 voxels: a 6 x 6 x 10 halo of x
// and the tile of g, one 16-channel block of each, in FP32) once, and thread
// (tap, ci) adds x[v + tap - 1][ci] g[v][0..15] for every voxel of the tile:
// one x value and a broadcast row of g (every thread of the block reads the
// same g row) per 16 FMAs. Thread (centre tap, ci 0) of the first ci block also
// sums g for the bias gradient. Grid: x = voxel-tile split (split s takes the
// tiles [s T / nsplit, (s + 1) T / nsplit)), y = ci block, z = co block; each
// split writes its partial sums to its own slice of part ([split][27 cin cout +
// cout]), which reduce_parts_kernel adds in split order.
constexpr int kDwD = 4, kDwH = 4, kDwW = 8, kDwVox = kDwD * kDwH * kDwW;
constexpr int kDwHD = kDwD + 2, kDwHH = kDwH + 2, kDwHW = kDwW + 2, kDwHalo = kDwHD * kDwHH * kDwHW;
constexpr int kDwThreads = 448;  // 27 taps x 16 ci = 432 accumulate; all stage

__global__ void __launch_bounds__(kDwThreads) dw_kernel(const __nv_bfloat16* __restrict__ x,
                                                        const __nv_bfloat16* __restrict__ g,
                                                        float* __restrict__ part, int B, int S, int cin, int cout,
                                                        int nsplit) {
    __shared__ float xs[kDwHalo][17];
    __shared__ __align__(16) float gs[kDwVox][16];
    const int cib = blockIdx.y, cob = blockIdx.z, split = blockIdx.x;
    const int tid = threadIdx.x;
    const int tap = tid >> 4, ci = tid & 15;
    const bool acc_thread = tid < 27 * 16;
    const bool bias_thread = cib == 0 && tap == 13 && ci == 0;
    const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;  // halo offsets of the tap
    const int td = (S + kDwD - 1) / kDwD, th = (S + kDwH - 1) / kDwH, tw = (S + kDwW - 1) / kDwW;
    const long long T = (long long)B * td * th * tw;
    const long long t0 = T * split / nsplit, t1 = T * (split + 1) / nsplit;
    float acc[16], bacc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = bacc[k] = 0.0f;
    for (long long t = t0; t < t1; ++t) {
        long long r = t;
        const int iw = (int)(r % tw);
        r /= tw;
        const int ih = (int)(r % th);
        r /= th;
        const int id = (int)(r % td);
        const int b = (int)(r / td);
        const int d0 = id * kDwD, h0 = ih * kDwH, w0 = iw * kDwW;
        __syncthreads();  // the previous tile's values are no longer read
        // stage: x halo (each item: 8 channels of one voxel) and the g tile
        for (int u = tid; u < 2 * kDwHalo + 2 * kDwVox; u += kDwThreads) {
            const bool isx = u < 2 * kDwHalo;
            const int uu = isx ? u : u - 2 * kDwHalo;
            const int half = uu & 1, vx = uu >> 1;
            int d, h, w;
            if (isx) {
                d = d0 - 1 + vx / (kDwHH * kDwHW);
                h = h0 - 1 + (vx / kDwHW) % kDwHH;
                w = w0 - 1 + vx % kDwHW;
            } else {
                d = d0 + vx / (kDwH * kDwW);
                h = h0 + (vx / kDwW) % kDwH;
                w = w0 + vx % kDwW;
            }
            float v8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (d >= 0 && d < S && h >= 0 && h < S && w >= 0 && w < S) {
                const long long vox = (((long long)b * S + d) * S + h) * S + w;
                const uint4 q = isx ? *reinterpret_cast<const uint4*>(x + vox * cin + cib * 16 + half * 8)
                                    : *reinterpret_cast<const uint4*>(g + vox * cout + cob * 16 + half * 8);
                const __nv_bfloat16* qb = reinterpret_cast<const __nv_bfloat16*>(&q);
#pragma unroll
                for (int e = 0; e < 8; ++e) v8[e] = bf2f(qb[e]);
            }
            float* dst = isx ? &xs[vx][half * 8] : &gs[vx][half * 8];
#pragma unroll
            for (int e = 0; e < 8; ++e) dst[e] = v8[e];
        }
        __syncthreads();
        if (acc_thread) {
            // row by row of the tile: the tap's halo row, then 8 voxels along w
            for (int vd = 0; vd < kDwD; ++vd)
                for (int vh = 0; vh < kDwH; ++vh) {
                    const float* xrow = &xs[((vd + dz) * kDwHH + (vh + dy)) * kDwHW + dx][ci];
                    const float4* grow = reinterpret_cast<const float4*>(gs[(vd * kDwH + vh) * kDwW]);
#pragma unroll
                    for (int vw = 0; vw < kDwW; ++vw) {
                        const float xv = xrow[vw * 17];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float4 gq = grow[vw * 4 + q];
                            acc[4 * q + 0] = fmaf(xv, gq.x, acc[4 * q + 0]);
                            acc[4 * q + 1] = fmaf(xv, gq.y, acc[4 * q + 1]);
                            acc[4 * q + 2] = fmaf(xv, gq.z, acc[4 * q + 2]);
                            acc[4 * q + 3] = fmaf(xv, gq.w, acc[4 * q + 3]);
                            if (bias_thread) {
                                bacc[4 * q + 0] += gq.x;
                                bacc[4 * q + 1] += gq.y;
                                bacc[4 * q + 2] += gq.z;
                                bacc[4 * q + 3] += gq.w;
                            }
                        }
                    }
                }
        }
    }
    if (acc_thread) {
        float* dw = part + (size_t)split * ((size_t)27 * cin * cout + cout);
        float* row = dw + ((size_t)tap * cin + cib * 16 + ci) * cout + cob * 16;
#pragma unroll
        for (int k = 0; k < 16; ++k) row[k] = acc[k];
        if (bias_thread) {
#pragma unroll
            for (int k = 0; k < 16; ++k) dw[(size_t)27 * cin * cout + cob * 16 + k] = bacc[k];
        }
    }
}

// Weight gradient of the FP32 input layer: 27 x kIn x 16 weights and 16
// biases; voxels split over blocks, each block's partial sums in
// part[block][27 * kIn * 16 + 16] (added in block order afterwards).
__global__ void dw_first_kernel(const float* __restrict__ in, const __nv_bfloat16* __restrict__ g,
                                float* __restrict__ part, int B, int S, int nsplit) {
    constexpr int CI = kCin[0], NW = 27 * CI * 16;
    const long long nv = (long long)B * S * S * S;
    const long long per = (nv + nsplit - 1) / nsplit;
    const long long v0 = blockIdx.x * per, v1 = v0 + per < nv ? v0 + per : nv;
    for (int t = threadIdx.x; t < NW + 16; t += blockDim.x) {
        float acc = 0.0f;
        if (t < NW) {
            const int tap = t / (CI * 16), ci = (t / 16) % CI, co = t % 16;
            const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
            for (long long v = v0; v < v1; ++v) {
                const int xx = (int)(v % S), yy = (int)((v / S) % S), zz = (int)((v / ((long long)S * S)) % S);
                const long long bb = v / ((long long)S * S * S);
                const int z2 = zz + dz, y2 = yy + dy, x2 = xx + dx;
                if (z2 < 0 || z2 >= S || y2 < 0 || y2 >= S || x2 < 0 || x2 >= S) continue;
                const long long u = ((bb * S + z2) * S + y2) * S + x2;
                acc = fmaf(in[CI * u + ci], bf2f(g[v * 16 + co]), acc);
            }
        } else {
            const int co = t - NW;
            for (long long v = v0; v < v1; ++v) acc += bf2f(g[v * 16 + co]);
        }
        part[(size_t)blockIdx.x * (NW + 16) + t] = acc;
    }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

__global__ void zero_f32_kernel(float* p, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = 0.0f;
}

int grid_for(long long n, int n_sm) {
    long long g = (n + 255) / 256;
    const long long cap = 16LL * n_sm;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

#define UCK(x)                            \
    do {                                  \
        cudaError_t e_ = (x);             \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

}  // namespace

size_t param_offset(int layer) {
    size_t off = 0;
    for (int l = 0; l < layer; ++l)
        off += (l == kHead ? (size_t)kCin[l] : (size_t)27 * kCin[l]) * kCout[l] + kCout[l];
    return off;
}
size_t param_count() { return param_offset(kLayers); }

// Whether a convolution with n_out output channels folds its depth taps (one
// MMA of N = 3 n_out per (dh, dw)): N <= 256 and the depth-shifted TMEM slices
// of a tile within 256 columns (two CTAs per SM).
static bool conv_folds(int n_out) { return n_out <= 32; }

cudaError_t pack_weights(const float* w, __nv_bfloat16* wp, int cin, int cout, int flip, cudaStream_t st) {
    const long long total = 27LL * cin * cout;
    pack_kernel<<<(int)((total + 255) / 256), 256, 0, st>>>(w, wp, cin, cout, flip,
                                                            conv_folds(flip ? cin : cout) ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t conv3_tc(const __nv_bfloat16* x, const __nv_bfloat16* wp, const float* bias, const __nv_bfloat16* mask,
                     __nv_bfloat16* y, int B, int D, int H, int W, int cin, int cout, int epi, int* err, int n_sm,
                     cudaStream_t st) {
    (void)n_sm;
    if (cin % 16 || cout % 16 || cout < 16 || cout > 256 || B < 1) return cudaErrorInvalidValue;
    ConvArgs a;
    a.x = x;
    a.wp = wp;
    a.bias = bias;
    a.mask = mask;
    a.y = y;
    a.B = B;
    a.D = D;
    a.H = H;
    a.W = W;
    a.cin = cin;
    a.cout = cout;
    a.epi = epi;
    // Output depth per CTA: 4 D slices (fewer when the accumulators need more
    // than 512 TMEM columns). Deeper tiles reuse the staged halo tile more but
    // leave one CTA per SM whose 128 threads stage too slowly to keep the
    // tensor cores fed (measured slower on GB300); double-buffered chunks when
    // the input has more than one chunk and two stages fit.
    // Folded layers: 8 (16 outputs) or 4 (32 outputs) slices per tile, the
    // tile's DT + 4 accumulator slices (two of them on each side only collect
    // halo contributions) in at most 256 TMEM columns.
    a.fold = conv_folds(cout) ? 1 : 0;
    int DT = a.fold ? (cout <= 16 ? 8 : 4) : 4;
    while (!a.fold && DT > 1 && DT * cout > 512) --DT;
    if (DT > D) DT = D;
    const size_t stage_b = (size_t)2 * (DT + 2) * kHH * kWW * 16 + (size_t)27 * cout * 32;
    const int nbuf = (2 * stage_b + 128 <= 200 * 1024 && cin > 16) ? 2 : 1;
    if (DT < 1) return cudaErrorInvalidValue;
    a.DT = DT;
    int nc = 32;
    while (nc < (DT + (a.fold ? 4 : 0)) * cout) nc *= 2;
    a.ncols = nc;
    a.itile = (uint32_t)(DT + 2) * kHH * kWW * 16;
    a.wtile = 27u * (uint32_t)cout * 32u;
    a.stage = 2 * a.itile + a.wtile;
    a.nbuf = nbuf;
    a.tiles_w = (W + kTW - 1) / kTW;
    a.tiles_h = (H + kTH - 1) / kTH;
    a.tiles_d = (D + DT - 1) / DT;
    a.err = err;
    size_t smem = (size_t)a.nbuf * a.stage + 128;
    // keep (CTAs per SM) x (TMEM columns) within the 512 columns of an SM
    const size_t sm_bytes = 228 * 1024, per_cta_reserve = 1024 + 64;
    const int max_ctas = 512 / nc;
    if ((sm_bytes / (smem + per_cta_reserve)) > (size_t)max_ctas) smem = sm_bytes / max_ctas - per_cta_reserve + 1;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    UCK(cudaFuncSetAttribute(conv3_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long long nblk = (long long)a.tiles_w * a.tiles_h * a.tiles_d * B;
    if (nblk > 0x7fffffffLL) return cudaErrorInvalidValue;
    conv3_tc_kernel<<<(unsigned)nblk, 128, smem, st>>>(a);
    return cudaGetLastError();
}

// ---- network driver --------------------------------------------------------

// Voxel-tile splits of a weight-gradient launch: about eight blocks per SM
// over the (ci, co) blocks, and no split without a tile.
static int dw_splits(int B, int S, int cin, int cout, int n_sm) {
    const long long tiles = (long long)B * ((S + kDwD - 1) / kDwD) * ((S + kDwH - 1) / kDwH) * ((S + kDwW - 1) / kDwW);
    const long long cb = (long long)(cin / 16) * (cout / 16);
    const long long want = std::max(1LL, 8LL * n_sm / cb);
    return (int)std::max(1LL, std::min(tiles, want));
}

cudaError_t create(Net& n, int S, int Bmax) {
    n.S = S;
    n.Bmax = Bmax;
    int dev = 0;
    UCK(cudaGetDevice(&dev));
    UCK(cudaDeviceGetAttribute(&n.n_sm, cudaDevAttrMultiProcessorCount, dev));
    n.nparam = param_count();
    auto alloc = [&](void** p, size_t bytes) -> cudaError_t {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) n.bufs.push_back(*p);
        return e;
    };
    UCK(alloc((void**)&n.params, n.nparam * 4));
    UCK(alloc((void**)&n.grads, n.nparam * 4));
    UCK(alloc((void**)&n.adam_m, n.nparam * 4));
    UCK(alloc((void**)&n.adam_v, n.nparam * 4));
    UCK(cudaMemset(n.adam_m, 0, n.nparam * 4));
    UCK(cudaMemset(n.adam_v, 0, n.nparam * 4));
    UCK(cudaMemset(n.params, 0, n.nparam * 4));
    for (int l = 1; l < kHead; ++l) {
        const size_t e = (size_t)27 * kCin[l] * kCout[l] * sizeof(__nv_bfloat16);
        UCK(alloc((void**)&n.wfwd[l], e));
        UCK(alloc((void**)&n.wbwd[l], e));
    }
    const size_t v0 = (size_t)Bmax * S * S * S, v1 = v0 / 8, v2 = v1 / 8, v3 = v2 / 8;
    auto act = [&](__nv_bfloat16** p, size_t vox, int C) { return alloc((void**)p, vox * C * 2); };
    UCK(act(&n.x0a, v0, 16));
    UCK(act(&n.x0, v0, 16));
    UCK(act(&n.p0, v1, 16));
    UCK(act(&n.x1a, v1, 32));
    UCK(act(&n.x1, v1, 32));
    UCK(act(&n.p1, v2, 32));
    UCK(act(&n.x2a, v2, 64));
    UCK(act(&n.x2, v2, 64));
    UCK(act(&n.p2, v3, 64));
    UCK(act(&n.x3a, v3, 128));
    UCK(act(&n.x3, v3, 128));
    UCK(act(&n.c2, v2, 192));
    UCK(act(&n.y2a, v2, 64));
    UCK(act(&n.y2, v2, 64));
    UCK(act(&n.c1, v1, 96));
    UCK(act(&n.y1a, v1, 32));
    UCK(act(&n.y1, v1, 32));
    UCK(act(&n.c0, v0, 48));
    UCK(act(&n.y0a, v0, 16));
    UCK(act(&n.y0, v0, 16));
    UCK(act(&n.g_y0, v0, 16));
    UCK(act(&n.g_y0a, v0, 16));
    UCK(act(&n.g_c0, v0, 48));
    UCK(act(&n.g_y1, v1, 32));
    UCK(act(&n.g_y1a, v1, 32));
    UCK(act(&n.g_c1, v1, 96));
    UCK(act(&n.g_y2, v2, 64));
    UCK(act(&n.g_y2a, v2, 64));
    UCK(act(&n.g_c2, v2, 192));
    UCK(act(&n.g_x3, v3, 128));
    UCK(act(&n.g_x3a, v3, 128));
    UCK(act(&n.g_p2, v3, 64));
    UCK(act(&n.g_x2, v2, 64));
    UCK(act(&n.g_x2a, v2, 64));
    UCK(act(&n.g_p1, v2, 32));
    UCK(act(&n.g_x1, v1, 32));
    UCK(act(&n.g_x1a, v1, 32));
    UCK(act(&n.g_p0, v1, 16));
    UCK(act(&n.g_x0, v0, 16));
    UCK(act(&n.g_x0a, v0, 16));
    UCK(alloc((void**)&n.out, v0 * 4));
    // partial sums of the gradient reductions: the largest of the head's
    // per-block sums, the input layer's and every 3x3x3 layer's per-split sums
    {
        size_t need = (size_t)18 * 16 * n.n_sm;
        need = std::max(need, (size_t)4 * n.n_sm * (27 * kIn * 16 + 16));
        const int lvl[kLayers] = {0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0, 0};
        for (int l = 1; l < kHead; ++l)
            need = std::max(need, (size_t)dw_splits(Bmax, S >> lvl[l], kCin[l], kCout[l], n.n_sm) *
                                      ((size_t)27 * kCin[l] * kCout[l] + kCout[l]));
        UCK(alloc((void**)&n.gpart, need * 4));
    }
    UCK(alloc((void**)&n.d_loss, 4));
    UCK(alloc((void**)&n.d_err, 4));
    UCK(cudaMemset(n.d_err, 0, 4));
    return cudaSuccess;
}

void destroy(Net& n) {
    for (void* p : n.bufs) cudaFree(p);
    n.bufs.clear();
}

cudaError_t pack(Net& n, cudaStream_t st) {
    for (int l = 1; l < kHead; ++l) {
        const float* w = n.params + param_offset(l);
        UCK(pack_weights(w, n.wfwd[l], kCin[l], kCout[l], 0, st));
        UCK(pack_weights(w, n.wbwd[l], kCin[l], kCout[l], 1, st));
    }
    n.packed = true;
    return cudaSuccess;
}

static const float* bias_of(const Net& n, int l) { return n.params + param_offset(l) + (size_t)27 * kCin[l] * kCout[l]; }

cudaError_t forward(Net& n, const float* in, int B, cudaStream_t st) {
    if (B < 1 || B > n.Bmax) return cudaErrorInvalidValue;
    if (!n.packed) UCK(pack(n, st));
    const int S = n.S, S1 = S / 2, S2 = S / 4, S3 = S / 8;
    const long long v0 = (long long)B * S * S * S, v1 = v0 / 8, v2 = v1 / 8, v3 = v2 / 8;
    auto conv = [&](const __nv_bfloat16* x, __nv_bfloat16* y, int l, int s) {
        return conv3_tc(x, n.wfwd[l], bias_of(n, l), nullptr, y, B, s, s, s, kCin[l], kCout[l], 1, n.d_err, n.n_sm,
                        st);
    };
    conv_first_kernel<<<grid_for(v0, n.n_sm), 256, 0, st>>>(in, n.params, bias_of(n, 0), n.x0a, B, S);
    UCK(cudaGetLastError());
    UCK(conv(n.x0a, n.x0, 1, S));
    pool_kernel<<<grid_for(v1 * 2, n.n_sm), 256, 0, st>>>(n.x0, n.p0, B, S, 16);
    UCK(conv(n.p0, n.x1a, 2, S1));
    UCK(conv(n.x1a, n.x1, 3, S1));
    pool_kernel<<<grid_for(v2 * 4, n.n_sm), 256, 0, st>>>(n.x1, n.p1, B, S1, 32);
    UCK(conv(n.p1, n.x2a, 4, S2));
    UCK(conv(n.x2a, n.x2, 5, S2));
    pool_kernel<<<grid_for(v3 * 8, n.n_sm), 256, 0, st>>>(n.x2, n.p2, B, S2, 64);
    UCK(conv(n.p2, n.x3a, 6, S3));
    UCK(conv(n.x3a, n.x3, 7, S3));
    upcat_kernel<<<grid_for(v2 * 24, n.n_sm), 256, 0, st>>>(n.x3, n.x2, n.c2, B, S2, 128, 64);
    UCK(conv(n.c2, n.y2a, 8, S2));
    UCK(conv(n.y2a, n.y2, 9, S2));
    upcat_kernel<<<grid_for(v1 * 12, n.n_sm), 256, 0, st>>>(n.y2, n.x1, n.c1, B, S1, 64, 32);
    UCK(conv(n.c1, n.y1a, 10, S1));
    UCK(conv(n.y1a, n.y1, 11, S1));
    upcat_kernel<<<grid_for(v0 * 6, n.n_sm), 256, 0, st>>>(n.y1, n.x0, n.c0, B, S, 32, 16);
    UCK(conv(n.c0, n.y0a, 12, S));
    UCK(conv(n.y0a, n.y0, 13, S));
    head_kernel<<<grid_for(v0, n.n_sm), 256, 0, st>>>(n.y0, n.params + param_offset(kHead), n.out, v0);
    return cudaGetLastError();
}

cudaError_t backward(Net& n, const float* in, const float* target, int B, cudaStream_t st) {
    const int S = n.S, S1 = S / 2, S2 = S / 4, S3 = S / 8;
    const long long v0 = (long long)B * S * S * S, v1 = v0 / 8, v2 = v1 / 8, v3 = v2 / 8;
    zero_f32_kernel<<<grid_for((long long)n.nparam, n.n_sm), 256, 0, st>>>(n.grads, (long long)n.nparam);
    {
        const int nblk = grid_for(v0, n.n_sm);
        float* ghw = n.grads + param_offset(kHead);
        head_backward_kernel<<<nblk, 256, 0, st>>>(in, target, n.out, n.y0, n.params + param_offset(kHead), n.g_y0,
                                                   n.gpart, v0, 1.0f / (float)v0);
        reduce_parts_kernel<<<1, 32, 0, st>>>(n.gpart, nblk, 18, 17, ghw);
        reduce_parts_kernel<<<1, 32, 0, st>>>(n.gpart + 17, nblk, 18, 1, n.d_loss);
    }
    UCK(cudaGetLastError());
    // data gradient through layer l: from g (cout channels) to cin channels,
    // masked by ReLU of the layer's input when that input is a ReLU output
    auto dconv = [&](const __nv_bfloat16* g, const __nv_bfloat16* xmask, __nv_bfloat16* dx, int l, int s) {
        return conv3_tc(g, n.wbwd[l], nullptr, xmask, dx, B, s, s, s, kCout[l], kCin[l], xmask ? 2 : 0, n.d_err,
                        n.n_sm, st);
    };
    auto dweight = [&](const __nv_bfloat16* x, const __nv_bfloat16* g, int l, int s) {
        const int nsplit = dw_splits(B, s, kCin[l], kCout[l], n.n_sm);
        dim3 grid(nsplit, kCin[l] / 16, kCout[l] / 16);
        const int count = 27 * kCin[l] * kCout[l] + kCout[l];
        dw_kernel<<<grid, kDwThreads, 0, st>>>(x, g, n.gpart, B, s, kCin[l], kCout[l], nsplit);
        reduce_parts_kernel<<<grid_for(count, n.n_sm), 256, 0, st>>>(n.gpart, nsplit, count, count,
                                                                     n.grads + param_offset(l));
        return cudaGetLastError();
    };
    // level 0, up path
    UCK(dweight(n.y0a, n.g_y0, 13, S));
    UCK(dconv(n.g_y0, n.y0a, n.g_y0a, 13, S));
    UCK(dweight(n.c0, n.g_y0a, 12, S));
    UCK(dconv(n.g_y0a, nullptr, n.g_c0, 12, S));
    upcat_back_low_kernel<<<grid_for(v1 * 4, n.n_sm), 256, 0, st>>>(n.g_c0, n.y1, n.g_y1, B, S, 32, 16);
    // level 1, up path
    UCK(dweight(n.y1a, n.g_y1, 11, S1));
    UCK(dconv(n.g_y1, n.y1a, n.g_y1a, 11, S1));
    UCK(dweight(n.c1, n.g_y1a, 10, S1));
    UCK(dconv(n.g_y1a, nullptr, n.g_c1, 10, S1));
    upcat_back_low_kernel<<<grid_for(v2 * 8, n.n_sm), 256, 0, st>>>(n.g_c1, n.y2, n.g_y2, B, S1, 64, 32);
    // level 2, up path
    UCK(dweight(n.y2a, n.g_y2, 9, S2));
    UCK(dconv(n.g_y2, n.y2a, n.g_y2a, 9, S2));
    UCK(dweight(n.c2, n.g_y2a, 8, S2));
    UCK(dconv(n.g_y2a, nullptr, n.g_c2, 8, S2));
    upcat_back_low_kernel<<<grid_for(v3 * 16, n.n_sm), 256, 0, st>>>(n.g_c2, n.x3, n.g_x3, B, S2, 128, 64);
    // bottleneck
    UCK(dweight(n.x3a, n.g_x3, 7, S3));
    UCK(dconv(n.g_x3, n.x3a, n.g_x3a, 7, S3));
    UCK(dweight(n.p2, n.g_x3a, 6, S3));
    UCK(dconv(n.g_x3a, nullptr, n.g_p2, 6, S3));
    // level 2, down path
    skip_back_kernel<<<grid_for(v2 * 8, n.n_sm), 256, 0, st>>>(n.g_p2, n.g_c2, n.x2, n.g_x2, B, S2, 128, 64);
    UCK(dweight(n.x2a, n.g_x2, 5, S2));
    UCK(dconv(n.g_x2, n.x2a, n.g_x2a, 5, S2));
    UCK(dweight(n.p1, n.g_x2a, 4, S2));
    UCK(dconv(n.g_x2a, nullptr, n.g_p1, 4, S2));
    // level 1, down path
    skip_back_kernel<<<grid_for(v1 * 4, n.n_sm), 256, 0, st>>>(n.g_p1, n.g_c1, n.x1, n.g_x1, B, S1, 64, 32);
    UCK(dweight(n.x1a, n.g_x1, 3, S1));
    UCK(dconv(n.g_x1, n.x1a, n.g_x1a, 3, S1));
    UCK(dweight(n.p0, n.g_x1a, 2, S1));
    UCK(dconv(n.g_x1a, nullptr, n.g_p0, 2, S1));
    // level 0, down path
    skip_back_kernel<<<grid_for(v0 * 2, n.n_sm), 256, 0, st>>>(n.g_p0, n.g_c0, n.x0, n.g_x0, B, S, 32, 16);
    UCK(dweight(n.x0a, n.g_x0, 1, S));
    UCK(dconv(n.g_x0, n.x0a, n.g_x0a, 1, S));
    {
        const int nsplit = 4 * n.n_sm;
        const int count = 27 * kIn * 16 + 16;
        dw_first_kernel<<<nsplit, 256, 0, st>>>(in, n.g_x0a, n.gpart, B, S, nsplit);
        reduce_parts_kernel<<<grid_for(count, n.n_sm), 256, 0, st>>>(n.gpart, nsplit, count, count,
                                                                     n.grads + param_offset(0));
    }
    return cudaGetLastError();
}

cudaError_t adam_step(Net& n, float lr, cudaStream_t st) {
    n.adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f / (1.0f - std::pow(b1, (float)n.adam_t));
    const float c2 = 1.0f / (1.0f - std::pow(b2, (float)n.adam_t));
    adam_kernel<<<grid_for((long long)n.nparam, n.n_sm), 256, 0, st>>>(n.params, n.grads, n.adam_m, n.adam_v,
                                                                      (long long)n.nparam, lr, b1, b2, 1e-8f, c1, c2);
    UCK(cudaGetLastError());
    return pack(n, st);
}

cudaError_t check_error(Net& n, cudaStream_t st) {
    int h = 0;
    UCK(cudaMemcpyAsync(&h, n.d_err, 4, cudaMemcpyDeviceToHost, st));
    UCK(cudaStreamSynchronize(st));
    return h ? cudaErrorLaunchTimeout : cudaSuccess;
}

}  // namespace unet
}  // namespace exx

namespace exx {
namespace unet {

// ---- pair samples ------------------------------------------------------------

namespace {


// Index of the Cartesian monomial x^a y^b z^c, l = a + b + c, in the
// library's order (degree ascending, then a descending, then b descending).
__host__ __device__ constexpr int mono_index(int a, int b, int c) {
    return (a + b + c) * (a + b + c + 1) * (a + b + c + 2) / 6 + (b + c) * (b + c + 1) / 2 + c;
}

// One network sample per pair (one CTA of 256 threads per pair):
//   channel 0: rho / s on the PE ball (s = max |rho| there), 0 elsewhere;
//   channel 1: on the cube outside the PE ball, the multipole expansion of
//     Eq. me evaluated from the moments of rho / s on the ball (Eq. mepole,
//     l <= lmax; FP32, Cartesian form with the library's K_l matrices), over
//     delta^2: the boundary values the solver imposes, in the target's units;
//   channel 2: the ball mask;
// and with vcache the target v / (s delta^2) on the ball.
__global__ void __launch_bounds__(256) sample_prep_kernel(const double* __restrict__ phi, int N0, int N1, int N2,
                                                          const PairRec* __restrict__ pairs, int k0, int S,
                                                          const BallGeo G, float* __restrict__ input,
                                                          float* __restrict__ scale, float* __restrict__ target,
                                                          const float* __restrict__ vcache, double d2, float dx,
                                                          float dy, float dz, float dV, int lmax,
                                                          const int* __restrict__ box_org, int3 bdim,
                                                          long long ostride) {
    constexpr int NM = kNMono;
    __shared__ double red[8];
    __shared__ float s_Mw[8][NM];
    __shared__ float s_M[NM], s_T[NM];
    const int k = k0 + blockIdx.x;
    const PairRec pr = pairs[k];
    const double* pi = phi + (long long)pr.i * ostride;
    const double* pj = phi + (long long)pr.j * ostride;
    const int N[3] = {N0, N1, N2}, bd[3] = {bdim.x, bdim.y, bdim.z};
    // rho at offset o of the pair's grid point (zero where o leaves a box)
    auto rho_at = [&](int ox, int oy, int oz) -> double {
        const int packed = (ox + 128) | ((oy + 128) << 8) | ((oz + 128) << 16);
        const long long ii = orb_index(N, pr.g, packed, box_org, bd, pr.i);
        const long long ij = orb_index(N, pr.g, packed, box_org, bd, pr.j);
        return (ii >= 0 && ij >= 0) ? pi[ii] * pj[ij] : 0.0;
    };
    const int R = G.r_pe, h = S / 2, S3 = S * S * S;
    double mx = 0.0;
    for (int v = threadIdx.x; v < S3; v += blockDim.x) {
        const int ox = v / (S * S) - h, oy = (v / S) % S - h, oz = v % S - h;
        if (ox * ox + oy * oy + oz * oz > R * R) continue;
        mx = fmax(mx, fabs(rho_at(ox, oy, oz)));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    double s = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) s = fmax(s, red[w]);
    if (!(s > 0.0)) s = 1.0;
    const double inv = 1.0 / s, tinv = 1.0 / (s * d2);
    float* in = input + (size_t)blockIdx.x * S3 * kIn;
    float* tg = target ? target + (size_t)blockIdx.x * S3 : nullptr;
    const float* vc = vcache ? vcache + (size_t)k * G.n_pe : nullptr;
    const int W = 2 * R + 1;
    for (int v = threadIdx.x; v < S3; v += blockDim.x) {
        const int ox = v / (S * S) - h, oy = (v / S) % S - h, oz = v % S - h;
        float r = 0.0f, m = 0.0f, t = 0.0f;
        if (ox * ox + oy * oy + oz * oz <= R * R) {
            r = (float)(rho_at(ox, oy, oz) * inv);
            m = 1.0f;
            if (tg && vc) {
                const RowRec Rw = G.rows_pe[G.row_of[(ox + R) * W + (oy + R)]];
                t = (float)(vc[Rw.pe_start + oz + Rw.zpe] * tinv);
            }
        }
        in[kIn * v] = r;
        in[kIn * v + 1] = 0.0f;
        in[kIn * v + kMaskChannel] = m;
        if (tg) tg[v] = t;
    }
    if (threadIdx.x == 0) scale[blockIdx.x] = (float)s;
    __syncthreads();

    // Moments M_abc = sum rho/s x^a y^b z^c dV over the ball points of the
    // cube: one thread per cube row (x, y), row sums S_c = sum_z rho/s z^c,
    // then every monomial; per-thread partials added in a fixed order.
    float M[NM];
#pragma unroll
    for (int q = 0; q < NM; ++q) M[q] = 0.0f;
    for (int row = threadIdx.x; row < S * S; row += blockDim.x) {
        const int ox = row / S - h, oy = row % S - h;
        const int rem = R * R - ox * ox - oy * oy;
        if (rem < 0) continue;
        int zr = (int)sqrtf((float)rem);
        while ((zr + 1) * (zr + 1) <= rem) ++zr;
        while (zr * zr > rem) --zr;
        const int zlo = max(-zr, -h), zhi = min(zr, h - 1);
        float sc[kLmaxMax + 1];
#pragma unroll
        for (int c = 0; c <= kLmaxMax; ++c) sc[c] = 0.0f;
        const float* rp = in + (size_t)row * S * kIn;
        for (int z = zlo; z <= zhi; ++z) {
            float p = rp[(z + h) * kIn];
            const float zz = (float)z * dz;
#pragma unroll
            for (int c = 0; c <= kLmaxMax; ++c) {
                sc[c] += p;
                p *= zz;
            }
        }
        float xa[kLmaxMax + 1], yb[kLmaxMax + 1];
        xa[0] = yb[0] = 1.0f;
#pragma unroll
        for (int e = 1; e <= kLmaxMax; ++e) {
            xa[e] = xa[e - 1] * ((float)ox * dx);
            yb[e] = yb[e - 1] * ((float)oy * dy);
        }
#pragma unroll
        for (int l = 0; l <= kLmaxMax; ++l)
#pragma unroll
            for (int a = l; a >= 0; --a)
#pragma unroll
                for (int b = l - a; b >= 0; --b) {
                    const int c = l - a - b;
                    M[mono_index(a, b, c)] = fmaf(xa[a] * yb[b], sc[c], M[mono_index(a, b, c)]);
                }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NM; ++q) {
        float v = M[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) s_Mw[wid][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < NM) {
        const int q = threadIdx.x;
        float t = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_Mw[w][q];
        const int l = c_mp.mono[q][0] + c_mp.mono[q][1] + c_mp.mono[q][2];
        s_M[q] = l <= lmax ? t * dV : 0.0f;
    }
    __syncthreads();
    // T = K M (the polynomials P_l of the expansion, K_l from the host tables)
    if (threadIdx.x < NM) {
        const int q = threadIdx.x;
        const int l = c_mp.mono[q][0] + c_mp.mono[q][1] + c_mp.mono[q][2];
        const int nl = (l + 1) * (l + 2) / 2, r0 = c_mp.mono_off[l];
        const double* Kr = c_mp.K + c_mp.k_off[l] + (q - r0) * nl;
        float acc = 0.0f;
        for (int t = 0; t < nl; ++t) acc = fmaf((float)Kr[t], s_M[r0 + t], acc);
        s_T[q] = acc;
    }
    __syncthreads();
    // channel 1 on the cube points outside the ball: v = sum_l P_l / r^(2l+1),
    // with P_l = sum_c U_{l,c}(x, y) z^c formed once per row
    const float id2 = (float)(1.0 / d2);
    for (int row = threadIdx.x; row < S * S; row += blockDim.x) {
        const int ox = row / S - h, oy = row % S - h;
        const int rxy = ox * ox + oy * oy;
        if (rxy + h * h <= R * R) continue;  // the whole row inside the ball
        const float x = (float)ox * dx, y = (float)oy * dy;
        float xa[kLmaxMax + 1], yb[kLmaxMax + 1];
        xa[0] = yb[0] = 1.0f;
#pragma unroll
        for (int e = 1; e <= kLmaxMax; ++e) {
            xa[e] = xa[e - 1] * x;
            yb[e] = yb[e - 1] * y;
        }
        float U[kNU];
#pragma unroll
        for (int l = 0; l <= kLmaxMax; ++l)
#pragma unroll
            for (int c = 0; c <= l; ++c) {
                float u = 0.0f;
#pragma unroll
                for (int a = l - c; a >= 0; --a) u = fmaf(s_T[mono_index(a, l - c - a, c)], xa[a] * yb[l - c - a], u);
                U[l * (l + 1) / 2 + c] = u;
            }
        const float rxy2 = x * x + y * y;
        float* rp = in + (size_t)row * S * kIn;
        for (int z = -h; z < h; ++z) {
            if (rxy + z * z <= R * R) continue;
            const float zz = (float)z * dz;
            const float ir = rsqrtf(fmaf(zz, zz, rxy2));
            const float ir2 = ir * ir;
            float acc = 0.0f;
#pragma unroll
            for (int l = kLmaxMax; l >= 0; --l) {
                float pl = U[l * (l + 1) / 2 + l];
#pragma unroll
                for (int c = l - 1; c >= 0; --c) pl = fmaf(pl, zz, U[l * (l + 1) / 2 + c]);
                acc = fmaf(acc, ir2, pl);
            }
            rp[(z + h) * kIn + 1] = acc * ir * id2;
        }
    }
}

__global__ void __launch_bounds__(256) guess_scatter_kernel(const float* __restrict__ out,
                                                            const float* __restrict__ scale, int k0, int S,
                                                            const BallGeo G, double d2, float* __restrict__ vguess) {
    const int b = blockIdx.x, h = S / 2, S3 = S * S * S;
    const float f = (float)(scale[b] * d2);
    const float* o = out + (size_t)b * S3;
    float* vg = vguess + (size_t)(k0 + b) * G.n_pe;
    for (int p = threadIdx.x; p < G.n_pe; p += blockDim.x) {
        const int pk = G.pt_off[p];
        const int ox = (pk & 255) - 128 + h, oy = ((pk >> 8) & 255) - 128 + h, oz = ((pk >> 16) & 255) - 128 + h;
        float v = 0.0f;
        if (ox >= 0 && ox < S && oy >= 0 && oy < S && oz >= 0 && oz < S) v = o[(ox * S + oy) * S + oz] * f;
        vg[p] = v;
    }
}

}  // namespace

cudaError_t sample_prep(const double* phi, const int N[3], const PairRec* pairs, int k0, int nk, int S,
                        const BallGeo& G, float* input, float* scale, float* target, const float* vcache, double d2,
                        const double delta[3], double dV, int lmax, const int* box_org, const int bdim[3],
                        long long ostride, cudaStream_t st) {
    if (nk <= 0) return cudaSuccess;
    sample_prep_kernel<<<nk, 256, 0, st>>>(phi, N[0], N[1], N[2], pairs, k0, S, G, input, scale, target, vcache, d2,
                                           (float)delta[0], (float)delta[1], (float)delta[2], (float)dV, lmax,
                                           box_org, make_int3(bdim[0], bdim[1], bdim[2]), ostride);
    return cudaGetLastError();
}

cudaError_t set_multipole_const_unet(const MultipoleConst& mc) {
    return cudaMemcpyToSymbol(c_mp, &mc, sizeof(MultipoleConst));
}

cudaError_t guess_scatter(const float* out, const float* scale, int k0, int nk, int S, const BallGeo& G, double d2,
                          float* vguess, cudaStream_t st) {
    if (nk <= 0) return cudaSuccess;
    guess_scatter_kernel<<<nk, 256, 0, st>>>(out, scale, k0, S, G, d2, vguess);
    return cudaGetLastError();
}

}  // namespace unet
}  // namespace exx

// ---- C ABI -----------------------------------------------------------------

#include "exx_guess.h"
#include <string>

namespace exx {
void set_global_error(const std::string& msg);  // defined in exx_api.cu
}

struct exx_guess {
    exx::unet::Net net;
};

namespace {

exx_status gfail(exx_status s, const std::string& m) {
    exx::set_global_error(m);
    return s;
}

exx_status gcuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return EXX_OK;
    (void)cudaGetLastError();
    if (e == cudaErrorLaunchTimeout)
        return gfail(EXX_ECUDA, std::string(what) + ": a tensor-core wait timed out");
    return gfail(e == cudaErrorMemoryAllocation ? EXX_ENOMEM : EXX_ECUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

extern "C" size_t exx_guess_param_count(void) { return exx::unet::param_count(); }

extern "C" exx_status exx_guess_create(exx_guess** out, int S, int batch_max) {
    if (!out) return gfail(EXX_EINVAL, "exx_guess_create: out is NULL");
    *out = nullptr;
    if (S < 16 || S > 64 || S % 8) return gfail(EXX_EINVAL, "exx_guess_create: S must be a multiple of 8 in [16, 64]");
    if (batch_max < 1 || batch_max > 1024) return gfail(EXX_EINVAL, "exx_guess_create: batch_max must be in [1, 1024]");
    exx_guess* g = new exx_guess();
    cudaError_t e = exx::unet::create(g->net, S, batch_max);
    if (e != cudaSuccess) {
        exx::unet::destroy(g->net);
        delete g;
        return gcuda(e, "exx_guess_create");
    }
    *out = g;
    return EXX_OK;
}

extern "C" exx_status exx_guess_set_params(exx_guess* g, const float* params, size_t n) {
    if (!g || !params) return gfail(EXX_EINVAL, "exx_guess_set_params: NULL argument");
    if (n != g->net.nparam) return gfail(EXX_EINVAL, "exx_guess_set_params: wrong parameter count");
    exx_status s = gcuda(cudaMemcpy(g->net.params, params, n * 4, cudaMemcpyHostToDevice), "exx_guess_set_params");
    if (s != EXX_OK) return s;
    g->net.packed = false;
    return gcuda(exx::unet::pack(g->net, nullptr), "exx_guess_set_params");
}

extern "C" exx_status exx_guess_get_params(exx_guess* g, float* params, size_t n) {
    if (!g || !params) return gfail(EXX_EINVAL, "exx_guess_get_params: NULL argument");
    if (n != g->net.nparam) return gfail(EXX_EINVAL, "exx_guess_get_params: wrong parameter count");
    return gcuda(cudaMemcpy(params, g->net.params, n * 4, cudaMemcpyDeviceToHost), "exx_guess_get_params");
}

extern "C" exx_status exx_guess_forward(exx_guess* g, const float* input, float* output, int batch, void* stream) {
    if (!g || !input || !output) return gfail(EXX_EINVAL, "exx_guess_forward: NULL argument");
    if (batch < 1 || batch > g->net.Bmax) return gfail(EXX_EINVAL, "exx_guess_forward: batch out of range");
    cudaStream_t st = (cudaStream_t)stream;
    exx_status s = gcuda(exx::unet::forward(g->net, input, batch, st), "exx_guess_forward");
    if (s != EXX_OK) return s;
    const size_t bytes = (size_t)batch * g->net.S * g->net.S * g->net.S * 4;
    s = gcuda(cudaMemcpyAsync(output, g->net.out, bytes, cudaMemcpyDeviceToDevice, st), "exx_guess_forward");
    if (s != EXX_OK) return s;
    return gcuda(exx::unet::check_error(g->net, st), "exx_guess_forward");
}

extern "C" exx_status exx_guess_gradient(exx_guess* g, const float* input, const float* target, int batch, float* loss,
                                         float* grad, void* stream) {
    if (!g || !input || !target) return gfail(EXX_EINVAL, "exx_guess_gradient: NULL argument");
    if (batch < 1 || batch > g->net.Bmax) return gfail(EXX_EINVAL, "exx_guess_gradient: batch out of range");
    cudaStream_t st = (cudaStream_t)stream;
    exx_status s = gcuda(exx::unet::forward(g->net, input, batch, st), "exx_guess_gradient");
    if (s == EXX_OK) s = gcuda(exx::unet::backward(g->net, input, target, batch, st), "exx_guess_gradient");
    if (s == EXX_OK) s = gcuda(exx::unet::check_error(g->net, st), "exx_guess_gradient");
    if (s == EXX_OK && loss)
        s = gcuda(cudaMemcpy(loss, g->net.d_loss, 4, cudaMemcpyDeviceToHost), "exx_guess_gradient");
    if (s == EXX_OK && grad)
        s = gcuda(cudaMemcpy(grad, g->net.grads, g->net.nparam * 4, cudaMemcpyDeviceToHost), "exx_guess_gradient");
    return s;
}

extern "C" exx_status exx_guess_train_step(exx_guess* g, const float* input, const float* target, int batch, float lr,
                                           float* loss, void* stream) {
    if (!g || !input || !target) return gfail(EXX_EINVAL, "exx_guess_train_step: NULL argument");
    if (batch < 1 || batch > g->net.Bmax) return gfail(EXX_EINVAL, "exx_guess_train_step: batch out of range");
    if (!(lr > 0.0f)) return gfail(EXX_EINVAL, "exx_guess_train_step: lr must be positive");
    cudaStream_t st = (cudaStream_t)stream;
    exx_status s = gcuda(exx::unet::forward(g->net, input, batch, st), "exx_guess_train_step");
    if (s == EXX_OK) s = gcuda(exx::unet::backward(g->net, input, target, batch, st), "exx_guess_train_step");
    if (s == EXX_OK) s = gcuda(exx::unet::adam_step(g->net, lr, st), "exx_guess_train_step");
    if (s == EXX_OK && loss)
        s = gcuda(cudaMemcpyAsync(loss, g->net.d_loss, 4, cudaMemcpyDeviceToHost, st), "exx_guess_train_step");
    if (s == EXX_OK) s = gcuda(exx::unet::check_error(g->net, st), "exx_guess_train_step");
    return s;
}

extern "C" void exx_guess_destroy(exx_guess* g) {
    if (!g) return;
    exx::unet::destroy(g->net);
    delete g;
}

extern "C" exx_status exx_unet_conv3d(const void* x, const float* w, const float* bias, const void* mask, void* y,
                                      int batch, int D, int H, int W, int cin, int cout, int mode, void* stream) {
    if (!x || !w || !y) return gfail(EXX_EINVAL, "exx_unet_conv3d: NULL argument");
    if (cin % 16 || cout % 16 || cin < 16 || cout < 16 || cin > 256 || cout > 256)
        return gfail(EXX_EINVAL, "exx_unet_conv3d: channels must be multiples of 16 in [16, 256]");
    if (batch < 1 || D < 1 || H < 1 || W < 1 || mode < 0 || mode > 2)
        return gfail(EXX_EINVAL, "exx_unet_conv3d: bad size or mode");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    __nv_bfloat16* wp = nullptr;
    int* err = nullptr;
    exx_status s = gcuda(cudaMalloc(&wp, (size_t)27 * cin * cout * 2), "exx_unet_conv3d");
    if (s == EXX_OK) s = gcuda(cudaMalloc(&err, 4), "exx_unet_conv3d");
    if (s == EXX_OK) s = gcuda(cudaMemsetAsync(err, 0, 4, st), "exx_unet_conv3d");
    const int flip = mode == 2 ? 1 : 0;
    if (s == EXX_OK) s = gcuda(exx::unet::pack_weights(w, wp, cin, cout, flip, st), "exx_unet_conv3d");
    if (s == EXX_OK) {
        const int ci = flip ? cout : cin, co = flip ? cin : cout;
        const int epi = mode == 1 ? 1 : (mode == 2 && mask ? 2 : 0);
        s = gcuda(exx::unet::conv3_tc((const __nv_bfloat16*)x, wp, flip ? nullptr : bias,
                                      (const __nv_bfloat16*)mask, (__nv_bfloat16*)y, batch, D, H, W, ci, co, epi, err,
                                      nsm, st),
                  "exx_unet_conv3d");
    }
    int h = 0;
    if (s == EXX_OK) s = gcuda(cudaMemcpyAsync(&h, err, 4, cudaMemcpyDeviceToHost, st), "exx_unet_conv3d");
    if (s == EXX_OK) s = gcuda(cudaStreamSynchronize(st), "exx_unet_conv3d");
    if (s == EXX_OK && h) s = gfail(EXX_ECUDA, "exx_unet_conv3d: a tensor-core wait timed out");
    cudaFree(wp);
    cudaFree(err);
    return s;
}
