// exx_pairs.cu -- pair list (Sec. III.C Step II), D_xx zeroing, E_xx reduction.
//
// The pair list keeps i <= j with |minimg(C_j - C_i)| < R_pair (strict) and
// stores for each pair the grid point nearest the pair centre
// C_ij = C_i + minimg(C_j - C_i)/2 (the midpoint of Step III, snapped with NINT
// and wrapped by MOD as in Eq. l2g). The list is built in parallel (count per
// i, scan, ordered fill), so its order is i-major with j ascending. Doubles
// decide integers here, so every operation is an explicitly rounded IEEE op.
#include <cuda_runtime.h>

#include "exx_kernels.cuh"

namespace exx {

__device__ __forceinline__ double minimg_d(double x, double L) {
    double t = __dadd_rn(__ddiv_rn(x, L), 0.5);
    return __dsub_rn(x, __dmul_rn(L, floor(t)));
}

struct PairGeom {
    double L[3];
    double delta[3];
    int N[3];
    double r2cut;
    int r_pe, r_me;
    // per-pair radii (alphas != NULL): rule of the spread-dependent subdomains
    const double* alphas;
    double ln_inv_eps, delta_max;
    int r_min;
    // separate radii for non-self pairs (ns_pe > 0): self pairs keep r_pe,
    // r_me (geometry 1), non-self pairs take ns_pe, ns_me (geometry 0)
    int ns_pe, ns_me;
    int* bad;  // if set, counts orbitals whose centre is NaN or Inf
};

// R_PE = clamp(ceil((s_eps + |cbar - C_ij|)/delta), r_min, r_max) with
// s_eps = sqrt(max(0, (ln(1/eps) - mu d^2)/(a_i + a_j))), mu = a_i a_j/(a_i + a_j),
// |cbar - C_ij| = |a_j/(a_i + a_j) - 1/2| |d|; R_ME = R_PE + max(3, ceil(R_PE/3)).
// Every operation is explicitly rounded: doubles decide the integer radius.
__device__ __forceinline__ int pair_radius_d(double ai, double aj, double d2, const PairGeom& G, int* r_me) {
    const double beta = __dadd_rn(ai, aj);
    const double mu = __ddiv_rn(__dmul_rn(ai, aj), beta);
    const double t = __ddiv_rn(__dsub_rn(G.ln_inv_eps, __dmul_rn(mu, d2)), beta);
    const double s = t > 0.0 ? __dsqrt_rn(t) : 0.0;
    const double w = __dmul_rn(fabs(__dsub_rn(__ddiv_rn(aj, beta), 0.5)), __dsqrt_rn(d2));
    const double rf = ceil(__ddiv_rn(__dadd_rn(s, w), G.delta_max));
    const int r = rf < (double)G.r_min ? G.r_min : (rf > (double)G.r_pe ? G.r_pe : (int)rf);
    *r_me = r + ((r + 2) / 3 > 3 ? (r + 2) / 3 : 3);
    return r;
}

__device__ __forceinline__ bool pair_within(const double* __restrict__ C, int i, int j, const PairGeom& G,
                                            double d[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = minimg_d(__dsub_rn(C[3 * j + a], C[3 * i + a]), G.L[a]);
    double d2 = __dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1]));
    d2 = __dadd_rn(d2, __dmul_rn(d[2], d[2]));
    return d2 < G.r2cut;
}

// counts[i] = number of j >= i paired with i. One block per i.
__global__ void pairs_count_kernel(int n, const double* __restrict__ C, PairGeom G, int* __restrict__ counts) {
    const int i = blockIdx.x;
    if (G.bad && threadIdx.x == 0 && !(isfinite(C[3 * i]) && isfinite(C[3 * i + 1]) && isfinite(C[3 * i + 2])))
        atomicAdd(G.bad, 1);
    int cnt = 0;
    for (int j = i + threadIdx.x; j < n; j += blockDim.x) {
        double d[3];
        cnt += pair_within(C, i, j, G, d) ? 1 : 0;
    }
    __shared__ int s[32];
    cnt = warp_sum_int(cnt);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x < 32) {
        int t = threadIdx.x < (blockDim.x >> 5) ? s[threadIdx.x] : 0;
        t = warp_sum_int(t);
        if (threadIdx.x == 0) counts[i] = t;
    }
}

// Exclusive scan of counts into offsets[0..n]; offsets[n] = number of pairs.
// One block of 1024 threads, each owning a contiguous segment.
__global__ void pairs_scan_kernel(int n, const int* __restrict__ counts, int* __restrict__ offsets,
                                  int* __restrict__ n_pair, int* __restrict__ queue) {
    __shared__ int s[1024];
    const int t = threadIdx.x;
    const int seg = (n + 1023) / 1024;
    const int b = t * seg, e = min(n, b + seg);
    int sum = 0;
    for (int k = b; k < e; ++k) sum += counts[k];
    s[t] = sum;
    __syncthreads();
    // Hillis-Steele inclusive scan over the 1024 segment sums
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
    if (t == 1023) {
        offsets[n] = s[1023];
        *n_pair = s[1023];
        *queue = 0;
    }
}

// Where the fill kernel puts a pair: the pair records of exx_compute, or the
// five-int records (i, j, g0, g1, g2) of exx_pair_list_static, whose list
// positions at or beyond cap are skipped.
struct RecordOut {
    PairRec* pairs;
    __device__ __forceinline__ void put(int pos, const PairRec& r) const { pairs[pos] = r; }
};
struct PackedOut {
    int* out;
    int cap;
    __device__ __forceinline__ void put(int pos, const PairRec& r) const {
        if (pos >= cap) return;
        int* rec = out + 5 * (long long)pos;
        rec[0] = r.i;
        rec[1] = r.j;
        rec[2] = r.g[0];
        rec[3] = r.g[1];
        rec[4] = r.g[2];
    }
};

// Ordered fill: block i writes its pairs (i, j), j ascending, at offsets[i].
template <class Out>
__global__ void pairs_fill_kernel(int n, const double* __restrict__ C, PairGeom G, const int* __restrict__ offsets,
                                  Out out) {
    const int i = blockIdx.x;
    __shared__ int s_w[33];
    int base = offsets[i];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j0 = i; j0 < n; j0 += blockDim.x) {
        const int j = j0 + threadIdx.x;
        double d[3] = {0.0, 0.0, 0.0};
        bool keep = j < n && pair_within(C, i, j, G, d);
        unsigned m = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) s_w[w] = __popc(m);
        __syncthreads();
        if (threadIdx.x == 0) {
            int run = 0;
            for (int k = 0; k < nw; ++k) {
                int c = s_w[k];
                s_w[k] = run;
                run += c;
            }
            s_w[32] = run;
        }
        __syncthreads();
        if (keep) {
            int pos = base + s_w[w] + __popc(m & ((1u << lane) - 1u));
            PairRec r;
            r.i = i;
            r.j = j;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                double c = __dadd_rn(C[3 * i + a], __dmul_rn(0.5, d[a]));
                long long g = llround(__ddiv_rn(c, G.delta[a]));
                long long mm = g % G.N[a];
                r.g[a] = (int)(mm < 0 ? mm + G.N[a] : mm);
            }
            if (G.alphas) {
                double d2 = __dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1]));
                d2 = __dadd_rn(d2, __dmul_rn(d[2], d[2]));
                int rme;
                r.r_pe = pair_radius_d(G.alphas[i], G.alphas[j], d2, G, &rme);
                r.r_me = rme;
                r.geo = r.r_pe - G.r_min;
            } else if (G.ns_pe > 0) {
                const bool self = i == j;
                r.r_pe = self ? G.r_pe : G.ns_pe;
                r.r_me = self ? G.r_me : G.ns_me;
                r.geo = self ? 1 : 0;
            } else {
                r.r_pe = G.r_pe;
                r.r_me = G.r_me;
                r.geo = 0;
            }
            out.put(pos, r);
        }
        base += s_w[32];
        __syncthreads();
    }
}

// Largest pairs first: counting sort of the pair indices by geometry
// (descending radius). hist[0..n_geo) counts, hist[n_geo..2 n_geo) cursors.
__global__ void radii_count_kernel(const PairRec* __restrict__ pairs, const int* __restrict__ n_pair,
                                   int* __restrict__ hist, int n_geo) {
    const int np = *n_pair;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x)
        atomicAdd(hist + pairs[p].geo, 1);
}

__global__ void radii_scan_kernel(int* __restrict__ hist, int n_geo) {
    if (threadIdx.x != 0) return;
    int run = 0;
    for (int g = n_geo - 1; g >= 0; --g) {
        const int c = hist[g];
        hist[n_geo + g] = run;
        run += c;
    }
}

__global__ void radii_scatter_kernel(const PairRec* __restrict__ pairs, const int* __restrict__ n_pair,
                                     int* __restrict__ hist, int n_geo, int* __restrict__ order) {
    const int np = *n_pair;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x)
        order[atomicAdd(hist + n_geo + pairs[p].geo, 1)] = p;
}

// The radius classes of the sorted order: after the scatter, hist[n_geo + g]
// is the end of geometry g's run; cls[2 g] = its start, cls[2 g + 1] = its
// length, cls[2 n_geo + g] = 0 (the class launch's work counter).
__global__ void radii_classes_kernel(const int* __restrict__ hist, int n_geo, int* __restrict__ cls) {
    for (int g = threadIdx.x; g < n_geo; g += blockDim.x) {
        cls[2 * g] = hist[n_geo + g] - hist[g];
        cls[2 * g + 1] = hist[g];
        cls[2 * n_geo + g] = 0;
    }
}

// Compact boxes: counts the pairs whose ME ball (the bounding cube of side
// 2 R_ME + 1 around g_ij) is not inside both orbitals' boxes; for those the
// result differs from the full-grid one (the orbitals count as zero outside).
__global__ void box_clip_kernel(const PairRec* __restrict__ pairs, const int* __restrict__ n_pair,
                                const int* __restrict__ box_org, int3 bdim, int3 N, int* __restrict__ clipped) {
    const int np = *n_pair;
    int c = 0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
        const PairRec r = pairs[p];
        const int g[3] = {r.g[0], r.g[1], r.g[2]}, n[3] = {N.x, N.y, N.z}, b[3] = {bdim.x, bdim.y, bdim.z};
        bool in = true;
        for (int t = 0; t < 2; ++t) {
            const int o = t ? r.j : r.i;
            for (int a = 0; a < 3; ++a) {
                int s = (g[a] - r.r_me - box_org[3 * o + a]) % n[a];
                s += s < 0 ? n[a] : 0;
                in = in && s + 2 * r.r_me < b[a];
            }
        }
        c += in ? 0 : 1;
    }
    c = warp_sum_int(c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(clipped, c);
}

// D_xx = 0 (grid-stride fill; 16-byte stores when the pointer allows them).
__global__ void zero_kernel(double* __restrict__ p, long long n, int vec) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (!vec) {
        for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) p[k] = 0.0;
        return;
    }
    long long n2 = n >> 1;
    double2* p2 = reinterpret_cast<double2*>(p);
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n2; k += stride)
        p2[k] = make_double2(0.0, 0.0);
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) p[n - 1] = 0.0;
}

// D_xx accumulated as fixed-point integers (deterministic mode): each word
// holds a 64-bit integer sum; convert it to FP64 in place.
__global__ void dfix_convert_kernel(double* __restrict__ p, long long n, double inv) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long* q = reinterpret_cast<long long*>(p);
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride)
        p[k] = (double)q[k] * inv;
}

// E_xx = -(sum_i E_ii + 2 sum_{i<j} E_ij), in a fixed order (one block); pairs
// whose E_ij is NaN or Inf are added to *bad (non-finite input propagated).
__global__ void exx_reduce_kernel(const PairRec* __restrict__ pairs, const int* __restrict__ n_pair,
                                  const double* __restrict__ e_pair, double* __restrict__ out, int* __restrict__ bad) {
    __shared__ double red[2][33];
    __shared__ int nbad;
    int flip = 0;
    if (threadIdx.x == 0) nbad = 0;
    __syncthreads();
    const int np = *n_pair;
    double s = 0.0;
    int nb = 0;
    for (int p = threadIdx.x; p < np; p += 1024) {
        const PairRec r = pairs[p];
        const double e = e_pair[p];
        s += (r.i == r.j ? 1.0 : 2.0) * e;
        nb += isfinite(e) ? 0 : 1;
    }
    s = block_sum<1024, double>(s, red, flip);
    if (nb) atomicAdd(&nbad, nb);
    __syncthreads();
    if (threadIdx.x == 0) {
        out[0] = -s;
        if (bad && nbad) atomicAdd(bad, nbad);
    }
}

}  // namespace exx

// ---- host launchers (C++ linkage inside the library) ----
namespace exx {

cudaError_t launch_pair_list(int n, const double* centers, const double L[3], const double delta[3], const int N[3],
                             double r_pair, int r_pe, int r_me, int* counts, int* offsets, int* n_pair, int* queue,
                             PairRec* pairs, cudaStream_t st, const double* alphas, double ln_inv_eps,
                             double delta_max, int r_min, int ns_pe, int ns_me, int* bad) {
    PairGeom G;
    for (int a = 0; a < 3; ++a) {
        G.L[a] = L[a];
        G.delta[a] = delta[a];
        G.N[a] = N[a];
    }
    G.r2cut = r_pair * r_pair;
    G.r_pe = r_pe;
    G.r_me = r_me;
    G.alphas = alphas;
    G.ln_inv_eps = ln_inv_eps;
    G.delta_max = delta_max;
    G.r_min = r_min;
    G.ns_pe = ns_pe;
    G.ns_me = ns_me;
    G.bad = bad;
    pairs_count_kernel<<<n, 256, 0, st>>>(n, centers, G, counts);
    pairs_scan_kernel<<<1, 1024, 0, st>>>(n, counts, offsets, n_pair, queue);
    pairs_fill_kernel<<<n, 256, 0, st>>>(n, centers, G, offsets, RecordOut{pairs});
    return cudaGetLastError();
}

// The same count / scan / fill for exx_pair_list_static: fixed radii, records
// of five ints, positions at or beyond cap skipped; scratch holds counts[n],
// offsets[n + 1] and two ints (pair count, unused queue word), in that order.
cudaError_t launch_pair_list_packed(int n, const double* centers, const double L[3], const double delta[3],
                                    const int N[3], double r_pair, int* scratch, int* out, int cap, cudaStream_t st) {
    PairGeom G = {};
    for (int a = 0; a < 3; ++a) {
        G.L[a] = L[a];
        G.delta[a] = delta[a];
        G.N[a] = N[a];
    }
    G.r2cut = r_pair * r_pair;
    int* counts = scratch;
    int* offsets = scratch + n;
    int* tail = offsets + n + 1;
    pairs_count_kernel<<<n, 256, 0, st>>>(n, centers, G, counts);
    pairs_scan_kernel<<<1, 1024, 0, st>>>(n, counts, offsets, tail, tail + 1);
    pairs_fill_kernel<<<n, 256, 0, st>>>(n, centers, G, offsets, PackedOut{out, cap});
    return cudaGetLastError();
}

cudaError_t launch_radii_sort(const PairRec* pairs, const int* n_pair, int* hist, int n_geo, int* order, int num_sms,
                              cudaStream_t st, int* classes) {
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int) * 2 * n_geo, st);
    if (e != cudaSuccess) return e;
    radii_count_kernel<<<num_sms * 2, 256, 0, st>>>(pairs, n_pair, hist, n_geo);
    radii_scan_kernel<<<1, 32, 0, st>>>(hist, n_geo);
    radii_scatter_kernel<<<num_sms * 2, 256, 0, st>>>(pairs, n_pair, hist, n_geo, order);
    if (classes) radii_classes_kernel<<<1, 64, 0, st>>>(hist, n_geo, classes);
    return cudaGetLastError();
}

cudaError_t launch_box_clip(const PairRec* pairs, const int* n_pair, const int* box_org, const int bdim[3],
                            const int N[3], int* clipped, int num_sms, cudaStream_t st) {
    box_clip_kernel<<<num_sms, 256, 0, st>>>(pairs, n_pair, box_org, make_int3(bdim[0], bdim[1], bdim[2]),
                                             make_int3(N[0], N[1], N[2]), clipped);
    return cudaGetLastError();
}

cudaError_t launch_zero(double* p, long long n, int num_sms, cudaStream_t st) {
    const int vec = (reinterpret_cast<unsigned long long>(p) & 15ull) == 0 ? 1 : 0;
    zero_kernel<<<num_sms * 8, 256, 0, st>>>(p, n, vec);
    return cudaGetLastError();
}

// Copy of n2 16-byte words between device-visible buffers (one of them pinned
// host memory, read or written by the SMs over the chip-to-chip link): four
// independent words in flight per thread and step.
__global__ void copy16_kernel(const double2* __restrict__ src, double2* __restrict__ dst, long long n2) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; k + 3 * stride < n2; k += 4 * stride) {
        const double2 a = src[k], b = src[k + stride], c = src[k + 2 * stride], d = src[k + 3 * stride];
        dst[k] = a;
        dst[k + stride] = b;
        dst[k + 2 * stride] = c;
        dst[k + 3 * stride] = d;
    }
    for (; k < n2; k += stride) dst[k] = src[k];
}

cudaError_t launch_copy16(const void* src, void* dst, long long n2, int num_sms, cudaStream_t st) {
    copy16_kernel<<<num_sms * 8, 256, 0, st>>>(reinterpret_cast<const double2*>(src), reinterpret_cast<double2*>(dst),
                                                n2);
    return cudaGetLastError();
}

cudaError_t launch_dfix_convert(double* p, long long n, double inv, int num_sms, cudaStream_t st) {
    dfix_convert_kernel<<<num_sms * 8, 256, 0, st>>>(p, n, inv);
    return cudaGetLastError();
}

cudaError_t launch_exx_reduce(const PairRec* pairs, const int* n_pair, const double* e_pair, double* out,
                              cudaStream_t st, int* bad) {
    exx_reduce_kernel<<<1, 1024, 0, st>>>(pairs, n_pair, e_pair, out, bad);
    return cudaGetLastError();
}

}  // namespace exx
