// exx_cluster.cu -- one thread-block cluster per pair, FP32 inner CG state on chip.
//
// The C CTAs of a cluster share one pair. The PE ball is split into C slabs of
// whole x planes (balanced by point count, at least 3 planes each so a stencil
// leg reaches at most the adjacent CTA). Each CTA keeps the CG direction p of
// its slab in shared memory as planes of a box of 2 R_PE + 7 rows (zero outside
// the ball, so the stencil needs no bounds tests). The thread maps (MODE):
//   0  one point per thread slot; x legs that leave the slab read the
//      neighbour's slab through distributed shared memory; three cluster
//      barriers per iteration (pts_segment)
//   1  z runs, halo planes filled by plain remote stores (run_segment)
//   2  quads of 4 consecutive z positions per slot, every leg one 16-byte
//      load, x legs read remotely, mbarrier cluster sums (quad_segment)
//   3  quads with 3 halo planes per side filled by bulk copies counted on an
//      mbarrier, one cluster sum per iteration, no cluster barrier in the CG,
//      fixed-point FP64 residuals (quad_halo_segment; the fastest on GB300)
// In every map r and A p stay in registers; dot products are summed per CTA,
// exchanged through distributed shared memory and added in rank order, so
// every CTA holds the same value.
//
// The FP64 parts of the pair (gather, multipoles, shell potential, the FP64
// residual 4 pi rho + lap v of each refinement step, E_ij, the D_xx scatter)
// are spread over all threads of the cluster and keep their data in the
// cluster's global workspace slot.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "exx_mg.cuh"
#include "exx_phases.cuh"

namespace cg = cooperative_groups;

namespace exx {

// Sum over the cluster: warp sums into shared memory, one CTA barrier, warp 0
// forms the CTA total and its first C lanes push it into every CTA's part[]
// through distributed shared memory; after one cluster barrier each CTA sums
// part[] in rank order (the same value in every CTA, the same summation order
// as a block sum followed by the exchange).
template <int NT, int C, typename T>
__device__ __forceinline__ T cluster_sum(T v, T (*red)[33], int& flip, T (*part)[16], int& cflip,
                                         cg::cluster_group& cl, int rank) {
    v = warp_sum(v);
    T* buf = red[flip];
    flip ^= 1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) buf[w] = v;
    __syncthreads();
    if (w == 0) {
        T t = lane < NT / 32 ? buf[lane] : T(0);
        t = warp_sum(t);
        if (lane < C) {
            T* dst = cl.map_shared_rank(&part[cflip][0], lane);
            dst[rank] = t;
        }
    }
    cl.sync();
    T s = T(0);
#pragma unroll
    for (int r = 0; r < C; ++r) s += part[cflip][r];
    cflip ^= 1;
    return s;
}

// Max over the cluster (same pattern and buffers as cluster_sum).
template <int NT, int C>
__device__ __forceinline__ double cluster_max(double v, double (*red)[33], int& flip, double (*part)[16], int& cflip,
                                              cg::cluster_group& cl, int rank) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    double* buf = red[flip];
    flip ^= 1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) buf[w] = v;
    __syncthreads();
    if (w == 0) {
        double t = lane < NT / 32 ? buf[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
        if (lane < C) {
            double* dst = cl.map_shared_rank(&part[cflip][0], lane);
            dst[rank] = t;
        }
    }
    cl.sync();
    double m = 0.0;
#pragma unroll
    for (int r = 0; r < C; ++r) m = fmax(m, part[cflip][r]);
    cflip ^= 1;
    return m;
}

// Fixed-point residuals (isotropic grids). 180 delta^2 times the weights of
// Eq. d2_1 (n = 3) are the integers -490, 270, -27, 2 per axis, so with v held
// as the integers round(v 2^E) the Laplacian is an exact integer sum, and the
// FP64 residual costs one conversion and two FP64 operations per point instead
// of twenty (GB300 issues FP64 at 1/64 of the FP32 rate). E is chosen per pair
// from a bound on |v| so that |v| 2^E < 2^50, which keeps every stencil sum
// below 2^62; a value outside the bound marks the pair, which then takes the
// FP64 stencil. The integer stencil rounds v to a multiple of 2^-E, so each
// value errs by at most 2^-51 of twice the bound and the Laplacian by at most
// 18.13 (the sum of |weights| / 180) times that over delta^2: one to two orders
// above the rounding of the FP64 sums it replaces, and for an R_PE 24 ball about
// 1e-11 of ||b||, three orders below the stop rule's tol 1e-8.
__device__ __forceinline__ long long to_fix(double v, double s2E, int& ovf) {
    const double x = v * s2E;
    if (!(fabs(x) <= 1125899906842624.0)) {  // 2^50
        ovf = 1;
        return 0;
    }
    return __double2ll_rn(x);
}

__device__ __forceinline__ long long lap_fix(const long long* __restrict__ f, long long c, int S, long long S2) {
    const long long s1 = (f[c + 1] + f[c - 1]) + (f[c + S] + f[c - S]) + (f[c + S2] + f[c - S2]);
    const long long s2 = (f[c + 2] + f[c - 2]) + (f[c + 2 * S] + f[c - 2 * S]) + (f[c + 2 * S2] + f[c - 2 * S2]);
    const long long s3 = (f[c + 3] + f[c - 3]) + (f[c + 3 * S] + f[c - 3 * S]) + (f[c + 3 * S2] + f[c - 3 * S2]);
    return 270 * s1 - 27 * s2 + 2 * s3 - 1470 * f[c];
}

// FP64 residual r = 4 pi rho + lap v on the CTA's points k0 + tid + j NT;
// writes r64 (and the debug copy); returns the thread's sum of r^2.
// With vf set, lap v comes from the fixed-point copy (lap_fix times finv).
__device__ __noinline__ double cta_residual(const SolveParams& P, const int* __restrict__ cube,
                                            const double* __restrict__ rho, const double* __restrict__ vc,
                                            double* __restrict__ r64, int k0, int k1, int nt, bool dbg,
                                            const long long* __restrict__ vf = nullptr, double finv = 0.0) {
    const Stencil<double> st = P.st64;  // into registers (see gather_rho)
    const int S = P.S;
    const long long S2 = P.S2;
    double* __restrict__ db = P.dbg_b;
    double acc = 0.0;
    for (int k = k0 + (int)threadIdx.x; k < k1; k += nt) {
        const double lap = vf ? (double)lap_fix(vf, cube[k], S, S2) * finv : lap19<double>(vc, cube[k], S, S2, st);
        const double rk = fma(kFourPi, rho[k], lap);
        r64[k] = rk;
        acc = fma(rk, rk, acc);
        if (dbg) db[k] = rk;
    }
    return acc;
}

// The first FP64 residual of a pair, while v is zero on the PE ball: the
// CTA's rim points (list[0 .. nrim)) take the full stencil, the interior ones
// r = 4 pi rho (lap v = 0 there exactly), each group in dense warps.
__device__ __noinline__ double cta_residual0(const SolveParams& P, const int* __restrict__ cube,
                                             const double* __restrict__ rho, const double* __restrict__ vc,
                                             double* __restrict__ r64, const int* __restrict__ list, int n, int nrim,
                                             int nt, bool dbg, const long long* __restrict__ vf = nullptr,
                                             double finv = 0.0) {
    const Stencil<double> st = P.st64;
    const int S = P.S;
    const long long S2 = P.S2;
    double* __restrict__ db = P.dbg_b;
    double acc = 0.0;
    for (int t = (int)threadIdx.x; t < n; t += nt) {
        const int k = list[t];
        double rk;
        if (t < nrim) {
            const double lap =
                vf ? (double)lap_fix(vf, cube[k], S, S2) * finv : lap19<double>(vc, cube[k], S, S2, st);
            rk = fma(kFourPi, rho[k], lap);
        } else {
            rk = kFourPi * rho[k];
        }
        r64[k] = rk;
        acc = fma(rk, rk, acc);
        if (dbg) db[k] = rk;
    }
    return acc;
}

// Eq. mepole, stages 2-4 on the cluster: each CTA forms the plane sums of its
// own slab's planes [pl0, pl0 + npl) into the cluster's shared array sYc
// [(2 R_PE + 1)][28] (global workspace); after a cluster barrier every CTA
// forms the moments M (times dV) and T = K M from all planes, as moment_finish.
template <int NT>
__device__ void moment_finish_cluster(const SolveParams& P, const BallGeo& G, const double* __restrict__ rowS,
                                      const double* __restrict__ xp, const double* __restrict__ yp,
                                      double* __restrict__ sYc, int pl0, int npl, double* __restrict__ s_M,
                                      double* __restrict__ s_T, cg::cluster_group& cl) {
    const int L = P.lmax;
    const int Rc = P.Rc;
    const int nplane = 2 * G.r_pe + 1;
    const int nbc = (L + 1) * (L + 2) / 2;
    for (int item = threadIdx.x; item < npl * nbc; item += NT) {
        const int pl = pl0 + item / nbc, bc = item % nbc;
        int dgr = 0;
        while ((dgr + 1) * (dgr + 2) / 2 <= bc) ++dgr;
        const int c = bc - dgr * (dgr + 1) / 2, b = dgr - c;
        double acc = 0.0;
        for (int row = G.plane_pe[pl]; row < G.plane_pe[pl + 1]; ++row) {
            const int oy = G.rows_pe[row].oy;
            acc = fma(yp[(oy + Rc) * 8 + b], rowS[row * 8 + c], acc);
        }
        sYc[pl * 28 + bc] = acc;
    }
    cl.sync();
    for (int m = threadIdx.x; m < kNMono; m += NT) {
        const int a = c_mp.mono[m][0], b = c_mp.mono[m][1], c = c_mp.mono[m][2];
        double acc = 0.0;
        if (a + b + c <= L) {
            const int dgr = b + c, bc = dgr * (dgr + 1) / 2 + c;
            for (int pl = 0; pl < nplane; ++pl) acc = fma(xp[(pl - G.r_pe + Rc) * 8 + a], sYc[pl * 28 + bc], acc);
        }
        s_M[m] = acc * P.dV;
    }
    __syncthreads();
    for (int m = threadIdx.x; m < kNMono; m += NT) {
        const int l = c_mp.mono[m][0] + c_mp.mono[m][1] + c_mp.mono[m][2];
        double acc = 0.0;
        if (l <= L) {
            const int nl = (l + 1) * (l + 2) / 2, r0 = c_mp.mono_off[l];
            const double* Kr = c_mp.K + c_mp.k_off[l] + (m - r0) * nl;
            for (int t = 0; t < nl; ++t) acc = fma(Kr[t], s_M[r0 + t], acc);
        }
        s_T[m] = acc;
    }
    __syncthreads();
}

// sum of rho v over the CTA's points.
__device__ __noinline__ double cta_energy(const int* __restrict__ cube, const double* __restrict__ rho,
                                          const double* __restrict__ vc, int k0, int k1, int nt) {
    double e = 0.0;
    for (int k = k0 + (int)threadIdx.x; k < k1; k += nt) e = fma(rho[k], vc[cube[k]], e);
    return e;
}

// The previous call's list position of pair (i, j), or -1 (lists are i-major, j ascending).
__device__ __forceinline__ int find_prev_pair(const PairRec* __restrict__ prev, int n, int i, int j) {
    int lo = 0, hi = n - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const PairRec q = prev[mid];
        if (q.i == i && q.j == j) return mid;
        if (q.i < i || (q.i == i && q.j < j)) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

// Warm start: v on the CTA's PE points from the previous call's potential of
// the same pair. Its grid centre moved by dlt, so the point at offset o now
// held the old offset o + dlt; where that leaves the PE ball the old value at
// o itself is taken.
__device__ __noinline__ void cta_warm_insert(const BallGeo& G, const int* __restrict__ cube, double* __restrict__ vc,
                                             const float* __restrict__ vold, int dx, int dy, int dz, int k0, int k1,
                                             int nt) {
    const int R = G.r_pe, W = 2 * G.r_pe + 1;
    const int* __restrict__ off = G.pt_off;
    const int* __restrict__ row_of = G.row_of;
    const RowRec* __restrict__ rows = G.rows_pe;
    for (int k = k0 + (int)threadIdx.x; k < k1; k += nt) {
        const int o = off[k];
        const int x = off_x(o) + dx, y = off_y(o) + dy, z = off_z(o) + dz;
        int src = k;
        if (x >= -R && x <= R && y >= -R && y <= R) {
            const int rr = row_of[(x + R) * W + (y + R)];
            if (rr >= 0) {
                const RowRec Rw = rows[rr];
                if (z >= -Rw.zpe && z <= Rw.zpe) src = Rw.pe_start + z + Rw.zpe;
            }
        }
        vc[cube[k]] = (double)vold[src];
    }
}

// Polynomial extrapolation from the last m calls (warm 3): v(o) = sum_s
// coef[s] v_s(o + dlt_s), each v_s read as in cta_warm_insert.
__device__ __noinline__ void cta_warm_extrapolate(const BallGeo& G, const int* __restrict__ cube,
                                                  double* __restrict__ vc, int m, const float* const* vold,
                                                  const int (*dlt)[3], const double* coef, int k0, int k1, int nt) {
    const int R = G.r_pe, W = 2 * G.r_pe + 1;
    const int* __restrict__ off = G.pt_off;
    const int* __restrict__ row_of = G.row_of;
    const RowRec* __restrict__ rows = G.rows_pe;
    for (int k = k0 + (int)threadIdx.x; k < k1; k += nt) {
        const int o = off[k];
        double acc = 0.0;
        for (int s = 0; s < m; ++s) {
            const int x = off_x(o) + dlt[s][0], y = off_y(o) + dlt[s][1], z = off_z(o) + dlt[s][2];
            int src = k;
            if (x >= -R && x <= R && y >= -R && y <= R) {
                const int rr = row_of[(x + R) * W + (y + R)];
                if (rr >= 0) {
                    const RowRec Rw = rows[rr];
                    if (z >= -Rw.zpe && z <= Rw.zpe) src = Rw.pe_start + z + Rw.zpe;
                }
            }
            acc = fma(coef[s], (double)vold[s][src], acc);
        }
        vc[cube[k]] = acc;
    }
}

// Stores v on the CTA's PE points (FP32) for the next call's warm start.
__device__ __noinline__ void cta_warm_store(const int* __restrict__ cube, const double* __restrict__ vc,
                                            float* __restrict__ vdst, int k0, int k1, int nt) {
    for (int k = k0 + (int)threadIdx.x; k < k1; k += nt) vdst[k] = (float)vc[cube[k]];
}

// The z-run CG of one pair (MODE 1), in segments between FP64 residual
// replacements, each in its own register allocation: a segment (re)starts
// from r = r64 / scale (p = r, or p = carry p + r after a replacement), runs
// FP32 CG iterations until the recursive residual has dropped by update_drop
// (or looks converged), adds scale d to v and returns; the caller then forms
// the FP64 residual. The arrays and scalars a segment does not touch in its
// inner loop come from a per-CTA block in shared memory, the reduction
// buffers are file-scope shared arrays and the stencil is the isotropic one
// (4 coefficients), so the run's registers fit the 64 a thread has at 1024
// threads per CTA.
struct RunSeg {
    int iters, maxed;  // maxed: stopped at max_iter
    float rr;          // r.r (in the segment's units) before the last iteration
    int flip32, cflip32;
    int hphase;        // halo mbarrier phases so far (quad_halo_segment)
};

struct RunCgCtx {
    const int* cube;
    double* vc;
    const double* r64;
    int max_iter;
    double target2;
    float drop2;
    int* fault;  // the call's time-out count, incremented when a bounded wait gives up
    long long* vfix;  // fixed-point copy of v (when fix)
    double s2E;       // its scale 2^E
    int fix;          // keep vfix current at the end of each segment
};

__shared__ float g_rc_red32[2][33];
__shared__ float g_rc_part32[2][16];
__shared__ RunCgCtx g_rc;
// one mbarrier per buffer of g_rc_mpart (cluster_sum_mb)
__shared__ __align__(8) unsigned long long g_rc_mbar[2];
__shared__ float g_rc_mpart[2][16];
__shared__ int g_rc_late;  // set once a wait has given up
__shared__ int g_fix_ovf;  // a fixed-point conversion of this CTA left the bound (this pair)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t cluster_addr(uint32_t a, int rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

// Polls the given phase parity of a CTA-local mbarrier at most limit times;
// returns whether the phase completed. Every wait of the cluster solver is one
// of these, so none can spin forever.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mb, uint32_t parity, int limit) {
    uint32_t done = 0;
    for (int it = 0; it < limit && !done; ++it)
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mb), "r"(parity)
            : "memory");
    return done != 0;
}

// Sum over the cluster without a cluster barrier: the CTA total goes to every
// CTA's g_rc_mpart[b][rank] by st.async, which counts its bytes on that CTA's
// mbarrier b; each CTA announces the C x 4 bytes it expects and waits for the
// phase to complete. Buffer b = n & 1 and its phase parity (n >> 1) & 1 follow
// from the running count n of these sums. A CTA refills buffer b (sum n + 2)
// only after every CTA has sent sum n + 1, which each does after all of its
// threads have read sum n, so the two buffers suffice. A wait that gives up
// (it never should) bumps the call's time-out count (*g_rc.fault) and takes
// what has arrived.
template <int NT, int C>
__device__ __forceinline__ float cluster_sum_mb(float v, int& flip, int& n, int rank) {
    v = warp_sum(v);
    float* buf = g_rc_red32[flip];
    flip ^= 1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) buf[w] = v;
    __syncthreads();
    const int b = n & 1;
    const uint32_t parity = (uint32_t)(n >> 1) & 1u;
    ++n;
    const uint32_t mb = smem_u32(&g_rc_mbar[b]);
    if (w == 0) {
        float t = lane < NT / 32 ? buf[lane] : 0.0f;
        t = warp_sum(t);
        if (lane == 0)
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(C * 4) : "memory");
        if (lane < C) {
            const uint32_t dst = cluster_addr(smem_u32(&g_rc_mpart[b][rank]), lane);
            const uint32_t rmb = cluster_addr(mb, lane);
            asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];" ::"r"(dst),
                         "f"(t), "r"(rmb)
                         : "memory");
        }
    }
    if (!mbar_wait_bounded(mb, parity, g_rc_late ? 1 : (1 << 16))) {
        g_rc_late = 1;  // later waits of this CTA give up at once
        if (threadIdx.x == 0) atomicAdd(g_rc.fault, 1);
    }
    float s = 0.0f;
#pragma unroll
    for (int r = 0; r < C; ++r) s += g_rc_mpart[b][r];
    return s;
}

// Four sums at once, as cluster_sum_mb (same mbarriers and phase count, one
// 16-byte st.async per CTA pair).
__shared__ __align__(16) float4 g_rc_red4[2][32];
__shared__ __align__(16) float4 g_rc_mpart4[2][16];

__device__ __forceinline__ float4 warp_sum4(float4 v) {
    v.x = warp_sum(v.x);
    v.y = warp_sum(v.y);
    v.z = warp_sum(v.z);
    v.w = warp_sum(v.w);
    return v;
}

template <int NT, int C>
__device__ __forceinline__ float4 cluster_sum4_mb(float4 v, int& flip, int& n, int rank) {
    v = warp_sum4(v);
    float4* buf = g_rc_red4[flip];
    flip ^= 1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) buf[w] = v;
    __syncthreads();
    const int b = n & 1;
    const uint32_t parity = (uint32_t)(n >> 1) & 1u;
    ++n;
    const uint32_t mb = smem_u32(&g_rc_mbar[b]);
    if (w == 0) {
        float4 t = lane < NT / 32 ? buf[lane] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        t = warp_sum4(t);
        if (lane == 0)
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(C * 16) : "memory");
        if (lane < C) {
            const uint32_t dst = cluster_addr(smem_u32(&g_rc_mpart4[b][rank]), lane);
            const uint32_t rmb = cluster_addr(mb, lane);
            asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(dst),
                         "f"(t.x), "f"(t.y), "f"(t.z), "f"(t.w), "r"(rmb)
                         : "memory");
        }
    }
    if (!mbar_wait_bounded(mb, parity, g_rc_late ? 1 : (1 << 16))) {
        g_rc_late = 1;
        if (threadIdx.x == 0) atomicAdd(g_rc.fault, 1);
    }
    float4 s = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
    for (int r = 0; r < C; ++r) {
        const float4 q = g_rc_mpart4[b][r];
        s.x += q.x;
        s.y += q.y;
        s.z += q.z;
        s.w += q.w;
    }
    return s;
}

template <int NT, int C, int PTS, int SYZ>
__device__ __noinline__ RunSeg run_segment(float* pcr, float* dst, float* hm, float* hp, int rk0, int rlen,
                                           double scale, float carry, float c0, float c1, float c2, float c3,
                                           int iters, int flip32, int cflip32) {
    constexpr int Syz = SYZ, Sp2 = SYZ * SYZ;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    // p of the run: own slab plus the neighbours' halo copies
    auto put_p = [&](int j, float v) {
        pcr[j] = v;
        if (hm) hm[j] = v;
        if (hp) hp[j] = v;
    };
    float r[PTS], ap[PTS], pz[PTS + 6];
    float a32 = 0.0f;
    {
        const double inv = 1.0 / scale;
        const double* r64 = g_rc.r64;
#pragma unroll
        for (int j = 0; j < PTS; ++j) {
            r[j] = 0.0f;
            ap[j] = 0.0f;
            dst[j * NT] = 0.0f;
            if (j < rlen) {
                r[j] = (float)(r64[rk0 + j] * inv);
                put_p(j, carry < 0.0f ? r[j] : fmaf(carry, pcr[j], r[j]));
                a32 = fmaf(r[j], r[j], a32);
            }
        }
    }
    float rr = cluster_sum<NT, C, float>(a32, g_rc_red32, flip32, g_rc_part32, cflip32, cl, rank);
    const float lim = g_rc.drop2 * rr;
    const float conv_thr = (float)(0.25 * g_rc.target2 / (scale * scale));
    RunSeg out;
    for (;;) {
        if (iters >= g_rc.max_iter) {
            out.maxed = 1;
            break;
        }
        float pa = 0.0f;
        if (rlen > 0) {
#pragma unroll
            for (int m = 0; m < PTS + 6; ++m) pz[m] = pcr[m - 3];
#pragma unroll
            for (int j = 0; j < PTS; ++j) {
                const float x1 = pcr[j + Sp2] + pcr[j - Sp2];
                const float x2 = pcr[j + 2 * Sp2] + pcr[j - 2 * Sp2];
                const float x3 = pcr[j + 3 * Sp2] + pcr[j - 3 * Sp2];
                const float s1 = (pz[j + 4] + pz[j + 2]) + (pcr[j + Syz] + pcr[j - Syz]) + x1;
                const float s2 = (pz[j + 5] + pz[j + 1]) + (pcr[j + 2 * Syz] + pcr[j - 2 * Syz]) + x2;
                const float s3 = (pz[j + 6] + pz[j]) + (pcr[j + 3 * Syz] + pcr[j - 3 * Syz]) + x3;
                const float a = fmaf(c0, pz[j + 3], fmaf(c1, s1, fmaf(c2, s2, c3 * s3)));
                ap[j] = -a;
                if (j < rlen) pa = fmaf(pz[j + 3], -a, pa);
            }
        }
        const float pap = cluster_sum<NT, C, float>(pa, g_rc_red32, flip32, g_rc_part32, cflip32, cl, rank);
        const float al = rr / pap;
        float ra = 0.0f;
#pragma unroll
        for (int j = 0; j < PTS; ++j) {
            if (j < rlen) {
                dst[j * NT] = fmaf(al, pz[j + 3], dst[j * NT]);
                r[j] = fmaf(-al, ap[j], r[j]);
                ra = fmaf(r[j], r[j], ra);
            }
        }
        const float rrn = cluster_sum<NT, C, float>(ra, g_rc_red32, flip32, g_rc_part32, cflip32, cl, rank);
        ++iters;
        if (rrn <= lim || rrn <= conv_thr || !(rrn == rrn)) {
            out.maxed = 0;
            break;
        }
        const float be = rrn / rr;
        rr = rrn;
#pragma unroll
        for (int j = 0; j < PTS; ++j)
            if (j < rlen) put_p(j, fmaf(be, pz[j + 3], r[j]));
        cl.sync();
    }
    // v += scale d
    const int* cube = g_rc.cube;
    double* vc = g_rc.vc;
#pragma unroll
    for (int j = 0; j < PTS; ++j) {
        if (j < rlen) {
            const int c = cube[rk0 + j];
            vc[c] = fma(scale, (double)dst[j * NT], vc[c]);
        }
    }
    out.iters = iters;
    out.rr = rr;
    out.flip32 = flip32;
    out.cflip32 = cflip32;
    return out;
}

// The point-map CG of one pair in segments, like run_segment: each thread
// slot j holds one point (slab offset | plane << 24 in spk, compact index in
// slot_k); x legs leaving the slab read the neighbour's slab (pm, pp). SYZ > 0
// makes the box pitches compile-time constants and ISO selects the isotropic
// stencil (4 coefficients), both to keep the loop within 64 registers.
struct StencilArgs {
    float c0, cx[3], cy[3], cz[3];
};

template <int NT, int C, int PTS, int SYZ, bool ISO>
__device__ __noinline__ RunSeg pts_segment(float* ps, const float* pm, const float* pp, float* dst, const int* spt,
                                           const int* skt, int planes, int planes_prev, int syz_rt, double scale,
                                           float carry, StencilArgs sa, int iters, int flip32, int cflip32) {
    const int Syz = SYZ > 0 ? SYZ : syz_rt;
    const int Sp2 = Syz * Syz;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    float r[PTS], ap[PTS];
    float a32 = 0.0f;
    {
        const double inv = 1.0 / scale;
        const double* r64 = g_rc.r64;
#pragma unroll
        for (int j = 0; j < PTS; ++j) {
            r[j] = 0.0f;
            ap[j] = 0.0f;
            dst[j * NT] = 0.0f;
            const int pkj = spt[j * NT];
            if (pkj >= 0) {
                const int off = pkj & 0xffffff;
                r[j] = (float)(r64[skt[j * NT]] * inv);
                ps[off] = carry < 0.0f ? r[j] : fmaf(carry, ps[off], r[j]);
                a32 = fmaf(r[j], r[j], a32);
            }
        }
    }
    float rr = cluster_sum<NT, C, float>(a32, g_rc_red32, flip32, g_rc_part32, cflip32, cl, rank);
    const float lim = g_rc.drop2 * rr;
    const float conv_thr = (float)(0.25 * g_rc.target2 / (scale * scale));
    RunSeg out;
    for (;;) {
        if (iters >= g_rc.max_iter) {
            out.maxed = 1;
            break;
        }
        float pa = 0.0f;
#pragma unroll
        for (int j = 0; j < PTS; ++j) {
            const int pkj = spt[j * NT];
            if (pkj >= 0) {
                const int off = pkj & 0xffffff, xl = pkj >> 24;
                const float pc = ps[off];
                float sz[3], sy[3], sx[3];
#pragma unroll
                for (int q = 1; q <= 3; ++q) {
                    sz[q - 1] = ps[off + q] + ps[off - q];
                    sy[q - 1] = ps[off + q * Syz] + ps[off - q * Syz];
                    const float xpv = xl + q < planes ? ps[off + q * Sp2] : (pp ? pp[off + (q - planes) * Sp2] : 0.0f);
                    const float xmv = xl - q >= 0 ? ps[off - q * Sp2] : (pm ? pm[off + (planes_prev - q) * Sp2] : 0.0f);
                    sx[q - 1] = xpv + xmv;
                }
                float a;
                if constexpr (ISO) {
                    a = fmaf(sa.c0, pc, fmaf(sa.cz[0], (sz[0] + sy[0]) + sx[0],
                                             fmaf(sa.cz[1], (sz[1] + sy[1]) + sx[1], sa.cz[2] * ((sz[2] + sy[2]) + sx[2]))));
                } else {
                    const float az = fmaf(sa.cz[0], sz[0], fmaf(sa.cz[1], sz[1], sa.cz[2] * sz[2]));
                    const float ay = fmaf(sa.cy[0], sy[0], fmaf(sa.cy[1], sy[1], sa.cy[2] * sy[2]));
                    const float ax = fmaf(sa.cx[0], sx[0], fmaf(sa.cx[1], sx[1], sa.cx[2] * sx[2]));
                    a = fmaf(sa.c0, pc, (az + ay) + ax);
                }
                ap[j] = -a;
                pa = fmaf(pc, -a, pa);
            }
        }
        const float pap = cluster_sum<NT, C, float>(pa, g_rc_red32, flip32, g_rc_part32, cflip32, cl, rank);
        const float al = rr / pap;
        float ra = 0.0f;
#pragma unroll
        for (int j = 0; j < PTS; ++j) {
            const int pkj = spt[j * NT];
            if (pkj >= 0) {
                dst[j * NT] = fmaf(al, ps[pkj & 0xffffff], dst[j * NT]);
                r[j] = fmaf(-al, ap[j], r[j]);
                ra = fmaf(r[j], r[j], ra);
            }
        }
        const float rrn = cluster_sum<NT, C, float>(ra, g_rc_red32, flip32, g_rc_part32, cflip32, cl, rank);
        ++iters;
        if (rrn <= lim || rrn <= conv_thr || !(rrn == rrn)) {
            out.maxed = 0;
            break;
        }
        const float be = rrn / rr;
        rr = rrn;
#pragma unroll
        for (int j = 0; j < PTS; ++j) {
            const int pkj = spt[j * NT];
            if (pkj >= 0) {
                const int off = pkj & 0xffffff;
                ps[off] = fmaf(be, ps[off], r[j]);
            }
        }
        cl.sync();
    }
    // v += scale d
    const int* cube = g_rc.cube;
    double* vc = g_rc.vc;
#pragma unroll
    for (int j = 0; j < PTS; ++j) {
        if (spt[j * NT] >= 0) {
            const int c = cube[skt[j * NT]];
            vc[c] = fma(scale, (double)dst[j * NT], vc[c]);
        }
    }
    out.iters = iters;
    out.rr = rr;
    out.flip32 = flip32;
    out.cflip32 = cflip32;
    return out;
}

// The quad-map CG of one pair in segments (MODE 2), like pts_segment: thread
// slot j holds a 16-byte aligned quad of 4 consecutive z positions of a slab
// row (spt: slab offset | valid mask << 20 | plane << 24; skt: compact index
// of element 0), and a warp covers consecutive quads. Every stencil leg is one
// 16-byte load: the quad itself and the quads before and after it (the z legs),
// and the quads one to three rows or planes away (the y and x legs; x legs
// past the slab come from the neighbour's slab). Elements outside the ball
// keep r = 0 (their A p is masked) and therefore p = 0. SY > 0 is the box side
// 2 R_PE + 7 the pitches are specialised for (row pitch rounded up to 4).
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

template <int NT, int C, int Q, int SY, bool ISO>
__device__ __noinline__ RunSeg quad_segment(float* ps, const float* pm, const float* pp, float4* dst, const int* spt,
                                            const int* skt, int planes, int planes_prev, int syz_rt, int sp2_rt,
                                            double scale, float carry, StencilArgs sa, int iters, int flip32,
                                            int cflip32) {
    constexpr int PZ = (SY + 3) & ~3;
    const int Syz = SY > 0 ? PZ : syz_rt;
    const int Sp2 = SY > 0 ? SY * PZ : sp2_rt;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    float4 r[Q], ap[Q];
    float a32 = 0.0f;
    {
        const double inv = 1.0 / scale;
        const double* r64 = g_rc.r64;
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const int pk = spt[j * NT];
            const int off = pk & 0xfffff, m = (pk >> 20) & 15;
            const int k = skt[j * NT];
            float4 rv;
            rv.x = (m & 1) ? (float)(r64[k] * inv) : 0.0f;
            rv.y = (m & 2) ? (float)(r64[k + 1] * inv) : 0.0f;
            rv.z = (m & 4) ? (float)(r64[k + 2] * inv) : 0.0f;
            rv.w = (m & 8) ? (float)(r64[k + 3] * inv) : 0.0f;
            r[j] = rv;
            ap[j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            dst[j * NT] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            float4 pv = rv;
            if (carry >= 0.0f) {
                const float4 po = ld4(ps + off);
                pv.x = fmaf(carry, po.x, rv.x);
                pv.y = fmaf(carry, po.y, rv.y);
                pv.z = fmaf(carry, po.z, rv.z);
                pv.w = fmaf(carry, po.w, rv.w);
            }
            st4(ps + off, pv);
            a32 = fmaf(rv.x, rv.x, fmaf(rv.y, rv.y, fmaf(rv.z, rv.z, fmaf(rv.w, rv.w, a32))));
        }
    }
    float rr = cluster_sum_mb<NT, C>(a32, flip32, cflip32, rank);
    const float lim = g_rc.drop2 * rr;
    const float conv_thr = (float)(0.25 * g_rc.target2 / (scale * scale));
    const float4 zero4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    RunSeg out;
    float al = 0.0f;
    for (;;) {
        if (iters >= g_rc.max_iter) {
            out.maxed = 1;
            break;
        }
        float pa = 0.0f;
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const int pk = spt[j * NT];
            const int off = pk & 0xfffff, m = (pk >> 20) & 15, xl = (int)((unsigned)pk >> 24);
            const float* b = ps + off;
            const float4 c = ld4(b), zl = ld4(b - 4), zh = ld4(b + 4);
            // z window: w[i + 3] is element i, i = -3 .. 6
            const float w[10] = {zl.y, zl.z, zl.w, c.x, c.y, c.z, c.w, zh.x, zh.y, zh.z};
            const float cz1 = sa.cz[0], cz2 = sa.cz[1], cz3 = sa.cz[2];
            float a[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                a[i] = fmaf(cz1, w[i + 4] + w[i + 2],
                            fmaf(cz2, w[i + 5] + w[i + 1], fmaf(cz3, w[i + 6] + w[i], sa.c0 * w[i + 3])));
#pragma unroll
            for (int q = 1; q <= 3; ++q) {
                const float cyq = ISO ? sa.cz[q - 1] : sa.cy[q - 1];
                const float4 ym = ld4(b - q * Syz), yp = ld4(b + q * Syz);
                a[0] = fmaf(cyq, ym.x + yp.x, a[0]);
                a[1] = fmaf(cyq, ym.y + yp.y, a[1]);
                a[2] = fmaf(cyq, ym.z + yp.z, a[2]);
                a[3] = fmaf(cyq, ym.w + yp.w, a[3]);
            }
#pragma unroll
            for (int q = 1; q <= 3; ++q) {
                const float cxq = ISO ? sa.cz[q - 1] : sa.cx[q - 1];
                const float4 xp = xl + q < planes ? ld4(b + q * Sp2)
                                                  : (pp ? ld4(pp + off + (q - planes) * Sp2) : zero4);
                const float4 xm = xl - q >= 0 ? ld4(b - q * Sp2)
                                              : (pm ? ld4(pm + off + (planes_prev - q) * Sp2) : zero4);
                a[0] = fmaf(cxq, xm.x + xp.x, a[0]);
                a[1] = fmaf(cxq, xm.y + xp.y, a[1]);
                a[2] = fmaf(cxq, xm.z + xp.z, a[2]);
                a[3] = fmaf(cxq, xm.w + xp.w, a[3]);
            }
            // A p = -lap p on the ball's elements, 0 elsewhere
            float4 av;
            av.x = (m & 1) ? -a[0] : 0.0f;
            av.y = (m & 2) ? -a[1] : 0.0f;
            av.z = (m & 4) ? -a[2] : 0.0f;
            av.w = (m & 8) ? -a[3] : 0.0f;
            ap[j] = av;
            pa = fmaf(c.x, av.x, fmaf(c.y, av.y, fmaf(c.z, av.z, fmaf(c.w, av.w, pa))));
        }
        const float pap = cluster_sum_mb<NT, C>(pa, flip32, cflip32, rank);
        al = rr / pap;
        float ra = 0.0f;
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            r[j].x = fmaf(-al, ap[j].x, r[j].x);
            r[j].y = fmaf(-al, ap[j].y, r[j].y);
            r[j].z = fmaf(-al, ap[j].z, r[j].z);
            r[j].w = fmaf(-al, ap[j].w, r[j].w);
            ra = fmaf(r[j].x, r[j].x, fmaf(r[j].y, r[j].y, fmaf(r[j].z, r[j].z, fmaf(r[j].w, r[j].w, ra))));
        }
        const float rrn = cluster_sum_mb<NT, C>(ra, flip32, cflip32, rank);
        ++iters;
        if (rrn <= lim || rrn <= conv_thr || !(rrn == rrn)) {
            out.maxed = 0;
            break;
        }
        const float be = rrn / rr;
        rr = rrn;
        // d += alpha p and p = r + beta p in one pass over the quads
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            float* b = ps + (spt[j * NT] & 0xfffff);
            const float4 po = ld4(b);
            float4 d = dst[j * NT];
            d.x = fmaf(al, po.x, d.x);
            d.y = fmaf(al, po.y, d.y);
            d.z = fmaf(al, po.z, d.z);
            d.w = fmaf(al, po.w, d.w);
            dst[j * NT] = d;
            st4(b, make_float4(fmaf(be, po.x, r[j].x), fmaf(be, po.y, r[j].y), fmaf(be, po.z, r[j].z),
                               fmaf(be, po.w, r[j].w)));
        }
        al = 0.0f;
        cl.sync();
    }
    // the last iteration's d += alpha p (p is unchanged since its stencil), then v += scale d
    const int* cube = g_rc.cube;
    double* vc = g_rc.vc;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const int pk = spt[j * NT];
        const int m = (pk >> 20) & 15;
        const float4 po = ld4(ps + (pk & 0xfffff));
        float4 d = dst[j * NT];
        d.x = fmaf(al, po.x, d.x);
        d.y = fmaf(al, po.y, d.y);
        d.z = fmaf(al, po.z, d.z);
        d.w = fmaf(al, po.w, d.w);
        const int k = skt[j * NT];
        const float dv[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (m & (1 << i)) {
                const int cc = cube[k + i];
                vc[cc] = fma(scale, (double)dv[i], vc[cc]);
            }
        }
    }
    out.iters = iters;
    out.rr = rr;
    out.flip32 = flip32;
    out.cflip32 = cflip32;
    return out;
}

// The quad-map CG with halo planes (MODE 3). The slab array holds 3 halo planes
// on each side of the CTA's planes (pc = plane 0), so every stencil leg is a
// local 16-byte load at a fixed offset. Whenever a CTA has written p, one
// thread copies its first and last 3 planes into the neighbours' halos with
// two bulk copies (cp.async.bulk, shared::cta -> shared::cluster), counted in
// bytes on the neighbours' halo mbarriers (g_halo_mbar), and opens the next
// phase of its own, announcing the bytes the neighbours send in it. An
// iteration first applies the centre, z and y legs, which read only the CTA's
// own planes (complete after a CTA barrier), then waits for the phase and
// applies the x legs, so the exchange overlaps the first pass: no cluster
// barrier. The correction d stays in registers. A neighbour refills a halo
// only after the cluster sum of the iteration, to which this CTA contributed
// after its x legs, so one mbarrier suffices; its phase count hph runs for
// the whole launch, and every phase opened is waited for.
__shared__ __align__(8) unsigned long long g_halo_mbar;

// Test of the time-out path (exx_options.inject_wait_timeout): a bounded wait
// on a fresh mbarrier that nothing arrives on and no copy or store targets
// runs out; the count reaches the host as EXX_ETIMEOUT and the rest of the
// launch is unchanged. The barrier is a spare 8-byte word past the end of the
// launch's dynamic shared memory layout, and the code stays out of line, so
// the kernel's own code and static shared layout do not change.
__device__ __noinline__ void inject_wait_timeout(uint32_t mb, int* timeouts) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
    if (!mbar_wait_bounded(mb, 0u, 256)) atomicAdd(timeouts, 1);
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(mb) : "memory");
}

// Byte offset of that spare word in the dynamic shared memory of a launch
// (after the slab, d and the slot map as cluster_kernel_smem counts them).
__host__ __device__ inline size_t cluster_smem_test_offset(const ClusterLayout& CL, int mode, int pts, int nt) {
    const size_t per = (size_t)nt * pts;
    const bool runs = mode == 1, halo = mode == 1 || mode == 3;
    const size_t slab = (size_t)(CL.cap_planes + (halo ? 6 : 0)) * CL.Sp2;
    const size_t dsf = mode == 3 ? 0 : (mode == 2 ? 4 : 1) * per;
    const size_t b = sizeof(float) * (((slab + 3) & ~(size_t)3) + dsf) + (runs ? 0 : sizeof(int) * per);
    return (b + 7) & ~(size_t)7;
}

// Bounded wait for the given phase parity of a CTA-local mbarrier; a wait that
// gives up marks the CTA late (later waits give up at once) and bumps the fault count.
__device__ __forceinline__ void halo_wait(uint32_t mb, uint32_t parity) {
    if (!mbar_wait_bounded(mb, parity, g_rc_late ? 1 : (1 << 16))) {
        g_rc_late = 1;
        if (threadIdx.x == 0) atomicAdd(g_rc.fault, 1);
    }
}

template <int NT, int C, int Q, int SY, bool ISO>
__device__ __noinline__ RunSeg quad_halo_segment(float* pc, const int* spt, const int* skt, int planes, uint32_t nbl,
                                                 uint32_t nbr, uint32_t mbl, uint32_t mbr,
                                                 int syz_rt, int sp2_rt, double scale, float carry, StencilArgs sa,
                                                 int iters, int flip32, int cflip32, int hph) {
    constexpr int PZ = (SY + 3) & ~3;
    const int Syz = SY > 0 ? PZ : syz_rt;
    const int Sp2 = SY > 0 ? SY * PZ : sp2_rt;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const uint32_t hmb = smem_u32(&g_halo_mbar);
    float4 r[Q], ap[Q], d[Q];
    auto put_p = [&](int pk, float4 v) { st4(pc + (pk & 0xfffff), v); };
    // After a CTA barrier (this CTA's p complete), thread 0 copies the first
    // and last 3 planes into the neighbours' halos by bulk copies that count
    // their bytes on the neighbours' halo mbarriers, and opens the next phase
    // of its own, announcing the bytes the neighbours send.
    const uint32_t plane3 = 12u * (uint32_t)Sp2;  // bytes of 3 planes
    const uint32_t in_bytes = (rank > 0 ? plane3 : 0u) + (rank < C - 1 ? plane3 : 0u);
    auto publish = [&]() {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // p writes -> the bulk copies' reads
        __syncthreads();
        if (threadIdx.x == 0) {
            if (rank > 0)
                asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                             ::"r"(nbl), "r"(smem_u32(pc)), "r"(plane3), "r"(mbl) : "memory");
            if (rank < C - 1) {
                const uint32_t o = 4u * (uint32_t)((planes - 3) * Sp2);
                asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                             ::"r"(nbr + o), "r"(smem_u32(pc) + o), "r"(plane3), "r"(mbr) : "memory");
            }
            asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(hmb), "r"(in_bytes)
                         : "memory");
        }
    };
    float a32 = 0.0f;
    {
        const double inv = 1.0 / scale;
        const double* r64 = g_rc.r64;
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const int pk = spt[j * NT];
            const int off = pk & 0xfffff, m = (pk >> 20) & 15;
            const int k = skt[j * NT];
            float4 rv;
            rv.x = (m & 1) ? (float)(r64[k] * inv) : 0.0f;
            rv.y = (m & 2) ? (float)(r64[k + 1] * inv) : 0.0f;
            rv.z = (m & 4) ? (float)(r64[k + 2] * inv) : 0.0f;
            rv.w = (m & 8) ? (float)(r64[k + 3] * inv) : 0.0f;
            r[j] = rv;
            d[j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            float4 pv = rv;
            if (carry >= 0.0f) {
                const float4 po = ld4(pc + off);
                pv.x = fmaf(carry, po.x, rv.x);
                pv.y = fmaf(carry, po.y, rv.y);
                pv.z = fmaf(carry, po.z, rv.z);
                pv.w = fmaf(carry, po.w, rv.w);
            }
            put_p(pk, pv);
            a32 = fmaf(rv.x, rv.x, fmaf(rv.y, rv.y, fmaf(rv.z, rv.z, fmaf(rv.w, rv.w, a32))));
        }
    }
    publish();
    float rr = cluster_sum4_mb<NT, C>(make_float4(a32, 0.0f, 0.0f, 0.0f), flip32, cflip32, rank).x;
    const float lim = g_rc.drop2 * rr;
    const float conv_thr = (float)(0.25 * g_rc.target2 / (scale * scale));
    RunSeg out;
    float al = 0.0f;
    for (;;) {
        if (iters >= g_rc.max_iter) {
            halo_wait(hmb, (uint32_t)hph & 1u);  // complete the pending phase
            ++hph;
            out.maxed = 1;
            break;
        }
        // p.Ap, r.Ap, Ap.Ap and r.r in one cluster sum: alpha = r.r / p.Ap and
        // r.r after the update = r.r - 2 alpha r.Ap + alpha^2 Ap.Ap, all four from
        // this iteration's vectors. (Carrying the predicted r.r into the next
        // iteration instead of summing it afresh lets its rounding errors add up
        // while r.r falls, and the solve diverges.)
        float pa = 0.0f, ra = 0.0f, aa = 0.0f, rq = 0.0f;
        // pass 1, while the neighbours' planes are still on their way: the
        // centre, z and y legs, which read only this CTA's planes
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const float* b = pc + (spt[j * NT] & 0xfffff);
            const float4 c = ld4(b), zl = ld4(b - 4), zh = ld4(b + 4);
            const float w[10] = {zl.y, zl.z, zl.w, c.x, c.y, c.z, c.w, zh.x, zh.y, zh.z};
            float a[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                a[i] = fmaf(sa.cz[0], w[i + 4] + w[i + 2],
                            fmaf(sa.cz[1], w[i + 5] + w[i + 1], fmaf(sa.cz[2], w[i + 6] + w[i], sa.c0 * w[i + 3])));
#pragma unroll
            for (int q = 1; q <= 3; ++q) {
                const float cyq = ISO ? sa.cz[q - 1] : sa.cy[q - 1];
                const float4 ym = ld4(b - q * Syz), yp = ld4(b + q * Syz);
                a[0] = fmaf(cyq, ym.x + yp.x, a[0]);
                a[1] = fmaf(cyq, ym.y + yp.y, a[1]);
                a[2] = fmaf(cyq, ym.z + yp.z, a[2]);
                a[3] = fmaf(cyq, ym.w + yp.w, a[3]);
            }
            ap[j] = make_float4(a[0], a[1], a[2], a[3]);
        }
        halo_wait(hmb, (uint32_t)hph & 1u);  // the halos hold the neighbours' p
        ++hph;
        // pass 2: the x legs, the mask and the dot products
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const int pk = spt[j * NT];
            const int m = (pk >> 20) & 15;
            const float* b = pc + (pk & 0xfffff);
            const float4 c = ld4(b);
            float a[4] = {ap[j].x, ap[j].y, ap[j].z, ap[j].w};
#pragma unroll
            for (int q = 1; q <= 3; ++q) {
                const float cxq = ISO ? sa.cz[q - 1] : sa.cx[q - 1];
                const float4 xm = ld4(b - q * Sp2), xp = ld4(b + q * Sp2);
                a[0] = fmaf(cxq, xm.x + xp.x, a[0]);
                a[1] = fmaf(cxq, xm.y + xp.y, a[1]);
                a[2] = fmaf(cxq, xm.z + xp.z, a[2]);
                a[3] = fmaf(cxq, xm.w + xp.w, a[3]);
            }
            float4 av;
            av.x = (m & 1) ? -a[0] : 0.0f;
            av.y = (m & 2) ? -a[1] : 0.0f;
            av.z = (m & 4) ? -a[2] : 0.0f;
            av.w = (m & 8) ? -a[3] : 0.0f;
            ap[j] = av;
            pa = fmaf(c.x, av.x, fmaf(c.y, av.y, fmaf(c.z, av.z, fmaf(c.w, av.w, pa))));
            ra = fmaf(r[j].x, av.x, fmaf(r[j].y, av.y, fmaf(r[j].z, av.z, fmaf(r[j].w, av.w, ra))));
            aa = fmaf(av.x, av.x, fmaf(av.y, av.y, fmaf(av.z, av.z, fmaf(av.w, av.w, aa))));
            rq = fmaf(r[j].x, r[j].x, fmaf(r[j].y, r[j].y, fmaf(r[j].z, r[j].z, fmaf(r[j].w, r[j].w, rq))));
        }
        const float4 sums = cluster_sum4_mb<NT, C>(make_float4(pa, ra, aa, rq), flip32, cflip32, rank);
        rr = sums.w;
        al = rr / sums.x;
        const float rrn = fmaf(al, fmaf(al, sums.z, -2.0f * sums.y), rr);
        ++iters;
        if (rrn <= lim || rrn <= conv_thr || !(rrn == rrn)) {
            out.maxed = 0;
            break;
        }
        const float be = rrn / rr;
        // d += alpha p, r -= alpha Ap and p = r + beta p, then publish p
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const int pk = spt[j * NT];
            const float4 po = ld4(pc + (pk & 0xfffff));
            d[j].x = fmaf(al, po.x, d[j].x);
            d[j].y = fmaf(al, po.y, d[j].y);
            d[j].z = fmaf(al, po.z, d[j].z);
            d[j].w = fmaf(al, po.w, d[j].w);
            r[j].x = fmaf(-al, ap[j].x, r[j].x);
            r[j].y = fmaf(-al, ap[j].y, r[j].y);
            r[j].z = fmaf(-al, ap[j].z, r[j].z);
            r[j].w = fmaf(-al, ap[j].w, r[j].w);
            put_p(pk, make_float4(fmaf(be, po.x, r[j].x), fmaf(be, po.y, r[j].y), fmaf(be, po.z, r[j].z),
                                  fmaf(be, po.w, r[j].w)));
        }
        al = 0.0f;
        publish();  // also makes this CTA's p complete for pass 1 of the next iteration
    }
    // the last iteration's d += alpha p (p is unchanged since its stencil), then v += scale d
    const int* cube = g_rc.cube;
    double* vc = g_rc.vc;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const int pk = spt[j * NT];
        const int m = (pk >> 20) & 15;
        const float4 po = ld4(pc + (pk & 0xfffff));
        const float dv[4] = {fmaf(al, po.x, d[j].x), fmaf(al, po.y, d[j].y), fmaf(al, po.z, d[j].z),
                             fmaf(al, po.w, d[j].w)};
        const int k = skt[j * NT];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (m & (1 << i)) {
                const int cc = cube[k + i];
                const double nv = fma(scale, (double)dv[i], vc[cc]);
                vc[cc] = nv;
                if (g_rc.fix) {
                    int o = 0;
                    g_rc.vfix[cc] = to_fix(nv, g_rc.s2E, o);
                    if (o) g_fix_ovf = 1;
                }
            }
        }
    }
    out.iters = iters;
    out.rr = rr;
    out.flip32 = flip32;
    out.cflip32 = cflip32;
    out.hphase = hph;
    return out;
}

// MODE 0: thread slot j of a thread holds one point of the slab (the
// [PTS][NT] point map); x legs that leave the slab read the neighbour's slab.
// MODE 1: the thread owns one run of at most PTS consecutive points of a
// slab row, and the slab carries 3 halo planes on each side that the
// neighbours fill with remote stores whenever they write p; the stencil then
// reads only the CTA's own shared memory at fixed offsets, the run's p values
// and z neighbours stay in registers (a point costs 12 shared loads plus a
// share of the run's PTS + 6), and the thread map puts the runs of a warp in
// distinct banks.
// MODE 2: thread slot j holds a quad of 4 consecutive z positions (PTS quads
// per thread, rows padded to a multiple of 4 points), so every stencil leg
// is one 16-byte load for 4 points (quad_segment).
template <int NT, int C, int PTS, int MODE, int SYZ, bool ISO>
__global__ void __launch_bounds__(NT, 1) cluster_pair_kernel(const __grid_constant__ SolveParams P,
                                                             const __grid_constant__ ClusterLayout CL) {
    constexpr bool RUNS = MODE == 1, HALO = MODE == 1 || MODE == 3, QUADS = MODE == 2 || MODE == 3;
    constexpr bool QHALO = MODE == 3;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    extern __shared__ __align__(16) double smem[];
    __shared__ double red[2][33];
    __shared__ double part[2][16];
    __shared__ double s_M[kNMono], s_T[kNMono];
    __shared__ int s_item;
    int flip = 0, cflip = 0;
    // FP32 reduction state, kept for the whole launch: the quad segments' mbarrier
    // phases advance with every sum (cluster_sum_mb), across segments and pairs
    int f32 = 0, cf32 = 0, hph = 0;

    const int Rc = P.Rc;
    // FP64 power tables (global, read-only) and this CTA's plane sums (global slot)
    const double* xp = P.pow_tab;
    const double* yp = xp + (2 * Rc + 1) * 8;
    const double* zp = yp + (2 * Rc + 1) * 8;
    // shared memory: the p slab, then the CG correction d and the point map, [PTS][NT] each
    float* ps = reinterpret_cast<float*>(smem);
    const int slab_floats = (CL.cap_planes + (HALO ? 6 : 0)) * CL.Sp2;
    float* ds = ps + ((slab_floats + 3) & ~3);  // 16-byte aligned
    // MODE 3 keeps d in registers (no ds)
    constexpr int ds_floats = QHALO ? 0 : (QUADS ? 4 : 1) * PTS * NT;
    int* spk = RUNS ? nullptr : reinterpret_cast<int*>(ds + ds_floats);
    const int Syz = CL.Syz;
    const int Sp2 = CL.Sp2;

    for (int t = threadIdx.x; t < slab_floats; t += NT) ps[t] = 0.0f;

    float* pm = rank > 0 ? cl.map_shared_rank(ps, rank - 1) : nullptr;
    float* pp = rank < C - 1 ? cl.map_shared_rank(ps, rank + 1) : nullptr;
    const int4 me = CL.rank_info[rank];
    const int planes = me.y;
    const int planes_prev = rank > 0 ? CL.rank_info[rank - 1].y : 0;
    const int k0 = me.z, k1 = me.w;
    const int* slot_k = RUNS ? nullptr : CL.slot_k + (size_t)rank * PTS * NT;
    // RUNS: this thread's run (slab offset, plane, first compact index, length)
    // and where its p values go in the neighbours' halo planes
    int roff = 0, rxl = 0, rk0 = 0, rlen = 0;
    float* pc = ps;                               // plane 0 of the CTA's slab
    float *hm = nullptr, *hp = nullptr;
    if constexpr (RUNS) {
        pc = ps + 3 * Sp2;
        const int rpk = CL.slot_pk[(size_t)rank * NT + threadIdx.x];
        const int rk = CL.slot_k[(size_t)rank * NT + threadIdx.x];
        if (rpk >= 0) {
            roff = rpk & 0xffffff;
            rxl = rpk >> 24;
            rlen = rk >> 24;
            rk0 = rk & 0xffffff;
        }
        const int pl = CL.rank_info[rank].y, plp = rank > 0 ? CL.rank_info[rank - 1].y : 0;
        const int rest = roff - rxl * Sp2;  // row and column within the plane
        if (rlen > 0 && rank > 0 && rxl < 3)
            hm = cl.map_shared_rank(ps, rank - 1) + (3 + plp + rxl) * Sp2 + rest;
        if (rlen > 0 && rank < C - 1 && rxl >= pl - 3)
            hp = cl.map_shared_rank(ps, rank + 1) + (3 + rxl - pl) * Sp2 + rest;
    } else {
        if constexpr (QHALO) pc = ps + 3 * Sp2;
#pragma unroll
        for (int j = 0; j < PTS; ++j)
            spk[j * NT + threadIdx.x] = CL.slot_pk[(size_t)rank * PTS * NT + j * NT + threadIdx.x];
    }
    // MODE 3: where this CTA's first and last planes go in the neighbours'
    // halos (shared::cluster addresses of the image of pc) and their halo mbarriers
    uint32_t nbl = 0, nbr = 0, mbl = 0, mbr = 0;
    if constexpr (QHALO) {
        const uint32_t base = smem_u32(ps), hm0 = smem_u32(&g_halo_mbar);
        if (rank > 0) {
            nbl = cluster_addr(base, rank - 1) + 4u * (uint32_t)((3 + planes_prev) * Sp2);
            mbl = cluster_addr(hm0, rank - 1);
        }
        if (rank < C - 1) {
            nbr = cluster_addr(base, rank + 1) + 4u * (uint32_t)((3 - planes) * Sp2);
            mbr = cluster_addr(hm0, rank + 1);
        }
    }

    const int cid = blockIdx.x / C;
    char* slot = P.ws + (size_t)cid * P.slot_bytes;
    double* vc = reinterpret_cast<double*>(slot + P.off_vcube);
    double* rho = reinterpret_cast<double*>(slot + P.off_rho);
    double* r64 = reinterpret_cast<double*>(slot + P.off_r);
    double* rowS = reinterpret_cast<double*>(slot + P.off_rows);
    double* sYc = reinterpret_cast<double*>(slot + P.off_sy);  // plane sums of the whole ball (cluster-shared)
    long long* vfix = reinterpret_cast<long long*>(slot + P.off_vfix);  // fixed-point v (mode 3)
    // the shell's row coefficients U_{l,c}: FP64, then the FP32 copy (shell_rows)
    double* U64 = reinterpret_cast<double*>(slot + P.off_ush);
    float* U32 = reinterpret_cast<float*>(U64 + (size_t)kNU * P.geos[P.n_geo - 1].n_rows_me);

    const int gt = rank * NT + (int)threadIdx.x, gn = C * NT;
    const int np = *P.n_pair;
    if (QUADS && threadIdx.x == 0) {
        // the quad segments' reduction barriers (count 1: this CTA's own arrive)
        for (int b = 0; b < 2; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&g_rc_mbar[b])) : "memory");
        if (QHALO)  // thread 0 arrives once per phase; the neighbours' bytes complete it
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&g_halo_mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        g_rc_late = 0;
    }
    cl.sync();

    for (;;) {
        if (rank == 0 && threadIdx.x == 0) {
            const int it = atomicAdd(P.queue, 1);
            for (int r = 0; r < C; ++r) *cl.map_shared_rank(&s_item, r) = it;
        }
        cl.sync();
        const int item = s_item;
        if (item >= np) break;
        const int pidx = P.order ? P.order[(P.item_base ? *P.item_base : 0) + item] : item;
        const PairRec pr = P.pairs[pidx];
        const BallGeo G = P.geos[pr.geo];
        const int* cube = G.pt_cube;

        const bool clk = P.phase_clk && rank == 0 && threadIdx.x == 0;
        long long t0 = clk ? clock64() : 0, tr = 0;

        // gather, multipoles, shell potential (FP64, spread over the cluster)
        gather_rho(P, G, pr, rho, vc, gt, gn);
        cl.sync();
        moment_rows(P, G, rho, rowS, zp, gt, gn);
        cl.sync();
        moment_finish_cluster<NT>(P, G, rowS, xp, yp, sYc, me.x + G.r_pe, planes, s_M, s_T, cl);
        shell_rows(P, G, xp, yp, s_T, U64, U32, gt, gn);
        cl.sync();
        const double vnear = shell_points<true>(P, G, vc, U64, U32, G.sh_near, G.n_near, gt, gn);
        shell_points<false>(P, G, vc, U64, U32, G.sh_far, G.n_far, gt, gn);
        // fixed-point copy of v for the FP64 residuals (mode 3, isotropic grids):
        // |v| <= max |v| on the shell layer + (2 pi / 3) max |rho| (R_PE delta)^2
        // (the ball's maximum-principle bound), taken twice over
        bool fix = QHALO && P.fixres;
        double s2E = 0.0, finvE = 0.0;
        if (fix) {
            double rm = 0.0;
            for (int k = gt; k < G.n_pe; k += gn) rm = fmax(rm, fabs(rho[k]));
            const double a2 = (double)G.r_pe * G.r_pe * P.delta[0] * P.delta[0];
            const double vb = 2.0 * cluster_max<NT, C>(fmax(vnear, (kFourPi / 3.0) * rm * a2), red, flip, part,
                                                      cflip, cl, rank);
            int e = 0;
            (void)frexp(vb, &e);  // vb < 2^e
            if (P.fixres == 2) e -= 60;  // test mode: the copy overflows, the pair falls back
            if (!(vb < 1e300)) fix = false;
            s2E = ldexp(1.0, 50 - e);
            finvE = ldexp(P.fix_inv, e - 50);
            if (threadIdx.x == 0) g_fix_ovf = 0;
            __syncthreads();
            if (fix) {
                int o = 0;
                for (int k = k0 + (int)threadIdx.x; k < k1; k += NT) vfix[cube[k]] = 0;
                const long long S2 = P.S2, S = P.S;
                for (int q = gt; q < G.n_near; q += gn) {
                    const int pk = G.sh_near[q];
                    const RowRec R = G.rows_me[pk >> 8];
                    const long long c = (long long)(R.ox + Rc) * S2 + (long long)(R.oy + Rc) * S + Rc + (pk & 255) - 128;
                    vfix[c] = to_fix(vc[c], s2E, o);
                }
                if (o) g_fix_ovf = 1;
            }
        }
        cl.sync();
        const long long t1 = clk ? clock64() : 0;

        // CG in FP32 with reliable updates: the FP32 recursive residual is
        // replaced by the FP64 residual 4 pi rho + lap v whenever it has
        // dropped by update_drop (or looks converged); the search direction is
        // kept, rescaled to the new residual norm, so the Krylov progress
        // survives each replacement. The stop test is the FP64 residual.
        double acc = cta_residual0(P, cube, rho, vc, r64, CL.res_list + k0, k1 - k0, CL.res_nrim[rank], NT,
                                   P.dbg_b != nullptr, fix ? vfix : nullptr, finvE);
        if (fix && g_fix_ovf) acc = __longlong_as_double(0x7ff8000000000000LL);  // NaN: the cluster falls back
        double bb = cluster_sum<NT, C, double>(acc, red, flip, part, cflip, cl, rank);
        if (fix && !(bb == bb)) {
            fix = false;
            acc = cta_residual0(P, cube, rho, vc, r64, CL.res_list + k0, k1 - k0, CL.res_nrim[rank], NT,
                                P.dbg_b != nullptr);
            bb = cluster_sum<NT, C, double>(acc, red, flip, part, cflip, cl, rank);
        }
        const double target2 = P.tol * P.tol * bb;
        if (clk) tr += clock64() - t1;
        int iters = 0, refines = 1;
        bool conv = true;
        double rn_start = bb;
        if (P.warm && bb > target2 && bb == bb) {
            // warm 3: extrapolate from the last calls that all hold the pair
            // (order = their number, up to 3: v1; 2 v1 - v2; 3 v1 - 3 v2 + v3)
            int xm = 0;
            int xdl[3][3];
            const float* xsrc[3];
            if (P.warm == 3) {
                for (int h = 0; h < P.xk; ++h) {
                    const int q = find_prev_pair(P.xp[h], *P.xn[h], pr.i, pr.j);
                    if (q < 0) break;
                    const PairRec po = P.xp[h][q];
                    bool ok = true;
                    for (int a = 0; a < 3; ++a) {
                        int d = pr.g[a] - po.g[a];
                        if (d > P.N[a] / 2) d -= P.N[a];
                        if (d < -(P.N[a] - 1) / 2) d += P.N[a];
                        xdl[h][a] = d;
                        ok = ok && abs(d) <= 3;
                    }
                    if (!ok) break;
                    xsrc[h] = P.xv[h] + (size_t)q * G.n_pe;
                    xm = h + 1;
                }
            }
            // warm 1: the same pair in the previous call's list; warm 2: this
            // pair's learned guess (same list position, no shift)
            const int prev = P.warm == 3 ? (xm > 0 ? 0 : -1)
                             : P.warm == 2 ? pidx
                                           : find_prev_pair(P.prev_pairs, *P.n_prev, pr.i, pr.j);
            if (prev >= 0) {
                int dlt[3] = {0, 0, 0};
                if (P.warm == 1) {
                    const PairRec po = P.prev_pairs[prev];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        int d = pr.g[a] - po.g[a];
                        if (d > P.N[a] / 2) d -= P.N[a];
                        if (d < -(P.N[a] - 1) / 2) d += P.N[a];
                        dlt[a] = d;
                    }
                }
                if (abs(dlt[0]) <= 3 && abs(dlt[1]) <= 3 && abs(dlt[2]) <= 3) {
                    const long long tu = clk ? clock64() : 0;
                    if (P.warm == 3) {
                        const double c1[3] = {1.0, 0.0, 0.0}, c2[3] = {2.0, -1.0, 0.0}, c3[3] = {3.0, -3.0, 1.0};
                        cta_warm_extrapolate(G, cube, vc, xm, xsrc, xdl, xm == 1 ? c1 : (xm == 2 ? c2 : c3), k0, k1,
                                             NT);
                    } else {
                        cta_warm_insert(G, cube, vc, P.vprev + (size_t)prev * G.n_pe, dlt[0], dlt[1], dlt[2], k0, k1,
                                        NT);
                    }
                    if (fix) {  // the warm values into the fixed-point copy
                        int o = 0;
                        for (int k = k0 + (int)threadIdx.x; k < k1; k += NT) vfix[cube[k]] = to_fix(vc[cube[k]], s2E, o);
                        if (o) g_fix_ovf = 1;
                    }
                    cl.sync();
                    acc = cta_residual(P, cube, rho, vc, r64, k0, k1, NT, false, fix ? vfix : nullptr, finvE);
                    if (fix && g_fix_ovf) acc = __longlong_as_double(0x7ff8000000000000LL);
                    rn_start = cluster_sum<NT, C, double>(acc, red, flip, part, cflip, cl, rank);
                    if (fix && !(rn_start == rn_start)) {
                        fix = false;
                        acc = cta_residual(P, cube, rho, vc, r64, k0, k1, NT, false);
                        rn_start = cluster_sum<NT, C, double>(acc, red, flip, part, cflip, cl, rank);
                    }
                    ++refines;
                    if (clk) tr += clock64() - tu;
                }
            }
        }
        if (rn_start > target2 && rn_start == rn_start) {
            if (threadIdx.x == 0) {
                g_rc.cube = cube;
                g_rc.vc = vc;
                g_rc.r64 = r64;
                g_rc.max_iter = P.max_iter;
                g_rc.target2 = target2;
                g_rc.drop2 = (float)(P.update_drop * P.update_drop);
                g_rc.fault = P.timeouts;
                g_rc.vfix = vfix;
                g_rc.s2E = s2E;
                g_rc.fix = fix ? 1 : 0;
            }
            __syncthreads();
            double scale = sqrt(rn_start);
            float carry = -1.0f;
            StencilArgs sa;
            sa.c0 = P.st32.c0;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                sa.cx[q] = P.st32.cx[q];
                sa.cy[q] = P.st32.cy[q];
                sa.cz[q] = P.st32.cz[q];
            }
            for (;;) {
                RunSeg sg;
                if constexpr (RUNS)
                    sg = run_segment<NT, C, PTS, SYZ>(pc + roff, ds + threadIdx.x, hm, hp, rk0, rlen, scale, carry,
                                                      sa.c0, sa.cz[0], sa.cz[1], sa.cz[2], iters, f32, cf32);
                else if constexpr (QHALO)
                    sg = quad_halo_segment<NT, C, PTS, SYZ, ISO>(pc, spk + threadIdx.x, slot_k + threadIdx.x, planes,
                                                                 nbl, nbr, mbl, mbr, Syz, Sp2, scale, carry,
                                                                 sa, iters, f32, cf32, hph);
                else if constexpr (QUADS)
                    sg = quad_segment<NT, C, PTS, SYZ, ISO>(ps, pm, pp, reinterpret_cast<float4*>(ds) + threadIdx.x,
                                                            spk + threadIdx.x, slot_k + threadIdx.x, planes,
                                                            planes_prev, Syz, Sp2, scale, carry, sa, iters, f32, cf32);
                else
                    sg = pts_segment<NT, C, PTS, SYZ, ISO>(ps, pm, pp, ds + threadIdx.x, spk + threadIdx.x,
                                                           slot_k + threadIdx.x, planes, planes_prev, Syz, scale,
                                                           carry, sa, iters, f32, cf32);
                iters = sg.iters;
                f32 = sg.flip32;
                cf32 = sg.cflip32;
                if constexpr (QHALO) hph = sg.hphase;
                if (sg.maxed) {
                    conv = false;
                    break;
                }
                const long long tu = clk ? clock64() : 0;
                cl.sync();
                acc = cta_residual(P, cube, rho, vc, r64, k0, k1, NT, false, fix ? vfix : nullptr, finvE);
                if (fix && g_fix_ovf) acc = __longlong_as_double(0x7ff8000000000000LL);
                double rn2 = cluster_sum<NT, C, double>(acc, red, flip, part, cflip, cl, rank);
                if (fix && !(rn2 == rn2)) {  // a conversion left the bound (or the solve broke down): FP64 stencil
                    fix = false;
                    if (threadIdx.x == 0) g_rc.fix = 0;
                    acc = cta_residual(P, cube, rho, vc, r64, k0, k1, NT, false);
                    rn2 = cluster_sum<NT, C, double>(acc, red, flip, part, cflip, cl, rank);
                }
                ++refines;
                if (clk) tr += clock64() - tu;
                if (rn2 <= target2) break;
                if (refines > P.max_refine || !(rn2 < scale * scale)) {
                    conv = false;
                    break;
                }
                const double ns = sqrt(rn2);
                carry = (float)(ns / scale) / sg.rr;
                scale = ns;
            }
        }
        const long long t2 = clk ? clock64() : 0;

        // E_ij, the warm-start cache and the scatter
        if (P.vcur) cta_warm_store(cube, vc, P.vcur + (size_t)pidx * G.n_pe, k0, k1, NT);
        double e = cta_energy(cube, rho, vc, k0, k1, NT);
        e = cluster_sum<NT, C, double>(e, red, flip, part, cflip, cl, rank);
        if (rank == 0 && threadIdx.x == 0) {
            P.e_pair[pidx] = e * P.dV;
            P.iters[pidx] = iters;
            if (P.refines) P.refines[pidx] = refines;
            if (!conv) atomicAdd(P.nonconv, 1);
        }
        scatter_dxx(P, G, pr, vc, gt, gn);
        cl.sync();
        if (clk) {
            const long long t3 = clock64();
            atomicAdd(P.phase_clk + 0, (unsigned long long)(t1 - t0));
            atomicAdd(P.phase_clk + 1, (unsigned long long)tr);
            atomicAdd(P.phase_clk + 2, (unsigned long long)(t2 - t1 - tr));
            atomicAdd(P.phase_clk + 3, (unsigned long long)(t3 - t2));
        }
    }
    // the time-out test's wait comes after the pair loop: placed before it, it
    // slowed the loop by 7 % on the water-64 workload (measured)
    if (P.test_wait && threadIdx.x == 0)
        inject_wait_timeout(smem_u32(smem) + (uint32_t)cluster_smem_test_offset(CL, MODE, PTS, NT), P.timeouts);
}

// ---------------------------------------------------------------------------
// The multigrid-preconditioned CG on a thread-block cluster (precision 1 with
// preconditioner 1). The C CTAs of a cluster share one pair and keep all its
// vectors in the cluster's workspace slot. One CTA per pair keeps about 300
// pairs in flight, whose FP32 vectors (about 2 MB each) are far beyond the
// 129 MB L2, and waits on DRAM; a cluster per pair keeps the vectors of the
// pairs in flight in L2. Each CTA sweeps a contiguous range of the PE ball's
// compact points (the points are ordered plane by plane, so a range is a slab
// and the stencil's reach into the neighbours' ranges is short); a cluster
// barrier separates two sweeps whenever the second reads what other CTAs
// wrote in the first. The V-cycle's level 0 and the restriction to level 1
// run on the whole cluster, the coarser levels (an eighth of the points and
// less) on CTA 0 while the others wait. Setup, FP64 residuals, E_ij and the
// scatter are the cluster solver's phases.
// ---------------------------------------------------------------------------

// Two FP32 sums over the cluster at once (as cluster_sum).
template <int NT, int C>
__device__ __forceinline__ float2 cluster_sum2(float2 v, float2 (*red)[33], int& flip, float2 (*part)[16], int& cflip,
                                               cg::cluster_group& cl, int rank) {
    v.x = warp_sum(v.x);
    v.y = warp_sum(v.y);
    float2* buf = red[flip];
    flip ^= 1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) buf[w] = v;
    __syncthreads();
    if (w == 0) {
        float2 t = lane < NT / 32 ? buf[lane] : make_float2(0.0f, 0.0f);
        t.x = warp_sum(t.x);
        t.y = warp_sum(t.y);
        if (lane < C) {
            float2* dst = cl.map_shared_rank(&part[cflip][0], lane);
            dst[rank] = t;
        }
    }
    cl.sync();
    float2 s = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int r = 0; r < C; ++r) {
        s.x += part[cflip][r].x;
        s.y += part[cflip][r].y;
    }
    cflip ^= 1;
    return s;
}

struct MGSums {
    float (*red)[33];
    float (*part)[16];
    float2 (*red2)[33];
    float2 (*part2)[16];
    int flip, cflip, flip2, cflip2;
};

// The preconditioner z = M r after the sweep that wrote r and the V-cycle's
// first Jacobi sweep (Z = w D^-1 r on level 0): the rest of the V-cycle, z into
// the level-0 Tc cube; returns this thread's r.z.
template <int NT, int C>
__device__ __noinline__ float cluster_mg_precondition(const SolveParams& P, const BallGeo& G, const MGGeo& M,
                                                      char* slot, int k0, int k1) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int kb = k0 + (int)threadIdx.x;
    const float* r = reinterpret_cast<const float*>(slot + P.off_r32);
    const MGView<float> v0 = mg_view<float>(P, G, M, slot, 0, r);
    const int n1 = M.lv[1].n;
    cl.sync();  // Z
    mg_residual(P, v0, kb, k1, NT);
    cl.sync();  // Tc
    mg_restrict(v0, M.lv[1], n1 * rank / C + (int)threadIdx.x, n1 * (rank + 1) / C, NT);
    cl.sync();  // level-1 right-hand side
    if (rank == 0) mg_vcycle<NT, float>(P, G, M, slot, r, 1);
    cl.sync();  // level-1 correction
    const MGView<float> v1 = mg_view<float>(P, G, M, slot, 1, r);
    mg_prolong(v0, v1, M.L == 1 ? v1.Z : v1.Tc, kb, k1, NT);
    cl.sync();  // Z
    return mg_smooth(P, v0, kb, k1, NT);
}

// One inner solve of the refinement loop: the FP32 PCG for A d = r64 / rn on
// the CTA's points [k0, k1), from d = 0, until r.r <= eta2 (r0.r0) or after
// max_iter iterations; d goes to the slot's FP32 d. Returns the iterations.
// The stop test comes after the preconditioner (its r.r is summed with r.z),
// so an iteration has one sum fewer and a solve one V-cycle more. Without
// coarse levels (a ball of radius <= 3) the preconditioner is the identity.
template <int NT, int C>
__device__ __noinline__ int cluster_mg_pcg(const SolveParams& P, const BallGeo& G, const MGGeo& M, char* slot, int k0,
                                           int k1, double inv_rn, float eta2, int max_iter, MGSums& sm) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int kb = k0 + (int)threadIdx.x;
    const int* cube = G.pt_cube;
    const double* r64 = reinterpret_cast<const double*>(slot + P.off_r);
    float* pc = reinterpret_cast<float*>(slot + P.off_p32);
    float* r = reinterpret_cast<float*>(slot + P.off_r32);
    float* d = reinterpret_cast<float*>(slot + P.off_d32);
    float* ap = reinterpret_cast<float*>(slot + P.off_ap32);
    float* Z0 = reinterpret_cast<float*>(slot + P.off_zc);
    float* T0 = reinterpret_cast<float*>(slot + P.off_tc);  // z
    const int S = P.S;
    const long long S2 = P.S2;
    const Stencil<float> A = negated(P.st32);
    const bool mg = M.L > 0;
    const float wd = (float)P.mg_omega / A.c0;
    float* zw = mg ? Z0 : T0;  // the sweep that writes r writes Z = wd r, or z = r
    const float zs = mg ? wd : 1.0f;
    float rr_part = 0.0f;
    for (int k = kb; k < k1; k += NT) {
        const float rk = (float)(r64[k] * inv_rn);
        r[k] = rk;
        d[k] = 0.0f;
        zw[cube[k]] = zs * rk;
        rr_part = fmaf(rk, rk, rr_part);
    }
    float rz_part = mg ? cluster_mg_precondition<NT, C>(P, G, M, slot, k0, k1) : rr_part;
    float2 s = cluster_sum2<NT, C>(make_float2(rz_part, rr_part), sm.red2, sm.flip2, sm.part2, sm.cflip2, cl, rank);
    float rz = s.x;
    const float target = eta2 * s.y;
    for (int k = kb; k < k1; k += NT) pc[cube[k]] = T0[cube[k]];
    int it = 0;
    while (it < max_iter) {
        cl.sync();  // p
        float pap = 0.0f;
        for (int k = kb; k < k1; k += NT) {
            const int c = cube[k];
            const float a = lap19<float>(pc, c, S, S2, A);
            ap[k] = a;
            pap = fmaf(pc[c], a, pap);
        }
        pap = cluster_sum<NT, C, float>(pap, sm.red, sm.flip, sm.part, sm.cflip, cl, rank);
        const float al = rz / pap;
        rr_part = 0.0f;
        for (int k = kb; k < k1; k += NT) {
            const int c = cube[k];
            d[k] = fmaf(al, pc[c], d[k]);
            const float rk = fmaf(-al, ap[k], r[k]);
            r[k] = rk;
            rr_part = fmaf(rk, rk, rr_part);
            zw[c] = zs * rk;
        }
        ++it;
        rz_part = mg ? cluster_mg_precondition<NT, C>(P, G, M, slot, k0, k1) : rr_part;
        s = cluster_sum2<NT, C>(make_float2(rz_part, rr_part), sm.red2, sm.flip2, sm.part2, sm.cflip2, cl, rank);
        if (s.y <= target || !(s.y == s.y)) break;
        const float be = s.x / rz;
        rz = s.x;
        for (int k = kb; k < k1; k += NT) {
            const int c = cube[k];
            pc[c] = fmaf(be, pc[c], T0[c]);
        }
    }
    return it;
}

template <int NT, int C, int MINB>
__global__ void __launch_bounds__(NT, MINB) cluster_mg_kernel(const __grid_constant__ SolveParams P) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    __shared__ double red[2][33];
    __shared__ double part[2][16];
    __shared__ float red32[2][33];
    __shared__ float part32[2][16];
    __shared__ float2 red2[2][33];
    __shared__ float2 part2[2][16];
    __shared__ double s_M[kNMono], s_T[kNMono];
    __shared__ int s_item;
    int flip = 0, cflip = 0;
    MGSums sm{red32, part32, red2, part2, 0, 0, 0, 0};

    const int Rc = P.Rc;
    const double* xp = P.pow_tab;
    const double* yp = xp + (2 * Rc + 1) * 8;
    const double* zp = yp + (2 * Rc + 1) * 8;
    const int cid = blockIdx.x / C;
    char* slot = P.ws + (size_t)cid * P.slot_bytes;
    double* vc = reinterpret_cast<double*>(slot + P.off_vcube);
    double* rho = reinterpret_cast<double*>(slot + P.off_rho);
    double* r64 = reinterpret_cast<double*>(slot + P.off_r);
    double* rowS = reinterpret_cast<double*>(slot + P.off_rows);
    double* sYc = reinterpret_cast<double*>(slot + P.off_sy);
    float* d32 = reinterpret_cast<float*>(slot + P.off_d32);
    float* p32 = reinterpret_cast<float*>(slot + P.off_p32);
    double* U64 = reinterpret_cast<double*>(slot + P.off_ush);
    float* U32 = reinterpret_cast<float*>(U64 + (size_t)kNU * P.geos[P.n_geo - 1].n_rows_me);
    const int t = threadIdx.x;
    const int gt = rank * NT + t, gn = C * NT;
    const int np = *P.n_pair;

    for (;;) {
        if (rank == 0 && t == 0) {
            const int it = atomicAdd(P.queue, 1);
            for (int r = 0; r < C; ++r) *cl.map_shared_rank(&s_item, r) = it;
        }
        cl.sync();
        const int item = s_item;
        if (item >= np) break;
        const int pidx = P.order ? P.order[(P.item_base ? *P.item_base : 0) + item] : item;
        const PairRec pr = P.pairs[pidx];
        const BallGeo G = P.geos[pr.geo];
        const MGGeo& M = P.mg[pr.geo];
        const int* cube = G.pt_cube;
        const int n_pe = G.n_pe;
        const int k0 = n_pe * rank / C, k1 = n_pe * (rank + 1) / C;
        const int npl = 2 * G.r_pe + 1;
        const int pl0 = npl * rank / C, pl1 = npl * (rank + 1) / C;
        const bool clk = P.phase_clk && rank == 0 && t == 0;
        const long long t0 = clk ? clock64() : 0;
        long long tr = 0;

        // gather, multipoles, shell potential (FP64, spread over the cluster)
        gather_rho(P, G, pr, rho, vc, gt, gn);
        cl.sync();
        moment_rows(P, G, rho, rowS, zp, gt, gn);
        cl.sync();
        moment_finish_cluster<NT>(P, G, rowS, xp, yp, sYc, pl0, pl1 - pl0, s_M, s_T, cl);
        shell_rows(P, G, xp, yp, s_T, U64, U32, gt, gn);
        cl.sync();
        shell_points<true>(P, G, vc, U64, U32, G.sh_near, G.n_near, gt, gn);
        shell_points<false>(P, G, vc, U64, U32, G.sh_far, G.n_far, gt, gn);
        cl.sync();
        const long long t1 = clk ? clock64() : 0;

        // FP64 refinement: r = 4 pi rho + lap v, then the FP32 PCG on r / ||r||
        int iters = 0, refines = 0;
        bool conv = true;
        double bb = -1.0, rn_prev = 1e300;
        for (;;) {
            const long long tu = clk ? clock64() : 0;
            double acc = cta_residual(P, cube, rho, vc, r64, k0, k1, NT, bb < 0.0 && P.dbg_b != nullptr);
            const double rn2 = cluster_sum<NT, C, double>(acc, red, flip, part, cflip, cl, rank);
            if (clk) tr += clock64() - tu;
            if (bb < 0.0) bb = rn2;
            if (rn2 <= P.tol * P.tol * bb) break;
            const double rn = sqrt(rn2);
            if (refines >= P.max_refine || iters >= P.max_iter || !(rn < rn_prev)) {
                conv = false;
                break;
            }
            rn_prev = rn;
            double eta = 0.3 * P.tol * sqrt(bb) / rn;
            eta = eta > P.inner_tol ? eta : P.inner_tol;
            const int budget = min(P.inner_max_iter, P.max_iter - iters);
            iters += cluster_mg_pcg<NT, C>(P, G, M, slot, k0, k1, 1.0 / rn, (float)(eta * eta), budget, sm);
            for (int k = k0 + t; k < k1; k += NT) vc[cube[k]] = fma(rn, (double)d32[k], vc[cube[k]]);
            ++refines;
            cl.sync();  // v
        }
        const long long t2 = clk ? clock64() : 0;

        // E_ij and the D_xx scatter
        double e = cta_energy(cube, rho, vc, k0, k1, NT);
        e = cluster_sum<NT, C, double>(e, red, flip, part, cflip, cl, rank);
        if (rank == 0 && t == 0) {
            P.e_pair[pidx] = e * P.dV;
            P.iters[pidx] = iters;
            if (P.refines) P.refines[pidx] = refines;
            if (!conv) atomicAdd(P.nonconv, 1);
        }
        scatter_dxx(P, G, pr, vc, gt, gn);
        if (P.n_geo > 1) {
            // the next pair may have other balls: every cube must be zero off them
            for (int k = k0 + t; k < k1; k += NT) p32[cube[k]] = 0.0f;
            mg_clear<float>(P, G, M, slot, k0 + t, k1, rank == 0 ? t : -1, NT);
        }
        cl.sync();
        if (clk) {
            const long long t3 = clock64();
            atomicAdd(P.phase_clk + 0, (unsigned long long)(t1 - t0));
            atomicAdd(P.phase_clk + 1, (unsigned long long)tr);
            atomicAdd(P.phase_clk + 2, (unsigned long long)(t2 - t1 - tr));
            atomicAdd(P.phase_clk + 3, (unsigned long long)(t3 - t2));
        }
    }
}

// ---- host side ----
cudaError_t set_multipole_const_cluster(const MultipoleConst& mc) {
    return cudaMemcpyToSymbol(c_mp, &mc, sizeof(MultipoleConst));
}

size_t cluster_kernel_smem(int Rc, const ClusterLayout& CL, int variant);

// Supported (threads, cluster size, points per thread) instantiations.
struct ClusterVariant {
    int nt, c, pts;
    int mode;  // 0 point map, 1 z runs with halo planes, 2 quad map, 3 quad map with halo planes
    int syz;   // modes 0, 1: slab row pitch the variant is specialised for;
               // mode 2: box side 2 R_PE + 7 (0 = any)
    bool iso;  // isotropic stencil only
    const void* fn;
    cudaError_t (*launch)(const SolveParams&, const ClusterLayout&, int, size_t, cudaStream_t);
};

template <int NT, int C, int PTS, int MODE, int SYZ, bool ISO>
static cudaError_t launch_cluster_t(const SolveParams& P, const ClusterLayout& CL, int n_clusters, size_t smem,
                                    cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_clusters * C, 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, cluster_pair_kernel<NT, C, PTS, MODE, SYZ, ISO>, P, CL);
}

#define EXX_CLUSTER_VARIANT(NT, C, PTS, MODE, SYZ, ISO)                                             \
    {NT, C, PTS, MODE, SYZ, ISO, (const void*)cluster_pair_kernel<NT, C, PTS, MODE, SYZ, ISO>,       \
     launch_cluster_t<NT, C, PTS, MODE, SYZ, ISO>}
static const ClusterVariant kVariants[] = {
    // point map, any radius and spacing
    EXX_CLUSTER_VARIANT(512, 2, 8, 0, 0, false),   EXX_CLUSTER_VARIANT(512, 2, 18, 0, 0, false),
    EXX_CLUSTER_VARIANT(512, 4, 10, 0, 0, false),  EXX_CLUSTER_VARIANT(512, 4, 18, 0, 0, false),
    EXX_CLUSTER_VARIANT(512, 8, 17, 0, 0, false),  EXX_CLUSTER_VARIANT(1024, 8, 9, 0, 0, false),
    EXX_CLUSTER_VARIANT(1024, 9, 8, 0, 0, false),
    // point map specialised for R_PE = 24 (pitch 55) on isotropic grids
    EXX_CLUSTER_VARIANT(1024, 9, 8, 0, 55, true),  EXX_CLUSTER_VARIANT(1024, 8, 9, 0, 55, true),
    // z runs with halo planes, specialised for R_PE = 24 (pitch 55) and 16 (39)
    EXX_CLUSTER_VARIANT(1024, 9, 8, 1, 55, true),  EXX_CLUSTER_VARIANT(1024, 4, 8, 1, 39, true),
    // quad map (PTS = quads per thread): R_PE = 24 on isotropic grids, and any radius
    EXX_CLUSTER_VARIANT(1024, 9, 2, 2, 55, true),  EXX_CLUSTER_VARIANT(512, 9, 4, 2, 55, true),
    EXX_CLUSTER_VARIANT(1024, 8, 3, 2, 55, true),
    EXX_CLUSTER_VARIANT(1024, 9, 2, 2, 0, false),  EXX_CLUSTER_VARIANT(1024, 4, 2, 2, 0, false),
    EXX_CLUSTER_VARIANT(512, 2, 4, 2, 0, false),
    // quad map with halo planes: R_PE = 24 on isotropic grids, and any radius
    EXX_CLUSTER_VARIANT(512, 9, 4, 3, 55, true),   EXX_CLUSTER_VARIANT(512, 9, 4, 3, 0, false),
    EXX_CLUSTER_VARIANT(512, 2, 4, 3, 0, false),
    // quad map with halo planes, 6 quads per thread: the radius classes of
    // per-pair radii (one CTA holds a whole small ball; 2, 4, 9 or 16 CTAs
    // share a larger one)
    EXX_CLUSTER_VARIANT(512, 1, 6, 3, 0, false),   EXX_CLUSTER_VARIANT(512, 2, 6, 3, 0, false),
    EXX_CLUSTER_VARIANT(512, 4, 6, 3, 0, false),   EXX_CLUSTER_VARIANT(512, 9, 6, 3, 0, false),
    EXX_CLUSTER_VARIANT(512, 16, 6, 3, 0, false),
};
#undef EXX_CLUSTER_VARIANT
constexpr int kNumVariants = (int)(sizeof(kVariants) / sizeof(kVariants[0]));

// Picks the point-map instantiation for (C, max points per CTA, threads):
// the one specialised for this slab pitch and an isotropic stencil when there
// is one, else the generic one with the most threads and the fewest points
// per thread. Returns the index into kVariants or -1.
int cluster_variant(int C, int max_pts, int threads, int syz, bool iso) {
    int best = -1;
    for (int v = 0; v < kNumVariants; ++v) {
        const ClusterVariant& K = kVariants[v];
        if (K.mode != 0 || K.c != C || K.nt * K.pts < max_pts) continue;
        if (threads && K.nt != threads) continue;
        if (K.syz && (K.syz != syz || !iso)) continue;
        if (best < 0) {
            best = v;
            continue;
        }
        const ClusterVariant& B = kVariants[best];
        const bool spec = K.syz != 0, bspec = B.syz != 0;
        if (spec != bspec) {
            if (spec) best = v;
            continue;
        }
        if (K.nt > B.nt || (K.nt == B.nt && K.pts < B.pts)) best = v;
    }
    return best;
}

cudaError_t cluster_prepare(int variant, size_t smem, int* max_clusters) {
    const ClusterVariant& K = kVariants[variant];
    cudaError_t e = cudaFuncSetAttribute(K.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (K.c > 8) {  // clusters beyond the portable size of 8 need the opt-in
        e = cudaFuncSetAttribute(K.fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(K.c, 1, 1);
    cfg.blockDim = dim3(K.nt, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = K.c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(max_clusters, K.fn, &cfg);
}

// Raises the variant's dynamic shared-memory limit (launch shapes of several
// radius classes can share one variant).
cudaError_t cluster_set_smem(int variant, size_t smem) {
    return cudaFuncSetAttribute(kVariants[variant].fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_cluster_kernel(int variant, const SolveParams& P, const ClusterLayout& CL, int n_clusters,
                                  size_t smem, cudaStream_t st) {
    return kVariants[variant].launch(P, CL, n_clusters, smem, st);
}

int cluster_variant_threads(int variant) { return kVariants[variant].nt; }
int cluster_variant_mode(int variant) { return kVariants[variant].mode; }
int cluster_variant_iso(int variant) { return kVariants[variant].iso ? 1 : 0; }
int cluster_variant_syz(int variant) { return kVariants[variant].syz; }
int cluster_variant_count() { return kNumVariants; }
int cluster_variant_size(int variant) { return kVariants[variant].c; }
int cluster_variant_pts(int variant) { return kVariants[variant].pts; }

size_t cluster_kernel_smem(int Rc, const ClusterLayout& CL, int variant) {
    (void)Rc;
    // slab (with 3 halo planes per side for modes 1 and 3), d ([PTS][NT]
    // points, or quads for mode 2; none for mode 3), the slot map (point or
    // quad slots), as laid out by cluster_pair_kernel, then the spare word of
    // the time-out test
    const ClusterVariant& K = kVariants[variant];
    return cluster_smem_test_offset(CL, K.mode, K.pts, K.nt) + 8;
}

// The cluster multigrid kernel: 512 threads per CTA, C = 2, 4, 8 or 16 CTAs per
// pair, built for one (128 registers) or two (64 registers) CTAs per SM.
template <int C, int MINB>
static cudaError_t mg_cluster_cfg(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, int n_clusters,
                                  cudaStream_t st) {
    cfg = {};
    cfg.gridDim = dim3(n_clusters * C, 1, 1);
    cfg.blockDim = dim3(512, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (C > 8)
        return cudaFuncSetAttribute(cluster_mg_kernel<512, C, MINB>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return cudaSuccess;
}

template <int C, int MINB>
static cudaError_t mg_cluster_prepare_t(int* max_clusters) {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    cudaError_t e = mg_cluster_cfg<C, MINB>(cfg, attr, 1, nullptr);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveClusters(max_clusters, cluster_mg_kernel<512, C, MINB>, &cfg);
}

template <int C, int MINB>
static cudaError_t mg_cluster_launch_t(const SolveParams& P, int n_clusters, cudaStream_t st) {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    cudaError_t e = mg_cluster_cfg<C, MINB>(cfg, attr, n_clusters, st);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, cluster_mg_kernel<512, C, MINB>, P);
}

bool mg_cluster_size_ok(int C) { return C == 2 || C == 4 || C == 8 || C == 16; }

#define EXX_MG_SWITCH(CALL2, CALL1)                          \
    switch (C * 4 + (minb == 1 ? 1 : 2)) {                   \
        case 2 * 4 + 2: return CALL2(2);                     \
        case 4 * 4 + 2: return CALL2(4);                     \
        case 8 * 4 + 2: return CALL2(8);                     \
        case 16 * 4 + 2: return CALL2(16);                   \
        case 8 * 4 + 1: return CALL1(8);                     \
        case 16 * 4 + 1: return CALL1(16);                   \
        default: return cudaErrorInvalidValue;               \
    }

cudaError_t mg_cluster_prepare(int C, int minb, int* max_clusters) {
#define P2(c) mg_cluster_prepare_t<c, 2>(max_clusters)
#define P1(c) mg_cluster_prepare_t<c, 1>(max_clusters)
    EXX_MG_SWITCH(P2, P1)
#undef P2
#undef P1
}

cudaError_t launch_cluster_mg(int C, int minb, const SolveParams& P, int n_clusters, cudaStream_t st) {
#define L2(c) mg_cluster_launch_t<c, 2>(P, n_clusters, st)
#define L1(c) mg_cluster_launch_t<c, 1>(P, n_clusters, st)
    EXX_MG_SWITCH(L2, L1)
#undef L2
#undef L1
}
#undef EXX_MG_SWITCH

}  // namespace exx
