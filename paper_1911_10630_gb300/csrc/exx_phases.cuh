// exx_phases.cuh -- per-pair phases shared by the one-CTA and the cluster
// pair kernels. Work is split over (tid, nthr) so that a phase can run on one
// CTA or on all CTAs of a thread-block cluster; the caller synchronises.
#pragma once

#include "exx_kernels.cuh"

namespace exx {

// Each translation unit that includes this header has its own copy, set by
// its own set_multipole_const_* function.
static __constant__ MultipoleConst c_mp;

constexpr double kFourPi = 12.566370614359172953850573533118;

// FP64 power tables x^e, y^e, z^e (e < 8) for offsets -Rc..Rc, in smem.
__device__ __forceinline__ void fill_power_tables(const SolveParams& P, double* xp, double* yp, double* zp,
                                                  int tid, int nthr) {
    const int Rc = P.Rc;
    for (int t = tid; t < (2 * Rc + 1) * 8; t += nthr) {
        const int o = t / 8 - Rc, e = t % 8;
        double px = 1.0, py = 1.0, pz = 1.0;
        const double x = o * P.delta[0], y = o * P.delta[1], z = o * P.delta[2];
        for (int k = 0; k < e; ++k) {
            px *= x;
            py *= y;
            pz *= z;
        }
        xp[t] = px;
        yp[t] = py;
        zp[t] = pz;
    }
}

// Step III: rho = phi_i phi_j on the PE ball (Eq. l2g indices); v = 0 there.
// Parameters are copied into registers first: P and G live in local memory,
// and stores through generic pointers would otherwise force their reload.
static __device__ __noinline__ void gather_rho(const SolveParams& P, const BallGeo& G, const PairRec& pr,
                                               double* __restrict__ rho, double* __restrict__ vc, int tid, int nthr) {
    const double* __restrict__ phi_i = P.phi + (long long)pr.i * P.ostride;
    const double* __restrict__ phi_j = P.phi + (long long)pr.j * P.ostride;
    const int N[3] = {P.N[0], P.N[1], P.N[2]};
    const int g[3] = {pr.g[0], pr.g[1], pr.g[2]};
    const int n_pe = G.n_pe;
    const int* __restrict__ off = G.pt_off;
    const int* __restrict__ cube = G.pt_cube;
    if (!P.box_org) {
        for (int k = tid; k < n_pe; k += nthr) {
            const long long gi = grid_index(N, g, off[k]);
            rho[k] = phi_i[gi] * phi_j[gi];
            vc[cube[k]] = 0.0;
        }
        return;
    }
    const int bd[3] = {P.bdim[0], P.bdim[1], P.bdim[2]};
    for (int k = tid; k < n_pe; k += nthr) {
        const long long ii = orb_index(N, g, off[k], P.box_org, bd, pr.i);
        const long long ij = orb_index(N, g, off[k], P.box_org, bd, pr.j);
        rho[k] = (ii >= 0 && ij >= 0) ? phi_i[ii] * phi_j[ij] : 0.0;
        vc[cube[k]] = 0.0;
    }
}

// Eq. mepole, stage 1: row sums S_c(x, y) = sum_z z^c rho(x, y, z), c <= 6,
// one thread per (row, c).
static __device__ __noinline__ void moment_rows(const SolveParams& P, const BallGeo& G,
                                                const double* __restrict__ rho, double* __restrict__ rowS,
                                                const double* __restrict__ zp, int tid, int nthr) {
    const int Rc = P.Rc;
    const int items = G.n_rows_pe * (kLmaxMax + 1);
    const RowRec* __restrict__ rows = G.rows_pe;
    for (int it = tid; it < items; it += nthr) {
        const int row = it / (kLmaxMax + 1), c = it - row * (kLmaxMax + 1);
        const RowRec R = rows[row];
        const double* rr = rho + R.pe_start + R.zpe;
        double s = 0.0;
        for (int z = -R.zpe; z <= R.zpe; ++z) s = fma(rr[z], zp[(z + Rc) * 8 + c], s);
        rowS[row * 8 + c] = s;
    }
}

// Eq. mepole, stages 2-4 (one CTA, NT threads, rowS complete and visible):
// plane sums, Cartesian moments M (times dV), and T = K M. Leaves T in s_T.
template <int NT>
__device__ void moment_finish(const SolveParams& P, const BallGeo& G, const double* __restrict__ rowS,
                              const double* __restrict__ xp, const double* __restrict__ yp, double* __restrict__ sY,
                              double* __restrict__ s_M, double* __restrict__ s_T) {
    const int L = P.lmax;
    const int Rc = P.Rc;
    const int nplane = 2 * G.r_pe + 1;
    const int nbc = (L + 1) * (L + 2) / 2;
    for (int item = threadIdx.x; item < nplane * nbc; item += NT) {
        const int pl = item / nbc, bc = item - pl * nbc;
        int dgr = 0;
        while ((dgr + 1) * (dgr + 2) / 2 <= bc) ++dgr;
        const int c = bc - dgr * (dgr + 1) / 2, b = dgr - c;
        double acc = 0.0;
        for (int row = G.plane_pe[pl]; row < G.plane_pe[pl + 1]; ++row) {
            const int oy = G.rows_pe[row].oy;
            acc = fma(yp[(oy + Rc) * 8 + b], rowS[row * 8 + c], acc);
        }
        sY[pl * 28 + bc] = acc;
    }
    __syncthreads();
    for (int m = threadIdx.x; m < kNMono; m += NT) {
        const int a = c_mp.mono[m][0], b = c_mp.mono[m][1], c = c_mp.mono[m][2];
        double acc = 0.0;
        if (a + b + c <= L) {
            const int dgr = b + c, bc = dgr * (dgr + 1) / 2 + c;
            for (int pl = 0; pl < nplane; ++pl) acc = fma(xp[(pl - G.r_pe + Rc) * 8 + a], sY[pl * 28 + bc], acc);
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

// Eq. me on the shell: v = sum_l P_l(r) / r^(2l+1), one warp per ME row.
// The lanes form the row's coefficients U_{l,c} = sum T_abc x^a y^b of
// P_l(z) together (ub: 2 x 28 values per warp in shared memory, FP64 and FP32
// copies), then evaluate the row's shell points. Points within zn of the row
// centre (the boundary layer that the stencil legs of the PE ball read) are
// evaluated in FP64; the rest of the shell only feeds the D_xx scatter and is
// evaluated in FP32.
static __device__ __noinline__ void shell_potential(const SolveParams& P, const BallGeo& G, double* __restrict__ vc,
                                                    const double* __restrict__ xp, const double* __restrict__ yp,
                                                    const double* __restrict__ s_T, double* ub, int wid, int nw) {
    const int lane = threadIdx.x & 31;
    const int Rc = P.Rc;
    const double dx = P.delta[0], dy = P.delta[1], dz = P.delta[2];
    const float dzf = (float)dz;
    const long long S2 = P.S2;
    const long long S = P.S;
    const int nrows = G.n_rows_me;
    const RowRec* __restrict__ rows = G.rows_me;
    float* ub32 = reinterpret_cast<float*>(ub + kNU);
    for (int row = wid; row < nrows; row += nw) {
        const RowRec R = rows[row];
        if (lane < kNU) {
            const double* xa = xp + (R.ox + Rc) * 8;
            const double* yb = yp + (R.oy + Rc) * 8;
            double u = 0.0;
            for (int t = 0; t < c_mp.uterm_n[lane]; ++t)
                u = fma(s_T[c_mp.uterm[lane][t][0]], xa[c_mp.uterm[lane][t][1]] * yb[c_mp.uterm[lane][t][2]], u);
            ub[lane] = u;
            ub32[lane] = (float)u;
        }
        __syncwarp();
        const double x = R.ox * dx, y = R.oy * dy;
        const double rxy2 = x * x + y * y;
        const float rxy2f = (float)rxy2;
        const long long base = (long long)(R.ox + Rc) * S2 + (long long)(R.oy + Rc) * S + Rc;
        // shell points of the row: z in [-zme, -zpe-1] and [zpe+1, zme] (or all when zpe < 0)
        const int zin = R.zpe >= 0 ? R.zpe + 1 : 0;      // first |z| on the shell
        const int nseg = R.zme - zin + 1;                 // points per half (z >= 0 side counts z = 0 once)
        const int npts = R.zpe >= 0 ? 2 * nseg : 2 * R.zme + 1;
        for (int t = lane; t < npts; t += 32) {
            int z;
            if (R.zpe >= 0) z = t < nseg ? -(zin + t) : zin + (t - nseg);
            else z = t - R.zme;
            const int az = z < 0 ? -z : z;
            if (az <= R.zn) {
                const double zz = z * dz;
                const double r2 = fma(zz, zz, rxy2);
                const double ir = rsqrt(r2);
                const double ir2 = ir * ir;
                double acc = 0.0;
#pragma unroll
                for (int l = kLmaxMax; l >= 0; --l) {
                    const double* Ul = ub + l * (l + 1) / 2;
                    double pl = Ul[l];
#pragma unroll
                    for (int c = l - 1; c >= 0; --c) pl = fma(pl, zz, Ul[c]);
                    acc = fma(acc, ir2, pl);
                }
                vc[base + z] = acc * ir;
            } else {
                const float zz = (float)z * dzf;
                const float r2 = fmaf(zz, zz, rxy2f);
                const float ir = rsqrtf(r2);
                const float ir2 = ir * ir;
                float acc = 0.0f;
#pragma unroll
                for (int l = kLmaxMax; l >= 0; --l) {
                    const float* Ul = ub32 + l * (l + 1) / 2;
                    float pl = Ul[l];
#pragma unroll
                    for (int c = l - 1; c >= 0; --c) pl = fmaf(pl, zz, Ul[c]);
                    acc = fmaf(acc, ir2, pl);
                }
                vc[base + z] = (double)(acc * ir);
            }
        }
        __syncwarp();
    }
}

// Eq. me on the shell, in two dense stages for the cluster kernel (the
// per-row form above leaves most lanes of its FP64 instructions idle, and
// GB300 issues FP64 at 1/64 of the FP32 rate). Stage 1: the coefficients
// U_{l,c}(x, y) of every ME row, one item per (u, row), u-major so that the
// lanes of a warp share u and its terms; FP64 into U64[u][row] with an FP32
// copy in U32[u][row].
static __device__ __noinline__ void shell_rows(const SolveParams& P, const BallGeo& G, const double* __restrict__ xp,
                                               const double* __restrict__ yp, const double* __restrict__ s_T,
                                               double* __restrict__ U64, float* __restrict__ U32, int tid, int nthr) {
    const int Rc = P.Rc;
    const int nr = G.n_rows_me;
    const RowRec* __restrict__ rows = G.rows_me;
    for (int it = tid; it < kNU * nr; it += nthr) {
        const int u = it / nr, row = it - u * nr;
        const RowRec R = rows[row];
        const double* xa = xp + (R.ox + Rc) * 8;
        const double* yb = yp + (R.oy + Rc) * 8;
        double acc = 0.0;
        for (int t = 0; t < c_mp.uterm_n[u]; ++t)
            acc = fma(s_T[c_mp.uterm[u][t][0]], xa[c_mp.uterm[u][t][1]] * yb[c_mp.uterm[u][t][2]], acc);
        U64[it] = acc;
        U32[it] = (float)acc;
    }
}

// Stage 2: v = sum_l P_l(z) / r^(2l+1) at the listed shell points (ME row << 8
// | (z + 128)), one point per thread: FP64 for the boundary layer the stencil
// reads (sh_near), FP32 with the FP32 copy of U for the rest (sh_far).
template <bool F64>
static __device__ __noinline__ double shell_points(const SolveParams& P, const BallGeo& G, double* __restrict__ vc,
                                                 const double* __restrict__ U64, const float* __restrict__ U32,
                                                 const int* __restrict__ list, int n, int tid, int nthr) {
    const int Rc = P.Rc;
    const int nr = G.n_rows_me;
    const double dx = P.delta[0], dy = P.delta[1], dz = P.delta[2];
    const long long S2 = P.S2, S = P.S;
    const RowRec* __restrict__ rows = G.rows_me;
    double vmax = 0.0;  // largest |v| written (FP64 points)
    for (int q = tid; q < n; q += nthr) {
        const int pk = list[q];
        const int row = pk >> 8, z = (pk & 255) - 128;
        const RowRec R = rows[row];
        const long long base = (long long)(R.ox + Rc) * S2 + (long long)(R.oy + Rc) * S + Rc;
        const double x = R.ox * dx, y = R.oy * dy;
        if constexpr (F64) {
            const double zz = z * dz;
            const double r2 = fma(zz, zz, x * x + y * y);
            const double ir = rsqrt(r2);
            const double ir2 = ir * ir;
            double acc = 0.0;
#pragma unroll
            for (int l = kLmaxMax; l >= 0; --l) {
                const double* Ul = U64 + (size_t)(l * (l + 1) / 2) * nr + row;
                double pl = Ul[(size_t)l * nr];
#pragma unroll
                for (int c = l - 1; c >= 0; --c) pl = fma(pl, zz, Ul[(size_t)c * nr]);
                acc = fma(acc, ir2, pl);
            }
            vc[base + z] = acc * ir;
            vmax = fmax(vmax, fabs(acc * ir));
        } else {
            const float zz = (float)z * (float)dz;
            const float r2 = fmaf(zz, zz, (float)(x * x + y * y));
            const float ir = rsqrtf(r2);
            const float ir2 = ir * ir;
            float acc = 0.0f;
#pragma unroll
            for (int l = kLmaxMax; l >= 0; --l) {
                const float* Ul = U32 + (size_t)(l * (l + 1) / 2) * nr + row;
                float pl = Ul[(size_t)l * nr];
#pragma unroll
                for (int c = l - 1; c >= 0; --c) pl = fmaf(pl, zz, Ul[(size_t)c * nr]);
                acc = fmaf(acc, ir2, pl);
            }
            vc[base + z] = (double)(acc * ir);
        }
    }
    return vmax;
}

// Step V scatter: D^i += v phi_j, D^j += v phi_i on the ME ball.
static __device__ __noinline__ void scatter_dxx(const SolveParams& P, const BallGeo& G, const PairRec& pr,
                                                const double* __restrict__ vc, int tid, int nthr) {
    if (!P.dxx) return;
    const long long ng = P.ostride;
    const double* __restrict__ phi_i = P.phi + (long long)pr.i * ng;
    const double* __restrict__ phi_j = P.phi + (long long)pr.j * ng;
    double* Di = P.dxx + (long long)pr.i * ng;
    double* Dj = P.dxx + (long long)pr.j * ng;
    const bool two = pr.i != pr.j;
    const int N[3] = {P.N[0], P.N[1], P.N[2]};
    const int g[3] = {pr.g[0], pr.g[1], pr.g[2]};
    const int n_me = G.n_me;
    const int* __restrict__ off = G.pt_off;
    const int* __restrict__ cube = G.pt_cube;
    const double dfix = P.dfix;
    const int bd[3] = {P.bdim[0], P.bdim[1], P.bdim[2]};
    for (int q = tid; q < n_me; q += nthr) {
        long long ii, ij;
        if (!P.box_org) {
            ii = ij = grid_index(N, g, off[q]);
        } else {  // a point outside a box: that orbital is zero there, and its D is not kept there
            ii = orb_index(N, g, off[q], P.box_org, bd, pr.i);
            ij = orb_index(N, g, off[q], P.box_org, bd, pr.j);
        }
        const double v = vc[cube[q]];
        const double pj = ij >= 0 ? phi_j[ij] : 0.0, pi = ii >= 0 ? phi_i[ii] : 0.0;
        if (dfix != 0.0) {  // integer adds: the sum is the same in any order
            // a contribution at or beyond 2^22 (2^62 at the scale 2^40) would
            // wrap: it is dropped and counted (the call then fails)
            const double xi = v * pj * dfix, xj = v * pi * dfix;
            const bool oki = fabs(xi) < 4611686018427387904.0, okj = fabs(xj) < 4611686018427387904.0;  // 2^62
            if (ii >= 0 && oki)
                atomicAdd(reinterpret_cast<unsigned long long*>(Di + ii), (unsigned long long)__double2ll_rn(xi));
            if (two && ij >= 0 && okj)
                atomicAdd(reinterpret_cast<unsigned long long*>(Dj + ij), (unsigned long long)__double2ll_rn(xj));
            if (!oki || (two && !okj)) atomicAdd(P.dfix_range, 1);
        } else {
            if (ii >= 0) atomicAdd(Di + ii, v * pj);
            if (two && ij >= 0) atomicAdd(Dj + ij, v * pi);
        }
    }
}

__device__ __forceinline__ Stencil<double> negated(const Stencil<double>& s) {
    Stencil<double> n;
    n.c0 = -s.c0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        n.cx[q] = -s.cx[q];
        n.cy[q] = -s.cy[q];
        n.cz[q] = -s.cz[q];
    }
    return n;
}

__device__ __forceinline__ Stencil<float> negated(const Stencil<float>& s) {
    Stencil<float> n;
    n.c0 = -s.c0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        n.cx[q] = -s.cx[q];
        n.cy[q] = -s.cy[q];
        n.cz[q] = -s.cz[q];
    }
    return n;
}

}  // namespace exx
