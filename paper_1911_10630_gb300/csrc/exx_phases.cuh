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
static __device__ __noinline__ void gather_rho(const SolveParams& P, const BallGeo& G, const PairRec& pr,
                                           double* __restrict__ rho, double* __restrict__ vc, int tid, int nthr) {
    const double* phi_i = P.phi + (long long)pr.i * P.ngrid;
    const double* phi_j = P.phi + (long long)pr.j * P.ngrid;
    for (int k = tid; k < G.n_pe; k += nthr) {
        const long long g = grid_index(P.N, pr.g, G.pt_off[k]);
        rho[k] = phi_i[g] * phi_j[g];
        vc[G.pt_cube[k]] = 0.0;
    }
}

// Eq. mepole, stage 1: row sums S_c(x, y) = sum_z z^c rho(x, y, z), c <= 6.
static __device__ __noinline__ void moment_rows(const SolveParams& P, const BallGeo& G, const double* __restrict__ rho,
                                            double* __restrict__ rowS, const double* __restrict__ zp, int tid,
                                            int nthr) {
    const int Rc = P.Rc;
    for (int row = tid; row < G.n_rows_pe; row += nthr) {
        const RowRec R = G.rows_pe[row];
        double s[kLmaxMax + 1];
#pragma unroll
        for (int c = 0; c <= kLmaxMax; ++c) s[c] = 0.0;
        const double* rr = rho + R.pe_start;
        for (int z = -R.zpe; z <= R.zpe; ++z) {
            const double v = rr[z + R.zpe];
            const double* zz = zp + (z + Rc) * 8;
#pragma unroll
            for (int c = 0; c <= kLmaxMax; ++c) s[c] = fma(v, zz[c], s[c]);
        }
#pragma unroll
        for (int c = 0; c <= kLmaxMax; ++c) rowS[row * 8 + c] = s[c];
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

// Eq. me on the shell: v = sum_l P_l(r) / r^(2l+1), one thread per ME row.
static __device__ __noinline__ void shell_potential(const SolveParams& P, const BallGeo& G, double* __restrict__ vc,
                                                const double* __restrict__ xp, const double* __restrict__ yp,
                                                const double* __restrict__ s_T, int tid, int nthr) {
    const int Rc = P.Rc;
    for (int row = tid; row < G.n_rows_me; row += nthr) {
        const RowRec R = G.rows_me[row];
        const double* xa = xp + (R.ox + Rc) * 8;
        const double* yb = yp + (R.oy + Rc) * 8;
        double U[kNU];  // U_{l,c} = sum_{a+b=l-c} T_abc x^a y^b
#pragma unroll
        for (int u = 0; u < kNU; ++u) U[u] = 0.0;
        {
            int m = 0;
#pragma unroll
            for (int l = 0; l <= kLmaxMax; ++l)
#pragma unroll
                for (int a = l; a >= 0; --a)
#pragma unroll
                    for (int b = l - a; b >= 0; --b) {
                        const int c = l - a - b;
                        U[l * (l + 1) / 2 + c] = fma(s_T[m], xa[a] * yb[b], U[l * (l + 1) / 2 + c]);
                        ++m;
                    }
        }
        const double x = R.ox * P.delta[0], y = R.oy * P.delta[1];
        const double rxy2 = x * x + y * y;
        const long long base = (long long)(R.ox + Rc) * P.S2 + (long long)(R.oy + Rc) * P.S + Rc;
        const int zlo_hi = R.zpe >= 0 ? -R.zpe - 1 : R.zme;
        for (int z = -R.zme; z <= R.zme; ++z) {
            if (R.zpe >= 0 && z > zlo_hi && z <= R.zpe) continue;
            const double zz = z * P.delta[2];
            const double r2 = fma(zz, zz, rxy2);
            const double ir = rsqrt(r2);
            const double ir2 = ir * ir;
            double acc = 0.0;
#pragma unroll
            for (int l = kLmaxMax; l >= 0; --l) {
                const double* Ul = U + l * (l + 1) / 2;
                double pl = Ul[l];
#pragma unroll
                for (int c = l - 1; c >= 0; --c) pl = fma(pl, zz, Ul[c]);
                acc = fma(acc, ir2, pl);
            }
            vc[base + z] = acc * ir;
        }
    }
}

// Step V scatter: D^i += v phi_j, D^j += v phi_i on the ME ball.
static __device__ __noinline__ void scatter_dxx(const SolveParams& P, const BallGeo& G, const PairRec& pr,
                                            const double* __restrict__ vc, int tid, int nthr) {
    if (!P.dxx) return;
    const double* phi_i = P.phi + (long long)pr.i * P.ngrid;
    const double* phi_j = P.phi + (long long)pr.j * P.ngrid;
    double* Di = P.dxx + (long long)pr.i * P.ngrid;
    double* Dj = P.dxx + (long long)pr.j * P.ngrid;
    const bool two = pr.i != pr.j;
    for (int q = tid; q < G.n_me; q += nthr) {
        const long long g = grid_index(P.N, pr.g, G.pt_off[q]);
        const double v = vc[G.pt_cube[q]];
        atomicAdd(Di + g, v * phi_j[g]);
        if (two) atomicAdd(Dj + g, v * phi_i[g]);
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
