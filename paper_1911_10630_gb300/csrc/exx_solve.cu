// exx_solve.cu -- the per-pair pipeline, one CTA per pair (Sec. III.C Steps III-V).
//
// A persistent grid pops pairs from a device work counter. For each pair the
// CTA, using a workspace slot of its own:
//   1. gathers rho_ij = phi_i phi_j on the PE ball through the wrapped indices
//      of Eq. l2g (coalesced along z);
//   2. forms the multipole moments of Eq. mepole in Cartesian form: row sums
//      S_c = sum_z z^c rho, plane sums, then M_abc = sum rho x^a y^b z^c dV,
//      and the coefficients T = K M of the degree-l polynomials P_l (K is the
//      host-built Legendre-addition-theorem matrix);
//   3. evaluates the far-field potential of Eq. me on the shell as
//      v = sum_l P_l(r) / r^(2l+1), one thread per (x, y) row;
//   4. builds the right-hand side of Eq. pe_mat_red as the residual
//      b = 4 pi rho + lap v of the full 19-point stencil (Eq. d2_1) with v = 0
//      on the PE ball and the multipole values on the shell;
//   5. solves A d = b with A = -lap restricted to the PE ball by conjugate
//      gradient, either in FP64 or as FP32 inner CG with FP64 refinement
//      (r = 4 pi rho + lap v recomputed in FP64 after each inner solve);
//   6. E_ij = sum_PE rho v dV (Eq. exx_omega) and the scatter
//      D^i += v phi_j, D^j += v phi_i on the ME ball (Eqs. Dxx_mlwf_omega).
// The potential lives in an FP64 cube of side 2 R_ME + 1 (shell values around
// the PE ball); the CG direction lives in a zero-padded cube so the stencil
// needs no bounds checks; the other CG vectors are compact over the PE ball.
#include <cuda_runtime.h>

#include "exx_phases.cuh"

namespace exx {

// --------------------------------------------------------------------------
// Conjugate gradient on the PE ball (Step IV). On entry: r = rhs, p = rhs on
// the PE ball (0 elsewhere in the cube), d = 0, rr = ||rhs||^2. Returns the
// iteration count; rr_out receives the final recursive ||r||^2.
// --------------------------------------------------------------------------
template <typename T, int NT>
__device__ int cg_ball(T* __restrict__ pc, T* __restrict__ r, T* __restrict__ d, T* __restrict__ ap,
                       const int* __restrict__ cube, int n_pe, int S, long long S2, const Stencil<T>& neg_st,
                       T rr, T target2, int max_iter, T (*red)[33], int& flip, T& rr_out) {
    // Dot products, alpha and beta stay in T: in the FP32 solve no FP64
    // instruction runs per iteration (FP64 is 1/64 of the FP32 rate here).
    int it = 0;
    while (rr > target2 && it < max_iter) {
        T pap = T(0);
        for (int k = threadIdx.x; k < n_pe; k += NT) {
            const int c = cube[k];
            const T a = lap19<T>(pc, c, S, S2, neg_st);
            ap[k] = a;
            pap = fma(pc[c], a, pap);
        }
        pap = block_sum<NT, T>(pap, red, flip);
        const T al = rr / pap;
        T rrn = T(0);
        for (int k = threadIdx.x; k < n_pe; k += NT) {
            const int c = cube[k];
            d[k] = fma(al, pc[c], d[k]);
            const T rk = fma(-al, ap[k], r[k]);
            r[k] = rk;
            rrn = fma(rk, rk, rrn);
        }
        rrn = block_sum<NT, T>(rrn, red, flip);
        ++it;
        if (rrn <= target2 || !(rrn == rrn)) {
            rr = rrn;
            break;
        }
        const T be = rrn / rr;
        rr = rrn;
        for (int k = threadIdx.x; k < n_pe; k += NT) {
            const int c = cube[k];
            pc[c] = fma(be, pc[c], r[k]);
        }
        __syncthreads();
    }
    rr_out = rr;
    return it;
}

// --------------------------------------------------------------------------
// Multigrid-preconditioned CG (FP64, one CTA per pair). The preconditioner is
// one symmetric V-cycle of the geometric hierarchy of MGGeo: on each level a
// weighted-Jacobi sweep from zero, the residual, full-weighting restriction
// (R = P^T / 8) down to the coarsest ball, which is solved with its dense
// inverse, then trilinear prolongation (P) and one more Jacobi sweep on the
// way up. Every level's operator is the 19-point stencil of Eq. d2_1 at the
// level's spacing with zero outside its ball, so the V-cycle is a fixed
// symmetric positive definite operator and the CG stays a CG. Vectors that a
// stencil or a transfer reads live in zero-padded cubes of the workspace slot.
// --------------------------------------------------------------------------
template <typename T>
struct MGView {
    const int* cube;
    const int* off;
    int n, S, c;       // points, cube side, cube centre
    long long S2;
    T* Z;              // smoothed correction (cube)
    T* Tc;             // residual, then the post-smoothed correction (cube)
    const T* rhs;      // right-hand side (compact)
    T* rnext;          // the next level's right-hand side (compact), NULL on the coarsest
    Stencil<T> A;      // -lap at the level's spacing
};

template <typename T>
__device__ __forceinline__ long long mg_idx(const MGView<T>& v, int x, int y, int z) {
    return ((long long)(x + v.c) * v.S + (y + v.c)) * v.S + (z + v.c);
}

// z of level 0 (in its Tc cube) from the right-hand side r0 (compact): the
// down and up halves of the V-cycle, in T (FP64, or FP32 on a normalised r0).
template <int NT, typename T>
__device__ __noinline__ void mg_vcycle(const SolveParams& P, const BallGeo& G, const MGGeo& M, char* slot,
                                       const T* __restrict__ r0) {
    const T w = (T)P.mg_omega;
    auto view = [&](int l) {
        MGView<T> v;
        Stencil<T> base;
        if constexpr (sizeof(T) == 8) base = negated(P.st64);
        else base = negated(P.st32);
        if (l == 0) {
            v.cube = G.pt_cube;
            v.off = G.pt_off;
            v.n = G.n_pe;
            v.S = P.S;
            v.c = P.Rc;
            v.S2 = P.S2;
            v.Z = reinterpret_cast<T*>(slot + P.off_zc);
            v.Tc = reinterpret_cast<T*>(slot + P.off_tc);
            v.rhs = r0;
            v.A = base;
        } else {
            const MGLevel& lv = M.lv[l];
            v.cube = lv.cube;
            v.off = lv.off;
            v.n = lv.n;
            v.S = lv.side;
            v.c = lv.R + 3;
            v.S2 = (long long)lv.side * lv.side;
            v.Z = reinterpret_cast<T*>(slot + P.off_mgz[l]);
            v.Tc = reinterpret_cast<T*>(slot + P.off_mgt[l]);
            v.rhs = reinterpret_cast<const T*>(slot + P.off_mgr[l]);
            const T sc = (T)ldexp(1.0, -2 * l);  // spacing 2^l delta
            v.A = base;
            v.A.c0 *= sc;
            for (int q = 0; q < 3; ++q) {
                v.A.cx[q] *= sc;
                v.A.cy[q] *= sc;
                v.A.cz[q] *= sc;
            }
        }
        v.rnext = l < M.L ? reinterpret_cast<T*>(slot + P.off_mgr[l + 1]) : nullptr;
        return v;
    };
    // down: Jacobi from zero, residual, restriction
    for (int l = 0; l < M.L; ++l) {
        const MGView<T> v = view(l);
        const T wd = w / v.A.c0;
        for (int k = threadIdx.x; k < v.n; k += NT) v.Z[v.cube[k]] = wd * v.rhs[k];
        __syncthreads();
        for (int k = threadIdx.x; k < v.n; k += NT) {
            const int c = v.cube[k];
            v.Tc[c] = v.rhs[k] - lap19<T>(v.Z, c, v.S, v.S2, v.A);
        }
        __syncthreads();
        const MGLevel& cl = M.lv[l + 1];
        for (int k = threadIdx.x; k < cl.n; k += NT) {
            const int pk = cl.off[k];
            const int X = 2 * off_x(pk), Y = 2 * off_y(pk), Z = 2 * off_z(pk);
            T acc = T(0);
#pragma unroll
            for (int ex = -1; ex <= 1; ++ex)
#pragma unroll
                for (int ey = -1; ey <= 1; ++ey)
#pragma unroll
                    for (int ez = -1; ez <= 1; ++ez) {
                        const T wt = (ex ? T(0.5) : T(1)) * (ey ? T(0.5) : T(1)) * (ez ? T(0.5) : T(1));
                        acc = fma(wt, v.Tc[mg_idx(v, X + ex, Y + ey, Z + ez)], acc);
                    }
            v.rnext[k] = T(0.125) * acc;
        }
        __syncthreads();
    }
    // the coarsest level: its dense inverse
    {
        const MGView<T> v = view(M.L);
        const T* minv;
        if constexpr (sizeof(T) == 8) minv = M.minv;
        else minv = M.minv32;
        for (int k = threadIdx.x; k < v.n; k += NT) {
            const T* row = minv + (size_t)k * v.n;
            T acc = T(0);
            for (int j = 0; j < v.n; ++j) acc = fma(row[j], v.rhs[j], acc);
            v.Z[v.cube[k]] = acc;
        }
        __syncthreads();
    }
    // up: prolongation of the coarser correction, then a Jacobi sweep into Tc
    for (int l = M.L - 1; l >= 0; --l) {
        const MGView<T> v = view(l), vc = view(l + 1);
        const T* zc = (l + 1 == M.L) ? vc.Z : vc.Tc;
        for (int k = threadIdx.x; k < v.n; k += NT) {
            const int pk = v.off[k];
            const int o[3] = {off_x(pk), off_y(pk), off_z(pk)};
            int lo[3], hi[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                lo[a] = (o[a] - (o[a] & 1)) / 2;  // floor(o / 2)
                hi[a] = lo[a] + (o[a] & 1);
            }
            T acc = T(0);
#pragma unroll
            for (int cx = 0; cx < 2; ++cx)
#pragma unroll
                for (int cy = 0; cy < 2; ++cy)
#pragma unroll
                    for (int cz = 0; cz < 2; ++cz) {
                        if ((cx && hi[0] == lo[0]) || (cy && hi[1] == lo[1]) || (cz && hi[2] == lo[2])) continue;
                        const T wt = (hi[0] != lo[0] ? T(0.5) : T(1)) * (hi[1] != lo[1] ? T(0.5) : T(1)) *
                                     (hi[2] != lo[2] ? T(0.5) : T(1));
                        acc = fma(wt, zc[mg_idx(vc, cx ? hi[0] : lo[0], cy ? hi[1] : lo[1], cz ? hi[2] : lo[2])],
                                  acc);
                    }
            v.Z[v.cube[k]] += acc;
        }
        __syncthreads();
        const T wd = w / v.A.c0;
        for (int k = threadIdx.x; k < v.n; k += NT) {
            const int c = v.cube[k];
            v.Tc[c] = fma(wd, v.rhs[k] - lap19<T>(v.Z, c, v.S, v.S2, v.A), v.Z[c]);
        }
        __syncthreads();
    }
}

// Clears what a pair wrote into the multigrid cubes (per-pair radii: the next
// pair's balls may have other sizes, and every cube must be zero off its ball).
template <int NT, typename T>
__device__ void mg_clear(const SolveParams& P, const BallGeo& G, const MGGeo& M, char* slot) {
    T* Z0 = reinterpret_cast<T*>(slot + P.off_zc);
    T* T0 = reinterpret_cast<T*>(slot + P.off_tc);
    for (int k = threadIdx.x; k < G.n_pe; k += NT) Z0[G.pt_cube[k]] = T0[G.pt_cube[k]] = T(0);
    for (int l = 1; l <= M.L; ++l) {
        T* Z = reinterpret_cast<T*>(slot + P.off_mgz[l]);
        T* Tc = reinterpret_cast<T*>(slot + P.off_mgt[l]);
        for (int k = threadIdx.x; k < M.lv[l].n; k += NT) Z[M.lv[l].cube[k]] = Tc[M.lv[l].cube[k]] = T(0);
    }
}

// PCG on the PE ball with the V-cycle as the preconditioner. On entry: r = rhs,
// d = 0, rr = ||rhs||^2; p goes to the cube pc (zero off the ball). Returns
// the iteration count; rr_out receives the final recursive ||r||^2.
//   T = double: the FP64 solve (precision 0), every level in FP64.
//   T = float: the inner solve of the FP64 refinement loop (precision 1): the
//   recurrence and the V-cycle in FP32 on the normalised residual, the stop
//   test of the refinement loop on the FP64 residual.
template <int NT, typename T>
__device__ __noinline__ int mg_pcg(const SolveParams& P, const BallGeo& G, const MGGeo& M, char* slot,
                                   T* __restrict__ pc, T* __restrict__ r, T* __restrict__ d, T* __restrict__ ap, T rr,
                                   T target2, int max_iter, T (*red)[33], int& flip, T& rr_out) {
    const int* cube = G.pt_cube;
    const int n_pe = G.n_pe, S = P.S;
    const long long S2 = P.S2;
    Stencil<T> A;
    if constexpr (sizeof(T) == 8) A = negated(P.st64);
    else A = negated(P.st32);
    const T* Z = reinterpret_cast<const T*>(slot + P.off_tc);  // z = M r (level-0 cube)
    mg_vcycle<NT, T>(P, G, M, slot, r);
    T rz = T(0);
    for (int k = threadIdx.x; k < n_pe; k += NT) {
        const int c = cube[k];
        const T z = Z[c];
        pc[c] = z;
        rz = fma(r[k], z, rz);
    }
    rz = block_sum<NT, T>(rz, red, flip);
    int it = 0;
    while (rr > target2 && it < max_iter) {
        T pap = T(0);
        for (int k = threadIdx.x; k < n_pe; k += NT) {
            const int c = cube[k];
            const T a = lap19<T>(pc, c, S, S2, A);
            ap[k] = a;
            pap = fma(pc[c], a, pap);
        }
        pap = block_sum<NT, T>(pap, red, flip);
        const T al = rz / pap;
        T rrn = T(0);
        for (int k = threadIdx.x; k < n_pe; k += NT) {
            const int c = cube[k];
            d[k] = fma(al, pc[c], d[k]);
            const T rk = fma(-al, ap[k], r[k]);
            r[k] = rk;
            rrn = fma(rk, rk, rrn);
        }
        rrn = block_sum<NT, T>(rrn, red, flip);
        ++it;
        rr = rrn;
        if (rrn <= target2 || !(rrn == rrn)) break;
        mg_vcycle<NT, T>(P, G, M, slot, r);
        T rzn = T(0);
        for (int k = threadIdx.x; k < n_pe; k += NT) rzn = fma(r[k], Z[cube[k]], rzn);
        rzn = block_sum<NT, T>(rzn, red, flip);
        const T be = rzn / rz;
        rz = rzn;
        for (int k = threadIdx.x; k < n_pe; k += NT) {
            const int c = cube[k];
            pc[c] = fma(be, pc[c], Z[c]);
        }
        __syncthreads();
    }
    rr_out = rr;
    return it;
}

// --------------------------------------------------------------------------
// The persistent pair kernel.
// --------------------------------------------------------------------------
template <int NT, bool MIXED, bool MG = false>
__global__ void __launch_bounds__(NT, (MIXED && !MG) ? 1 : 2) pair_kernel(const __grid_constant__ SolveParams P) {
    extern __shared__ double smem[];
    __shared__ double red[2][33];
    __shared__ float red32[2][33];
    __shared__ double s_M[kNMono], s_T[kNMono];
    __shared__ int s_item;
    __shared__ double s_ub[NT / 32][kNU + kNU / 2];
    int flip = 0, flip32 = 0;

    const int Rc = P.Rc;
    const int S = P.S;
    const long long S2 = P.S2;
    double* xp = smem;                      // [(2Rc+1)*8] x^a
    double* yp = xp + (2 * Rc + 1) * 8;     // y^b
    double* zp = yp + (2 * Rc + 1) * 8;     // z^c
    double* sY = zp + (2 * Rc + 1) * 8;     // [(2 Rmax_pe + 1) * 28]

    fill_power_tables(P, xp, yp, zp, threadIdx.x, NT);
    __syncthreads();

    char* slot = P.ws + (size_t)blockIdx.x * P.slot_bytes;
    double* vc = reinterpret_cast<double*>(slot + P.off_vcube);
    double* pc = reinterpret_cast<double*>(slot + P.off_pcube);
    double* rho = reinterpret_cast<double*>(slot + P.off_rho);
    double* r = reinterpret_cast<double*>(slot + P.off_r);
    double* d = reinterpret_cast<double*>(slot + P.off_d);
    double* ap = reinterpret_cast<double*>(slot + P.off_ap);
    float* p32 = reinterpret_cast<float*>(slot + P.off_p32);
    float* r32 = reinterpret_cast<float*>(slot + P.off_r32);
    float* d32 = reinterpret_cast<float*>(slot + P.off_d32);
    float* ap32 = reinterpret_cast<float*>(slot + P.off_ap32);
    double* rowS = reinterpret_cast<double*>(slot + P.off_rows);

    const Stencil<double> neg64 = negated(P.st64);
    const Stencil<float> neg32 = negated(P.st32);
    const double four_pi = kFourPi;
    const int np = *P.n_pair;

    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(P.queue, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= np) break;
        const int pidx = P.order ? P.order[(P.item_base ? *P.item_base : 0) + item] : item;
        const PairRec pr = P.pairs[pidx];
        const BallGeo G = P.geos[pr.geo];
        const int* cube = G.pt_cube;
        const int n_pe = G.n_pe;

        // 1. gather rho on the PE ball; v = 0 there
        gather_rho(P, G, pr, rho, vc, threadIdx.x, NT);
        __syncthreads();

        // 2. multipole moments and polynomial coefficients
        moment_rows(P, G, rho, rowS, zp, threadIdx.x, NT);
        __syncthreads();
        moment_finish<NT>(P, G, rowS, xp, yp, sY, s_M, s_T);

        // 3. far-field potential on the shell
        shell_potential(P, G, vc, xp, yp, s_T, s_ub[threadIdx.x >> 5], threadIdx.x >> 5, NT / 32);
        __syncthreads();

        // 4./5. right-hand side and solve
        int iters = 0, refines = 0;
        bool conv = true;
        if (!MIXED) {
            double acc = 0.0;
            for (int k = threadIdx.x; k < n_pe; k += NT) {
                const int c = cube[k];
                const double b = fma(four_pi, rho[k], lap19<double>(vc, c, S, S2, P.st64));
                r[k] = b;
                pc[c] = b;
                d[k] = 0.0;
                acc = fma(b, b, acc);
                if (P.dbg_b) P.dbg_b[k] = b;
            }
            const double bb = block_sum<NT, double>(acc, red, flip);
            double rr_fin;
            const double target2 = P.tol * P.tol * bb;
            if (MG && P.mg[pr.geo].L > 0)
                iters = mg_pcg<NT, double>(P, G, P.mg[pr.geo], slot, pc, r, d, ap, bb, target2, P.max_iter, red,
                                           flip, rr_fin);
            else
                iters = cg_ball<double, NT>(pc, r, d, ap, cube, n_pe, S, S2, neg64, bb, target2, P.max_iter, red,
                                            flip, rr_fin);
            conv = rr_fin <= target2;
            for (int k = threadIdx.x; k < n_pe; k += NT) vc[cube[k]] += d[k];
            refines = 1;
        } else {
            double bb = -1.0, rn_prev = 1e300;
            for (;;) {
                // FP64 residual r = 4 pi rho + lap v (v: current iterate on PE, shell values outside)
                double acc = 0.0;
                for (int k = threadIdx.x; k < n_pe; k += NT) {
                    const int c = cube[k];
                    const double rk = fma(four_pi, rho[k], lap19<double>(vc, c, S, S2, P.st64));
                    r[k] = rk;
                    acc = fma(rk, rk, acc);
                    if (bb < 0.0 && P.dbg_b) P.dbg_b[k] = rk;
                }
                const double rn2 = block_sum<NT, double>(acc, red, flip);
                if (bb < 0.0) bb = rn2;
                if (rn2 <= P.tol * P.tol * bb) break;
                const double rn = sqrt(rn2);
                if (refines >= P.max_refine || iters >= P.max_iter || !(rn < rn_prev)) {
                    conv = false;
                    break;
                }
                rn_prev = rn;
                const double inv = 1.0 / rn;
                float acc32 = 0.0f;
                for (int k = threadIdx.x; k < n_pe; k += NT) {
                    const int c = cube[k];
                    const float rk = (float)(r[k] * inv);
                    r32[k] = rk;
                    p32[c] = rk;
                    d32[k] = 0.0f;
                    acc32 = fmaf(rk, rk, acc32);
                }
                const float rr32 = block_sum<NT, float>(acc32, red32, flip32);
                double eta = 0.3 * P.tol * sqrt(bb) / rn;
                eta = eta > P.inner_tol ? eta : P.inner_tol;
                float rr_fin;
                const int budget = min(P.inner_max_iter, P.max_iter - iters);
                if (MG && P.mg[pr.geo].L > 0)
                    iters += mg_pcg<NT, float>(P, G, P.mg[pr.geo], slot, p32, r32, d32, ap32, rr32,
                                               (float)(eta * eta) * rr32, budget, red32, flip32, rr_fin);
                else
                    iters += cg_ball<float, NT>(p32, r32, d32, ap32, cube, n_pe, S, S2, neg32, rr32,
                                                (float)(eta * eta) * rr32, budget, red32, flip32, rr_fin);
                for (int k = threadIdx.x; k < n_pe; k += NT) vc[cube[k]] = fma(rn, (double)d32[k], vc[cube[k]]);
                ++refines;
                __syncthreads();
            }
        }
        __syncthreads();

        // 6. E_ij over the PE ball and the D_xx scatter over the ME ball
        double e = 0.0;
        for (int k = threadIdx.x; k < n_pe; k += NT) e = fma(rho[k], vc[cube[k]], e);
        e = block_sum<NT, double>(e, red, flip);
        if (threadIdx.x == 0) {
            P.e_pair[pidx] = e * P.dV;
            P.iters[pidx] = iters;
            if (P.refines) P.refines[pidx] = refines;
            if (!conv) atomicAdd(P.nonconv, 1);
        }
        scatter_dxx(P, G, pr, vc, threadIdx.x, NT);
        if (P.n_geo > 1) {
            // the next pair may have another ball: the direction cube must be
            // zero outside it, so clear the points this pair wrote
            for (int k = threadIdx.x; k < n_pe; k += NT) {
                if (MIXED) p32[cube[k]] = 0.0f;
                else pc[cube[k]] = 0.0;
            }
            if (MG && P.mg[pr.geo].L > 0) {
                if (MIXED) mg_clear<NT, float>(P, G, P.mg[pr.geo], slot);
                else mg_clear<NT, double>(P, G, P.mg[pr.geo], slot);
            }
        }
        __syncthreads();
    }
}

// Debug: rho on the whole ME ball and v read back from slot 0.
__global__ void debug_pair_readback(const SolveParams P, PairRec pr, double* rho_me, double* v_me) {
    const BallGeo G = P.geos[pr.geo];
    const double* vc = reinterpret_cast<const double*>(P.ws + P.off_vcube);
    const double* phi_i = P.phi + (long long)pr.i * P.ostride;
    const double* phi_j = P.phi + (long long)pr.j * P.ostride;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < G.n_me; q += gridDim.x * blockDim.x) {
        const long long ii = orb_index(P.N, pr.g, G.pt_off[q], P.box_org, P.bdim, pr.i);
        const long long ij = orb_index(P.N, pr.g, G.pt_off[q], P.box_org, P.bdim, pr.j);
        rho_me[q] = (ii >= 0 && ij >= 0) ? phi_i[ii] * phi_j[ij] : 0.0;
        v_me[q] = vc[G.pt_cube[q]];
    }
}

// A p on the PE ball: scatter p into the (zeroed) slot-0 cube, then apply.
__global__ void apply_scatter(const SolveParams P, const double* p) {
    const BallGeo G = P.geos[P.n_geo - 1];
    double* pc = reinterpret_cast<double*>(P.ws + P.off_pcube);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < G.n_pe; k += gridDim.x * blockDim.x)
        pc[G.pt_cube[k]] = p[k];
}

__global__ void apply_stencil(const SolveParams P, double* ap) {
    const BallGeo G = P.geos[P.n_geo - 1];
    const double* pc = reinterpret_cast<const double*>(P.ws + P.off_pcube);
    const Stencil<double> neg = negated(P.st64);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < G.n_pe; k += gridDim.x * blockDim.x)
        ap[k] = lap19<double>(pc, G.pt_cube[k], P.S, P.S2, neg);
}

__global__ void apply_unscatter(const SolveParams P) {
    const BallGeo G = P.geos[P.n_geo - 1];
    double* pc = reinterpret_cast<double*>(P.ws + P.off_pcube);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < G.n_pe; k += gridDim.x * blockDim.x)
        pc[G.pt_cube[k]] = 0.0;
}

// ---- host side ----
cudaError_t set_multipole_const_solve(const MultipoleConst& mc) {
    return cudaMemcpyToSymbol(c_mp, &mc, sizeof(MultipoleConst));
}

size_t pair_kernel_smem(int Rc, int r_pe_max) {
    return sizeof(double) * ((size_t)3 * (2 * Rc + 1) * 8 + (size_t)(2 * r_pe_max + 1) * 28);
}

template <int NT, bool MIXED>
static cudaError_t launch_t(const SolveParams& P, int grid, size_t smem, cudaStream_t st) {
    pair_kernel<NT, MIXED><<<grid, NT, smem, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_pair_kernel(const SolveParams& P, int threads, bool mixed, int grid, size_t smem, cudaStream_t st) {
    if (P.mg) {  // the multigrid-preconditioned CG (512 threads): FP64, or FP32 inside FP64 refinement
        if (mixed) pair_kernel<512, true, true><<<grid, 512, smem, st>>>(P);
        else pair_kernel<512, false, true><<<grid, 512, smem, st>>>(P);
        return cudaGetLastError();
    }
    if (threads == 256) return mixed ? launch_t<256, true>(P, grid, smem, st) : launch_t<256, false>(P, grid, smem, st);
    if (threads == 1024)
        return mixed ? launch_t<1024, true>(P, grid, smem, st) : launch_t<1024, false>(P, grid, smem, st);
    return mixed ? launch_t<512, true>(P, grid, smem, st) : launch_t<512, false>(P, grid, smem, st);
}

cudaError_t pair_kernel_occupancy(int threads, bool mixed, bool mg, size_t smem, int* blocks_per_sm) {
    const void* f;
    if (mg) f = mixed ? (const void*)pair_kernel<512, true, true> : (const void*)pair_kernel<512, false, true>;
    else if (threads == 256) f = mixed ? (const void*)pair_kernel<256, true> : (const void*)pair_kernel<256, false>;
    else if (threads == 1024) f = mixed ? (const void*)pair_kernel<1024, true> : (const void*)pair_kernel<1024, false>;
    else f = mixed ? (const void*)pair_kernel<512, true> : (const void*)pair_kernel<512, false>;
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, threads, smem);
}

cudaError_t launch_debug_readback(const SolveParams& P, const PairRec& pr, double* rho_me, double* v_me,
                                  cudaStream_t st) {
    debug_pair_readback<<<64, 256, 0, st>>>(P, pr, rho_me, v_me);
    return cudaGetLastError();
}

cudaError_t launch_apply(const SolveParams& P, const double* p, double* ap, cudaStream_t st) {
    apply_scatter<<<64, 256, 0, st>>>(P, p);
    apply_stencil<<<64, 256, 0, st>>>(P, ap);
    apply_unscatter<<<64, 256, 0, st>>>(P);
    return cudaGetLastError();
}

}  // namespace exx
