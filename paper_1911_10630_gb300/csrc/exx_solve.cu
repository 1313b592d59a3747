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

#include "exx_mg.cuh"
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

// PCG on the PE ball with the V-cycle as the preconditioner. On entry: r = rhs,
// d = 0, rr = ||rhs||^2; p goes to the cube pc (zero off the ball). Returns
// the iteration count; rr_out receives the final recursive ||r||^2.
//   T = double: the FP64 solve (precision 0), every level in FP64.
//   T = float: the inner solve of the FP64 refinement loop (precision 1): the
//   recurrence and the V-cycle in FP32 on the normalised residual, the stop
//   test of the refinement loop on the FP64 residual.
// Inlined into the kernel with P its own parameter block, so that the sweeps
// read the level operators as parameter constants; U unrolls the sweeps.
template <int NT, typename T, int U>
__device__ __forceinline__ int mg_pcg(const SolveParams& P, const BallGeo& G, const MGGeo& M, char* slot,
                                      T* __restrict__ pc, T* __restrict__ r, T* __restrict__ d, T* __restrict__ ap, T rr,
                                      T target2, int max_iter, T (*red)[33], int& flip, T& rr_out) {
    const int* cube = G.pt_cube;
    const int n_pe = G.n_pe, S = P.S;
    const long long S2 = P.S2;
    const Stencil<T>& A = mg_stencil<T>(P, 0);
    const T* __restrict__ Z = reinterpret_cast<const T*>(slot + P.off_tc);  // z = M r (level-0 cube)
    T* __restrict__ Zj = reinterpret_cast<T*>(slot + P.off_zc);             // the V-cycle's first Jacobi sweep
    const T wd = mg_wd<T>(P, 0);
    T rz = block_sum<NT, T>(mg_vcycle<NT, T, U>(P, G, M, slot, r), red, flip);
    for (int k = threadIdx.x; k < n_pe; k += NT) {
        const int c = cube[k];
        pc[c] = Z[c];
    }
    int it = 0;
    while (rr > target2 && it < max_iter) {
        __syncthreads();  // p
        T pap = T(0);
#pragma unroll (U)
        for (int k = threadIdx.x; k < n_pe; k += NT) {
            const int c = cube[k];
            const T a = lap19<T>(pc, c, S, S2, A);
            ap[k] = a;
            pap = fma(pc[c], a, pap);
        }
        pap = block_sum<NT, T>(pap, red, flip);
        const T al = rz / pap;
        T rrn = T(0);
        // d, r and the V-cycle's first sweep Z = w D^-1 r in one pass
#pragma unroll (U)
        for (int k = threadIdx.x; k < n_pe; k += NT) {
            const int c = cube[k];
            d[k] = fma(al, pc[c], d[k]);
            const T rk = fma(-al, ap[k], r[k]);
            r[k] = rk;
            Zj[c] = wd * rk;
            rrn = fma(rk, rk, rrn);
        }
        rrn = block_sum<NT, T>(rrn, red, flip);
        ++it;
        rr = rrn;
        if (rrn <= target2 || !(rrn == rrn)) break;
        const T rzn = block_sum<NT, T>(mg_vcycle<NT, T, U>(P, G, M, slot, r, 0, true), red, flip);
        const T be = rzn / rz;
        rz = rzn;
#pragma unroll (U)
        for (int k = threadIdx.x; k < n_pe; k += NT) {
            const int c = cube[k];
            pc[c] = fma(be, pc[c], Z[c]);
        }
    }
    rr_out = rr;
    return it;
}

// --------------------------------------------------------------------------
// The persistent pair kernel.
// --------------------------------------------------------------------------
// Resident CTAs per SM the launch bounds ask for: two of the FP64 and the
// 512-thread kernels; for the multigrid kernels 1024 threads per SM, except
// the 256-thread FP32 one: the sweeps wait on DRAM, and more CTAs keep more
// loads in flight at the price of registers (spills) and of cache space per
// pair. ONE_BALL (every pair on one PE ball, fixed radii): six CTAs, 40
// registers, the sweeps unrolled by 2; per-pair radii, whose largest balls
// then thrash the caches at six: five CTAs, 48 registers, no unrolling.
// Measured on one box, water-64 workload: five 0.512 s (unrolled) / 0.507
// (not), six 0.488 (unrolled); batched-uneven workload: five 0.331 / 0.328,
// six 0.467 (unrolled).
template <int NT, bool ONE_BALL>
constexpr int mg_min_blocks() { return NT == 256 ? (ONE_BALL ? 6 : 5) : 1024 / NT; }

template <int NT, bool MIXED, bool MG = false, bool ONE_BALL = false>
__global__ void __launch_bounds__(NT, MG ? mg_min_blocks<NT, ONE_BALL>() : (MIXED ? 1 : 2)) pair_kernel(const __grid_constant__ SolveParams P) {
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
        const bool clk = P.phase_clk && threadIdx.x == 0;
        const long long t0 = clk ? clock64() : 0;
        long long tr = 0;

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
        const long long t1 = clk ? clock64() : 0;
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
                iters = mg_pcg<NT, double, 2>(P, G, P.mg[pr.geo], slot, pc, r, d, ap, bb, target2, P.max_iter, red,
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
                const long long tu = clk ? clock64() : 0;
                double acc = 0.0;
                for (int k = threadIdx.x; k < n_pe; k += NT) {
                    const int c = cube[k];
                    const double rk = fma(four_pi, rho[k], lap19<double>(vc, c, S, S2, P.st64));
                    r[k] = rk;
                    acc = fma(rk, rk, acc);
                    if (bb < 0.0 && P.dbg_b) P.dbg_b[k] = rk;
                }
                const double rn2 = block_sum<NT, double>(acc, red, flip);
                if (clk) tr += clock64() - tu;
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
                    iters += mg_pcg<NT, float, ONE_BALL ? 2 : 1>(P, G, P.mg[pr.geo], slot, p32, r32, d32, ap32, rr32,
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
        const long long t2 = clk ? clock64() : 0;

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
                const int t = threadIdx.x;
                if (MIXED) mg_clear<float>(P, G, P.mg[pr.geo], slot, t, n_pe, t, NT);
                else mg_clear<double>(P, G, P.mg[pr.geo], slot, t, n_pe, t, NT);
            }
        }
        __syncthreads();
        if (clk) {
            const long long t3 = clock64();
            atomicAdd(P.phase_clk + 0, (unsigned long long)(t1 - t0));
            atomicAdd(P.phase_clk + 1, (unsigned long long)tr);
            atomicAdd(P.phase_clk + 2, (unsigned long long)(t2 - t1 - tr));
            atomicAdd(P.phase_clk + 3, (unsigned long long)(t3 - t2));
        }
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
    if (P.mg) {  // the multigrid-preconditioned CG: FP64, or FP32 inside FP64 refinement
        if (!mixed) pair_kernel<512, false, true><<<grid, 512, smem, st>>>(P);
        else if (threads == 256 && P.n_geo == 1) pair_kernel<256, true, true, true><<<grid, 256, smem, st>>>(P);
        else if (threads == 256) pair_kernel<256, true, true><<<grid, 256, smem, st>>>(P);
        else if (threads == 1024) pair_kernel<1024, true, true><<<grid, 1024, smem, st>>>(P);
        else pair_kernel<512, true, true><<<grid, 512, smem, st>>>(P);
        return cudaGetLastError();
    }
    if (threads == 256) return mixed ? launch_t<256, true>(P, grid, smem, st) : launch_t<256, false>(P, grid, smem, st);
    if (threads == 1024)
        return mixed ? launch_t<1024, true>(P, grid, smem, st) : launch_t<1024, false>(P, grid, smem, st);
    return mixed ? launch_t<512, true>(P, grid, smem, st) : launch_t<512, false>(P, grid, smem, st);
}

cudaError_t pair_kernel_occupancy(int threads, bool mixed, bool mg, bool one_ball, size_t smem, int* blocks_per_sm) {
    const void* f;
    if (mg && !mixed) f = (const void*)pair_kernel<512, false, true>;
    else if (mg && threads == 256 && one_ball) f = (const void*)pair_kernel<256, true, true, true>;
    else if (mg && threads == 256) f = (const void*)pair_kernel<256, true, true>;
    else if (mg && threads == 1024) f = (const void*)pair_kernel<1024, true, true>;
    else if (mg) f = (const void*)pair_kernel<512, true, true>;
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
