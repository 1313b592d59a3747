// exx_mg.cuh -- the geometric-multigrid V-cycle that preconditions the CG of
// Step IV (Sec. III.C), shared by the one-CTA and the cluster pair kernels.
//
// Levels: the PE ball of radius R (level 0), then balls of radius ceil(R / 2),
// ... down to radius <= 3, each at twice the previous spacing. Every level's
// operator is the 19-point stencil of Eq. d2_1 at the level's spacing with
// zero outside its ball, so one symmetric V-cycle is a fixed symmetric
// positive definite operator and the CG stays a CG. Down: a weighted-Jacobi
// sweep from zero, the residual, full-weighting restriction (R = P^T / 8) to
// the next level's right-hand side; bottom: the coarsest ball's dense inverse;
// up: trilinear prolongation of the coarser correction, then one more Jacobi
// sweep. Vectors that a stencil or a transfer reads live in zero-padded cubes
// of the pair's workspace slot; right-hand sides are compact.
//
// Each stage runs over the level's compact points k = kb, kb + step, ... < ke
// and the caller synchronises between stages: one CTA strides over all points
// (kb = threadIdx.x, step = NT), a cluster gives each CTA a range of them.
#pragma once

#include "exx_kernels.cuh"  // lap19, off_x / off_y / off_z

namespace exx {

// U: unrolling of a stage's loop over its points (over restrict-qualified
// arrays the loads of the unrolled points overlap, at the price of registers).
// The default, 2, is the cluster kernels'; the one-CTA kernel picks its own
// by its residency.

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
    int l;             // level (its operator: mg_stencil)
};

// -lap at level l's spacing and the Jacobi factor omega / diagonal, read from
// the kernel parameters (the caller passes the kernel's own parameter block).
template <typename T>
__device__ __forceinline__ const Stencil<T>& mg_stencil(const SolveParams& P, int l) {
    if constexpr (sizeof(T) == 8) return P.mg_a64[l];
    else return P.mg_a32[l];
}
template <typename T>
__device__ __forceinline__ T mg_wd(const SolveParams& P, int l) {
    if constexpr (sizeof(T) == 8) return P.mg_wd64[l];
    else return P.mg_wd32[l];
}

template <typename T>
__device__ __forceinline__ long long mg_idx(const MGView<T>& v, int x, int y, int z) {
    return ((long long)(x + v.c) * v.S + (y + v.c)) * v.S + (z + v.c);
}

// Level l of hierarchy M in the workspace slot; level 0 is the PE ball with
// right-hand side r0 (compact), the levels below read theirs from the slot.
template <typename T>
__device__ __forceinline__ MGView<T> mg_view(const SolveParams& P, const BallGeo& G, const MGGeo& M, char* slot,
                                             int l, const T* r0) {
    MGView<T> v;
    v.l = l;
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
    }
    v.rnext = l < M.L ? reinterpret_cast<T*>(slot + P.off_mgr[l + 1]) : nullptr;
    return v;
}

// Jacobi from zero: Z = w D^-1 rhs.
template <typename T, int U = 2>
__device__ __forceinline__ void mg_jacobi0(const SolveParams& P, const MGView<T>& v, int kb, int ke, int step) {
    const T wd = mg_wd<T>(P, v.l);
    const int* __restrict__ cube = v.cube;
    const T* __restrict__ rhs = v.rhs;
    T* __restrict__ Zs = v.Z;
#pragma unroll (U)
    for (int k = kb; k < ke; k += step) Zs[cube[k]] = wd * rhs[k];
}

// Residual into Tc: rhs - A Z.
template <typename T, int U = 2>
__device__ __forceinline__ void mg_residual(const SolveParams& P, const MGView<T>& v, int kb, int ke, int step) {
    const Stencil<T>& A = mg_stencil<T>(P, v.l);
    const int* __restrict__ cube = v.cube;
    const T* __restrict__ rhs = v.rhs;
    const T* __restrict__ Zs = v.Z;
    T* __restrict__ Tcs = v.Tc;
#pragma unroll (U)
    for (int k = kb; k < ke; k += step) {
        const int c = cube[k];
        Tcs[c] = rhs[k] - lap19<T>(Zs, c, v.S, v.S2, A);
    }
}

// Full weighting of Tc onto the points kb.. of the next level cl (its rhs).
template <typename T, int U = 2>
__device__ __forceinline__ void mg_restrict(const MGView<T>& v, const MGLevel& cl, int kb, int ke, int step) {
    const int* __restrict__ off = cl.off;
    const T* __restrict__ Tcs = v.Tc;
    T* __restrict__ rn = v.rnext;
#pragma unroll (U)
    for (int k = kb; k < ke; k += step) {
        const int pk = off[k];
        const int X = 2 * off_x(pk), Y = 2 * off_y(pk), Z = 2 * off_z(pk);
        T acc = T(0);
#pragma unroll
        for (int ex = -1; ex <= 1; ++ex)
#pragma unroll
            for (int ey = -1; ey <= 1; ++ey)
#pragma unroll
                for (int ez = -1; ez <= 1; ++ez) {
                    const T wt = (ex ? T(0.5) : T(1)) * (ey ? T(0.5) : T(1)) * (ez ? T(0.5) : T(1));
                    acc = fma(wt, Tcs[mg_idx(v, X + ex, Y + ey, Z + ez)], acc);
                }
        rn[k] = T(0.125) * acc;
    }
}

// The coarsest level: Z = M^-1 rhs with the dense inverse minv.
template <typename T>
__device__ __forceinline__ void mg_bottom(const MGView<T>& v, const T* minv, int kb, int ke, int step) {
    for (int k = kb; k < ke; k += step) {
        const T* row = minv + (size_t)k * v.n;
        T acc = T(0);
        for (int j = 0; j < v.n; ++j) acc = fma(row[j], v.rhs[j], acc);
        v.Z[v.cube[k]] = acc;
    }
}

// Z += P zc: trilinear prolongation of the coarser correction zc (level vc's cube).
template <typename T, int U = 2>
__device__ __forceinline__ void mg_prolong(const MGView<T>& v, const MGView<T>& vc, const T* zc, int kb, int ke,
                                           int step) {
    const int* __restrict__ off = v.off;
    const int* __restrict__ cube = v.cube;
    T* __restrict__ Zs = v.Z;
    const T* __restrict__ zcs = zc;
#pragma unroll (U)
    for (int k = kb; k < ke; k += step) {
        const int pk = off[k];
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
                    acc = fma(wt, zcs[mg_idx(vc, cx ? hi[0] : lo[0], cy ? hi[1] : lo[1], cz ? hi[2] : lo[2])], acc);
                }
        Zs[cube[k]] += acc;
    }
}

// Post-smoothing: Tc = Z + w D^-1 (rhs - A Z); returns this thread's sum of
// rhs . Tc (on level 0: r . z for the PCG).
template <typename T, int U = 2>
__device__ __forceinline__ T mg_smooth(const SolveParams& P, const MGView<T>& v, int kb, int ke, int step) {
    const T wd = mg_wd<T>(P, v.l);
    const Stencil<T>& A = mg_stencil<T>(P, v.l);
    const int* __restrict__ cube = v.cube;
    const T* __restrict__ rhs = v.rhs;
    const T* __restrict__ Zs = v.Z;
    T* __restrict__ Tcs = v.Tc;
    T rz = T(0);
#pragma unroll (U)
    for (int k = kb; k < ke; k += step) {
        const int c = cube[k];
        const T t = fma(wd, rhs[k] - lap19<T>(Zs, c, v.S, v.S2, A), Zs[c]);
        Tcs[c] = t;
        rz = fma(rhs[k], t, rz);
    }
    return rz;
}

// The V-cycle from level l0 down and back up to it, on one CTA (CTA barriers
// between the stages). With l0 = 0 this is the whole preconditioner z = M r0
// (z in the level-0 Tc cube); with l0 = 1 it continues a cycle whose level-1
// right-hand side is already in the slot, leaving level 1's correction in its
// Tc cube (its Z cube when level 1 is the coarsest). With z0_ready the caller
// has already written level l0's first Jacobi sweep (Z = w D^-1 rhs) and
// synchronised. Returns this thread's share of rhs . z on level l0.
template <int NT, typename T, int U = 2>
__device__ __forceinline__ T mg_vcycle(const SolveParams& P, const BallGeo& G, const MGGeo& M, char* slot,
                                       const T* __restrict__ r0, int l0 = 0, bool z0_ready = false) {
    const int t = threadIdx.x;
    for (int l = l0; l < M.L; ++l) {
        const MGView<T> v = mg_view<T>(P, G, M, slot, l, r0);
        if (!(l == l0 && z0_ready)) {
            mg_jacobi0<T, U>(P, v, t, v.n, NT);
            __syncthreads();
        }
        mg_residual<T, U>(P, v, t, v.n, NT);
        __syncthreads();
        mg_restrict<T, U>(v, M.lv[l + 1], t, M.lv[l + 1].n, NT);
        __syncthreads();
    }
    {
        const MGView<T> v = mg_view<T>(P, G, M, slot, M.L, r0);
        const T* minv;
        if constexpr (sizeof(T) == 8) minv = M.minv;
        else minv = M.minv32;
        mg_bottom(v, minv, t, v.n, NT);
        __syncthreads();
    }
    T rz = T(0);
    for (int l = M.L - 1; l >= l0; --l) {
        const MGView<T> v = mg_view<T>(P, G, M, slot, l, r0), vc = mg_view<T>(P, G, M, slot, l + 1, r0);
        mg_prolong<T, U>(v, vc, (l + 1 == M.L) ? vc.Z : vc.Tc, t, v.n, NT);
        __syncthreads();
        rz = mg_smooth<T, U>(P, v, t, v.n, NT);
        __syncthreads();
    }
    return rz;
}

// Zeroes the level cubes' points kb.. (per-pair radii: the next pair's balls
// may have other sizes, and every cube must be zero off its ball). Level 0
// over [kb0, ke0), the coarse levels over [kbc, n_l) when kbc >= 0.
template <typename T>
__device__ __forceinline__ void mg_clear(const SolveParams& P, const BallGeo& G, const MGGeo& M, char* slot, int kb0,
                                         int ke0, int kbc, int step) {
    T* Z0 = reinterpret_cast<T*>(slot + P.off_zc);
    T* T0 = reinterpret_cast<T*>(slot + P.off_tc);
    for (int k = kb0; k < ke0; k += step) Z0[G.pt_cube[k]] = T0[G.pt_cube[k]] = T(0);
    if (kbc < 0) return;
    for (int l = 1; l <= M.L; ++l) {
        T* Z = reinterpret_cast<T*>(slot + P.off_mgz[l]);
        T* Tc = reinterpret_cast<T*>(slot + P.off_mgt[l]);
        for (int k = kbc; k < M.lv[l].n; k += step) Z[M.lv[l].cube[k]] = Tc[M.lv[l].cube[k]] = T(0);
    }
}

}  // namespace exx
