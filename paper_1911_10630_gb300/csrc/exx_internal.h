// exx_internal.h -- types shared by the host orchestration and the kernels of
// the pair-Poisson exact-exchange library (not part of the public ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace exx {

// Multipole order limit and the Cartesian monomial count for l <= 6:
// sum_{l=0..6} (l+1)(l+2)/2 = 84.
constexpr int kLmaxMax = 6;
constexpr int kNMono = 84;
constexpr int kNU = 28;  // sum_{l<=6} (l+1): per-row polynomial coefficients U_{l,c}

// One pair of the list (Sec. III.C Step II). 32 bytes.
struct PairRec {
    int i, j;       // orbitals, i <= j
    int g[3];       // grid point nearest the pair centre, in [0, N)
    int r_pe, r_me; // radii in grid points for this pair
    int geo;        // index of the ball geometry used (radii table)
};

// One (x, y) row of a ball: z runs over [-zme, zme]; the PE part is
// [-zpe, zpe] (zpe < 0 when the row has no PE points).
struct RowRec {
    short ox, oy;
    short zpe, zme;
    int pe_start;   // compact PE index of (ox, oy, -zpe), or -1
    int zn;         // shell points with |z| <= zn are read by stencil legs of PE points (-1: none)
};

// Device tables of one ball geometry (R_PE, R_ME); points in Algorithm 2
// order: PE points lexicographic, then shell points lexicographic.
struct BallGeo {
    int r_pe, r_me;
    int n_pe, n_me;
    int n_rows_pe, n_rows_me;
    const int* pt_cube;      // [n_me] index in the workspace cube
    const int* pt_off;       // [n_me] packed offsets: (ox+128) | (oy+128)<<8 | (oz+128)<<16
    const RowRec* rows_pe;   // [n_rows_pe]
    const RowRec* rows_me;   // [n_rows_me]
    const int* plane_pe;     // [2 r_pe + 2] first PE row of each x plane (last = n_rows_pe)
    const int* row_of;       // [(2 r_pe + 1)^2] PE row index of (ox, oy), -1 outside
    // shell points split by the precision of their boundary value (|z| <= zn
    // of the row: FP64, read by the stencil; else FP32), ME row << 8 | (z + 128)
    const int* sh_near;
    const int* sh_far;
    int n_near, n_far;
};

// 19-point Laplacian coefficients of Eq. d2_1 on an orthorhombic grid:
// lap f(c) = c0 f(c) + sum_a sum_q ca[q-1] (f(c + q s_a) + f(c - q s_a)).
template <typename T>
struct Stencil {
    T c0;
    T cx[3], cy[3], cz[3];
};

constexpr int kMaxGeo = 64;

// Geometric multigrid of the preconditioned CG (one CTA per pair): level 0 is
// the PE ball of R_PE at spacing delta in the workspace cube; level l >= 1 is
// the ball of R_l = ceil(R_{l-1} / 2) at spacing 2^l delta, stored in its own
// zero-padded cube of side 2 R_l + 7 (centre R_l + 3), down to R_L <= 3, where
// the coarse problem is solved with its dense inverse.
constexpr int kMGMax = 6;  // coarse levels at most (R_PE <= 64)
struct MGLevel {
    int R, n, side;         // radius, points, cube side
    const int* cube;        // [n] index of each point in the level cube (Algorithm 2 order)
    const int* off;         // [n] packed offsets, as BallGeo::pt_off
};
struct MGGeo {
    int L;                  // coarse levels (1..L)
    MGLevel lv[kMGMax + 1]; // lv[1..L]
    const double* minv;     // [n_L][n_L] inverse of the coarsest operator
    const float* minv32;    // the same in FP32 (FP32 V-cycle)
};

// Everything the pair kernel needs, passed by value.
struct SolveParams {
    // inputs / outputs
    const double* phi;
    double* dxx;
    long long ngrid;    // N0 N1 N2
    // compact orbital boxes (exx_compute_boxes): orbital i holds the grid
    // points (box_org[i] + b) mod N, b in [0, bdim), in C order; the points
    // outside count as zero for it. NULL = full grids.
    const int* box_org;
    int bdim[3];
    long long ostride;  // values per orbital in phi and dxx: ngrid, or the box volume
    int N[3];
    double delta[3];
    double dV;
    Stencil<double> st64;
    Stencil<float> st32;

    // pairs
    const PairRec* pairs;
    const int* n_pair;  // device scalar
    const int* order;   // processing order (NULL = list order)
    const int* item_base;  // if set, the launch takes order[*item_base + item] (one radius class per launch)
    int* queue;         // device work counter

    // geometry
    const BallGeo* geos;  // device array of geometries
    int n_geo;
    int S, Rc;            // cube side and cube radius of the workspace
    long long S2;

    // workspace: n_slots slots of slot_bytes each
    char* ws;
    size_t slot_bytes;
    size_t off_vcube, off_pcube, off_rho, off_r, off_d, off_ap;  // FP64 parts
    size_t off_p32, off_r32, off_d32, off_ap32;                  // FP32 parts
    size_t off_rows;                                             // [n_rows_pe][8] row sums
    size_t off_sy;                                               // [C][(2 r_pe + 1) * 28] plane sums (cluster)
    size_t off_ush;                                              // [28][n_rows_me] FP64 then FP32 row coefficients U_{l,c} (cluster)
    size_t off_vfix;                                             // [S^3] int64 fixed-point copy of v (cluster, fixres)
    int fixres;               // cluster kernel: FP64 residuals from an exact integer stencil on a fixed-point v
                              // (1; 2: bound made too small, every pair falls back, for tests)
    double fix_inv;           // 1 / (180 delta^2): the integer stencil's weights are 180 delta^2 x Eq. d2_1's
    double dfix;              // D_xx as fixed-point integers with this scale (2^40; 0 = FP64 atomics)
    int* dfix_range;          // counts fixed-point D_xx contributions beyond the range (dropped)
    // multigrid-preconditioned CG (one-CTA FP64 solver): per geometry, NULL = plain CG
    const MGGeo* mg;
    double mg_omega;          // weight of the Jacobi smoothing sweeps
    // per level l: -lap at spacing 2^l delta (the negated weights of Eq. d2_1
    // times 4^-l, exact in either precision) and the Jacobi factor omega over
    // its diagonal; in the parameters, the sweeps read them as constants
    Stencil<double> mg_a64[kMGMax + 1];
    Stencil<float> mg_a32[kMGMax + 1];
    double mg_wd64[kMGMax + 1];
    float mg_wd32[kMGMax + 1];
    size_t off_zc, off_tc;    // level-0 cubes (the workspace cube's size): smoothed correction, residual
    size_t off_mgz[kMGMax + 1], off_mgt[kMGMax + 1], off_mgr[kMGMax + 1];  // levels 1..: cubes and right-hand side
    const double* pow_tab;  // [3][2 Rc + 1][8] x^e, y^e, z^e (cluster kernel; global, read-only)

    // solver
    double tol;
    int max_iter;
    int inner_max_iter;
    double inner_tol;
    int max_refine;
    double update_drop;       // reliable-update trigger of the cluster solver
    unsigned long long* phase_clk;  // [4] cycles: setup, FP64 residuals, FP32 CG, finish (cluster solver)
    int lmax;
    int n_mono;
    int warm_start;       // 1: take x0 from the cache when valid
    const double* x0_cache;   // [n_pair_cap][n_pe] previous solutions (fixed radii)
    double* x_cache_out;      // write solutions here (may alias nothing)
    const int* x0_valid;      // [n_pair] 1 when x0_cache row is this pair's previous solution

    // warm start from the previous call (cluster solver, fixed radii)
    int warm;                     // 1: look the pair up in prev_pairs and start from its cached v
    const PairRec* prev_pairs;    // previous call's pair list (i-major, j ascending)
    const int* n_prev;            // its length (device)
    const float* vprev;           // [n_prev][n_pe] previous PE potentials
    float* vcur;                  // [n_pair][n_pe] this call's PE potentials (written)
    // polynomial extrapolation (warm 3): the potentials, pair lists and pair
    // counts of the last xk calls, newest first (xv[0] = vprev)
    const float* xv[3];
    const PairRec* xp[3];
    const int* xn[3];
    int xk;

    // outputs
    double* e_pair;
    int* iters;
    int* refines;
    int* nonconv;
    int* timeouts;        // bounded device waits that ran out
    int test_wait;        // 1: thread 0 of every CTA makes one extra bounded wait run out (test of the time-out path)
    // debug
    double* dbg_b;        // if set, the RHS b of the processed pair (slot 0)
};

// Slab decomposition of the PE ball over the C CTAs of a cluster (FP32 inner
// CG kept in shared memory): CTA r owns the whole x planes x0[r] .. x0[r] +
// planes[r] - 1 and the compact PE points k0[r] .. k1[r] - 1.
constexpr int kMaxCluster = 16;
struct ClusterLayout {
    int C;
    int Syz, Sp2;        // slab box side 2 R_PE + 7 and its square
    int cap_planes;      // max planes of a slab (shared memory per CTA)
    int sy_doubles;      // doubles reserved for the plane sums before the slab
    int max_pts;         // max points of a CTA
    int x0[kMaxCluster], planes[kMaxCluster], k0[kMaxCluster], k1[kMaxCluster];  // host copy
    const int* pt_slab;  // [n_pe] slab offset | (plane within slab) << 24
    const int4* rank_info;  // device [C]: x0, planes, k0, k1 (read by the kernel)
    const int* slot_pk;     // device [C][PTS][NT]: packed slab offset of each thread slot, or -1
    const int* slot_k;      // device [C][PTS][NT]: compact PE index of each thread slot, or -1
    const int* res_list;    // device [n_pe]: per rank, rim points then interior points (first residual)
    const int* res_nrim;    // device [C]: rim points of each rank
};

// Host-built constants of the Cartesian form of the multipole expansion.
struct MultipoleConst {
    double K[1596];        // block-diagonal K_l, l = 0..6, row-major per block
    int k_off[8];          // offset of block l in K
    int mono_off[8];       // first monomial of degree l
    unsigned char mono[kNMono][3];  // (a, b, c) of each monomial
    // U_{l,c} = sum over a + b = l - c of T_abc x^a y^b: for u = l(l+1)/2 + c,
    // the terms (monomial m, a, b) and their count
    unsigned char uterm[kNU][kLmaxMax + 1][3];
    unsigned char uterm_n[kNU];
};

}  // namespace exx
