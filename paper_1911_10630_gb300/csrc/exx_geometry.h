// exx_geometry.h -- host-side table builders (ball geometry, multipole matrices).
#pragma once

#include <vector>

#include "exx_internal.h"

namespace exx {

struct HostBall {
    int r_pe = 0, r_me = 0, n_pe = 0, n_me = 0;
    std::vector<int> cube;          // [n_me] cube index (cube radius Rc)
    std::vector<int> off;           // [n_me] packed offsets
    std::vector<RowRec> rows_pe;    // PE rows, lexicographic
    std::vector<RowRec> rows_me;    // ME rows, lexicographic
    std::vector<int> plane_pe;      // [2 r_pe + 2]
    std::vector<int> row_of;        // [(2 r_pe + 1)^2] PE row of (ox, oy) or -1
    std::vector<int> sh_near;       // shell points with |z| <= zn of their ME row: row << 8 | (z + 128)
    std::vector<int> sh_far;        // the other shell points, same packing
};

void build_multipole_const(MultipoleConst& mc);

// Splits the PE ball of B into C slabs of whole x planes (each >= 3 planes),
// minimising the largest point count. Fills L (without the device pointer) and
// the per-point slab offsets. The slab box has 2 R_PE + 7 rows of 2 R_PE + 7
// points per plane; pitch4 pads the row pitch to a multiple of 4 (16-byte rows
// for the quad map). max_planes >= 3 caps the planes of a slab (the shared
// memory a CTA can hold). Returns false if no such split exists.
bool build_cluster_layout(const HostBall& B, int C, ClusterLayout& L, std::vector<int>& pt_slab, bool pitch4 = false,
                          int max_planes = 0);
void build_ball(HostBall& B, int r_pe, int r_me, int Rc);

// Thread-slot maps of the cluster solver for NT threads x PTS points per CTA:
// slot (j, t) of CTA r holds one point of the CTA's slab. Points are dealt so
// that the 32 lanes of every warp read 32 different shared-memory banks
// (distinct slab offsets mod 32); every stencil leg shifts all lanes by the
// same amount, so the whole stencil is conflict-free. slot_pk gets the packed
// slab offset (or -1), slot_k the compact PE index (or -1), [C][PTS][NT].
// Returns the number of warps in which two lanes share a bank.
// bank_aware = 0 keeps the natural order (slot (j, t) = point k0 + t + j NT),
// whose warps read contiguous addresses (coalesced remote loads, at most a
// two-row bank conflict).
int build_slot_maps(const ClusterLayout& L, const std::vector<int>& pt_slab, int NT, int PTS, int bank_aware,
                    std::vector<int>& slot_pk, std::vector<int>& slot_k);
// Thread map of the z-run cluster solver: every thread owns one run of at
// most ZL consecutive points of one slab row. run_pk[rank][t] = slab offset
// of the run's first point | plane << 24 (-1: idle thread); run_k[rank][t] =
// first compact PE index | length << 24. Returns the largest run count of a
// rank, or -1 if a rank has more runs than NT.
int build_run_maps(const ClusterLayout& L, const std::vector<int>& pt_slab, int NT, int ZL,
                   std::vector<int>& run_pk, std::vector<int>& run_k);
// Thread map of the quad cluster solver (a layout built with pitch4): every
// row of a slab is cut into 16-byte aligned quads of 4 consecutive z
// positions, and quad s of CTA r goes to slot (j, t) = (s / NT, s % NT), so a
// warp covers consecutive quads. quad_pk[r][j][t] = slab offset of the quad
// | valid-element mask << 20 | plane << 24; quad_k = compact PE index of the
// quad's element 0 (element i is k + i when mask bit i is set). Idle slots
// point at a quad that lies outside the ball in every plane, with mask 0.
// bank_aware (only for the layout with halo planes, whose idle quads sit in
// rows 0..2 of plane 0) deals the quads so that every 8 consecutive slots hold
// quads of 8 distinct bank groups ((offset / 4) mod 8), which makes every
// 16-byte stencil load conflict-free. Returns the largest quad count of a
// rank, or -1 if the quads do not fit Q x NT slots or the slab offsets do not
// fit 20 bits.
int build_quad_maps(const ClusterLayout& L, const std::vector<int>& pt_slab, int NT, int Q, std::vector<int>& quad_pk,
                    std::vector<int>& quad_k, int bank_aware = 0);
// Order of the first FP64 residual of a pair, when v is still zero on the PE
// ball: per rank, its points whose stencil reaches the shell (|o| > R_PE - 3,
// the rim) first, then the interior ones, where lap v = 0 and r = 4 pi rho.
// list[k0 .. k1) holds rank r's compact indices, nrim[r] its rim count.
void build_residual_order(const HostBall& B, const ClusterLayout& L, std::vector<int>& list, std::vector<int>& nrim);

// The coarse levels of the multigrid preconditioner for a PE ball of radius
// r_pe: R_l = ceil(R_{l-1} / 2) while R_{l-1} > 3; for each level its radius,
// points (lexicographic), cube side 2 R + 7 and cube indices, packed offsets;
// minv the inverse of the coarsest level's operator -lap (Eq. d2_1 at spacing
// 2^L delta_a, zero outside the ball), row-major. Returns false on failure.
struct HostMGLevel {
    int R = 0, side = 0;
    std::vector<int> cube, off;
};
bool build_mg_levels(int r_pe, const double delta[3], std::vector<HostMGLevel>& levels, std::vector<double>& minv);

}  // namespace exx
