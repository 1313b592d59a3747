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
};

void build_multipole_const(MultipoleConst& mc);

// Splits the PE ball of B into C slabs of whole x planes (each >= 3 planes),
// minimising the largest point count. Fills L (without the device pointer) and
// the per-point slab offsets. Returns false if no such split exists.
bool build_cluster_layout(const HostBall& B, int C, ClusterLayout& L, std::vector<int>& pt_slab);
void build_ball(HostBall& B, int r_pe, int r_me, int Rc);

}  // namespace exx
