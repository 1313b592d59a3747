// exx_geometry.cpp -- host-built tables: ball geometry (Algorithm 2) and the
// Cartesian form of the multipole expansion (Eqs. me, mepole).
//
// Multipoles in Cartesian form. The expansion of Eq. me, summed over m with
// the addition theorem of spherical harmonics, is the Legendre series
//     v(r) = sum_l sum_q rho_q dV (r r_q)^l P_l(cos g) / r^(2l+1),
// and (r r_q)^l P_l(cos g) = sum_k c_lk (r . r_q)^(l-2k) (r^2)^k (r_q^2)^k with
// c_lk = (-1)^k (2l-2k)! / (2^l k! (l-k)! (l-2k)!). Expanding the powers with
// multinomial coefficients gives, for each degree l, a symmetric matrix K_l
// over the degree-l monomials with
//     P_l(r) = sum_alpha T_alpha r^alpha,   T = K_l M,
//     M_beta = sum_q rho_q dV r_q^beta      (Cartesian moments of degree l),
// so the device never evaluates a spherical harmonic: it forms the 84
// Cartesian moments of degree <= 6 and the polynomial P_l on the shell.
#include "exx_geometry.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

namespace exx {

static double fact(int n) {
    double f = 1.0;
    for (int k = 2; k <= n; ++k) f *= k;
    return f;
}

static double multinom(int n, int a, int b, int c) { return fact(n) / (fact(a) * fact(b) * fact(c)); }

void build_multipole_const(MultipoleConst& mc) {
    std::memset(&mc, 0, sizeof(mc));
    int m = 0;
    int idx[kLmaxMax + 1][kLmaxMax + 1][kLmaxMax + 1];
    for (int l = 0; l <= kLmaxMax; ++l) {
        mc.mono_off[l] = m;
        for (int a = l; a >= 0; --a)
            for (int b = l - a; b >= 0; --b) {
                const int c = l - a - b;
                mc.mono[m][0] = (unsigned char)a;
                mc.mono[m][1] = (unsigned char)b;
                mc.mono[m][2] = (unsigned char)c;
                idx[a][b][c] = m - mc.mono_off[l];
                ++m;
            }
    }
    mc.mono_off[kLmaxMax + 1] = m;
    for (int l = 0; l <= kLmaxMax; ++l)
        for (int c = 0; c <= l; ++c) {
            const int u = l * (l + 1) / 2 + c;
            int n = 0;
            for (int a = l - c; a >= 0; --a) {
                const int b = l - c - a;
                mc.uterm[u][n][0] = (unsigned char)(mc.mono_off[l] + idx[a][b][c]);
                mc.uterm[u][n][1] = (unsigned char)a;
                mc.uterm[u][n][2] = (unsigned char)b;
                ++n;
            }
            mc.uterm_n[u] = (unsigned char)n;
        }
    int koff = 0;
    for (int l = 0; l <= kLmaxMax; ++l) {
        const int nl = (l + 1) * (l + 2) / 2;
        mc.k_off[l] = koff;
        double* K = mc.K + koff;
        for (int k = 0; 2 * k <= l; ++k) {
            const double clk = ((k & 1) ? -1.0 : 1.0) * fact(2 * l - 2 * k) /
                               (std::pow(2.0, l) * fact(k) * fact(l - k) * fact(l - 2 * k));
            const int md = l - 2 * k;
            for (int g0 = 0; g0 <= md; ++g0)
                for (int g1 = 0; g0 + g1 <= md; ++g1) {
                    const int g2 = md - g0 - g1;
                    const double mg = multinom(md, g0, g1, g2);
                    for (int d0 = 0; d0 <= k; ++d0)
                        for (int d1 = 0; d0 + d1 <= k; ++d1) {
                            const int d2 = k - d0 - d1;
                            const double mdl = multinom(k, d0, d1, d2);
                            for (int e0 = 0; e0 <= k; ++e0)
                                for (int e1 = 0; e0 + e1 <= k; ++e1) {
                                    const int e2 = k - e0 - e1;
                                    const double me = multinom(k, e0, e1, e2);
                                    const int ra = idx[g0 + 2 * d0][g1 + 2 * d1][g2 + 2 * d2];
                                    const int cb = idx[g0 + 2 * e0][g1 + 2 * e1][g2 + 2 * e2];
                                    K[ra * nl + cb] += clk * mg * mdl * me;
                                }
                        }
                }
        }
        koff += nl * nl;
    }
    mc.k_off[kLmaxMax + 1] = koff;
}

static int isqrt_floor(long v) {
    if (v < 0) return -1;
    long r = (long)std::sqrt((double)v);
    while (r * r > v) --r;
    while ((r + 1) * (r + 1) <= v) ++r;
    return (int)r;
}

static int pack_off(int x, int y, int z) { return (x + 128) | ((y + 128) << 8) | ((z + 128) << 16); }

void build_ball(HostBall& B, int r_pe, int r_me, int Rc) {
    const int S = 2 * Rc + 1;
    const long rpe2 = (long)r_pe * r_pe, rme2 = (long)r_me * r_me;
    B.r_pe = r_pe;
    B.r_me = r_me;
    B.cube.clear();
    B.off.clear();
    B.rows_pe.clear();
    B.rows_me.clear();
    B.row_of.clear();
    B.sh_near.clear();
    B.sh_far.clear();
    B.plane_pe.assign(2 * r_pe + 2, 0);
    auto cube = [&](int x, int y, int z) { return ((x + Rc) * S + (y + Rc)) * S + (z + Rc); };
    // PE ball, lexicographic (Algorithm 2, first list)
    for (int x = -r_pe; x <= r_pe; ++x) {
        B.plane_pe[x + r_pe] = (int)B.rows_pe.size();
        for (int y = -r_pe; y <= r_pe; ++y) {
            const long s2 = (long)x * x + (long)y * y;
            if (s2 > rpe2) continue;
            const int zpe = isqrt_floor(rpe2 - s2);
            RowRec R;
            R.ox = (short)x;
            R.oy = (short)y;
            R.zpe = (short)zpe;
            R.zme = (short)isqrt_floor(rme2 - s2);
            R.pe_start = (int)B.cube.size();
            R.zn = -1;
            B.rows_pe.push_back(R);
            for (int z = -zpe; z <= zpe; ++z) {
                B.cube.push_back(cube(x, y, z));
                B.off.push_back(pack_off(x, y, z));
            }
        }
    }
    B.plane_pe[2 * r_pe + 1] = (int)B.rows_pe.size();
    B.n_pe = (int)B.cube.size();
    B.row_of.assign((size_t)(2 * r_pe + 1) * (2 * r_pe + 1), -1);
    for (int rr = 0; rr < (int)B.rows_pe.size(); ++rr)
        B.row_of[(size_t)(B.rows_pe[rr].ox + r_pe) * (2 * r_pe + 1) + (B.rows_pe[rr].oy + r_pe)] = rr;
    // shell, lexicographic (Algorithm 2, second list); rows of the ME ball
    int pe_row = 0;
    for (int x = -r_me; x <= r_me; ++x)
        for (int y = -r_me; y <= r_me; ++y) {
            const long s2 = (long)x * x + (long)y * y;
            if (s2 > rme2) continue;
            RowRec R;
            R.ox = (short)x;
            R.oy = (short)y;
            R.zme = (short)isqrt_floor(rme2 - s2);
            R.zpe = (short)(s2 <= rpe2 ? isqrt_floor(rpe2 - s2) : -1);
            R.pe_start = R.zpe >= 0 ? B.rows_pe[pe_row++].pe_start : -1;
            // boundary layer: shell points (x, y, z) with a PE point within three
            // steps along an axis: |z| <= zpe + 3 of the row itself, or |z| <= zpe
            // of a row (x +- q, y) or (x, y +- q), q <= 3
            int zn = R.zpe >= 0 ? R.zpe + 3 : -1;
            for (int q = 1; q <= 3; ++q) {
                const int nb[4][2] = {{x + q, y}, {x - q, y}, {x, y + q}, {x, y - q}};
                for (int t = 0; t < 4; ++t) {
                    const long n2 = (long)nb[t][0] * nb[t][0] + (long)nb[t][1] * nb[t][1];
                    if (n2 <= rpe2) zn = std::max(zn, isqrt_floor(rpe2 - n2));
                }
            }
            R.zn = zn;
            const int row = (int)B.rows_me.size();
            B.rows_me.push_back(R);
            for (int z = -R.zme; z <= R.zme; ++z) {
                if (z >= -R.zpe && z <= R.zpe) continue;
                B.cube.push_back(cube(x, y, z));
                B.off.push_back(pack_off(x, y, z));
                (std::abs(z) <= zn ? B.sh_near : B.sh_far).push_back((row << 8) | (z + 128));
            }
        }
    B.n_me = (int)B.cube.size();
}

bool build_cluster_layout(const HostBall& B, int C, ClusterLayout& L, std::vector<int>& pt_slab, bool pitch4,
                          int max_planes) {
    const int R = B.r_pe, P = 2 * R + 1;
    if (C < 1 || C > kMaxCluster || P < 3 * C) return false;
    if (max_planes < 3) max_planes = P;
    std::vector<long> n(P, 0), cum(P + 1, 0);
    for (const RowRec& row : B.rows_pe) n[row.ox + R] += 2 * row.zpe + 1;
    for (int i = 0; i < P; ++i) cum[i + 1] = cum[i] + n[i];
    // f[r][i]: smallest max load of the first i planes in r slabs of >= 3 planes
    const long INF = 1L << 60;
    std::vector<std::vector<long>> f(C + 1, std::vector<long>(P + 1, INF));
    std::vector<std::vector<int>> arg(C + 1, std::vector<int>(P + 1, -1));
    f[0][0] = 0;
    for (int r = 1; r <= C; ++r)
        for (int i = 3 * r; i <= P; ++i)
            for (int j = std::max(3 * (r - 1), i - max_planes); j <= i - 3; ++j) {
                if (f[r - 1][j] >= INF) continue;
                const long v = std::max(f[r - 1][j], cum[i] - cum[j]);
                if (v < f[r][i]) {
                    f[r][i] = v;
                    arg[r][i] = j;
                }
            }
    if (f[C][P] >= INF) return false;
    std::vector<int> bounds(C + 1);
    bounds[C] = P;
    for (int r = C; r >= 1; --r) bounds[r - 1] = arg[r][bounds[r]];
    std::memset(&L, 0, sizeof(L));
    L.C = C;
    L.Syz = pitch4 ? (2 * R + 7 + 3) & ~3 : 2 * R + 7;  // row pitch (z)
    L.Sp2 = (2 * R + 7) * L.Syz;                         // plane pitch
    L.sy_doubles = ((2 * R + 1) * 28 + 1) & ~1;
    int cap = 0, maxp = 0;
    for (int r = 0; r < C; ++r) {
        L.x0[r] = bounds[r] - R;
        L.planes[r] = bounds[r + 1] - bounds[r];
        L.k0[r] = (int)cum[bounds[r]];
        L.k1[r] = (int)cum[bounds[r + 1]];
        cap = std::max(cap, L.planes[r]);
        maxp = std::max(maxp, L.k1[r] - L.k0[r]);
    }
    L.cap_planes = cap;
    L.max_pts = maxp;
    if ((long)cap * L.Sp2 >= (1L << 24)) return false;
    pt_slab.assign(B.n_pe, 0);
    int r = 0;
    for (int k = 0; k < B.n_pe; ++k) {
        while (k >= L.k1[r]) ++r;
        const int packed = B.off[k];
        const int ox = (packed & 0xff) - 128, oy = ((packed >> 8) & 0xff) - 128, oz = ((packed >> 16) & 0xff) - 128;
        const int xl = ox - L.x0[r];
        pt_slab[k] = (xl << 24) | (xl * L.Sp2 + (oy + R + 3) * L.Syz + (oz + R + 3));
    }
    return true;
}

int build_slot_maps(const ClusterLayout& L, const std::vector<int>& pt_slab, int NT, int PTS, int bank_aware,
                    std::vector<int>& slot_pk, std::vector<int>& slot_k) {
    const int per = NT * PTS, warps_per_j = NT / 32, n_ws = PTS * warps_per_j;
    slot_pk.assign((size_t)L.C * per, -1);
    slot_k.assign((size_t)L.C * per, -1);
    if (!bank_aware) {
        for (int r = 0; r < L.C; ++r) {
            if (L.k1[r] - L.k0[r] > per) return -1;
            for (int k = L.k0[r]; k < L.k1[r]; ++k) {
                const int s = k - L.k0[r];
                slot_pk[(size_t)r * per + s] = pt_slab[k];
                slot_k[(size_t)r * per + s] = k;
            }
        }
        return 0;
    }
    int conflicted = 0;
    for (int r = 0; r < L.C; ++r) {
        int ws = 0;  // next warp slot: j = ws / warps_per_j, warp = ws % warps_per_j
        auto place = [&](int slot_ws, int lane, int k) {
            const int j = slot_ws / warps_per_j, t = (slot_ws % warps_per_j) * 32 + lane;
            slot_pk[(size_t)r * per + (size_t)j * NT + t] = pt_slab[k];
            slot_k[(size_t)r * per + (size_t)j * NT + t] = k;
        };
        // 1) plane by plane: whole warps of one plane, one point per bank, so the
        //    lanes of a warp agree on which x legs leave the slab
        std::vector<int> pool;
        int k = L.k0[r];
        while (k < L.k1[r]) {
            const int xl = pt_slab[k] >> 24;
            std::vector<std::vector<int>> bucket(32);
            while (k < L.k1[r] && (pt_slab[k] >> 24) == xl) {
                bucket[(pt_slab[k] & 0xffffff) & 31].push_back(k);
                ++k;
            }
            std::vector<size_t> head(32, 0);
            for (;;) {
                bool full = true;
                for (int b = 0; b < 32; ++b) full = full && head[b] < bucket[b].size();
                if (!full || ws >= n_ws) break;
                for (int b = 0; b < 32; ++b) place(ws, b, bucket[b][head[b]++]);
                ++ws;
            }
            for (int b = 0; b < 32; ++b)
                for (size_t h = head[b]; h < bucket[b].size(); ++h) pool.push_back(bucket[b][h]);
        }
        // 2) the per-plane remainders: distinct banks within a warp where possible
        std::vector<std::vector<int>> bucket(32);
        for (int q : pool) bucket[(pt_slab[q] & 0xffffff) & 31].push_back(q);
        std::vector<size_t> head(32, 0);
        size_t left = pool.size();
        while (left > 0 && ws < n_ws) {
            int lane = 0;
            for (int b = 0; b < 32 && left > 0; ++b)
                if (head[b] < bucket[b].size()) {
                    place(ws, lane++, bucket[b][head[b]++]);
                    --left;
                }
            ++ws;
        }
        // 3) anything still left shares banks in free slots
        for (int s2 = 0; s2 < n_ws && left > 0; ++s2)
            for (int lane = 0; lane < 32 && left > 0; ++lane) {
                const int j = s2 / warps_per_j, t = (s2 % warps_per_j) * 32 + lane;
                if (slot_k[(size_t)r * per + (size_t)j * NT + t] >= 0) continue;
                for (int b = 0; b < 32; ++b)
                    if (head[b] < bucket[b].size()) {
                        place(s2, lane, bucket[b][head[b]++]);
                        --left;
                        ++conflicted;
                        break;
                    }
            }
        if (left > 0) return -1;
    }
    return conflicted;
}

int build_run_maps(const ClusterLayout& L, const std::vector<int>& pt_slab, int NT, int ZL,
                   std::vector<int>& run_pk, std::vector<int>& run_k) {
    run_pk.assign((size_t)L.C * NT, -1);
    run_k.assign((size_t)L.C * NT, 0);
    int max_runs = 0;
    struct Run {
        int pk, k, len;
    };
    for (int r = 0; r < L.C; ++r) {
        // rows of the slab: maximal stretches of consecutive points whose slab
        // offsets are consecutive (same plane and row, z ascending)
        std::vector<Run> runs;
        int hist[32] = {0};  // runs starting in each bank
        int k = L.k0[r];
        while (k < L.k1[r]) {
            int e = k + 1;
            while (e < L.k1[r] && (pt_slab[e] & 0xffffff) == (pt_slab[e - 1] & 0xffffff) + 1 &&
                   (pt_slab[e] >> 24) == (pt_slab[k] >> 24))
                ++e;
            // the row [k, e) in n = ceil(len / ZL) pieces of at most ZL points;
            // each later piece starts where its bank is least used so far
            // (near the even split on ties), so warps can draw distinct banks
            const int len = e - k, n = (len + ZL - 1) / ZL;
            int at = k;
            for (int q = 0; q < n; ++q) {
                int next = e;
                if (q + 1 < n) {
                    const int lo = std::max(at + 1, e - (n - q - 1) * ZL), hi = std::min(at + ZL, e - (n - q - 1));
                    const int even = k + (int)((long)len * (q + 1) / n);
                    next = -1;
                    for (int c = lo; c <= hi; ++c) {
                        const int b = (pt_slab[c] & 0xffffff) & 31;
                        if (next < 0 || hist[b] < hist[(pt_slab[next] & 0xffffff) & 31] ||
                            (hist[b] == hist[(pt_slab[next] & 0xffffff) & 31] && std::abs(c - even) < std::abs(next - even)))
                            next = c;
                    }
                }
                runs.push_back({pt_slab[at], at, next - at});
                ++hist[(pt_slab[at] & 0xffffff) & 31];
                at = next;
            }
            k = e;
        }
        if ((int)runs.size() > NT) return -1;
        max_runs = std::max(max_runs, (int)runs.size());
        // lanes: each warp takes runs whose first points lie in distinct banks
        // (then every load of the warp hits 32 banks), drawing from the
        // fullest banks first so that the banks run out evenly
        std::vector<std::vector<int>> bucket(32);
        for (size_t q = 0; q < runs.size(); ++q) bucket[(runs[q].pk & 0xffffff) & 31].push_back((int)q);
        std::vector<int> lane_run;
        size_t left = runs.size();
        while (left > 0) {
            std::vector<int> order(32);
            for (int b = 0; b < 32; ++b) order[b] = b;
            std::stable_sort(order.begin(), order.end(),
                             [&](int a, int b) { return bucket[a].size() > bucket[b].size(); });
            int got = 0;
            for (int pass = 0; pass < 32 && got < 32 && left > 0; ++pass)
                for (int q = 0; q < 32 && got < 32 && left > 0; ++q) {
                    std::vector<int>& bk = bucket[order[q]];
                    if ((int)bk.size() <= pass) continue;
                    lane_run.push_back(bk.back());
                    bk.pop_back();
                    ++got;
                    --left;
                }
        }
        for (size_t t = 0; t < lane_run.size(); ++t) {
            const Run& R = runs[lane_run[t]];
            run_pk[(size_t)r * NT + t] = R.pk;
            run_k[(size_t)r * NT + t] = (R.len << 24) | R.k;
        }
    }
    return max_runs;
}


int build_quad_maps(const ClusterLayout& L, const std::vector<int>& pt_slab, int NT, int Q, std::vector<int>& quad_pk,
                    std::vector<int>& quad_k, int bank_aware) {
    const int per = NT * Q;
    // idle slots: the quad at row 3, z 0..3 of plane 0 (outside the ball in
    // every plane, so it stays zero), with no valid element
    const int idle = 3 * L.Syz;
    quad_pk.assign((size_t)L.C * per, idle);
    quad_k.assign((size_t)L.C * per, 0);
    if ((L.Syz & 3) || (long)L.cap_planes * L.Sp2 >= (1L << 20) || (bank_aware && (per & 7))) return -1;
    // bank-aware idle quads: one per bank group (offset / 4) mod 8 from rows
    // 0..2 of plane 0, which lie outside the ball in every plane
    int idle_of[8];
    for (int c = 0; c < 8; ++c) idle_of[c] = -1;
    for (int row = 0; row < 3; ++row)
        for (int q = 0; 4 * q + 3 < L.Syz; ++q) {
            const int off = row * L.Syz + 4 * q;
            if (idle_of[(off >> 2) & 7] < 0) idle_of[(off >> 2) & 7] = off;
        }
    int max_quads = 0;
    for (int r = 0; r < L.C; ++r) {
        std::vector<int> qpk, qk;  // the rank's quads, row by row
        int k = L.k0[r];
        while (k < L.k1[r]) {
            // one row of the slab: consecutive offsets within one plane
            int e = k + 1;
            while (e < L.k1[r] && (pt_slab[e] & 0xffffff) == (pt_slab[e - 1] & 0xffffff) + 1 &&
                   (pt_slab[e] >> 24) == (pt_slab[k] >> 24))
                ++e;
            const int off0 = pt_slab[k] & 0xffffff, xl = pt_slab[k] >> 24;
            const int z0 = off0 % L.Syz, z1 = z0 + (e - k) - 1;  // z positions of the row's ends in the box
            for (int qz = z0 & ~3; qz <= z1; qz += 4) {
                int mask = 0;
                for (int i = 0; i < 4; ++i)
                    if (qz + i >= z0 && qz + i <= z1) mask |= 1 << i;
                qpk.push_back((off0 - z0 + qz) | (mask << 20) | (xl << 24));
                qk.push_back(k + (qz - z0));
            }
            k = e;
        }
        const int nq = (int)qpk.size();
        int* dpk = quad_pk.data() + (size_t)r * per;
        int* dk = quad_k.data() + (size_t)r * per;
        if (!bank_aware) {
            if (nq > per) return -1;
            for (int s = 0; s < nq; ++s) {
                dpk[s] = qpk[s];
                dk[s] = qk[s];
            }
        } else {
            // every 8 consecutive slots (the lanes of one phase of a 16-byte
            // shared-memory access) take quads of 8 distinct bank groups, so
            // every stencil leg, shifted alike for all lanes, is conflict-free
            for (int c = 0; c < 8; ++c)
                if (idle_of[c] < 0) return -1;
            std::vector<std::vector<int>> bucket(8);
            for (int q = 0; q < nq; ++q) bucket[((qpk[q] & 0xfffff) >> 2) & 7].push_back(q);
            size_t groups = 0;
            for (int c = 0; c < 8; ++c) groups = std::max(groups, bucket[c].size());
            if ((long)groups * 8 > per) return -1;
            for (int s = 0; s < per; ++s) dpk[s] = idle_of[s & 7];
            for (int c = 0; c < 8; ++c)
                for (size_t g = 0; g < bucket[c].size(); ++g) {
                    dpk[8 * g + c] = qpk[bucket[c][g]];
                    dk[8 * g + c] = qk[bucket[c][g]];
                }
        }
        max_quads = std::max(max_quads, nq);
    }
    return max_quads;
}


void build_residual_order(const HostBall& B, const ClusterLayout& L, std::vector<int>& list, std::vector<int>& nrim) {
    const long in2 = (long)(B.r_pe - 3) * (B.r_pe - 3);
    list.assign(B.n_pe, 0);
    nrim.assign(L.C, 0);
    for (int r = 0; r < L.C; ++r) {
        int at = L.k0[r];
        for (int pass = 0; pass < 2; ++pass)
            for (int k = L.k0[r]; k < L.k1[r]; ++k) {
                const int p = B.off[k];
                const long x = (p & 0xff) - 128, y = ((p >> 8) & 0xff) - 128, z = ((p >> 16) & 0xff) - 128;
                const bool rim = B.r_pe < 3 || x * x + y * y + z * z > in2;
                if (rim != (pass == 0)) continue;
                list[at++] = k;
                if (rim) ++nrim[r];
            }
    }
}

bool build_mg_levels(int r_pe, const double delta[3], std::vector<HostMGLevel>& levels, std::vector<double>& minv) {
    levels.clear();
    minv.clear();
    int R = r_pe;
    int l = 0;
    while (R > 3) {
        R = (R + 1) / 2;
        ++l;
        if (l > kMGMax) return false;
        HostMGLevel H;
        H.R = R;
        H.side = 2 * R + 7;
        const int c = R + 3;
        for (int x = -R; x <= R; ++x)
            for (int y = -R; y <= R; ++y)
                for (int z = -R; z <= R; ++z) {
                    if (x * x + y * y + z * z > R * R) continue;
                    H.cube.push_back(((x + c) * H.side + (y + c)) * H.side + (z + c));
                    H.off.push_back((x + 128) | ((y + 128) << 8) | ((z + 128) << 16));
                }
        levels.push_back(H);
    }
    if (levels.empty()) return false;
    // the coarsest operator, dense: A = -lap at spacing 2^L delta (Eq. d2_1, n = 3)
    const HostMGLevel& C = levels.back();
    const int n = (int)C.off.size();
    const double Wt[4] = {-49.0 / 18.0, 3.0 / 2.0, -3.0 / 20.0, 1.0 / 90.0};
    double ih2[3];
    for (int a = 0; a < 3; ++a) {
        const double h = std::ldexp(delta[a], l);
        ih2[a] = 1.0 / (h * h);
    }
    std::vector<int> pos((size_t)C.side * C.side * C.side, -1);
    for (int k = 0; k < n; ++k) pos[C.cube[k]] = k;
    std::vector<double> A((size_t)n * n, 0.0);
    const int st[3] = {C.side * C.side, C.side, 1};
    for (int k = 0; k < n; ++k) {
        A[(size_t)k * n + k] = -Wt[0] * (ih2[0] + ih2[1] + ih2[2]);
        for (int a = 0; a < 3; ++a)
            for (int q = 1; q <= 3; ++q)
                for (int sgn = -1; sgn <= 1; sgn += 2) {
                    const int j = pos[C.cube[k] + sgn * q * st[a]];
                    if (j >= 0) A[(size_t)k * n + j] -= Wt[q] * ih2[a];
                }
    }
    // Cholesky A = U^T U (A is symmetric positive definite on the ball), then
    // the inverse column by column from the two triangular solves
    std::vector<double> U((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) {
        double d = A[(size_t)i * n + i];
        for (int k = 0; k < i; ++k) d -= U[(size_t)k * n + i] * U[(size_t)k * n + i];
        if (!(d > 0.0)) return false;
        d = std::sqrt(d);
        U[(size_t)i * n + i] = d;
        for (int j = i + 1; j < n; ++j) {
            double t = A[(size_t)i * n + j];
            for (int k = 0; k < i; ++k) t -= U[(size_t)k * n + i] * U[(size_t)k * n + j];
            U[(size_t)i * n + j] = t / d;
        }
    }
    minv.assign((size_t)n * n, 0.0);
    std::vector<double> y(n);
    for (int col = 0; col < n; ++col) {
        for (int i = 0; i < n; ++i) {  // U^T y = e_col
            double t = i == col ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) t -= U[(size_t)k * n + i] * y[k];
            y[i] = t / U[(size_t)i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {  // U x = y
            double t = y[i];
            for (int k = i + 1; k < n; ++k) t -= U[(size_t)i * n + k] * minv[(size_t)k * n + col];
            minv[(size_t)i * n + col] = t / U[(size_t)i * n + i];
        }
    }
    return true;
}

}  // namespace exx
