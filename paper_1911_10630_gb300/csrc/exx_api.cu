// exx_api.cu -- the C ABI (include/exx.h): context, validation, workspace,
// launch sequence and CUDA-graph replay.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/exx.h"
#include "exx_geometry.h"
#include "exx_internal.h"
#include "exx_unet.cuh"

namespace exx {
cudaError_t launch_pair_list(int n, const double* centers, const double L[3], const double delta[3], const int N[3],
                             double r_pair, int r_pe, int r_me, int* counts, int* offsets, int* n_pair, int* queue,
                             PairRec* pairs, cudaStream_t st, const double* alphas, double ln_inv_eps,
                             double delta_max, int r_min, int ns_pe = 0, int ns_me = 0, int* bad = nullptr);
cudaError_t launch_radii_sort(const PairRec* pairs, const int* n_pair, int* hist, int n_geo, int* order, int num_sms,
                              cudaStream_t st, int* classes = nullptr);
cudaError_t cluster_set_smem(int variant, size_t smem);
cudaError_t launch_zero(double* p, long long n, int num_sms, cudaStream_t st);
cudaError_t launch_box_clip(const PairRec* pairs, const int* n_pair, const int* box_org, const int bdim[3],
                            const int N[3], int* clipped, int num_sms, cudaStream_t st);
cudaError_t launch_dfix_convert(double* p, long long n, double inv, int num_sms, cudaStream_t st);
cudaError_t launch_copy16(const void* src, void* dst, long long n2, int num_sms, cudaStream_t st);
cudaError_t launch_exx_reduce(const PairRec* pairs, const int* n_pair, const double* e_pair, double* out,
                              cudaStream_t st, int* bad = nullptr);
cudaError_t set_multipole_const_solve(const MultipoleConst& mc);
cudaError_t set_multipole_const_cluster(const MultipoleConst& mc);
size_t pair_kernel_smem(int Rc, int r_pe_max);
cudaError_t launch_pair_kernel(const SolveParams& P, int threads, bool mixed, int grid, size_t smem, cudaStream_t st);
cudaError_t pair_kernel_occupancy(int threads, bool mixed, bool mg, bool one_ball, size_t smem, int* blocks_per_sm);
cudaError_t launch_mg_apply(const SolveParams& P, int geo, const double* r, double* z, cudaStream_t st);  // exx_debug.cu
cudaError_t launch_debug_readback(const SolveParams& P, const PairRec& pr, double* rho_me, double* v_me,
                                  cudaStream_t st);
cudaError_t launch_apply(const SolveParams& P, const double* p, double* ap, cudaStream_t st);
size_t cluster_kernel_smem(int Rc, const ClusterLayout& CL, int variant);
int cluster_variant(int C, int max_pts, int threads, int syz, bool iso);
cudaError_t cluster_prepare(int variant, size_t smem, int* max_clusters);
cudaError_t launch_cluster_kernel(int variant, const SolveParams& P, const ClusterLayout& CL, int n_clusters,
                                  size_t smem, cudaStream_t st);
int cluster_variant_threads(int variant);
int cluster_variant_pts(int variant);
int cluster_variant_mode(int variant);
int cluster_variant_iso(int variant);
int cluster_variant_syz(int variant);
int cluster_variant_count();
int cluster_variant_size(int variant);
bool mg_cluster_size_ok(int C);
cudaError_t mg_cluster_prepare(int C, int minb, int* max_clusters);
cudaError_t launch_cluster_mg(int C, int minb, const SolveParams& P, int n_clusters, cudaStream_t st);
}  // namespace exx

using namespace exx;

struct exx_ctx {
    // parameters
    double cell[3];
    int grid[3];
    double delta[3];
    double dV;
    double r_pair;
    int r_pe, r_me, lmax;
    double tol;
    exx_options opt;
    long long ngrid;

    // device
    int device = 0;
    int num_sms = 0;

    // geometry: one ball per radius (fixed radii: one; per-pair radii: r_min .. r_pe)
    HostBall hb;                  // the largest ball (sizes the workspace)
    std::vector<HostBall> balls;  // balls[geo], R_PE = r_min + geo
    int r_min = 0, n_geo = 1;
    int ns_pe = 0, ns_me = 0;     // radii_mode 2: non-self radii (geometry 0; self pairs use geometry 1)
    double ln_inv_eps = 0.0, delta_max = 0.0;
    void* geo_mem = nullptr;  // device tables
    BallGeo* d_geos = nullptr;
    void* mg_mem = nullptr;   // multigrid hierarchies (preconditioner 1)
    MGGeo* d_mg = nullptr;
    BallGeo geo_host;

    // workspace
    char* ws = nullptr;
    size_t slot_bytes = 0;
    int n_slots = 0;
    int threads = 512;
    size_t smem = 0;
    SolveParams P;

    // cluster solver (precision 1): one thread-block cluster per pair. Every
    // launch shape that fits is a candidate; the autotuner times them on the
    // first call and keeps the fastest.
    struct ClusterCand {
        int C = 0, variant = -1, lane_map = 0, n_clusters = 0;
        size_t smem = 0;
        ClusterLayout L;
        double pairs_per_s = 0.0;
    };
    bool use_cluster = false;
    std::vector<ClusterCand> cands;
    int cand = -1;  // candidate in use
    bool tuned = false;
    double tune_ms = 0.0;
    int cl_variant = -1;
    int n_clusters = 0;
    ClusterLayout CL;
    std::vector<void*> cl_mem;  // device tables of all candidates
    // per-pair radii on the cluster solver: one launch per radius class
    // (geometry), largest first, each with the launch shape that fits it
    // (kind 2: cluster kernel candidate; kind 1: the one-CTA pair kernel)
    struct RadiusClass {
        int geo = 0, kind = 1;
        ClusterCand cand;
    };
    bool per_class = false;
    std::vector<RadiusClass> classes;
    // the multigrid-preconditioned CG on clusters (preconditioner 1, precision 1):
    // mg_C CTAs per pair, mg_minb CTAs per SM, up to mg_clusters resident clusters
    int mg_C = 0, mg_minb = 2, mg_clusters = 0;
    // exx_compute_async: the last call's counters are read (after waiting for
    // the call) by the next exx_get_stats; box of that call
    bool stats_pending = false;
    bool pending_box = false;
    // the classes alternate between the context stream (lane 0) and aux
    // (lane 1), forked and joined inside the graph, so that one class's tail
    // overlaps the next class's work; each lane has its own workspace slots
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int lane_slots[2] = {0, 0};
    int* d_class = nullptr;  // [2 n_geo] start and length of each class in the order, [n_geo] work counters
    double* d_pow = nullptr;
    unsigned long long* d_phase = nullptr;  // [4] phase cycles of the cluster solver
    int clock_khz = 0;

    // pair buffers
    int cap_n = 0;
    long long cap_pairs = 0;
    int* d_counts = nullptr;
    int* d_offsets = nullptr;
    PairRec* d_pairs = nullptr;
    double* d_epair = nullptr;
    int* d_iters = nullptr;
    int* d_refines = nullptr;
    int* d_order = nullptr;  // largest-first processing order (per-pair radii)
    int* d_hist = nullptr;
    int* d_scalars = nullptr;  // [0] n_pair, [1] queue, [2] nonconv
    double* d_exx = nullptr;
    double* h_exx = nullptr;   // pinned

    // warm start (previous call's potentials)
    PairRec* d_prev_pairs = nullptr;
    long long prev_cap = 0;
    float* d_vcache[2] = {nullptr, nullptr};
    // warm 3: the potentials and pair lists of the two calls before the previous one
    float* hv[2] = {nullptr, nullptr};
    PairRec* hp[2] = {nullptr, nullptr};
    int hk = 0;  // valid history levels beyond the previous call (0..2)
    long long hv_pairs = 0, hp_cap = 0;  // capacities of the history buffers
    long long vcache_pairs = 0;
    int parity = 0;
    bool have_prev = false;

    // learned warm start (warm_start 2): the U-Net and its per-pair guesses
    exx::unet::Net* gnet = nullptr;
    float* d_guess = nullptr;   // [guess_cap][n_pe] FP32 guesses, list order
    long long guess_cap = 0;
    float* d_gin = nullptr;     // [Bmax][S^3][2] network input
    float* d_gscale = nullptr;  // [Bmax] per-pair density scale
    cudaEvent_t ev_g[2] = {nullptr, nullptr};
    double guess_ms = 0.0;

    // host-buffer path
    double* d_orb = nullptr;
    double* d_dxx = nullptr;
    double* d_cent = nullptr;
    double* d_alpha = nullptr;
    size_t host_cap_bytes = 0;
    int host_cap_n = 0;

    // test of the time-out path: calls left that inject one run-out wait, and
    // whether the current call does
    int inject_left = 0;
    int inject_now = 0;
    int g_inject = -1;  // injection state the cached graph was captured with

    // the current call's orbital storage: full grids (cur_box NULL) or
    // compact boxes (exx_compute_boxes)
    const int* cur_box = nullptr;
    int cur_bdim[3] = {0, 0, 0};
    long long cur_ostride = 0;
    int g_bdim[3] = {0, 0, 0};  // box dimensions the cached graph was captured with

    // graph cache
    cudaGraphExec_t gexec = nullptr;
    const void* g_key[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int g_n = -1;
    cudaStream_t g_stream = nullptr;

    // internal stream (graph capture is not allowed on the legacy stream)
    cudaStream_t work = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;

    // timing
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool timed = false;

    // last call
    int last_n = 0;
    const double* last_orb = nullptr;
    exx_stats stats;
    std::string err;
};

static thread_local std::string g_init_err;

namespace exx {
// Error text for entry points without a context (read by exx_last_error(NULL)).
void set_global_error(const std::string& msg) { g_init_err = msg; }
}  // namespace exx

static exx_status fail(exx_ctx* c, exx_status s, const std::string& msg) {
    if (c) c->err = msg;
    else g_init_err = msg;
    return s;
}

static exx_status cuda_fail(exx_ctx* c, cudaError_t e, const char* where) {
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%s: %s (%s)", where, cudaGetErrorString(e), cudaGetErrorName(e));
    return fail(c, e == cudaErrorMemoryAllocation ? EXX_ENOMEM : EXX_ECUDA, buf);
}

#define CK(call, where)                                  \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
    } while (0)

extern "C" exx_options exx_default_options(void) {
    exx_options o;
    std::memset(&o, 0, sizeof(o));
    o.precision = 0;
    o.batched = 1;
    o.warm_start = 0;
    o.radii_mode = 0;
    o.r_pe_nonself = 0;
    o.r_me_nonself = 0;
    o.fixed_residual = 0;
    o.deterministic = 0;
    o.max_iter = 20000;
    o.inner_max_iter = 4000;
    o.inner_tol = 0.0;  // library choice
    o.threads = 0;
    o.ctas_per_sm = 0;
    o.solver_kind = 0;
    o.cluster_size = 0;
    o.update_drop = 1e-4;
    o.lane_map = 0;
    o.autotune = 1;
    return o;
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

static void apply_cand(exx_ctx* cc, int k) {
    const exx_ctx::ClusterCand& K = cc->cands[k];
    cc->cand = k;
    cc->CL = K.L;
    cc->cl_variant = K.variant;
    cc->smem = K.smem;
    cc->threads = cluster_variant_threads(K.variant);
    cc->n_clusters = std::min(K.n_clusters, cc->n_slots > 0 ? cc->n_slots : K.n_clusters);
}

// One quad-map cluster candidate with halo planes (mode 3, bank-aware
// dealing) for ball B on variant v: slab layout, thread map and first-residual
// order, with their tables uploaded. fits = false when the slabs, the quads
// or the shared memory do not fit, or no cluster of this size can be resident.
static exx_status make_quad_cand(exx_ctx* c, const HostBall& B, int v, int max_optin, exx_ctx::ClusterCand& K,
                                 bool& fits) {
    fits = false;
    const int C = cluster_variant_size(v);
    ClusterLayout L;
    std::vector<int> pt;
    // planes a CTA can hold besides its 6 halo planes, the slot map and the
    // static shared memory (4 KiB kept free)
    const long plane_bytes = 4L * (((2 * B.r_pe + 7 + 3) & ~3) * (2 * B.r_pe + 7));
    const long budget = (long)max_optin - 4096 - 4L * cluster_variant_threads(v) * cluster_variant_pts(v);
    const int max_planes = (int)(budget / plane_bytes) - 6;
    if (max_planes < 3 || !build_cluster_layout(B, C, L, pt, true, max_planes)) return EXX_OK;
    std::vector<int> spk, sk, res_list, res_nrim;
    // bank-aware dealing (lane map 5) when the slab's quads allow it, else
    // the natural order (lane map 4): the dealing needs every bank group in
    // every run of 8 slots, which some pitches do not offer
    int lane_map = 5;
    if (build_quad_maps(L, pt, cluster_variant_threads(v), cluster_variant_pts(v), spk, sk, 1) < 0) {
        lane_map = 4;
        if (build_quad_maps(L, pt, cluster_variant_threads(v), cluster_variant_pts(v), spk, sk, 0) < 0) return EXX_OK;
    }
    const size_t sm = cluster_kernel_smem(B.r_me, L, v);
    if ((long)sm + 4096 > (long)max_optin) return EXX_OK;
    int nclu = 0;
    cudaError_t e = cluster_prepare(v, sm, &nclu);
    if (e != cudaSuccess || nclu < 1) {
        (void)cudaGetLastError();
        return EXX_OK;
    }
    build_residual_order(B, L, res_list, res_nrim);
    int4 ri[kMaxCluster];
    for (int r = 0; r < C; ++r) ri[r] = make_int4(L.x0[r], L.planes[r], L.k0[r], L.k1[r]);
    const size_t n_int = pt.size() + 4 * (size_t)C + spk.size() + sk.size() + res_list.size() + res_nrim.size();
    int* d = nullptr;
    e = cudaMalloc(&d, sizeof(int) * n_int);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMalloc(class tables)");
    c->cl_mem.push_back(d);
    int* at = d;
    auto put = [&](const void* src, size_t n) -> int* {
        int* here = at;
        if (e == cudaSuccess && n) e = cudaMemcpy(here, src, sizeof(int) * n, cudaMemcpyHostToDevice);
        at += n;
        return here;
    };
    L.rank_info = reinterpret_cast<const int4*>(put(ri, 4 * (size_t)C));  // first: 16-byte aligned
    L.pt_slab = put(pt.data(), pt.size());
    L.slot_pk = put(spk.data(), spk.size());
    L.slot_k = put(sk.data(), sk.size());
    L.res_list = put(res_list.data(), res_list.size());
    L.res_nrim = put(res_nrim.data(), res_nrim.size());
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpy(class tables)");
    K.C = C;
    K.variant = v;
    K.lane_map = lane_map;
    K.n_clusters = nclu;
    K.smem = sm;
    K.L = L;
    fits = true;
    return EXX_OK;
}

static void free_pairs(exx_ctx* c) {
    cudaFree(c->d_counts);
    cudaFree(c->d_offsets);
    cudaFree(c->d_pairs);
    cudaFree(c->d_epair);
    cudaFree(c->d_iters);
    cudaFree(c->d_refines);
    cudaFree(c->d_order);
    c->d_order = nullptr;
    c->d_counts = c->d_offsets = nullptr;
    c->d_pairs = nullptr;
    c->d_epair = nullptr;
    c->d_iters = c->d_refines = nullptr;
    c->cap_n = 0;
    c->cap_pairs = 0;
}

static void drop_graph(exx_ctx* c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    c->g_n = -1;
}

extern "C" void exx_destroy(exx_ctx* c) {
    if (!c) return;
    drop_graph(c);
    free_pairs(c);
    cudaFree(c->d_scalars);
    cudaFree(c->d_hist);
    cudaFree(c->d_class);
    cudaFree(c->d_exx);
    if (c->h_exx) cudaFreeHost(c->h_exx);
    cudaFree(c->ws);
    cudaFree(c->geo_mem);
    cudaFree(c->mg_mem);
    cudaFree(c->d_orb);
    cudaFree(c->d_dxx);
    cudaFree(c->d_cent);
    cudaFree(c->d_alpha);
    for (void* m : c->cl_mem) cudaFree(m);
    cudaFree(c->d_prev_pairs);
    cudaFree(c->d_vcache[0]);
    cudaFree(c->d_vcache[1]);
    cudaFree(c->hv[0]);
    cudaFree(c->hv[1]);
    cudaFree(c->hp[0]);
    cudaFree(c->hp[1]);
    cudaFree(c->d_pow);
    cudaFree(c->d_phase);
    if (c->gnet) {
        exx::unet::destroy(*c->gnet);
        delete c->gnet;
    }
    cudaFree(c->d_guess);
    cudaFree(c->d_gin);
    cudaFree(c->d_gscale);
    for (auto& e : c->ev_g)
        if (e) cudaEventDestroy(e);
    for (auto& e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->aux) cudaStreamDestroy(c->aux);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    if (c->work) cudaStreamDestroy(c->work);
    delete c;
}

extern "C" exx_status exx_init(exx_ctx** out, const double cell[3], const int grid[3], double r_pair, int r_pe,
                               int r_me, int l_max, double tol, const exx_options* opt) {
    exx_ctx* c = nullptr;
    if (!out) return fail(nullptr, EXX_EINVAL, "exx_init: out is NULL");
    *out = nullptr;
    if (!cell || !grid) return fail(nullptr, EXX_EINVAL, "exx_init: cell or grid is NULL");
    for (int a = 0; a < 3; ++a) {
        if (!(cell[a] > 0.0) || !std::isfinite(cell[a])) return fail(nullptr, EXX_EINVAL, "exx_init: cell lengths must be finite and > 0");
        if (grid[a] < 1 || grid[a] > 4096) return fail(nullptr, EXX_EINVAL, "exx_init: grid sizes must be in [1, 4096]");
    }
    if (!(r_pair > 0.0)) return fail(nullptr, EXX_EINVAL, "exx_init: r_pair must be > 0 (INFINITY keeps all pairs)");
    if (r_pe < 1) return fail(nullptr, EXX_EINVAL, "exx_init: r_pe must be >= 1");
    if (r_me < r_pe + 3) return fail(nullptr, EXX_EINVAL, "exx_init: r_me must be >= r_pe + 3 (the shell holds the stencil reach)");
    if (r_me > 63) return fail(nullptr, EXX_EINVAL, "exx_init: r_me must be <= 63");
    for (int a = 0; a < 3; ++a)
        if (2 * r_me + 1 > grid[a]) return fail(nullptr, EXX_EINVAL, "exx_init: 2 r_me + 1 must not exceed any grid size");
    if (l_max < 0 || l_max > kLmaxMax) return fail(nullptr, EXX_EINVAL, "exx_init: l_max must be in [0, 6]");
    if (!(tol > 0.0 && tol < 1.0)) return fail(nullptr, EXX_EINVAL, "exx_init: tol must be in (0, 1)");
    exx_options o = opt ? *opt : exx_default_options();
    if (o.precision != 0 && o.precision != 1) return fail(nullptr, EXX_EINVAL, "exx_init: precision must be 0 or 1");
    if (o.radii_mode < 0 || o.radii_mode > 2) return fail(nullptr, EXX_EINVAL, "exx_init: radii_mode must be 0, 1 or 2");
    if (o.radii_mode == 2) {
        if (o.r_pe_nonself < 1 || o.r_pe_nonself > r_pe || o.r_me_nonself > r_me ||
            o.r_me_nonself < o.r_pe_nonself + 3)
            return fail(nullptr, EXX_EINVAL,
                        "exx_init: radii_mode 2 needs 1 <= r_pe_nonself <= r_pe, r_pe_nonself + 3 <= r_me_nonself <= r_me");
        if (o.solver_kind == 2 && o.preconditioner != 1)
            return fail(nullptr, EXX_EINVAL,
                        "exx_init: radii_mode 2 runs on solver_kind 1 (or on clusters with preconditioner 1)");
    }
    if (o.radii_mode == 1) {
        const int rme_rule = r_pe + std::max(3, (r_pe + 2) / 3);
        if (r_me < rme_rule)
            return fail(nullptr, EXX_EINVAL,
                        "exx_init: with radii_mode 1, r_me must be >= r_pe + max(3, ceil(r_pe/3)) (the largest pair's R_ME)");
    }
    if (o.warm_start < 0 || o.warm_start > 3)
        return fail(nullptr, EXX_EINVAL, "exx_init: warm_start must be 0, 1, 2 or 3");
    if (o.warm_start != 0 && (o.precision != 1 || o.radii_mode != 0 || o.solver_kind == 1))
        return fail(nullptr, EXX_EINVAL,
                    "exx_init: warm_start 1 and 2 run on the cluster solver (precision 1, fixed radii, solver_kind 0 or 2)");
    if (o.max_iter <= 0) o.max_iter = 20000;
    if (o.inner_max_iter <= 0) o.inner_max_iter = 4000;
    if (!(o.inner_tol > 0.0 && o.inner_tol < 1.0)) o.inner_tol = o.preconditioner == 1 ? 1e-4 : 1e-5;
    if (!(o.update_drop > 0.0 && o.update_drop < 1.0)) o.update_drop = 1e-4;
    if (o.threads != 0 && (o.threads < 256 || o.threads > 1024 || o.threads % 32))
        return fail(nullptr, EXX_EINVAL, "exx_init: threads must be 0 or a multiple of 32 in [256, 1024]");
    if (o.solver_kind < 0 || o.solver_kind > 2) return fail(nullptr, EXX_EINVAL, "exx_init: solver_kind must be 0, 1 or 2");
    if (o.solver_kind == 2 && o.precision != 1)
        return fail(nullptr, EXX_EINVAL, "exx_init: solver_kind 2 (cluster) runs the FP32 inner solver: precision must be 1");
    if (o.cluster_size != 0 && o.cluster_size != 2 && o.cluster_size != 4 && o.cluster_size != 8 &&
        o.cluster_size != 9 && !(o.cluster_size == 16 && o.preconditioner == 1))
        return fail(nullptr, EXX_EINVAL,
                    "exx_init: cluster_size must be 0, 2, 4, 8 or 9 (16 with the multigrid CG)");
    if (o.fixed_residual < 0 || o.fixed_residual > 2)
        return fail(nullptr, EXX_EINVAL, "exx_init: fixed_residual must be 0, 1 or 2");
    if (o.deterministic < 0 || o.deterministic > 1)
        return fail(nullptr, EXX_EINVAL, "exx_init: deterministic must be 0 or 1");
    if (o.inject_wait_timeout < 0) return fail(nullptr, EXX_EINVAL, "exx_init: inject_wait_timeout must be >= 0");
    if (o.preconditioner < 0 || o.preconditioner > 1)
        return fail(nullptr, EXX_EINVAL, "exx_init: preconditioner must be 0 or 1");
    if (o.preconditioner == 1 && o.warm_start != 0)
        return fail(nullptr, EXX_EINVAL, "exx_init: the multigrid-preconditioned CG takes no warm start");
    if (o.preconditioner == 1 && o.solver_kind == 2 && o.precision != 1)
        return fail(nullptr, EXX_EINVAL,
                    "exx_init: the multigrid-preconditioned CG on clusters (solver_kind 2) needs precision 1");
    if (o.preconditioner == 1 && o.solver_kind != 1 && o.precision == 1 && o.cluster_size != 0 &&
        !mg_cluster_size_ok(o.cluster_size))
        return fail(nullptr, EXX_EINVAL, "exx_init: the multigrid CG on clusters takes cluster_size 2, 4, 8 or 16");

    c = new exx_ctx();
    std::memset(&c->stats, 0, sizeof(c->stats));
    c->opt = o;
    c->inject_left = o.inject_wait_timeout;
    for (int a = 0; a < 3; ++a) {
        c->cell[a] = cell[a];
        c->grid[a] = grid[a];
        c->delta[a] = cell[a] / (double)grid[a];
    }
    c->dV = c->delta[0] * c->delta[1] * c->delta[2];
    c->ngrid = (long long)grid[0] * grid[1] * grid[2];
    c->r_pair = r_pair;
    c->r_pe = r_pe;
    c->r_me = r_me;
    c->lmax = l_max;
    c->tol = tol;

    auto bail = [&](exx_status s) {
        g_init_err = c->err;
        exx_destroy(c);
        return s;
    };
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaGetDevice"));
    e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaDeviceGetAttribute"));

    // constants of the multipole expansion (identical for every context)
    static MultipoleConst mc;
    static bool mc_built = false;
    if (!mc_built) {
        build_multipole_const(mc);
        mc_built = true;
    }
    e = set_multipole_const_solve(mc);
    if (e == cudaSuccess) e = set_multipole_const_cluster(mc);
    if (e == cudaSuccess) e = exx::unet::set_multipole_const_unet(mc);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMemcpyToSymbol(multipoles)"));

    // ball geometries (Algorithm 2), cube radius Rc = R_ME (the largest)
    const int Rc = r_me, S = 2 * Rc + 1;
    if (o.radii_mode == 1) {
        c->r_min = std::min(12, r_pe);
        c->n_geo = r_pe - c->r_min + 1;
    } else if (o.radii_mode == 2) {
        c->r_min = o.r_pe_nonself;
        c->n_geo = 2;
        c->ns_pe = o.r_pe_nonself;
        c->ns_me = o.r_me_nonself;
    } else {
        c->r_min = r_pe;
        c->n_geo = 1;
    }
    c->ln_inv_eps = std::log(1e14);
    c->delta_max = std::max(c->delta[0], std::max(c->delta[1], c->delta[2]));
    c->balls.resize(c->n_geo);
    for (int g = 0; g < c->n_geo; ++g) {
        int R = c->r_min + g;
        int Rm = o.radii_mode == 1 ? R + std::max(3, (R + 2) / 3) : r_me;
        if (o.radii_mode == 2) {  // geometry 0: non-self pairs, 1: self pairs
            R = g == 0 ? o.r_pe_nonself : r_pe;
            Rm = g == 0 ? o.r_me_nonself : r_me;
        }
        build_ball(c->balls[g], R, Rm, Rc);
    }
    c->hb = c->balls.back();
    const HostBall& B = c->hb;
    {
        std::vector<size_t> o_cube(c->n_geo), o_off(c->n_geo), o_rpe(c->n_geo), o_rme(c->n_geo), o_pl(c->n_geo),
            o_ro(c->n_geo), o_sn(c->n_geo), o_sf(c->n_geo);
        size_t at = 0;
        for (int g = 0; g < c->n_geo; ++g) {
            const HostBall& Bg = c->balls[g];
            o_cube[g] = at; at = align256(at + sizeof(int) * Bg.n_me);
            o_off[g] = at; at = align256(at + sizeof(int) * Bg.n_me);
            o_rpe[g] = at; at = align256(at + sizeof(RowRec) * Bg.rows_pe.size());
            o_rme[g] = at; at = align256(at + sizeof(RowRec) * Bg.rows_me.size());
            o_pl[g] = at; at = align256(at + sizeof(int) * Bg.plane_pe.size());
            o_ro[g] = at; at = align256(at + sizeof(int) * Bg.row_of.size());
            o_sn[g] = at; at = align256(at + sizeof(int) * Bg.sh_near.size());
            o_sf[g] = at; at = align256(at + sizeof(int) * Bg.sh_far.size());
        }
        const size_t o_geo = at;
        const size_t geo_bytes = align256(o_geo + sizeof(BallGeo) * c->n_geo);
        e = cudaMalloc(&c->geo_mem, geo_bytes);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMalloc(geometry)"));
        char* gm = (char*)c->geo_mem;
        std::vector<BallGeo> gv(c->n_geo);
        for (int g = 0; g < c->n_geo; ++g) {
            const HostBall& Bg = c->balls[g];
            BallGeo& G = gv[g];
            G.r_pe = Bg.r_pe;
            G.r_me = Bg.r_me;
            G.n_pe = Bg.n_pe;
            G.n_me = Bg.n_me;
            G.n_rows_pe = (int)Bg.rows_pe.size();
            G.n_rows_me = (int)Bg.rows_me.size();
            G.pt_cube = (const int*)(gm + o_cube[g]);
            G.pt_off = (const int*)(gm + o_off[g]);
            G.rows_pe = (const RowRec*)(gm + o_rpe[g]);
            G.rows_me = (const RowRec*)(gm + o_rme[g]);
            G.plane_pe = (const int*)(gm + o_pl[g]);
            G.row_of = (const int*)(gm + o_ro[g]);
            G.sh_near = (const int*)(gm + o_sn[g]);
            G.sh_far = (const int*)(gm + o_sf[g]);
            G.n_near = (int)Bg.sh_near.size();
            G.n_far = (int)Bg.sh_far.size();
            if ((e = cudaMemcpy(gm + o_ro[g], Bg.row_of.data(), sizeof(int) * Bg.row_of.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
                (e = cudaMemcpy(gm + o_cube[g], Bg.cube.data(), sizeof(int) * Bg.n_me, cudaMemcpyHostToDevice)) != cudaSuccess ||
                (e = cudaMemcpy(gm + o_off[g], Bg.off.data(), sizeof(int) * Bg.n_me, cudaMemcpyHostToDevice)) != cudaSuccess ||
                (e = cudaMemcpy(gm + o_rpe[g], Bg.rows_pe.data(), sizeof(RowRec) * Bg.rows_pe.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
                (e = cudaMemcpy(gm + o_rme[g], Bg.rows_me.data(), sizeof(RowRec) * Bg.rows_me.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
                (e = cudaMemcpy(gm + o_pl[g], Bg.plane_pe.data(), sizeof(int) * Bg.plane_pe.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
                (e = cudaMemcpy(gm + o_sn[g], Bg.sh_near.data(), sizeof(int) * Bg.sh_near.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
                (e = cudaMemcpy(gm + o_sf[g], Bg.sh_far.data(), sizeof(int) * Bg.sh_far.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
                return bail(cuda_fail(c, e, "cudaMemcpy(geometry)"));
        }
        c->geo_host = gv.back();
        c->d_geos = (BallGeo*)(gm + o_geo);
        e = cudaMemcpy(gm + o_geo, gv.data(), sizeof(BallGeo) * c->n_geo, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMemcpy(geometry records)"));
    }

    // multigrid hierarchies of every ball geometry (preconditioner 1)
    std::vector<std::vector<HostMGLevel>> mgl(c->n_geo);
    std::vector<std::vector<double>> mgi(c->n_geo);
    int mg_levels = 0;
    if (o.preconditioner == 1) {
        for (int g = 0; g < c->n_geo; ++g) {
            if (c->balls[g].r_pe <= 3) continue;  // nothing coarser: plain CG for this ball
            if (!build_mg_levels(c->balls[g].r_pe, c->delta, mgl[g], mgi[g]))
                return bail(fail(c, EXX_EINVAL, "exx_init: multigrid hierarchy could not be built"));
            mg_levels = std::max(mg_levels, (int)mgl[g].size());
        }
    }

    // workspace slots
    const long long S3 = (long long)S * S * S;
    SolveParams& P = c->P;
    std::memset(&P, 0, sizeof(P));
    size_t off = 0;
    P.off_vcube = off; off = align256(off + sizeof(double) * S3);
    P.off_pcube = off; off = align256(off + sizeof(double) * S3);
    P.off_p32 = off; off = align256(off + sizeof(float) * S3);
    P.off_rho = off; off = align256(off + sizeof(double) * B.n_pe);
    P.off_r = off; off = align256(off + sizeof(double) * B.n_pe);
    P.off_d = off; off = align256(off + sizeof(double) * B.n_pe);
    P.off_ap = off; off = align256(off + sizeof(double) * B.n_pe);
    P.off_r32 = off; off = align256(off + sizeof(float) * B.n_pe);
    P.off_d32 = off; off = align256(off + sizeof(float) * B.n_pe);
    P.off_ap32 = off; off = align256(off + sizeof(float) * B.n_pe);
    P.off_rows = off; off = align256(off + sizeof(double) * 8 * B.rows_pe.size());
    P.off_sy = off; off = align256(off + sizeof(double) * (size_t)kMaxCluster * (((2 * r_pe + 1) * 28 + 1) & ~1));
    P.off_ush = off; off = align256(off + (sizeof(double) + sizeof(float)) * kNU * B.rows_me.size());
    P.off_vfix = off; off = align256(off + sizeof(long long) * S3);
    if (mg_levels > 0) {
        P.off_zc = off; off = align256(off + sizeof(double) * S3);
        P.off_tc = off; off = align256(off + sizeof(double) * S3);
        for (int l = 1; l <= mg_levels; ++l) {
            size_t cube = 0, npts = 0;
            for (int g = 0; g < c->n_geo; ++g)
                if ((int)mgl[g].size() >= l) {
                    const HostMGLevel& H = mgl[g][l - 1];
                    cube = std::max(cube, (size_t)H.side * H.side * H.side);
                    npts = std::max(npts, H.off.size());
                }
            P.off_mgz[l] = off; off = align256(off + sizeof(double) * cube);
            P.off_mgt[l] = off; off = align256(off + sizeof(double) * cube);
            P.off_mgr[l] = off; off = align256(off + sizeof(double) * npts);
        }
    }
    c->slot_bytes = off;
    // x^e, y^e, z^e (e < 8) for offsets -Rc..Rc, by repeated multiplication
    {
        std::vector<double> tab((size_t)3 * (2 * Rc + 1) * 8);
        for (int a = 0; a < 3; ++a)
            for (int o = -Rc; o <= Rc; ++o) {
                const double x = o * c->delta[a];
                double px = 1.0;
                for (int e2 = 0; e2 < 8; ++e2) {
                    tab[((size_t)a * (2 * Rc + 1) + (o + Rc)) * 8 + e2] = px;
                    px *= x;
                }
            }
        e = cudaMalloc(&c->d_pow, sizeof(double) * tab.size());
        if (e == cudaSuccess) e = cudaMemcpy(c->d_pow, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "power table"));
        P.pow_tab = c->d_pow;
    }

    if (mg_levels > 0) {
        size_t bytes = align256(sizeof(MGGeo) * c->n_geo);
        for (int g = 0; g < c->n_geo; ++g) {
            for (const HostMGLevel& H : mgl[g]) bytes += align256(sizeof(int) * H.off.size()) * 2;
            bytes += align256(sizeof(double) * mgi[g].size()) + align256(sizeof(float) * mgi[g].size());
        }
        e = cudaMalloc(&c->mg_mem, bytes);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMalloc(multigrid tables)"));
        char* at = (char*)c->mg_mem + align256(sizeof(MGGeo) * c->n_geo);
        std::vector<MGGeo> mv(c->n_geo);
        for (int g = 0; g < c->n_geo && e == cudaSuccess; ++g) {
            MGGeo& M = mv[g];
            std::memset(&M, 0, sizeof(M));
            M.L = (int)mgl[g].size();
            for (int l = 1; l <= M.L && e == cudaSuccess; ++l) {
                const HostMGLevel& H = mgl[g][l - 1];
                MGLevel& lv = M.lv[l];
                lv.R = H.R;
                lv.n = (int)H.off.size();
                lv.side = H.side;
                lv.cube = (const int*)at;
                e = cudaMemcpy(at, H.cube.data(), sizeof(int) * H.cube.size(), cudaMemcpyHostToDevice);
                at += align256(sizeof(int) * H.cube.size());
                lv.off = (const int*)at;
                if (e == cudaSuccess) e = cudaMemcpy(at, H.off.data(), sizeof(int) * H.off.size(), cudaMemcpyHostToDevice);
                at += align256(sizeof(int) * H.off.size());
            }
            M.minv = (const double*)at;
            if (e == cudaSuccess && !mgi[g].empty())
                e = cudaMemcpy(at, mgi[g].data(), sizeof(double) * mgi[g].size(), cudaMemcpyHostToDevice);
            at += align256(sizeof(double) * mgi[g].size());
            std::vector<float> m32(mgi[g].begin(), mgi[g].end());
            M.minv32 = (const float*)at;
            if (e == cudaSuccess && !m32.empty())
                e = cudaMemcpy(at, m32.data(), sizeof(float) * m32.size(), cudaMemcpyHostToDevice);
            at += align256(sizeof(float) * m32.size());
        }
        c->d_mg = (MGGeo*)c->mg_mem;
        if (e == cudaSuccess) e = cudaMemcpy(c->d_mg, mv.data(), sizeof(MGGeo) * c->n_geo, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMemcpy(multigrid tables)"));
        P.mg = c->d_mg;
        P.mg_omega = 0.8;
    }

    // cluster solver candidates: every cluster size, thread count and lane map
    // whose slab layout, registers and shared memory fit
    if (o.precision == 1 && o.solver_kind != 1 && o.preconditioner == 0 && c->n_geo == 1) {
        int max_optin = 0;
        cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
        const int csizes[4] = {9, 8, 4, 2};
        for (int ci = 0; ci < 4; ++ci) {
            const int C = csizes[ci];
            if (o.cluster_size && o.cluster_size != C) continue;
            ClusterLayout L;
            std::vector<int> pt;
            if (!build_cluster_layout(B, C, L, pt)) continue;
            int* d_pt = nullptr;
            int4* d_ri = nullptr;
            int* d_res = nullptr;  // residual order and rim counts of this partition
            std::vector<int> res_list, res_nrim;
            build_residual_order(B, L, res_list, res_nrim);
            // one candidate: variant v with thread map (spk, sk) and lane map lm
            auto add_cand = [&](int v, int lm, const std::vector<int>& spk, const std::vector<int>& sk,
                                const ClusterLayout& LL) -> exx_status {
                const size_t sm = cluster_kernel_smem(Rc, LL, v);
                if ((long)sm + 2048 > (long)max_optin) return EXX_OK;
                int nclu = 0;
                e = cluster_prepare(v, sm, &nclu);
                if (e != cudaSuccess || nclu < 1) {
                    (void)cudaGetLastError();
                    return EXX_OK;
                }
                if (!d_pt) {
                    e = cudaMalloc(&d_pt, sizeof(int) * pt.size());
                    if (e == cudaSuccess) c->cl_mem.push_back(d_pt);
                    if (e == cudaSuccess) e = cudaMemcpy(d_pt, pt.data(), sizeof(int) * pt.size(), cudaMemcpyHostToDevice);
                    int4 ri[kMaxCluster];
                    for (int r = 0; r < C; ++r) ri[r] = make_int4(L.x0[r], L.planes[r], L.k0[r], L.k1[r]);
                    if (e == cudaSuccess) e = cudaMalloc(&d_ri, sizeof(int4) * C);
                    if (e == cudaSuccess) c->cl_mem.push_back(d_ri);
                    if (e == cudaSuccess) e = cudaMemcpy(d_ri, ri, sizeof(int4) * C, cudaMemcpyHostToDevice);
                    if (e == cudaSuccess) e = cudaMalloc(&d_res, sizeof(int) * (res_list.size() + res_nrim.size()));
                    if (e == cudaSuccess) c->cl_mem.push_back(d_res);
                    if (e == cudaSuccess)
                        e = cudaMemcpy(d_res, res_list.data(), sizeof(int) * res_list.size(), cudaMemcpyHostToDevice);
                    if (e == cudaSuccess)
                        e = cudaMemcpy(d_res + res_list.size(), res_nrim.data(), sizeof(int) * res_nrim.size(),
                                       cudaMemcpyHostToDevice);
                    if (e != cudaSuccess) return cuda_fail(c, e, "slab tables");
                }
                int* d_slot = nullptr;
                e = cudaMalloc(&d_slot, sizeof(int) * (spk.size() + sk.size()));
                if (e == cudaSuccess) c->cl_mem.push_back(d_slot);
                if (e == cudaSuccess) e = cudaMemcpy(d_slot, spk.data(), sizeof(int) * spk.size(), cudaMemcpyHostToDevice);
                if (e == cudaSuccess)
                    e = cudaMemcpy(d_slot + spk.size(), sk.data(), sizeof(int) * sk.size(), cudaMemcpyHostToDevice);
                if (e != cudaSuccess) return cuda_fail(c, e, "slot maps");
                exx_ctx::ClusterCand K;
                K.C = C;
                K.variant = v;
                K.lane_map = lm;
                K.n_clusters = nclu;
                K.smem = sm;
                K.L = LL;
                K.L.pt_slab = d_pt;
                K.L.rank_info = d_ri;
                K.L.slot_pk = d_slot;
                K.L.slot_k = d_slot + spk.size();
                K.L.res_list = d_res;
                K.L.res_nrim = d_res + res_list.size();
                c->cands.push_back(K);
                return EXX_OK;
            };
            const bool isotropic = c->delta[0] == c->delta[1] && c->delta[1] == c->delta[2];
            // z-run thread maps with halo planes (lane map 2): only on request;
            // on GB300 the point map is faster (the halo copies add a remote
            // store for nearly every point of a thin slab, and the cluster
            // barrier waits for them; reading the x legs of the runs remotely
            // instead was slower still, as a warp's remote loads scatter)
            for (int v = 0; v < cluster_variant_count(); ++v) {
                if (cluster_variant_mode(v) != 1 || cluster_variant_size(v) != C) continue;
                if (cluster_variant_syz(v) && cluster_variant_syz(v) != L.Syz) continue;
                if (!isotropic) continue;  // the run kernel's stencil has one spacing
                if (o.threads && o.threads != cluster_variant_threads(v)) continue;
                const int lm = 2;
                if (o.lane_map != lm) continue;
                std::vector<int> spk, sk;
                if (build_run_maps(L, pt, cluster_variant_threads(v), cluster_variant_pts(v), spk, sk) < 0) continue;
                const exx_status sa = add_cand(v, lm, spk, sk, L);
                if (sa != EXX_OK) return bail(sa);
            }
            // quads of 4 consecutive z positions per thread slot, on a layout
            // whose rows are padded to 16 bytes: x legs read from the
            // neighbours (lane map 3) or from halo planes (lane map 4)
            if (o.autotune || (o.lane_map >= 3 && o.lane_map <= 5)) {
                ClusterLayout Lq;
                std::vector<int> ptq;
                if (build_cluster_layout(B, C, Lq, ptq, true)) {
                    // per thread count the first fit (the table lists specialised before generic)
                    std::vector<int> have;  // (mode, thread count) pairs with a candidate
                    for (int v = 0; v < cluster_variant_count(); ++v) {
                        const int mode = cluster_variant_mode(v);
                        if ((mode != 2 && mode != 3) || cluster_variant_size(v) != C) continue;
                        if (cluster_variant_syz(v) && (cluster_variant_syz(v) != 2 * r_pe + 7 || !isotropic)) continue;
                        if (cluster_variant_iso(v) && !isotropic) continue;
                        const int nt = cluster_variant_threads(v);
                        if (o.threads && o.threads != nt) continue;
                        if (std::find(have.begin(), have.end(), mode * 4096 + nt) != have.end()) continue;
                        // lane map 3: mode 2; 4: mode 3; 5: mode 3 with bank-aware dealing
                        for (int ba = 0; ba <= (mode == 3 ? 1 : 0); ++ba) {
                            const int lm = mode == 2 ? 3 : 4 + ba;
                            if (!o.autotune && o.lane_map != lm) continue;
                            std::vector<int> spk, sk;
                            if (build_quad_maps(Lq, ptq, nt, cluster_variant_pts(v), spk, sk, ba) < 0) continue;
                            const exx_status sa = add_cand(v, lm, spk, sk, Lq);
                            if (sa != EXX_OK) return bail(sa);
                        }
                        have.push_back(mode * 4096 + nt);
                    }
                }
            }
            // one point per thread slot (lane maps 0 and 1)
            for (int nt : {1024, 512}) {
                if (o.threads && o.threads != nt) continue;
                const int v = cluster_variant(C, L.max_pts, nt, L.Syz, isotropic);
                if (v < 0) continue;
                for (int lm = 0; lm <= 1; ++lm) {
                    if (!o.autotune && lm != o.lane_map) continue;
                    std::vector<int> spk, sk;
                    if (build_slot_maps(L, pt, cluster_variant_threads(v), cluster_variant_pts(v), lm, spk, sk) < 0)
                        continue;
                    const exx_status sa = add_cand(v, lm, spk, sk, L);
                    if (sa != EXX_OK) return bail(sa);
                }
            }
        }
        if (!c->cands.empty()) {
            c->use_cluster = true;
            // default before tuning: the first candidate in preference order
            // (largest cluster, most threads, the requested lane map)
            int pick = 0;
            for (int k = 0; k < (int)c->cands.size(); ++k)
                if (c->cands[k].lane_map == o.lane_map) {
                    pick = k;
                    break;
                }
            c->cand = pick;
            c->tuned = !o.autotune || c->cands.size() == 1;
        }
        if (!c->use_cluster && o.solver_kind == 2)
            return bail(fail(c, EXX_EINVAL, "exx_init: no cluster layout fits these radii"));
    }
    // per-pair radii on the cluster solver: for every radius class the first
    // fitting quad-map launch shape in the order of increasing cluster size
    // (a small ball in one CTA's shared memory, larger ones over 2 to 16
    // CTAs; at a cluster size, the variant specialised for the slab pitch
    // first, then fewer quads per thread); the one-CTA pair kernel takes any
    // class that fits none
    if (o.precision == 1 && o.solver_kind != 1 && o.preconditioner == 0 && o.radii_mode == 1) {
        int max_optin = 0;
        cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
        const bool isotropic = c->delta[0] == c->delta[1] && c->delta[1] == c->delta[2];
        std::vector<int> order;  // mode-3 variants by cluster size, specialised first, then quads per thread
        for (int v = 0; v < cluster_variant_count(); ++v)
            if (cluster_variant_mode(v) == 3 && cluster_variant_threads(v) == 512) order.push_back(v);
        std::stable_sort(order.begin(), order.end(), [](int a, int b) {
            if (cluster_variant_size(a) != cluster_variant_size(b)) return cluster_variant_size(a) < cluster_variant_size(b);
            if ((cluster_variant_syz(a) != 0) != (cluster_variant_syz(b) != 0)) return cluster_variant_syz(a) != 0;
            return cluster_variant_pts(a) < cluster_variant_pts(b);
        });
        std::vector<size_t> need_smem(cluster_variant_count(), 0);
        c->classes.resize(c->n_geo);
        for (int g = 0; g < c->n_geo; ++g) {
            exx_ctx::RadiusClass& RC = c->classes[g];
            RC.geo = g;
            RC.kind = 1;
            const HostBall& Bg = c->balls[g];
            for (int v : order) {
                if (o.cluster_size && cluster_variant_size(v) != o.cluster_size) continue;
                if (cluster_variant_syz(v) && (cluster_variant_syz(v) != 2 * Bg.r_pe + 7 || !isotropic)) continue;
                if (cluster_variant_iso(v) && !isotropic) continue;
                bool fits = false;
                const exx_status sa = make_quad_cand(c, Bg, v, max_optin, RC.cand, fits);
                if (sa != EXX_OK) return bail(sa);
                if (fits) {
                    RC.kind = 2;
                    need_smem[v] = std::max(need_smem[v], RC.cand.smem);
                    break;
                }
            }
        }
        for (int v = 0; v < cluster_variant_count(); ++v)
            if (need_smem[v] && (e = cluster_set_smem(v, need_smem[v])) != cudaSuccess)
                return bail(cuda_fail(c, e, "cudaFuncSetAttribute(class shared memory)"));
        c->per_class = true;
        e = cudaMalloc(&c->d_class, sizeof(int) * 3 * (size_t)c->n_geo);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMalloc(radius classes)"));
    }
    // the multigrid-preconditioned CG on clusters (solver_kind 2 at precision 1)
    if (o.preconditioner == 1 && o.precision == 1 && o.solver_kind == 2 && mg_levels > 0) {
        const int C = o.cluster_size ? o.cluster_size : 8;
        const int minb = o.ctas_per_sm == 1 ? 1 : 2;
        int nclu = 0;
        e = mg_cluster_prepare(C, minb, &nclu);
        if (e != cudaSuccess || nclu < 1) {
            (void)cudaGetLastError();
            if (o.solver_kind == 2)
                return bail(fail(c, EXX_EINVAL, "exx_init: no cluster of this size can be resident for the multigrid CG"));
        } else {
            c->mg_C = C;
            c->mg_minb = minb;
            c->mg_clusters = nclu;
            c->threads = 512;
        }
    }
    if (o.warm_start != 0 && !c->use_cluster)
        return bail(fail(c, EXX_EINVAL, "exx_init: warm_start 1 and 2 need the cluster solver, which does not fit these radii"));
    if (c->use_cluster) apply_cand(c, c->cand);

    // one CTA per pair: 512 threads, or 256 (five or six CTAs per SM, measured fastest) for the FP32 multigrid CG
    const int def_threads = (o.preconditioner == 1 && o.precision == 1) ? 256 : 512;
    c->threads = c->use_cluster ? c->threads
                                : ((o.threads == 256 || o.threads == 512 || o.threads == 1024) ? o.threads : def_threads);
    if (!c->use_cluster) c->smem = pair_kernel_smem(Rc, r_pe);
    int bps = 0;
    long long want;
    if (c->use_cluster) {
        want = 0;
        for (const auto& K : c->cands) want = std::max<long long>(want, K.n_clusters);
    } else if (c->mg_C) {
        want = c->mg_clusters;
    } else if (c->per_class) {
        // the classes of a lane run one after another and share its slots
        e = pair_kernel_occupancy(c->threads, true, false, c->n_geo == 1, c->smem, &bps);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "occupancy query"));
        for (int g = 0; g < c->n_geo; ++g) {
            const exx_ctx::RadiusClass& RC = c->classes[g];
            const int lane = (c->n_geo - 1 - g) & 1;
            const int need = RC.kind == 2 ? RC.cand.n_clusters : c->num_sms * std::max(1, std::min(bps, 2));
            c->lane_slots[lane] = std::max(c->lane_slots[lane], need);
        }
        want = (long long)c->lane_slots[0] + c->lane_slots[1];
    } else {
        e = pair_kernel_occupancy(c->threads, o.precision == 1, o.preconditioner == 1, c->n_geo == 1, c->smem, &bps);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "occupancy query"));
        if (bps < 1) return bail(fail(c, EXX_ECUDA, "pair kernel does not fit on an SM"));
        // all resident (the launch bounds allow two CTAs per SM; the 256-thread
        // FP32 multigrid kernel six on one ball, five with per-pair radii)
        const int cap = (o.preconditioner == 1 && o.precision == 1) ? (c->n_geo == 1 ? 6 : 5) : 4;
        int per_sm = o.ctas_per_sm > 0 ? std::min(o.ctas_per_sm, bps) : std::min(bps, cap);
        want = (long long)c->num_sms * per_sm;
    }
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    long long fit = (long long)(0.25 * (double)free_b / (double)c->slot_bytes);
    c->n_slots = (int)std::max(1LL, std::min(want, fit));
    if (c->per_class && c->n_slots < want) {  // not enough memory for two lanes: one lane, shared slots
        c->lane_slots[0] = c->n_slots;
        c->lane_slots[1] = 0;
    }
    if (c->use_cluster) apply_cand(c, c->cand);
    e = cudaMalloc(&c->ws, c->slot_bytes * (size_t)c->n_slots);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMalloc(workspace)"));
    e = cudaMemset(c->ws, 0, c->slot_bytes * (size_t)c->n_slots);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMemset(workspace)"));

    cudaDeviceGetAttribute(&c->clock_khz, cudaDevAttrClockRate, c->device);
    e = cudaMalloc(&c->d_phase, sizeof(unsigned long long) * 4);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMalloc(phase clocks)"));
    e = cudaMalloc(&c->d_hist, sizeof(int) * 2 * (size_t)c->n_geo);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMalloc(radius histogram)"));
    e = cudaMalloc(&c->d_scalars, sizeof(int) * 16);  // [8], [9]: pair counts of the extrapolation history
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMalloc(scalars)"));
    e = cudaMalloc(&c->d_exx, sizeof(double) * 2);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMalloc(exx)"));
    e = cudaMallocHost(&c->h_exx, sizeof(double) * 2);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMallocHost"));
    for (auto& ev : c->ev) {
        e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaEventCreate"));
    }
    if ((e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&c->work, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(cuda_fail(c, e, "stream/event creation"));
    if (c->per_class && c->lane_slots[1] > 0 &&
        ((e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
         (e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming)) != cudaSuccess ||
         (e = cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking)) != cudaSuccess))
        return bail(cuda_fail(c, e, "stream/event creation (radius classes)"));

    // fixed kernel parameters
    for (int a = 0; a < 3; ++a) {
        P.N[a] = grid[a];
        P.delta[a] = c->delta[a];
    }
    P.ngrid = c->ngrid;
    P.ostride = c->ngrid;
    P.dV = c->dV;
    const double W[4] = {-49.0 / 18.0, 3.0 / 2.0, -3.0 / 20.0, 1.0 / 90.0};  // Eq. d2_1
    double inv2[3];
    for (int a = 0; a < 3; ++a) inv2[a] = 1.0 / (c->delta[a] * c->delta[a]);
    // isotropic grids: 180 delta^2 x the weights are the integers -490, 270, -27, 2
    P.fixres = (c->delta[0] == c->delta[1] && c->delta[1] == c->delta[2] && c->opt.fixed_residual != 1)
                   ? (c->opt.fixed_residual == 2 ? 2 : 1)
                   : 0;
    P.fix_inv = inv2[0] / 180.0;
    P.dfix = c->opt.deterministic ? 1099511627776.0 : 0.0;  // 2^40
    P.st64.c0 = W[0] * (inv2[0] + inv2[1] + inv2[2]);
    for (int q = 1; q <= 3; ++q) {
        P.st64.cx[q - 1] = W[q] * inv2[0];
        P.st64.cy[q - 1] = W[q] * inv2[1];
        P.st64.cz[q - 1] = W[q] * inv2[2];
    }
    P.st32.c0 = (float)P.st64.c0;
    for (int q = 0; q < 3; ++q) {
        P.st32.cx[q] = (float)P.st64.cx[q];
        P.st32.cy[q] = (float)P.st64.cy[q];
        P.st32.cz[q] = (float)P.st64.cz[q];
    }
    for (int l = 0; l <= kMGMax; ++l) {
        const double s64 = std::ldexp(1.0, -2 * l);
        const float s32 = (float)s64;
        Stencil<double>& a = P.mg_a64[l];
        Stencil<float>& b = P.mg_a32[l];
        a.c0 = -P.st64.c0 * s64;
        b.c0 = -P.st32.c0 * s32;
        for (int q = 0; q < 3; ++q) {
            a.cx[q] = -P.st64.cx[q] * s64;
            a.cy[q] = -P.st64.cy[q] * s64;
            a.cz[q] = -P.st64.cz[q] * s64;
            b.cx[q] = -P.st32.cx[q] * s32;
            b.cy[q] = -P.st32.cy[q] * s32;
            b.cz[q] = -P.st32.cz[q] * s32;
        }
        P.mg_wd64[l] = P.mg_omega / a.c0;
        P.mg_wd32[l] = (float)P.mg_omega / b.c0;
    }
    P.geos = c->d_geos;
    P.n_geo = c->n_geo;
    P.S = S;
    P.Rc = Rc;
    P.S2 = (long long)S * S;
    P.ws = c->ws;
    P.slot_bytes = c->slot_bytes;
    P.tol = tol;
    P.max_iter = o.max_iter;
    P.inner_max_iter = o.inner_max_iter;
    P.inner_tol = o.inner_tol;
    P.max_refine = 40;
    P.update_drop = o.update_drop;
    P.lmax = l_max;
    P.n_mono = (l_max + 1) * (l_max + 2) * (l_max + 3) / 6;
    P.n_pair = c->d_scalars;
    P.queue = c->d_scalars + 1;
    P.nonconv = c->d_scalars + 2;
    P.timeouts = c->d_scalars + 10;  // [11]: non-finite inputs (pair list, E_xx reduction), [12]: clipped pairs
    P.dfix_range = c->d_scalars + 13;

    c->stats.n_pe = B.n_pe;
    c->stats.n_me = B.n_me;
    c->stats.solver_kind = (c->use_cluster || c->per_class || c->mg_C) ? 2 : 1;
    c->stats.cluster_size = c->use_cluster ? c->CL.C : (c->mg_C ? c->mg_C : 1);
    c->stats.grid_ctas = c->use_cluster ? c->n_clusters * c->CL.C
                                        : (c->mg_C ? std::min(c->mg_clusters, c->n_slots) * c->mg_C : c->n_slots);
    c->stats.lane_map = c->use_cluster ? c->cands[c->cand].lane_map : 0;
    c->stats.n_candidates = (int)c->cands.size();
    c->stats.threads = c->threads;
    *out = c;
    return EXX_OK;
}

static exx_status ensure_pairs(exx_ctx* c, int n) {
    if (n <= c->cap_n) return EXX_OK;
    drop_graph(c);
    free_pairs(c);
    const long long np = (long long)n * (n + 1) / 2;
    CK(cudaMalloc(&c->d_counts, sizeof(int) * (size_t)n), "cudaMalloc(counts)");
    CK(cudaMalloc(&c->d_offsets, sizeof(int) * (size_t)(n + 1)), "cudaMalloc(offsets)");
    CK(cudaMalloc(&c->d_pairs, sizeof(PairRec) * (size_t)np), "cudaMalloc(pairs)");
    CK(cudaMalloc(&c->d_epair, sizeof(double) * (size_t)np), "cudaMalloc(e_pair)");
    CK(cudaMalloc(&c->d_iters, sizeof(int) * (size_t)np), "cudaMalloc(iters)");
    CK(cudaMalloc(&c->d_refines, sizeof(int) * (size_t)np), "cudaMalloc(refines)");
    if (c->n_geo > 1) CK(cudaMalloc(&c->d_order, sizeof(int) * (size_t)np), "cudaMalloc(order)");
    c->cap_n = n;
    c->cap_pairs = np;
    return EXX_OK;
}

// The launch sequence of one call (captured into a graph when batched).
static exx_status enqueue(exx_ctx* c, const double* orbitals, const double* centers, const double* alphas, int n,
                          double* d_xx, cudaStream_t st, bool capturing) {
    // inside a capture a plain event record only expresses a dependency; the
    // external flag turns it into an event-record node that can be timed
    const unsigned evf = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    SolveParams P = c->P;
    P.phi = orbitals;
    P.dxx = d_xx;
    P.pairs = c->d_pairs;
    P.order = c->n_geo > 1 ? c->d_order : nullptr;
    P.e_pair = c->d_epair;
    P.iters = c->d_iters;
    P.refines = c->d_refines;
    P.dbg_b = nullptr;
    P.phase_clk = c->d_phase;
    P.test_wait = c->inject_now;
    P.box_org = c->cur_box;
    for (int a = 0; a < 3; ++a) P.bdim[a] = c->cur_bdim[a];
    P.ostride = c->cur_ostride;
    CK(cudaEventRecordWithFlags(c->ev[0], st, evf), "cudaEventRecord");
    CK(launch_zero(d_xx, (long long)n * c->cur_ostride, c->num_sms, st), "zero D_xx");
    CK(cudaMemsetAsync(c->d_scalars + 2, 0, sizeof(int), st), "reset counters");
    CK(cudaMemsetAsync(c->d_scalars + 10, 0, 4 * sizeof(int), st), "reset counters");
    CK(cudaMemsetAsync(c->d_phase, 0, sizeof(unsigned long long) * 4, st), "reset phase clocks");
    CK(launch_pair_list(n, centers, c->cell, c->delta, c->grid, c->r_pair, c->r_pe, c->r_me, c->d_counts,
                        c->d_offsets, c->d_scalars, c->d_scalars + 1, c->d_pairs, st,
                        c->opt.radii_mode == 1 ? alphas : nullptr, c->ln_inv_eps, c->delta_max, c->r_min, c->ns_pe,
                        c->ns_me, c->d_scalars + 11),
       "pair list");
    if (c->n_geo > 1)
        CK(launch_radii_sort(c->d_pairs, c->d_scalars, c->d_hist, c->n_geo, c->d_order, c->num_sms, st,
                             c->per_class ? c->d_class : nullptr),
           "largest-first order");
    if (c->cur_box)
        CK(launch_box_clip(c->d_pairs, c->d_scalars, c->cur_box, c->cur_bdim, c->grid, c->d_scalars + 12, c->num_sms,
                           st),
           "box check");
    CK(cudaEventRecordWithFlags(c->ev[1], st, evf), "cudaEventRecord");
    if (c->per_class) {
        // one launch per radius class, the largest radius first, alternating
        // between the two lanes; each takes its run of the sorted order from
        // the device (start, length, work counter)
        const bool two = c->aux != nullptr;
        if (two) {
            CK(cudaEventRecord(c->ev_fork, st), "cudaEventRecord(fork)");
            CK(cudaStreamWaitEvent(c->aux, c->ev_fork, 0), "cudaStreamWaitEvent(fork)");
        }
        for (int g = c->n_geo - 1; g >= 0; --g) {
            const exx_ctx::RadiusClass& RC = c->classes[g];
            const int lane = two ? (c->n_geo - 1 - g) & 1 : 0;
            cudaStream_t ls = lane ? c->aux : st;
            const int slots = two ? c->lane_slots[lane] : c->n_slots;
            SolveParams Pg = P;
            Pg.ws = c->ws + (size_t)(lane ? c->lane_slots[0] : 0) * c->slot_bytes;
            Pg.item_base = c->d_class + 2 * g;
            Pg.n_pair = c->d_class + 2 * g + 1;
            Pg.queue = c->d_class + 2 * c->n_geo + g;
            if (RC.kind == 2)
                CK(launch_cluster_kernel(RC.cand.variant, Pg, RC.cand.L, std::min(RC.cand.n_clusters, slots),
                                         RC.cand.smem, ls),
                   "cluster pair kernel (radius class)");
            else
                CK(launch_pair_kernel(Pg, c->threads, true, slots, c->smem, ls), "pair kernel (radius class)");
        }
        if (two) {
            CK(cudaEventRecord(c->ev_join, c->aux), "cudaEventRecord(join)");
            CK(cudaStreamWaitEvent(st, c->ev_join, 0), "cudaStreamWaitEvent(join)");
        }
    } else if (c->use_cluster)
        CK(launch_cluster_kernel(c->cl_variant, P, c->CL, c->n_clusters, c->smem, st), "cluster pair kernel");
    else if (c->mg_C)
        CK(launch_cluster_mg(c->mg_C, c->mg_minb, P, std::min(c->mg_clusters, c->n_slots), st),
           "cluster multigrid kernel");
    else
        CK(launch_pair_kernel(P, c->threads, c->opt.precision == 1, c->n_slots, c->smem, st), "pair kernel");
    if (P.dfix != 0.0)
        CK(launch_dfix_convert(d_xx, (long long)n * c->cur_ostride, 1.0 / P.dfix, c->num_sms, st), "D_xx to FP64");
    CK(cudaEventRecordWithFlags(c->ev[2], st, evf), "cudaEventRecord");
    CK(launch_exx_reduce(c->d_pairs, c->d_scalars, c->d_epair, c->d_exx, st, c->d_scalars + 11), "E_xx reduction");
    CK(cudaMemcpyAsync(c->h_exx, c->d_exx, sizeof(double), cudaMemcpyDeviceToHost, st), "copy E_xx");
    CK(cudaEventRecordWithFlags(c->ev[3], st, evf), "cudaEventRecord");
    return EXX_OK;
}

// Warm-start call: eager launches, because the potential cache is sized from
// this call's pair count. The cluster kernel starts each pair kept from the
// previous call (same i, j) from its cached potential, shifted by the move of
// the pair's grid centre, and caches the new potential for the next call.
static exx_status compute_warm(exx_ctx* c, const double* orbitals, const double* centers, const double* alphas,
                               int n, double* d_xx, cudaStream_t st) {
    SolveParams P = c->P;
    P.phi = orbitals;
    P.dxx = d_xx;
    P.pairs = c->d_pairs;
    P.order = nullptr;
    P.e_pair = c->d_epair;
    P.iters = c->d_iters;
    P.refines = c->d_refines;
    P.dbg_b = nullptr;
    P.phase_clk = c->d_phase;
    P.test_wait = c->inject_now;
    P.box_org = c->cur_box;
    for (int a = 0; a < 3; ++a) P.bdim[a] = c->cur_bdim[a];
    P.ostride = c->cur_ostride;
    CK(cudaEventRecord(c->ev[0], st), "cudaEventRecord");
    CK(launch_zero(d_xx, (long long)n * c->cur_ostride, c->num_sms, st), "zero D_xx");
    CK(cudaMemsetAsync(c->d_scalars + 2, 0, sizeof(int), st), "reset counters");
    CK(cudaMemsetAsync(c->d_scalars + 10, 0, 4 * sizeof(int), st), "reset counters");
    CK(cudaMemsetAsync(c->d_phase, 0, sizeof(unsigned long long) * 4, st), "reset phase clocks");
    CK(launch_pair_list(n, centers, c->cell, c->delta, c->grid, c->r_pair, c->r_pe, c->r_me, c->d_counts,
                        c->d_offsets, c->d_scalars, c->d_scalars + 1, c->d_pairs, st, nullptr, c->ln_inv_eps,
                        c->delta_max, c->r_min, 0, 0, c->d_scalars + 11),
       "pair list");
    if (c->cur_box)
        CK(launch_box_clip(c->d_pairs, c->d_scalars, c->cur_box, c->cur_bdim, c->grid, c->d_scalars + 12, c->num_sms,
                           st),
           "box check");
    int np = 0;
    CK(cudaMemcpyAsync(&np, c->d_scalars, sizeof(int), cudaMemcpyDeviceToHost, st), "read n_pair");
    CK(cudaStreamSynchronize(st), "warm start synchronize");
    if (np > c->vcache_pairs) {  // grow the caches (the previous potentials are lost)
        cudaFree(c->d_vcache[0]);
        cudaFree(c->d_vcache[1]);
        c->d_vcache[0] = c->d_vcache[1] = nullptr;
        c->vcache_pairs = 0;
        c->have_prev = false;
        const long long want = (long long)(1.25 * np) + 16;
        const size_t bytes = sizeof(float) * (size_t)want * c->hb.n_pe;
        CK(cudaMalloc(&c->d_vcache[0], bytes), "cudaMalloc(warm-start cache)");
        CK(cudaMalloc(&c->d_vcache[1], bytes), "cudaMalloc(warm-start cache)");
        c->vcache_pairs = want;
    }
    if (np > c->prev_cap) {
        cudaFree(c->d_prev_pairs);
        c->d_prev_pairs = nullptr;
        c->have_prev = false;
        c->prev_cap = 0;
        CK(cudaMalloc(&c->d_prev_pairs, sizeof(PairRec) * (size_t)c->cap_pairs), "cudaMalloc(previous pairs)");
        c->prev_cap = c->cap_pairs;
    }
    if (c->opt.warm_start == 3) {  // history for the extrapolation, sized like the previous call's cache
        const size_t vbytes = sizeof(float) * (size_t)c->vcache_pairs * c->hb.n_pe;
        for (int h = 0; h < 2; ++h) {
            if (!c->hv[h] || c->hv_pairs < c->vcache_pairs) {
                cudaFree(c->hv[h]);
                c->hv[h] = nullptr;
                CK(cudaMalloc(&c->hv[h], vbytes), "cudaMalloc(extrapolation history)");
                c->hk = 0;
            }
            if (!c->hp[h] || c->hp_cap < c->prev_cap) {
                cudaFree(c->hp[h]);
                c->hp[h] = nullptr;
                CK(cudaMalloc(&c->hp[h], sizeof(PairRec) * (size_t)c->prev_cap), "cudaMalloc(extrapolation history)");
                c->hk = 0;
            }
        }
        c->hv_pairs = c->vcache_pairs;
        c->hp_cap = c->prev_cap;
        if (!c->have_prev) c->hk = 0;
    }
    P.warm = c->have_prev ? (c->opt.warm_start == 3 ? 3 : 1) : 0;
    P.prev_pairs = c->d_prev_pairs;
    P.xk = c->have_prev ? 1 + c->hk : 0;
    P.xv[0] = c->d_vcache[c->parity ^ 1];
    P.xp[0] = c->d_prev_pairs;
    P.xn[0] = c->d_scalars + 7;
    for (int h = 0; h < 2; ++h) {
        P.xv[h + 1] = c->hv[h];
        P.xp[h + 1] = c->hp[h];
        P.xn[h + 1] = c->d_scalars + 8 + h;
    }
    P.n_prev = c->d_scalars + 7;
    P.vprev = c->d_vcache[c->parity ^ 1];
    P.vcur = c->d_vcache[c->parity];
    if (c->opt.warm_start == 2) {
        // learned guesses: the network runs on batches of pairs, its output
        // is scattered to each pair's PE points and the CG starts from it
        exx::unet::Net& net = *c->gnet;
        if (np > c->guess_cap) {
            cudaFree(c->d_guess);
            c->d_guess = nullptr;
            c->guess_cap = 0;
            const long long want = (long long)(1.25 * np) + 16;
            CK(cudaMalloc(&c->d_guess, sizeof(float) * (size_t)want * c->hb.n_pe), "cudaMalloc(learned guesses)");
            c->guess_cap = want;
        }
        const double d2 = std::cbrt(c->delta[0] * c->delta[0] * c->delta[1] * c->delta[1] * c->delta[2] * c->delta[2]);
        CK(cudaEventRecord(c->ev_g[0], st), "cudaEventRecord");
        for (int k0 = 0; k0 < np; k0 += net.Bmax) {
            const int nk = std::min(net.Bmax, np - k0);
            CK(exx::unet::sample_prep(orbitals, c->grid, c->d_pairs, k0, nk, net.S, c->geo_host, c->d_gin,
                                      c->d_gscale, nullptr, nullptr, d2, c->delta, c->dV, c->lmax, c->cur_box,
                                      c->cur_bdim, c->cur_ostride, st),
               "guess input");
            CK(exx::unet::forward(net, c->d_gin, nk, st), "guess network");
            CK(exx::unet::guess_scatter(net.out, c->d_gscale, k0, nk, net.S, c->geo_host, d2, c->d_guess, st),
               "guess scatter");
        }
        CK(cudaEventRecord(c->ev_g[1], st), "cudaEventRecord");
        P.warm = 2;
        P.vprev = c->d_guess;
    }
    CK(cudaEventRecord(c->ev[1], st), "cudaEventRecord");
    CK(launch_cluster_kernel(c->cl_variant, P, c->CL, c->n_clusters, c->smem, st), "cluster pair kernel");
    if (P.dfix != 0.0)
        CK(launch_dfix_convert(d_xx, (long long)n * c->cur_ostride, 1.0 / P.dfix, c->num_sms, st), "D_xx to FP64");
    CK(cudaEventRecord(c->ev[2], st), "cudaEventRecord");
    CK(launch_exx_reduce(c->d_pairs, c->d_scalars, c->d_epair, c->d_exx, st, c->d_scalars + 11), "E_xx reduction");
    CK(cudaMemcpyAsync(c->h_exx, c->d_exx, sizeof(double), cudaMemcpyDeviceToHost, st), "copy E_xx");
    if (c->opt.warm_start == 3 && c->have_prev) {
        // the previous call moves one level back in the history (pointer
        // swaps; the oldest buffers are recycled for this call's successors)
        CK(cudaMemcpyAsync(c->d_scalars + 9, c->d_scalars + 8, sizeof(int), cudaMemcpyDeviceToDevice, st),
           "history counts");
        CK(cudaMemcpyAsync(c->d_scalars + 8, c->d_scalars + 7, sizeof(int), cudaMemcpyDeviceToDevice, st),
           "history counts");
        float* tv = c->hv[1];
        c->hv[1] = c->hv[0];
        c->hv[0] = c->d_vcache[c->parity ^ 1];
        c->d_vcache[c->parity ^ 1] = tv;
        PairRec* tp = c->hp[1];
        c->hp[1] = c->hp[0];
        c->hp[0] = c->d_prev_pairs;
        c->d_prev_pairs = tp;
        c->hk = std::min(c->hk + 1, 2);
    }
    // this call's list becomes the previous one
    CK(cudaMemcpyAsync(c->d_prev_pairs, c->d_pairs, sizeof(PairRec) * (size_t)np, cudaMemcpyDeviceToDevice, st),
       "keep pair list");
    CK(cudaMemcpyAsync(c->d_scalars + 7, c->d_scalars, sizeof(int), cudaMemcpyDeviceToDevice, st), "keep n_pair");
    CK(cudaEventRecord(c->ev[3], st), "cudaEventRecord");
    c->parity ^= 1;
    c->have_prev = true;
    if (c->opt.warm_start == 2) {
        int h = 0;
        CK(cudaMemcpyAsync(&h, c->gnet->d_err, sizeof(int), cudaMemcpyDeviceToHost, st), "guess status");
        CK(cudaStreamSynchronize(st), "guess status");
        if (h) return fail(c, EXX_ETIMEOUT, "exx_compute: a tensor-core wait of the guess network timed out");
        float ms = 0.f;
        c->guess_ms = cudaEventElapsedTime(&ms, c->ev_g[0], c->ev_g[1]) == cudaSuccess ? ms : -1.0;
    }
    return EXX_OK;
}

// Choices of the autotuner, kept for the process: contexts with the same grid,
// radii and solver options build the same candidate list and reuse the
// first context's choice (consistent launch shapes, no repeated tuning).
struct TuneKey {
    double cell[3], delta[3], r_pair, update_drop;
    int grid[3], r_pe, r_me, precision, cluster_size, threads, lane_map, radii_mode, n_cands;
    bool operator==(const TuneKey& o) const { return std::memcmp(this, &o, sizeof(TuneKey)) == 0; }
};
static std::mutex g_tune_mu;
static std::vector<std::pair<TuneKey, int>> g_tune_cache;

static TuneKey tune_key(const exx_ctx* c) {
    TuneKey k;
    std::memset(&k, 0, sizeof(k));
    for (int a = 0; a < 3; ++a) {
        k.cell[a] = c->cell[a];
        k.delta[a] = c->delta[a];
        k.grid[a] = c->grid[a];
    }
    k.r_pair = c->r_pair;
    k.update_drop = c->opt.update_drop;
    k.r_pe = c->r_pe;
    k.r_me = c->r_me;
    k.precision = c->opt.precision;
    k.cluster_size = c->opt.cluster_size;
    k.threads = c->opt.threads;
    k.lane_map = c->opt.lane_map;
    k.radii_mode = c->opt.radii_mode;
    k.n_cands = (int)c->cands.size();
    return k;
}

// The autotuner: on the first call, every cluster-solver candidate processes
// the same prefix of the pair queue (no D_xx scatter); the one with the most
// pairs per second is kept for the life of the context (and for later
// contexts with the same key).
static exx_status autotune(exx_ctx* c, const double* orbitals, const double* centers, const double* alphas, int n,
                           cudaStream_t st) {
    const TuneKey key = tune_key(c);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (const auto& e : g_tune_cache)
            if (e.first == key && e.second >= 0 && e.second < (int)c->cands.size()) {
                apply_cand(c, e.second);
                c->tuned = true;
                c->tune_ms = 0.0;
                drop_graph(c);
                return EXX_OK;
            }
    }
    CK(launch_pair_list(n, centers, c->cell, c->delta, c->grid, c->r_pair, c->r_pe, c->r_me, c->d_counts,
                        c->d_offsets, c->d_scalars, c->d_scalars + 1, c->d_pairs, st,
                        c->opt.radii_mode == 1 ? alphas : nullptr, c->ln_inv_eps, c->delta_max, c->r_min, c->ns_pe,
                        c->ns_me),
       "pair list (autotune)");
    int np = 0;
    CK(cudaMemcpyAsync(&np, c->d_scalars, sizeof(int), cudaMemcpyDeviceToHost, st), "read n_pair");
    CK(cudaStreamSynchronize(st), "autotune synchronize");
    int widest = 1;
    for (const auto& K : c->cands) widest = std::max(widest, std::min(K.n_clusters, c->n_slots));
    const int K = std::max(1, std::min(np, 8 * widest));  // 8 pairs per cluster: tail and noise small
    CK(cudaMemcpy(c->d_scalars + 4, &K, sizeof(int), cudaMemcpyHostToDevice), "tuning count");
    SolveParams P = c->P;
    P.phi = orbitals;
    P.dxx = nullptr;
    P.box_org = c->cur_box;
    for (int a = 0; a < 3; ++a) P.bdim[a] = c->cur_bdim[a];
    P.ostride = c->cur_ostride;
    P.pairs = c->d_pairs;
    P.order = nullptr;
    P.e_pair = c->d_epair;
    P.iters = c->d_iters;
    P.refines = c->d_refines;
    P.dbg_b = nullptr;
    P.phase_clk = nullptr;
    P.n_pair = c->d_scalars + 4;
    P.queue = c->d_scalars + 5;
    P.nonconv = c->d_scalars + 6;
    int best = c->cand;
    double best_rate = -1.0;
    auto t_start = std::chrono::steady_clock::now();
    for (int k = 0; k < (int)c->cands.size(); ++k) {
        apply_cand(c, k);
        float ms = 0.f;
        for (int rep = 0; rep < 2; ++rep) {  // the first launch also loads the kernel
            CK(cudaMemsetAsync(c->d_scalars + 5, 0, sizeof(int), st), "tuning queue");
            CK(cudaEventRecord(c->ev[1], st), "cudaEventRecord");
            CK(launch_cluster_kernel(c->cl_variant, P, c->CL, c->n_clusters, c->smem, st), "autotune launch");
            CK(cudaEventRecord(c->ev[2], st), "cudaEventRecord");
            CK(cudaStreamSynchronize(st), "autotune synchronize");
            CK(cudaEventElapsedTime(&ms, c->ev[1], c->ev[2]), "autotune timing");
        }
        c->cands[k].pairs_per_s = K / (ms * 1e-3);
        if (c->cands[k].pairs_per_s > best_rate) {
            best_rate = c->cands[k].pairs_per_s;
            best = k;
        }
    }
    apply_cand(c, best);
    c->tuned = true;
    c->tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache.push_back({key, best});
    }
    drop_graph(c);
    return EXX_OK;
}

// exx_compute and exx_compute_boxes: box = NULL for full grids, else the
// boxes' corners (device, [n][3]) and their dimensions (host, 3 ints).
static exx_status finish_stats(exx_ctx* c, bool box);

// After an exx_compute_async call: waits for its work and reads its counters
// (its outcome stays in them; a call's status is not returned here).
static cudaError_t wait_pending(exx_ctx* c) {
    if (!c->stats_pending) return cudaSuccess;
    const cudaError_t e = cudaStreamSynchronize(c->work);
    if (e != cudaSuccess) return e;
    (void)finish_stats(c, c->pending_box);
    return cudaSuccess;
}

// One call. With e_xx_dev set (exx_compute_async) E_xx goes to that device
// double and the call returns without waiting for its work; else E_xx goes to
// *e_xx on the host after the work has finished.
static exx_status compute_impl(exx_ctx* c, const double* orbitals, const double* centers, int n, const double* alphas,
                               double* e_xx, double* d_xx, void* stream, const int* box, const int* bdim,
                               double* e_xx_dev = nullptr) {
    if (!c) return fail(nullptr, EXX_EINVAL, "exx_compute: ctx is NULL");
    if (!orbitals || !centers || !(e_xx || e_xx_dev) || !d_xx)
        return fail(c, EXX_EINVAL, "exx_compute: NULL array argument");
    if (n < 1 || n > 65535) return fail(c, EXX_EINVAL, "exx_compute: n must be in [1, 65535]");
    if ((const void*)orbitals == (const void*)d_xx) return fail(c, EXX_EINVAL, "exx_compute: d_xx aliases orbitals");
    if (c->opt.radii_mode == 1 && !alphas)
        return fail(c, EXX_EINVAL, "exx_compute: radii_mode 1 needs the orbital exponents (alphas)");
    if (((reinterpret_cast<uintptr_t>(orbitals) | reinterpret_cast<uintptr_t>(centers) |
          reinterpret_cast<uintptr_t>(d_xx) | reinterpret_cast<uintptr_t>(alphas)) & 7u) != 0)
        return fail(c, EXX_EINVAL, "exx_compute: arrays must be 8-byte aligned");
    cudaStream_t user = (cudaStream_t)stream;
    c->cur_box = box;
    for (int a = 0; a < 3; ++a) c->cur_bdim[a] = box ? bdim[a] : 0;
    c->cur_ostride = box ? (long long)bdim[0] * bdim[1] * bdim[2] : c->ngrid;
    exx_status s = ensure_pairs(c, n);
    if (s != EXX_OK) return s;
    // all work runs on the context's stream, ordered after the caller's stream
    cudaStream_t st = c->work;
    CK(cudaEventRecord(c->ev_in, user), "cudaEventRecord(caller stream)");
    CK(cudaStreamWaitEvent(st, c->ev_in, 0), "cudaStreamWaitEvent");
    if (c->opt.warm_start == 2 && !c->gnet)
        return fail(c, EXX_EINVAL, "exx_compute: warm_start 2 needs a model (exx_load_guess_model)");
    if (c->use_cluster && !c->tuned) {
        s = autotune(c, orbitals, centers, alphas, n, st);
        if (s != EXX_OK) return s;
    }
    cudaError_t e;
    c->inject_now = c->inject_left > 0 ? 1 : 0;
    if (c->inject_now) --c->inject_left;
    if (c->opt.warm_start) {
        s = compute_warm(c, orbitals, centers, alphas, n, d_xx, st);
        if (s != EXX_OK) return s;
    } else if (c->opt.batched) {
        const void* key[5] = {orbitals, centers, d_xx, alphas, box};
        bool hit = c->gexec && c->g_n == n && std::equal(key, key + 5, c->g_key) && c->g_inject == c->inject_now &&
                   std::equal(c->cur_bdim, c->cur_bdim + 3, c->g_bdim);
        if (!hit) {
            drop_graph(c);
            cudaGraph_t g;
            e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamBeginCapture");
            s = enqueue(c, orbitals, centers, alphas, n, d_xx, st, true);
            e = cudaStreamEndCapture(st, &g);
            if (s != EXX_OK) {
                if (e == cudaSuccess) cudaGraphDestroy(g);
                return s;
            }
            if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&c->gexec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                c->gexec = nullptr;
                return cuda_fail(c, e, "cudaGraphInstantiate");
            }
            std::copy(key, key + 5, c->g_key);
            c->g_n = n;
            c->g_inject = c->inject_now;
            std::copy(c->cur_bdim, c->cur_bdim + 3, c->g_bdim);
        }
        e = cudaGraphLaunch(c->gexec, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphLaunch");
    } else {
        s = enqueue(c, orbitals, centers, alphas, n, d_xx, st, false);
        if (s != EXX_OK) return s;
    }
    if (e_xx_dev)
        CK(cudaMemcpyAsync(e_xx_dev, c->d_exx, sizeof(double), cudaMemcpyDeviceToDevice, st), "copy E_xx (device)");
    CK(cudaEventRecord(c->ev_out, st), "cudaEventRecord(done)");
    CK(cudaStreamWaitEvent(user, c->ev_out, 0), "cudaStreamWaitEvent(caller stream)");
    c->last_n = n;
    c->last_orb = orbitals;
    if (e_xx_dev) {  // no host synchronisation: the counters wait for exx_get_stats
        c->stats_pending = true;
        c->pending_box = box != nullptr;
        return EXX_OK;
    }
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "exx_compute (stream synchronize)");
    *e_xx = c->h_exx[0];
    return finish_stats(c, box != nullptr);
}

// Timings and counters of the last call, once its work has finished; the
// call's status from them (EXX_EINVAL for dropped deterministic D_xx
// contributions, EXX_ETIMEOUT, EXX_ENOCONV).
static exx_status finish_stats(exx_ctx* c, bool box) {
    c->stats_pending = false;
    float ms = 0.f;
    c->stats.solve_ms = cudaEventElapsedTime(&ms, c->ev[1], c->ev[2]) == cudaSuccess ? ms : -1.0;
    c->stats.total_ms = cudaEventElapsedTime(&ms, c->ev[0], c->ev[3]) == cudaSuccess ? ms : -1.0;
    (void)cudaGetLastError();  // a failed timing query must not leak into later status checks
    int sc[14];
    CK(cudaMemcpy(sc, c->d_scalars, sizeof(sc), cudaMemcpyDeviceToHost), "read counters");
    const int npair = sc[0], nonconv = sc[2];
    c->stats.n_pair = npair;
    c->stats.n_nonconv = nonconv;
    c->stats.n_timeouts = sc[10];
    c->stats.n_nonfinite = sc[11];
    c->stats.n_clipped = box ? sc[12] : 0;
    c->stats.n_dropped = sc[13];
    c->stats.iters_max = -1;  // filled lazily by exx_get_stats
    if (sc[13] > 0) {
        char buf[200];
        std::snprintf(buf, sizeof(buf),
                      "deterministic D_xx: %d contributions |v phi| >= 2^22 lie beyond the fixed-point range and were "
                      "dropped (D_xx incomplete; use deterministic = 0)",
                      sc[13]);
        return fail(c, EXX_EINVAL, buf);
    }
    if (sc[10] > 0) {
        char buf[160];
        std::snprintf(buf, sizeof(buf), "%d bounded device waits ran out (results written, not to be trusted)",
                      sc[10]);
        return fail(c, EXX_ETIMEOUT, buf);
    }
    if (nonconv > 0) {
        char buf[128];
        std::snprintf(buf, sizeof(buf), "%d of %d pair solves reached the iteration cap", nonconv, npair);
        return fail(c, EXX_ENOCONV, buf);
    }
    return EXX_OK;
}

extern "C" exx_status exx_compute(exx_ctx* c, const double* orbitals, const double* centers, int n,
                                  const double* alphas, double* e_xx, double* d_xx, void* stream) {
    return compute_impl(c, orbitals, centers, n, alphas, e_xx, d_xx, stream, nullptr, nullptr);
}

extern "C" exx_status exx_compute_async(exx_ctx* c, const double* orbitals, const double* centers, int n,
                                        const double* alphas, double* e_xx_dev, double* d_xx, void* stream) {
    if (!c) return fail(nullptr, EXX_EINVAL, "exx_compute_async: ctx is NULL");
    if (!e_xx_dev || (reinterpret_cast<uintptr_t>(e_xx_dev) & 7u) != 0)
        return fail(c, EXX_EINVAL, "exx_compute_async: e_xx_dev must be an 8-byte aligned device pointer");
    if (c->opt.warm_start != 0)
        return fail(c, EXX_EINVAL, "exx_compute_async: warm starts need exx_compute (host-side bookkeeping)");
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, e_xx_dev) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
        (void)cudaGetLastError();
        return fail(c, EXX_EINVAL, "exx_compute_async: e_xx_dev must be device memory");
    }
    return compute_impl(c, orbitals, centers, n, alphas, nullptr, d_xx, stream, nullptr, nullptr, e_xx_dev);
}

extern "C" exx_status exx_compute_boxes(exx_ctx* c, const double* boxes, const int* origin, const int box_dim[3],
                                        const double* centers, int n, const double* alphas, double* e_xx,
                                        double* d_boxes, void* stream) {
    if (!c) return fail(nullptr, EXX_EINVAL, "exx_compute_boxes: ctx is NULL");
    if (!origin || !box_dim) return fail(c, EXX_EINVAL, "exx_compute_boxes: NULL origin or box_dim");
    if ((reinterpret_cast<uintptr_t>(origin) & 3u) != 0)
        return fail(c, EXX_EINVAL, "exx_compute_boxes: origin must be 4-byte aligned");
    for (int a = 0; a < 3; ++a)
        if (box_dim[a] < 2 * c->r_me + 1 || box_dim[a] > c->grid[a])
            return fail(c, EXX_EINVAL, "exx_compute_boxes: box_dim must be in [2 r_me + 1, N] on every axis");
    return compute_impl(c, boxes, centers, n, alphas, e_xx, d_boxes, stream, origin, box_dim);
}

// The device address of pinned, device-mapped host memory at p (the whole
// range [p, p + bytes) inside one such allocation), or NULL for any other memory.
static void* mapped_host(const void* p, size_t bytes) {
    if (bytes == 0) return nullptr;
    cudaPointerAttributes a0, a1;
    if (cudaPointerGetAttributes(&a0, p) != cudaSuccess ||
        cudaPointerGetAttributes(&a1, (const char*)p + (bytes - 1)) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    if (a0.type != cudaMemoryTypeHost || a1.type != cudaMemoryTypeHost || !a0.devicePointer || !a1.devicePointer)
        return nullptr;
    // both ends mapped by one contiguous mapping
    if ((const char*)a1.devicePointer != (const char*)a0.devicePointer + (bytes - 1)) return nullptr;
    return a0.devicePointer;
}

static cudaError_t copy_from_host(exx_ctx* c, const void* host, void* dev, size_t bytes, cudaStream_t st) {
    void* mp = mapped_host(host, bytes);
    if (mp && bytes % 16 == 0 && ((uintptr_t)mp & 15u) == 0 && ((uintptr_t)dev & 15u) == 0)
        return launch_copy16(mp, dev, (long long)(bytes / 16), c->num_sms, st);
    return cudaMemcpyAsync(dev, host, bytes, cudaMemcpyHostToDevice, st);
}

static cudaError_t copy_to_host(exx_ctx* c, const void* dev, void* host, size_t bytes, cudaStream_t st) {
    void* mp = mapped_host(host, bytes);
    if (mp && bytes % 16 == 0 && ((uintptr_t)mp & 15u) == 0 && ((uintptr_t)dev & 15u) == 0)
        return launch_copy16(dev, mp, (long long)(bytes / 16), c->num_sms, st);
    return cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, st);
}

extern "C" exx_status exx_compute_host(exx_ctx* c, const double* orbitals_host, const double* centers_host, int n,
                                       const double* alphas_host, double* e_xx, double* d_xx_host, void* stream) {
    if (!c) return fail(nullptr, EXX_EINVAL, "exx_compute_host: ctx is NULL");
    if (!orbitals_host || !centers_host || !e_xx || !d_xx_host)
        return fail(c, EXX_EINVAL, "exx_compute_host: NULL array argument");
    if (n < 1 || n > 65535) return fail(c, EXX_EINVAL, "exx_compute_host: n must be in [1, 65535]");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = sizeof(double) * (size_t)n * (size_t)c->ngrid;
    if (bytes > c->host_cap_bytes || n > c->host_cap_n) {
        drop_graph(c);
        cudaFree(c->d_orb);
        cudaFree(c->d_dxx);
        cudaFree(c->d_cent);
        cudaFree(c->d_alpha);
        c->d_orb = c->d_dxx = c->d_cent = c->d_alpha = nullptr;
        c->host_cap_bytes = 0;
        c->host_cap_n = 0;
        CK(cudaMalloc(&c->d_orb, bytes), "cudaMalloc(orbitals copy)");
        CK(cudaMalloc(&c->d_dxx, bytes), "cudaMalloc(d_xx copy)");
        CK(cudaMalloc(&c->d_cent, sizeof(double) * 3 * (size_t)n), "cudaMalloc(centers copy)");
        CK(cudaMalloc(&c->d_alpha, sizeof(double) * (size_t)n), "cudaMalloc(alphas copy)");
        c->host_cap_bytes = bytes;
        c->host_cap_n = n;
    }
    // the orbitals: read by the SMs straight from pinned, device-mapped host
    // memory when the buffer is such (on the GB300's chip-to-chip link this
    // outruns the copy engine, measured), else by a copy-engine copy
    CK(copy_from_host(c, orbitals_host, c->d_orb, bytes, st), "copy orbitals");
    CK(cudaMemcpyAsync(c->d_cent, centers_host, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice, st),
       "copy centers");
    if (alphas_host)
        CK(cudaMemcpyAsync(c->d_alpha, alphas_host, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, st),
           "copy alphas");
    exx_status s = exx_compute(c, c->d_orb, c->d_cent, n, alphas_host ? c->d_alpha : nullptr, e_xx, c->d_dxx, stream);
    if (s != EXX_OK && s != EXX_ENOCONV && s != EXX_ETIMEOUT) return s;
    CK(copy_to_host(c, c->d_dxx, d_xx_host, bytes, st), "copy d_xx");
    CK(cudaStreamSynchronize(st), "exx_compute_host (stream synchronize)");
    return s;
}

extern "C" exx_status exx_get_stats(const exx_ctx* cc, exx_stats* out) {
    exx_ctx* c = const_cast<exx_ctx*>(cc);
    if (!c || !out) return fail(c, EXX_EINVAL, "exx_get_stats: NULL argument");
    CK(wait_pending(c), "exx_get_stats (waiting for the last call)");
    if (c->stats.iters_max < 0 && c->stats.n_pair > 0) {
        const int np = c->stats.n_pair;
        std::vector<int> it(np), rf(np);
        std::vector<PairRec> pr(np);
        CK(cudaMemcpy(it.data(), c->d_iters, sizeof(int) * np, cudaMemcpyDeviceToHost), "read iters");
        CK(cudaMemcpy(rf.data(), c->d_refines, sizeof(int) * np, cudaMemcpyDeviceToHost), "read refines");
        CK(cudaMemcpy(pr.data(), c->d_pairs, sizeof(PairRec) * np, cudaMemcpyDeviceToHost), "read pairs");
        long long tot = 0, pit = 0;
        int rmax = 0;
        for (int p = 0; p < np; ++p) {
            tot += it[p];
            const int g = std::min(std::max(pr[p].geo, 0), c->n_geo - 1);
            pit += (long long)it[p] * c->balls[g].n_pe;
            rmax = std::max(rmax, rf[p]);
        }
        std::vector<int> srt = it;
        std::sort(srt.begin(), srt.end());
        c->stats.iters_total = tot;
        c->stats.point_iters = pit;
        c->stats.iters_max = srt.back();
        c->stats.iters_p50 = srt[(np - 1) / 2];
        c->stats.iters_p99 = srt[std::min(np - 1, (int)std::ceil(0.99 * np) - 1)];
        c->stats.refine_max = rmax;
        unsigned long long ph[4] = {0, 0, 0, 0};
        CK(cudaMemcpy(ph, c->d_phase, sizeof(ph), cudaMemcpyDeviceToHost), "read phase clocks");
        // shares of the pair-kernel time (the clusters run side by side)
        const double cyc = (double)ph[0] + (double)ph[1] + (double)ph[2] + (double)ph[3];
        for (int k = 0; k < 4; ++k)
            c->stats.phase_ms[k] = cyc > 0.0 ? c->stats.solve_ms * (double)ph[k] / cyc : 0.0;
    }
    if (c->per_class) {  // radius classes: the largest cluster and grid of any class
        int cmax = 1, gmax = c->n_slots;
        for (const auto& RC : c->classes)
            if (RC.kind == 2) {
                cmax = std::max(cmax, RC.cand.C);
                gmax = std::max(gmax, std::min(RC.cand.n_clusters, c->n_slots) * RC.cand.C);
            }
        c->stats.solver_kind = 2;
        c->stats.cluster_size = cmax;
        c->stats.grid_ctas = gmax;
        c->stats.threads = 512;
        c->stats.lane_map = 5;
    }
    if (c->use_cluster) {
        c->stats.solver_kind = 2;
        c->stats.cluster_size = c->CL.C;
        c->stats.grid_ctas = c->n_clusters * c->CL.C;
        c->stats.threads = c->threads;
        c->stats.lane_map = c->cands[c->cand].lane_map;
        c->stats.tune_ms = c->tune_ms;
        c->stats.guess_ms = c->opt.warm_start == 2 ? c->guess_ms : 0.0;
    }
    *out = c->stats;
    if (out->iters_max < 0) out->iters_max = 0;
    return EXX_OK;
}

extern "C" exx_status exx_get_pairs(const exx_ctx* cc, int* pi, int* pj, int* g, int* radii, double* e_pair,
                                    int* iters, int cap, int* n_pair) {
    exx_ctx* c = const_cast<exx_ctx*>(cc);
    if (!c) return fail(nullptr, EXX_EINVAL, "exx_get_pairs: ctx is NULL");
    CK(wait_pending(c), "exx_get_pairs (waiting for the last call)");
    const int np = c->stats.n_pair;
    if (n_pair) *n_pair = np;
    if (np > cap && (pi || pj || g || radii || e_pair || iters))
        return fail(c, EXX_EINVAL, "exx_get_pairs: cap smaller than the pair count");
    if (np == 0) return EXX_OK;
    std::vector<PairRec> pr(np);
    CK(cudaMemcpy(pr.data(), c->d_pairs, sizeof(PairRec) * np, cudaMemcpyDeviceToHost), "read pairs");
    for (int p = 0; p < np; ++p) {
        if (pi) pi[p] = pr[p].i;
        if (pj) pj[p] = pr[p].j;
        if (g)
            for (int a = 0; a < 3; ++a) g[3 * p + a] = pr[p].g[a];
        if (radii) {
            radii[2 * p] = pr[p].r_pe;
            radii[2 * p + 1] = pr[p].r_me;
        }
    }
    if (e_pair) CK(cudaMemcpy(e_pair, c->d_epair, sizeof(double) * np, cudaMemcpyDeviceToHost), "read e_pair");
    if (iters) CK(cudaMemcpy(iters, c->d_iters, sizeof(int) * np, cudaMemcpyDeviceToHost), "read iters");
    return EXX_OK;
}

extern "C" exx_status exx_debug_pair(exx_ctx* c, const double* orbitals, int index, double* rho, double* v, double* b,
                                     void* stream) {
    if (!c) return fail(nullptr, EXX_EINVAL, "exx_debug_pair: ctx is NULL");
    if (!orbitals) return fail(c, EXX_EINVAL, "exx_debug_pair: orbitals is NULL");
    CK(wait_pending(c), "exx_debug_pair (waiting for the last call)");
    if (index < 0 || index >= c->stats.n_pair) return fail(c, EXX_ENOPAIR, "exx_debug_pair: index out of range");
    (void)cudaGetLastError();
    cudaStream_t st = (cudaStream_t)stream;
    const HostBall& B = c->hb;
    PairRec pr;
    CK(cudaMemcpy(&pr, c->d_pairs + index, sizeof(PairRec), cudaMemcpyDeviceToHost), "read pair");
    // a one-pair list in the spare tail of the scalars block
    PairRec* d_one = nullptr;
    double *d_rho = nullptr, *d_v = nullptr, *d_b = nullptr, *d_e = nullptr;
    int* d_sc = nullptr;
    CK(cudaMalloc(&d_one, sizeof(PairRec)), "cudaMalloc");
    CK(cudaMalloc(&d_rho, sizeof(double) * B.n_me), "cudaMalloc");
    CK(cudaMalloc(&d_v, sizeof(double) * B.n_me), "cudaMalloc");
    CK(cudaMalloc(&d_b, sizeof(double) * B.n_pe), "cudaMalloc");
    CK(cudaMalloc(&d_e, sizeof(double) * 2), "cudaMalloc");
    CK(cudaMalloc(&d_sc, sizeof(int) * 8), "cudaMalloc");
    int sc[8] = {1, 0, 0, 0, 0, 0, 0, 0};
    CK(cudaMemcpy(d_one, &pr, sizeof(PairRec), cudaMemcpyHostToDevice), "copy pair");
    CK(cudaMemcpy(d_sc, sc, sizeof(sc), cudaMemcpyHostToDevice), "copy scalars");
    SolveParams P = c->P;
    P.phi = orbitals;  // stored as in the last call (full grids or compact boxes)
    P.dxx = nullptr;
    P.box_org = c->cur_box;
    for (int a = 0; a < 3; ++a) P.bdim[a] = c->cur_bdim[a];
    P.ostride = c->cur_ostride ? c->cur_ostride : c->ngrid;
    P.pairs = d_one;
    P.n_pair = d_sc;
    P.queue = d_sc + 1;
    P.nonconv = d_sc + 2;
    P.order = nullptr;
    P.e_pair = d_e;
    P.iters = d_sc + 3;
    P.refines = d_sc + 4;
    P.dbg_b = d_b;
    exx_status s = EXX_OK;
    cudaError_t e = c->use_cluster ? launch_cluster_kernel(c->cl_variant, P, c->CL, 1, c->smem, st)
                                   : launch_pair_kernel(P, c->threads, c->opt.precision == 1, 1, c->smem, st);
    if (e == cudaSuccess) e = launch_debug_readback(P, pr, d_rho, d_v, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && rho) e = cudaMemcpy(rho, d_rho, sizeof(double) * B.n_me, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && v) e = cudaMemcpy(v, d_v, sizeof(double) * B.n_me, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && b) e = cudaMemcpy(b, d_b, sizeof(double) * B.n_pe, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) s = cuda_fail(c, e, "exx_debug_pair");
    cudaFree(d_one);
    cudaFree(d_rho);
    cudaFree(d_v);
    cudaFree(d_b);
    cudaFree(d_e);
    cudaFree(d_sc);
    return s;
}

extern "C" exx_status exx_apply_operator(exx_ctx* c, const double* p, double* ap, void* stream) {
    if (!c) return fail(nullptr, EXX_EINVAL, "exx_apply_operator: ctx is NULL");
    if (!p || !ap) return fail(c, EXX_EINVAL, "exx_apply_operator: NULL argument");
    (void)cudaGetLastError();
    cudaStream_t st = (cudaStream_t)stream;
    CK(launch_apply(c->P, p, ap, st), "apply operator");
    CK(cudaStreamSynchronize(st), "apply operator (synchronize)");
    return EXX_OK;
}

extern "C" exx_status exx_apply_preconditioner(exx_ctx* c, const double* r, double* z, void* stream) {
    if (!c) return fail(nullptr, EXX_EINVAL, "exx_apply_preconditioner: ctx is NULL");
    if (!r || !z) return fail(c, EXX_EINVAL, "exx_apply_preconditioner: NULL argument");
    const int geo = c->n_geo - 1;
    if (!c->P.mg || c->balls[geo].r_pe <= 3)
        return fail(c, EXX_EINVAL, "exx_apply_preconditioner: no multigrid hierarchy (needs preconditioner = 1 and R_PE > 3)");
    (void)cudaGetLastError();
    cudaStream_t st = (cudaStream_t)stream;
    // slot 0's multigrid cubes: the FP32 solver keeps floats there, which an
    // FP64 view does not see as zero off the ball; cleared before the cycle,
    // and after it for the solvers, which expect zero off every ball
    char* mg0 = c->ws + c->P.off_zc;
    const size_t mgb = c->slot_bytes - c->P.off_zc;
    CK(cudaMemsetAsync(mg0, 0, mgb, st), "apply preconditioner (clear)");
    CK(launch_mg_apply(c->P, geo, r, z, st), "apply preconditioner");
    CK(cudaMemsetAsync(mg0, 0, mgb, st), "apply preconditioner (clear)");
    CK(cudaStreamSynchronize(st), "apply preconditioner (synchronize)");
    return EXX_OK;
}

extern "C" exx_status exx_quad_map(int r_pe, int cluster_size, int threads, int quads, int bank_aware,
                                   int* quad_pk, int* quad_k, size_t cap, int* info) {
    if (r_pe < 1 || r_pe > 64 || cluster_size < 2 || cluster_size > kMaxCluster || threads < 32 || threads > 1024 ||
        threads % 32 || quads < 1 || quads > 16 || !quad_pk || !quad_k || !info)
        return fail(nullptr, EXX_EINVAL, "exx_quad_map: bad arguments");
    const size_t per = (size_t)threads * quads;
    if (cap < per * cluster_size) return fail(nullptr, EXX_EINVAL, "exx_quad_map: cap too small");
    HostBall B;
    build_ball(B, r_pe, r_pe + 3, r_pe + 3);
    ClusterLayout L;
    std::vector<int> pt, pk, kk;
    if (!build_cluster_layout(B, cluster_size, L, pt, true))
        return fail(nullptr, EXX_EINVAL, "exx_quad_map: no slab layout for these radii and cluster size");
    const int mq = build_quad_maps(L, pt, threads, quads, pk, kk, bank_aware ? 1 : 0);
    if (mq < 0) return fail(nullptr, EXX_EINVAL, "exx_quad_map: the quads do not fit the slots");
    std::memcpy(quad_pk, pk.data(), sizeof(int) * pk.size());
    std::memcpy(quad_k, kk.data(), sizeof(int) * kk.size());
    info[0] = mq;
    info[1] = L.Syz;
    info[2] = L.Sp2;
    info[3] = L.cap_planes;
    for (int r = 0; r < cluster_size; ++r) {
        info[4 + 4 * r] = L.x0[r];
        info[5 + 4 * r] = L.planes[r];
        info[6 + 4 * r] = L.k0[r];
        info[7 + 4 * r] = L.k1[r];
    }
    return EXX_OK;
}

extern "C" exx_status exx_ball_tables(int r_pe, int r_me, int* off, int* cube, int* near, size_t cap, int* n_pe,
                                      int* n_me) {
    if (r_pe < 1 || r_me <= r_pe || r_me > 64 || !off || !n_pe || !n_me)
        return fail(nullptr, EXX_EINVAL, "exx_ball_tables: bad arguments");
    HostBall B;
    build_ball(B, r_pe, r_me, r_me);
    *n_pe = B.n_pe;
    *n_me = B.n_me;
    if (cap < (size_t)B.n_me) return fail(nullptr, EXX_EINVAL, "exx_ball_tables: cap smaller than the ME ball");
    std::memcpy(off, B.off.data(), sizeof(int) * B.off.size());
    if (cube) std::memcpy(cube, B.cube.data(), sizeof(int) * B.cube.size());
    if (near) {
        // the near list holds (ME row << 8) | (z + 128); mark those points by
        // their cube index
        std::vector<char> is_near((size_t)(2 * r_me + 1) * (2 * r_me + 1) * (2 * r_me + 1), 0);
        const int S = 2 * r_me + 1;
        for (int e : B.sh_near) {
            const RowRec& R = B.rows_me[e >> 8];
            const int z = (e & 0xff) - 128;
            is_near[((size_t)(R.ox + r_me) * S + (R.oy + r_me)) * S + (z + r_me)] = 1;
        }
        for (int k = 0; k < B.n_me; ++k) near[k] = k < B.n_pe ? 0 : (int)is_near[B.cube[k]];
    }
    return EXX_OK;
}

extern "C" exx_status exx_mg_levels(int r_pe, const double delta[3], int* radius, int* points, int* side, int cap,
                                    int* levels, double* minv, size_t minv_cap) {
    if (r_pe < 4 || r_pe > 127 || !delta || !radius || !points || !side || !levels || cap < 0)
        return fail(nullptr, EXX_EINVAL, "exx_mg_levels: bad arguments");
    for (int a = 0; a < 3; ++a)
        if (!(delta[a] > 0.0) || !std::isfinite(delta[a]))
            return fail(nullptr, EXX_EINVAL, "exx_mg_levels: spacings must be finite and > 0");
    std::vector<HostMGLevel> lv;
    std::vector<double> mi;
    if (!build_mg_levels(r_pe, delta, lv, mi))
        return fail(nullptr, EXX_EINVAL, "exx_mg_levels: the hierarchy could not be built");
    *levels = (int)lv.size();
    if (cap < (int)lv.size()) return fail(nullptr, EXX_EINVAL, "exx_mg_levels: cap smaller than the level count");
    for (size_t l = 0; l < lv.size(); ++l) {
        radius[l] = lv[l].R;
        points[l] = (int)lv[l].off.size();
        side[l] = lv[l].side;
    }
    if (minv) {
        if (minv_cap < mi.size()) return fail(nullptr, EXX_EINVAL, "exx_mg_levels: minv_cap too small");
        std::memcpy(minv, mi.data(), sizeof(double) * mi.size());
    }
    return EXX_OK;
}

extern "C" exx_status exx_radius_classes(const exx_ctx* c, int* r_pe, int* cluster_size, int* resident, int cap,
                                         int* n_class) {
    if (!c || !n_class) return fail(const_cast<exx_ctx*>(c), EXX_EINVAL, "exx_radius_classes: NULL argument");
    const int n = c->per_class ? (int)c->classes.size() : 0;
    *n_class = n;
    if (n > cap && (r_pe || cluster_size || resident))
        return fail(const_cast<exx_ctx*>(c), EXX_EINVAL, "exx_radius_classes: cap smaller than the class count");
    for (int k = 0; k < n; ++k) {
        const exx_ctx::RadiusClass& RC = c->classes[k];
        if (r_pe) r_pe[k] = c->balls[RC.geo].r_pe;
        if (cluster_size) cluster_size[k] = RC.kind == 2 ? RC.cand.C : 0;
        const int lane = c->aux ? (c->n_geo - 1 - RC.geo) & 1 : 0;
        const int slots = c->aux ? c->lane_slots[lane] : c->n_slots;
        if (resident) resident[k] = RC.kind == 2 ? std::min(RC.cand.n_clusters, slots) : slots;
    }
    return EXX_OK;
}

extern "C" exx_status exx_ball_size(const exx_ctx* c, int* n_pe, int* n_me) {
    if (!c) return fail(nullptr, EXX_EINVAL, "exx_ball_size: ctx is NULL");
    if (n_pe) *n_pe = c->hb.n_pe;
    if (n_me) *n_me = c->hb.n_me;
    return EXX_OK;
}

extern "C" exx_status exx_load_guess_model(exx_ctx* c, const void* weights, size_t bytes) {
    if (!c) return fail(nullptr, EXX_EINVAL, "exx_load_guess_model: ctx is NULL");
    if (!weights || bytes < 16) return fail(c, EXX_EINVAL, "exx_load_guess_model: blob too short");
    int32_t hdr[4];
    std::memcpy(hdr, weights, sizeof(hdr));
    const size_t np = exx::unet::param_count();
    if (hdr[0] != 0x47585845 || hdr[1] != 2) return fail(c, EXX_EINVAL, "exx_load_guess_model: bad magic or version");
    if (hdr[2] < 16 || hdr[2] > 64 || hdr[2] % 8) return fail(c, EXX_EINVAL, "exx_load_guess_model: bad cube side");
    if ((size_t)hdr[3] != np || bytes != 16 + np * sizeof(float))
        return fail(c, EXX_EINVAL, "exx_load_guess_model: parameter count does not match the network");
    (void)cudaGetLastError();
    if (c->gnet) {
        exx::unet::destroy(*c->gnet);
        delete c->gnet;
        c->gnet = nullptr;
    }
    cudaFree(c->d_gin);
    cudaFree(c->d_gscale);
    c->d_gin = nullptr;
    c->d_gscale = nullptr;
    const int S = hdr[2];
    // batch: about 4 GB of activations
    const long long per = (long long)S * S * S * 1200;
    const int bmax = (int)std::max(1LL, std::min(256LL, (4LL << 30) / per));
    c->gnet = new exx::unet::Net();
    cudaError_t e = exx::unet::create(*c->gnet, S, bmax);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_gin, sizeof(float) * exx::unet::kIn * (size_t)bmax * S * S * S);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_gscale, sizeof(float) * (size_t)bmax);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->gnet->params, static_cast<const char*>(weights) + 16, np * sizeof(float),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = exx::unet::pack(*c->gnet, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    for (auto& ev : c->ev_g)
        if (e == cudaSuccess && !ev) e = cudaEventCreate(&ev);
    if (e != cudaSuccess) {
        exx::unet::destroy(*c->gnet);
        delete c->gnet;
        c->gnet = nullptr;
        return cuda_fail(c, e, "exx_load_guess_model");
    }
    return EXX_OK;
}

extern "C" exx_status exx_export_samples(exx_ctx* c, const double* orbitals, int S, float* input, float* target,
                                         int cap, int* count, void* stream) {
    if (!c) return fail(nullptr, EXX_EINVAL, "exx_export_samples: ctx is NULL");
    if (!orbitals || !input || !target || !count) return fail(c, EXX_EINVAL, "exx_export_samples: NULL argument");
    if (S < 8 || S > 128 || S % 2) return fail(c, EXX_EINVAL, "exx_export_samples: S must be even in [8, 128]");
    if (c->opt.warm_start != 1 || !c->have_prev)
        return fail(c, EXX_EINVAL, "exx_export_samples: needs a completed exx_compute call with warm_start 1");
    if (orbitals != c->last_orb) return fail(c, EXX_EINVAL, "exx_export_samples: orbitals differ from the last call's");
    (void)cudaGetLastError();
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaStreamSynchronize(c->work), "exx_export_samples");
    int np = 0;
    CK(cudaMemcpy(&np, c->d_scalars + 7, sizeof(int), cudaMemcpyDeviceToHost), "exx_export_samples");
    *count = np;
    const int nk = std::min(np, std::max(cap, 0));
    if (nk <= 0) return EXX_OK;
    float* d_scale = nullptr;
    CK(cudaMalloc(&d_scale, sizeof(float) * (size_t)nk), "exx_export_samples");
    const double d2 = std::cbrt(c->delta[0] * c->delta[0] * c->delta[1] * c->delta[1] * c->delta[2] * c->delta[2]);
    cudaError_t e = exx::unet::sample_prep(orbitals, c->grid, c->d_prev_pairs, 0, nk, S, c->geo_host, input, d_scale,
                                           target, c->d_vcache[c->parity ^ 1], d2, c->delta, c->dV, c->lmax,
                                           c->cur_box, c->cur_bdim, c->cur_ostride, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_scale);
    if (e != cudaSuccess) return cuda_fail(c, e, "exx_export_samples");
    return EXX_OK;
}

extern "C" const char* exx_last_error(const exx_ctx* c) { return c ? c->err.c_str() : g_init_err.c_str(); }
