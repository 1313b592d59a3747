/*
 * exx.h -- C ABI of the GB300 pair-Poisson exact-exchange library.
 *
 * The library evaluates the real-space exact exchange of localized orbitals
 * (Ko et al., arXiv:1911.10630): for every pair of orbitals whose centres are
 * closer than R_pair it forms rho_ij = phi_i phi_j on a ball of radius R_PE
 * around the pair centre, sets Dirichlet values from a multipole expansion on
 * the shell out to R_ME, solves the reduced Poisson system with the order-6,
 * 19-point Laplacian by conjugate gradient, and returns
 *     E_xx  = - sum over ordered pairs of int_PE rho_ij v_ij      (Eq. exx_omega)
 *     D^i  += v_ij phi_j   on the ME ball of each pair            (Eqs. Dxx_mlwf,
 *                                                                   Dxx_mlwf_omega)
 * The input and output contract is the exx module's (Sec. III: the orbitals on
 * the real-space grid in, E_xx and {D_xx^i} out).
 *
 * Conventions for every entry point:
 *   - Hartree atomic units; the hybrid fraction a_x is NOT applied.
 *   - Grids are orthorhombic, N0 x N1 x N2 points, numbered 0..N-1 along each
 *     axis (Eq. l2g), point g at r = g * delta with delta_a = L_a / N_a.
 *   - Orbital and force arrays are FP64, shape [n][N0][N1][N2], C order (the
 *     last index fastest), one full grid per orbital.
 *   - Radii R_PE and R_ME are in grid points; the balls are the integer sets
 *     |o|^2 <= R_PE^2 and R_PE^2 < |o|^2 <= R_ME^2 (Algorithm 2).
 *   - Every function returns an exx_status; none aborts, traps or exits.
 *     After an error, exx_last_error() describes it.
 *   - Pointers marked "device" must be CUDA device (or managed) memory of the
 *     current device; "host" pointers are ordinary host memory (pinned memory
 *     makes the host-buffer entry points faster).
 *   - The caller owns every array it passes; the library owns its workspace.
 *   - A context is not thread-safe: use one context per host thread.
 */
#ifndef EXX_GB300_H
#define EXX_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct exx_ctx exx_ctx;

typedef enum {
    EXX_OK = 0,
    EXX_EINVAL = -1,   /* invalid argument (shape, radius, pointer, option)          */
    EXX_ENOMEM = -2,   /* device or host allocation failed                           */
    EXX_ECUDA = -3,    /* a CUDA call failed (no device, launch error, ...)           */
    EXX_ENOCONV = -4,  /* some CG solves reached max_iter; all outputs still written */
    EXX_ENOPAIR = -5,  /* a query named a pair that is not in the current list       */
    EXX_ETIMEOUT = -6  /* a bounded device wait ran out (a cluster exchange or a
                          tensor-core completion did not arrive within its poll
                          limit); outputs are written but not to be trusted;
                          the context stays usable                            */
} exx_status;

/* Solver choices. exx_default_options() fills the defaults noted here. */
typedef struct {
    int precision;     /* 0: FP64 conjugate gradient (default).
                          1: FP32 inner CG with FP64 residual refinement: the
                             residual r = 4 pi rho + lap v is recomputed in FP64
                             after each inner solve, and the stop test is FP64. */
    int batched;       /* 0: pairs in list order. 1: largest pairs first from a
                          device work queue, the whole call captured once and
                          replayed as a CUDA graph (default 1).                  */
    int warm_start;    /* 0: CG from zero (default). 1: previous call's v_ij for
                          pairs kept from the previous call (same i and j), moved
                          with the pair's grid centre; other pairs start from
                          zero. 2: the learned guess of the model loaded with
                          exx_load_guess_model (include/exx_guess.h). 3:
                          polynomial extrapolation over the calls that hold the
                          pair (Step IV: guesses from earlier MD steps): v1,
                          2 v1 - v2 or 3 v1 - 3 v2 + v3 from the last one, two
                          or three calls, each moved with the pair's grid
                          centre. 1, 2 and 3 need precision 1, fixed radii and
                          the cluster solver;
                          the stop rule is unchanged, so a start only changes
                          the iteration count.                                  */
    int radii_mode;    /* 0: fixed R_PE / R_ME for all pairs (default).
                          1: per-pair radii from the orbital exponents passed to
                             exx_compute (alphas), clamped to [12, R_PE]; R_PE and
                             R_ME of exx_init are then the maxima.
                          2: separate radii for self and non-self pairs (the
                             paper's self / non-self proto-subdomains, Sec. IV):
                             self pairs use R_PE / R_ME of exx_init, non-self
                             pairs r_pe_nonself / r_me_nonself below.
                          1 with precision 1 runs the cluster solver in radius
                          classes: one launch per R_PE, the largest first, each
                          on the smallest cluster whose slab layout fits (one
                          CTA holds a ball up to R_PE 13; 2, 4, 9 or 16 CTAs
                          share larger ones), the one-CTA solver for a radius
                          that fits none; 1 with precision 0, or solver_kind 1,
                          and 2 run on the one-CTA solver.                      */
    int max_iter;      /* CG iteration cap per solve (default 20000).            */
    int inner_max_iter;/* FP32 inner iterations per refinement step (default 4000) */
    double inner_tol;  /* FP32 inner relative tolerance of the refinement loop;
                          0 = library choice: 1e-4 for the multigrid CG, 1e-5
                          otherwise (measured fastest on water-64 and the
                          batched-uneven workload).                           */
    int threads;       /* threads per CTA, 0 = library choice, else a multiple of
                          32 in [256, 1024]; the one-CTA solver runs 256, 512
                          or 1024 (other values: the library choice, 512, or
                          256 for the FP32 multigrid CG, which then keeps six
                          CTAs per SM, five with per-pair radii), the cluster
                          solver only the launch shapes it is built for.      */
    int ctas_per_sm;   /* resident CTAs per SM, 0 = library choice (the
                          multigrid CG on clusters: 1 or 2, default 2).         */
    int solver_kind;   /* 0 = library choice; 1 = one CTA per pair with state in
                          global memory; 2 = one thread-block cluster per pair
                          (plain CG: the FP32 inner state in shared memory;
                          multigrid CG: all state in the pair's workspace,
                          shared by the cluster's CTAs; only when requested). */
    int cluster_size;  /* CTAs per cluster for solver_kind 2: 0 = library choice,
                          else 2, 4, 8 or 9 (9 with the non-portable cluster
                          size opt-in; on GB300, 15 clusters of 9 CTAs fit
                          against 15 of 8); for the multigrid CG 2, 4, 8
                          (default) or 16.                                      */
    double update_drop;/* cluster solver: the FP64 residual replaces the FP32 one
                          each time the FP32 residual has dropped by this factor
                          (reliable updates; default 1e-4: tol 1e-8 in two
                          segments, measured fastest on the water-64 workload
                          among 1e-1 .. 1e-5; 0 or out of (0, 1) = default).    */
    int lane_map;      /* cluster solver thread-to-point map: 0 = natural order
                          (contiguous warps, default), 1 = bank-distinct lanes
                          dealt plane by plane, 2 = each thread owns a run of
                          consecutive points of a row (z neighbours in
                          registers, runs of a warp in distinct banks, halo
                          planes filled by the neighbours; isotropic grids
                          with R_PE 16 or 24; only when requested), 3 = each
                          thread slot holds a quad of 4 consecutive points of
                          a row (rows padded to 16 bytes, every stencil leg one
                          16-byte load; x legs past the slab read from the
                          neighbour), 4 = quads with 3 halo planes per side
                          that the neighbours fill by asynchronous remote
                          stores (all stencil loads local), 5 = as 4 with the
                          quads dealt so that the 8 lanes of each phase of a
                          16-byte shared-memory access hit distinct banks;
                          3, 4 and 5 are tried by the autotuner.               */
    int autotune;      /* cluster solver: 1 = on the first exx_compute of a context
                          time every fitting launch shape (cluster size, threads
                          per CTA, lane map) on a prefix of the pair queue and
                          keep the fastest (default); later contexts of the
                          process with the same grid, radii and options reuse
                          that choice; 0 = take the first fit.                  */
    int r_pe_nonself;  /* radii_mode 2: R_PE of non-self pairs, 1..R_PE        */
    int r_me_nonself;  /* radii_mode 2: R_ME of non-self pairs,
                          r_pe_nonself + 3 .. R_ME                              */
    int fixed_residual;/* cluster solver with lane map 4 or 5 on an isotropic
                          grid: 0 = the FP64 residuals of the refinement come
                          from an exact integer stencil on a fixed-point copy
                          of v (default), 1 = from the FP64 stencil, 2 = test
                          mode: the fixed-point bound is made too small, so
                          every pair takes the overflow fallback to the FP64
                          stencil.                                              */
    int deterministic; /* 0 = D_xx accumulated by FP64 atomic adds (the order of
                          the adds, hence the last bits, varies; default);
                          1 = accumulated as 64-bit fixed-point integers
                          (resolution 2^-40, |D_xx| < 2^22) by integer atomic
                          adds, whose sum does not depend on their order, then
                          converted to FP64 in place: bitwise reproducible. A
                          contribution |v phi| >= 2^22 is dropped and the call
                          returns EXX_EINVAL (outputs written, D_xx incomplete). */
    int preconditioner;/* 0: plain CG (default). 1: CG preconditioned by one
                          symmetric geometric-multigrid V-cycle per iteration
                          (the paper names preconditioners as the main future
                          speed-up, Sec. IV.B and the conclusions): the balls
                          of radius R_l = ceil(R_{l-1} / 2) at spacing
                          2^l delta down to R <= 3, the 19-point stencil on
                          every level, one weighted-Jacobi sweep (weight 0.8)
                          down and up, full-weighting restriction, trilinear
                          prolongation, the coarsest ball solved exactly. Not
                          with warm_start. With precision 0 the PCG and every
                          level are FP64, one CTA per pair; with precision 1
                          each inner solve of the FP64 refinement loop is this
                          PCG in FP32 (recurrence and V-cycle), on one CTA per
                          pair, or with solver_kind 2 on a cluster of CTAs per
                          pair whose vectors stay in L2. A ball of radius <= 3
                          has no coarse level: its CG is unpreconditioned.
                          The stop rule is unchanged: ||r|| <= tol ||b||.      */
    int inject_wait_timeout; /* test only (default 0): the next this-many calls
                          of the context each make one extra bounded device wait
                          run out (cluster solver: thread 0 of every CTA polls an
                          mbarrier that nothing arrives on, with no copy or store
                          in flight to it), so the call returns EXX_ETIMEOUT
                          while its results stay those of a normal call.       */
} exx_options;

typedef struct {
    int n_pair;            /* pairs in the last call                             */
    int n_nonconv;         /* solves that hit max_iter                           */
    int iters_max;         /* max CG iterations over pairs (inner, summed)        */
    int iters_p50;         /* median CG iterations                               */
    int iters_p99;         /* 99th percentile CG iterations                      */
    long long iters_total; /* sum of CG iterations over pairs                     */
    long long point_iters; /* sum over pairs of N_PE x CG iterations              */
    int refine_max;        /* max FP64 refinement steps (precision 1)             */
    double solve_ms;       /* device time of the pair kernel in the last call      */
    double total_ms;       /* device time of the whole call (events on the stream) */
    int n_pe, n_me;        /* ball sizes for the fixed radii                       */
    int solver_kind;       /* solver that ran                                      */
    int cluster_size;      /* CTAs per pair                                        */
    int grid_ctas;         /* CTAs launched for the pair kernel                    */
    int threads;           /* threads per CTA                                      */
    double phase_ms[4];    /* the pair-kernel time split by the cycle counts of
                              its CTAs (clusters) into setup (gather,
                              multipoles, shell), the FP64 residuals of the
                              refinement loop, the CG iterations (with the
                              V-cycles under preconditioner 1) and finish
                              (E_ij, scatter)                                    */
    int lane_map;          /* lane map in use (cluster solver)                      */
    int n_candidates;      /* launch shapes the autotuner could choose from          */
    double tune_ms;        /* host time spent by the autotuner (first call)          */
    double guess_ms;       /* device time of the learned guesses (warm_start 2)      */
    int n_timeouts;        /* bounded device waits that ran out (EXX_ETIMEOUT)       */
    int n_nonfinite;       /* non-finite inputs seen: centres that are NaN or Inf,
                              plus pairs whose E_ij came out NaN or Inf (a NaN or
                              Inf orbital value on the pair's PE ball propagates
                              into E_ij, E_xx and D_xx; nothing is masked)      */
    int n_clipped;         /* exx_compute_boxes: pairs whose ME ball is not inside
                              both orbitals' boxes (0 for full grids)           */
    int n_dropped;         /* deterministic D_xx: contributions beyond the
                              fixed-point range, dropped (the synchronous calls
                              return EXX_EINVAL for them)                        */
} exx_stats;

/* Defaults described in exx_options. */
exx_options exx_default_options(void);

/*
 * Creates a context for one grid and one set of method parameters.
 *   cell[3]   orthorhombic cell lengths L_a (bohr), > 0
 *   grid[3]   grid points N_a, >= 2 R_ME + 1 (a ball never overlaps its own
 *             periodic image)
 *   r_pair    pair cutoff in bohr, strict |C_i - C_j| < r_pair under the
 *             minimum image (Sec. III.C Step II); INFINITY keeps all pairs
 *   r_pe      PE ball radius in grid points, 1 <= r_pe
 *   r_me      ME ball radius in grid points, r_me >= r_pe + 3 (the shell must
 *             hold the stencil's reach, Sec. IV.A) and r_me <= 63
 *   l_max     multipole order of Eqs. me/mepole, 0 <= l_max <= 6
 *   tol       relative residual ||r||_2 <= tol ||b||_2 on the PE ball, where
 *             b = 4 pi rho + boundary charge (Eq. pe_mat_red); 0 < tol < 1
 *   opt       NULL for exx_default_options()
 * Allocates the device tables on the current device. On error *out is NULL.
 * Errors: EXX_EINVAL (checked before any CUDA call), EXX_ECUDA, EXX_ENOMEM.
 */
exx_status exx_init(exx_ctx **out, const double cell[3], const int grid[3], double r_pair, int r_pe,
                    int r_me, int l_max, double tol, const exx_options *opt);

/*
 * One evaluation of E_xx and {D_xx^i}.
 *   orbitals  device, [n][N0][N1][N2] FP64, read only
 *   centers   device, [n][3] FP64 orbital centres in bohr (any real values;
 *             they are used through the minimum image)
 *   n         number of orbitals, 1 <= n <= 65535
 *   alphas    device, [n] FP64 Gaussian-like exponents used only when
 *             radii_mode = 1, else ignored (may be NULL)
 *   e_xx      host, receives E_xx
 *   d_xx      device, [n][N0][N1][N2] FP64, overwritten with D_xx (zeroed by
 *             the library first); must not alias orbitals
 *   stream    cudaStream_t, NULL = the legacy default stream
 * Work is ordered on the stream; the call returns after E_xx is on the host,
 * so d_xx is complete when it returns. The arrays must stay valid until then.
 * Errors: EXX_EINVAL, EXX_ECUDA, EXX_ENOMEM, EXX_ENOCONV (outputs written),
 * EXX_ETIMEOUT (outputs written, not to be trusted). NaN or Inf inputs are not
 * an error: they propagate into the outputs and exx_get_stats counts them.
 */
exx_status exx_compute(exx_ctx *ctx, const double *orbitals, const double *centers, int n,
                       const double *alphas, double *e_xx, double *d_xx, void *stream);

/*
 * exx_compute on orbitals stored as compact boxes instead of full grids: the
 * paper's outlook redistributes the orbitals by their compact supports
 * (Sec. IV.B); here each orbital is kept only on a periodic box of grid points
 * around its support, which cuts the memory of orbitals and D_xx by the ratio
 * of box to grid volume (about 4x for 1024 orbitals on 190^3 points).
 *   boxes     device, [n][B0][B1][B2] FP64: orbital i on the grid points
 *             (origin_i + b) mod N, 0 <= b < box_dim, C order, read only
 *   origin    device, [n][3] int: the boxes' corners, each in [0, N)
 *   box_dim   host int[3]: B_a, 2 R_ME + 1 <= B_a <= N_a, the same for all
 *             orbitals
 *   centers, n, alphas, e_xx, stream: as for exx_compute
 *   d_boxes   device, same layout as boxes: D_xx^i on orbital i's box
 *             (zeroed by the library first)
 * An orbital counts as zero outside its box, and D_xx^i is kept only on it.
 * When every pair's ME ball lies inside both of its orbitals' boxes the
 * results equal exx_compute's on the full grids; boxes of side
 * 2 (ceil(R_pair / (2 delta)) + R_ME + 1) + 1 around the orbitals' nearest grid
 * points guarantee it. exx_get_stats reports the pairs for which it fails
 * (n_clipped). Errors: as exx_compute; EXX_EINVAL for bad box_dim.
 */
exx_status exx_compute_boxes(exx_ctx *ctx, const double *boxes, const int *origin, const int box_dim[3],
                             const double *centers, int n, const double *alphas, double *e_xx, double *d_boxes,
                             void *stream);

/*
 * exx_compute without any host synchronisation (no counterpart in the paper,
 * whose module returns to a CPU caller): the same work, enqueued after the
 * caller's stream, with E_xx written to e_xx_dev (one double in DEVICE memory)
 * and D_xx to d_xx; the caller's stream is ordered after the work, so a kernel
 * or copy the caller enqueues next sees both. The call returns EXX_OK once the
 * work is enqueued (errors in its arguments or launches as for exx_compute);
 * its outcome (non-converged solves, timed-out waits, non-finite inputs,
 * dropped deterministic D_xx contributions) is read with exx_get_stats, which
 * waits for the last call first, as exx_get_pairs and exx_debug_pair do. Only
 * the last call's counters are kept: an asynchronous call issued before the
 * previous one's counters were read replaces them. The first call of a context
 * on the cluster solver times its launch shapes (autotune) and so blocks.
 * Errors: EXX_EINVAL for a NULL, misaligned or non-device e_xx_dev and with
 * warm_start != 0 (those keep host-side state; use exx_compute).
 */
exx_status exx_compute_async(exx_ctx *ctx, const double *orbitals, const double *centers, int n,
                             const double *alphas, double *e_xx_dev, double *d_xx, void *stream);

/*
 * Same as exx_compute with HOST buffers: copies orbitals, centers (and alphas)
 * to the device, runs exx_compute and copies D_xx back into d_xx_host.
 *   orbitals_host [n][N0][N1][N2], centers_host [n][3], alphas_host [n] or NULL,
 *   d_xx_host [n][N0][N1][N2] (written). Device buffers are held by the
 *   context between calls and grown when n grows. An orbitals or d_xx buffer
 *   in pinned, device-mapped host memory (cudaHostAlloc, cudaMallocHost,
 *   cudaHostRegister with mapping), 16-byte aligned, is moved by the GPU's
 *   SMs reading or writing it directly; any other buffer by cudaMemcpyAsync.
 *   The call returns after D_xx has reached d_xx_host.
 */
exx_status exx_compute_host(exx_ctx *ctx, const double *orbitals_host, const double *centers_host,
                            int n, const double *alphas_host, double *e_xx, double *d_xx_host,
                            void *stream);

/* Statistics of the last exx_compute / exx_compute_host call. */
exx_status exx_get_stats(const exx_ctx *ctx, exx_stats *out);

/*
 * Pair list of the last call (Sec. III.C Step II), in list order (i-major, j
 * ascending), with per-pair results:
 *   pi, pj        orbital indices, i <= j
 *   g             3 ints per pair: grid point nearest the pair centre, in [0, N)
 *   radii         2 ints per pair: R_PE, R_ME used for the pair (may be NULL)
 *   e_pair        sum over the PE ball of rho_ij v_ij dV (may be NULL)
 *   iters         CG iterations of the pair (may be NULL)
 * All host arrays of capacity cap pairs; *n_pair receives the count. Any
 * output pointer may be NULL. EXX_EINVAL if cap is too small.
 */
exx_status exx_get_pairs(const exx_ctx *ctx, int *pi, int *pj, int *g, int *radii, double *e_pair,
                         int *iters, int cap, int *n_pair);

/*
 * Intermediates of one pair of the last call, for step-level checks:
 *   index     position in the pair list of the last call
 *   rho       host [N_ME]: phi_i phi_j on the ME ball, PE points first (may be NULL)
 *   v         host [N_ME]: the potential: CG solution on the PE ball, multipole
 *             expansion (Eq. me) on the shell (may be NULL)
 *   b         host [N_PE]: right-hand side 4 pi rho + boundary charge of
 *             Eq. pe_mat_red written as A v = b (may be NULL)
 * Ball points are in Algorithm 2 order (lexicographic (x, y, z) within the PE
 * ball, then within the shell). Re-solves the pair on the device with the
 * context's options. EXX_ENOPAIR if index is out of range.
 */
exx_status exx_debug_pair(exx_ctx *ctx, const double *orbitals, int index, double *rho, double *v,
                          double *b, void *stream);

/*
 * Applies A = -lap_PE (the 19-point stencil of Eq. d2_1 restricted to the PE
 * ball, zero outside it) to p on the PE ball of the context's R_PE.
 *   p, ap     device, [N_PE] FP64 in Algorithm 2 order
 */
exx_status exx_apply_operator(exx_ctx *ctx, const double *p, double *ap, void *stream);

/*
 * Applies the multigrid preconditioner of the PCG (preconditioner = 1; the
 * paper names preconditioning as the way to fewer iterations, Sec. IV.B and
 * Sec. V) once: z = M r, one symmetric V-cycle in FP64 over the levels of
 * exx_mg_levels, on the PE ball of the context's largest R_PE.
 *   r, z      device, [N_PE] FP64 in Algorithm 2 order
 * Uses workspace slot 0 and leaves it as the solvers expect; waits for the
 * stream. Must not overlap an exx_compute call on the same context.
 * EXX_EINVAL without a hierarchy (preconditioner 0, or R_PE <= 3).
 */
exx_status exx_apply_preconditioner(exx_ctx *ctx, const double *r, double *z, void *stream);

/*
 * The launch plan of per-pair radii on the cluster solver (radii_mode 1,
 * precision 1): one class per R_PE, launched largest first. The paper has no
 * counterpart (its subdomain sizes vary per pair, Sec. IV.A; how they map to
 * thread-block clusters is this library's). Host arrays of capacity cap:
 *   r_pe          the class's R_PE
 *   cluster_size  CTAs per pair (1 = the whole ball in one CTA's shared
 *                 memory), or 0 when the class runs on the one-CTA solver
 *                 with its state in global memory
 *   resident      clusters (or CTAs) the class's launch keeps resident
 * *n_class receives the class count (0 when the context has no classes). Any
 * output array may be NULL. EXX_EINVAL if cap is too small.
 */
exx_status exx_radius_classes(const exx_ctx *ctx, int *r_pe, int *cluster_size, int *resident, int cap,
                              int *n_class);

/* Ball sizes for the context's fixed radii. */
exx_status exx_ball_size(const exx_ctx *ctx, int *n_pe, int *n_me);

/*
 * Loads the learned warm-start model used by warm_start = 2: a blob of four
 * int32 {0x47585845, 2, S, count} followed by count FP32 parameters of the
 * U-Net described in include/exx_guess.h (S = side of the network's input
 * cube). weights: host. Allocates the network and its batch buffers (about
 * 4 GB). EXX_EINVAL if the header or the size does not match; a later load
 * replaces the model.
 */
exx_status exx_load_guess_model(exx_ctx *ctx, const void *weights, size_t bytes);

/*
 * Pair list without device allocation. The paper has no counterpart. It is
 * for callers that cannot call cudaMalloc: applications that route all device
 * memory through their own pool or arena (a framework's caching allocator, a
 * service held to a fixed per-process budget), where an allocation outside
 * the pool breaks the budget or fails near the memory limit, and latency-bound
 * loops that cannot afford cudaMalloc's implicit device synchronisation. It
 * returns the pair list exx_compute builds for the same centres (the same
 * count / scan / fill kernels, hence the same records in the same order).
 * Its scratch (per-orbital counts, prefix sums and the pair count) lives in
 * a static device array sized for 16384 orbitals; every GPU that loads the
 * library holds that array (about 128 KiB) until the process exits.
 *   centers   device, [n][3] FP64 orbital centres (bohr)
 *   n         1 <= n <= 16384, else EXX_EINVAL
 *   cell, grid, r_pair  as for exx_init
 *   pairs     device, [cap][5] int: i, j (i <= j) and the grid point nearest
 *             the pair centre (3 ints, in [0, N)), in list order
 *   cap       capacity of pairs in records
 *   n_pair    host, receives the number of pairs; if it exceeds cap only the
 *             first cap records are written and EXX_EINVAL is returned
 *   stream    cudaStream_t, NULL = legacy default stream; the call waits for it
 * The first call on a device looks up the array's device address (once per
 * device), so make that call before any stream capture. All calls share the
 * one array, which keeps the last call's contents (every word a call reads it
 * writes first): calls that overlap on the GPU race and must be serialised.
 * Allocates nothing. Errors are read with exx_last_error(NULL).
 */
exx_status exx_pair_list_static(const double *centers, int n, const double cell[3], const int grid[3],
                                double r_pair, int *pairs, int cap, int *n_pair, void *stream);

/*
 * The cluster solver's quad thread map (lane maps 4 and 5), built on the host
 * exactly as exx_init builds it, for tests of the layout; no device work. The
 * paper has no counterpart (the map is how this library lays the PE ball of
 * Sec. III.C Step IV out over a thread-block cluster).
 *   r_pe          PE radius in grid points (1..64)
 *   cluster_size  CTAs sharing a pair (2..16); slabs of >= 3 whole x planes
 *   threads       threads per CTA (a multiple of 32, <= 1024)
 *   quads         quad slots per thread (1..16)
 *   bank_aware    0: quads in row order; 1: dealt so that every 8
 *                 consecutive slots hold 8 distinct bank groups
 *   quad_pk       host [cluster_size][quads][threads] ints: slab offset of
 *                 the quad (floats from the CTA's plane 0, a multiple of 4)
 *                 | valid-element mask << 20 | plane << 24
 *   quad_k        host, same shape: compact PE index of the quad's element 0
 *                 (Algorithm 2 order; element i is k + i when mask bit i is set)
 *   cap           entries each of quad_pk and quad_k can hold
 *   info          host int[4 + 4 * cluster_size]: largest quad count of a CTA,
 *                 row pitch, plane pitch (floats), largest slab (planes), then per
 *                 CTA: first plane offset x0, planes, first and end compact index
 * Returns EXX_EINVAL on bad arguments or when the map does not fit; the
 * message is read with exx_last_error(NULL).
 */
exx_status exx_quad_map(int r_pe, int cluster_size, int threads, int quads, int bank_aware, int *quad_pk,
                        int *quad_k, size_t cap, int *info);

/*
 * The ball tables the kernels index, built on the host as exx_init builds
 * them, with no CUDA call: the proto-subdomain of Algorithm 2 (Sec. III.C,
 * Step III), the PE ball |o| <= r_pe followed by the shell r_pe < |o| <= r_me,
 * each in lexicographic (x, y, z) order.
 *   r_pe, r_me  radii in grid points, 1 <= r_pe < r_me <= 64
 *   off         host int[cap]: packed offsets (x + 128) | (y + 128) << 8 |
 *               (z + 128) << 16
 *   cube        host int[cap], or NULL: each point's index in the cube of side
 *               S = 2 r_me + 1 around the origin, ((x + r_me) S + y + r_me) S +
 *               z + r_me
 *   near        host int[cap], or NULL: 1 for a shell point whose far-field
 *               potential is evaluated in FP64 (the layer next to the PE ball
 *               that the stencil of Eq. d2_1 reads), 0 for the other shell
 *               points (FP32) and for the PE ball
 *   cap         entries each array can hold (at least the ME ball's points)
 *   n_pe, n_me  host: points of the PE ball and of the whole ME ball
 * Returns EXX_EINVAL on bad arguments or a cap too small (n_pe and n_me are
 * still written); the message is read with exx_last_error(NULL).
 */
exx_status exx_ball_tables(int r_pe, int r_me, int *off, int *cube, int *near, size_t cap, int *n_pe, int *n_me);

/*
 * The multigrid hierarchy that preconditions the CG (preconditioner = 1; the
 * paper names preconditioning as the way to fewer iterations, Sec. IV.B and
 * Sec. V), built on the host as exx_init builds it, with no CUDA call. For a
 * PE ball of radius r_pe at spacings delta, level l >= 1 is the ball of radius
 * R_l = ceil(R_{l-1} / 2) (R_0 = r_pe) at spacing 2^l delta, down to the first
 * R_l <= 3; its points are those of the ball in lexicographic (x, y, z)
 * order, held in a zero-padded cube of side 2 R_l + 7.
 *   r_pe      PE radius in grid points (4..127; a ball of radius 3 or less
 *             has no coarser level)
 *   delta     host double[3]: grid spacings in bohr (> 0)
 *   radius, points, side   host int[cap]: R_l, the ball's point count and the
 *             cube side of levels l = 1..L, level l at entry l - 1
 *   cap       entries each of radius, points and side can hold
 *   levels    host, receives L
 *   minv      host double[points[L-1]^2], or NULL: the inverse of the coarsest
 *             level's operator (-lap of Eq. d2_1 at spacing 2^L delta, zero
 *             outside the ball), row-major in the level's point order
 *   minv_cap  entries minv can hold
 * Returns EXX_EINVAL on bad arguments, a cap or minv_cap too small, or a
 * hierarchy that cannot be built; the message is read with exx_last_error(NULL).
 */
exx_status exx_mg_levels(int r_pe, const double delta[3], int *radius, int *points, int *side, int cap, int *levels,
                         double *minv, size_t minv_cap);

/*
 * Measures the FP64 FMA rate of the current device, the roofline denominator
 * of the plain FP64 CG (whose binding unit on this GPU is the FP64 pipe, not
 * HBM). The paper has no counterpart. Eight independent FMA chains per thread
 * on 8 CTAs of 256 threads per SM; the best of three timed launches.
 *   tflops   host, receives 2 x FMAs / s / 1e12
 *   stream   cudaStream_t, NULL = legacy default stream; the call waits for it
 * Allocates nothing on the device. Errors (EXX_EINVAL, EXX_ECUDA) are read
 * with exx_last_error(NULL).
 */
exx_status exx_probe_fp64_rate(double *tflops, void *stream);

/* Message of the last error on this context (or of the last failed exx_init
 * when ctx is NULL); owned by the library, valid until the next call. */
const char *exx_last_error(const exx_ctx *ctx);

/* Frees the context and its device memory. NULL is ignored. */
void exx_destroy(exx_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* EXX_GB300_H */
