/*
 * oracle_exx.c -- plain, slow, FP64 CPU oracle for the MLWF pair-Poisson exact
 * exchange of Ko, Jia, Santra, Wu, Car and DiStasio (arXiv:1911.10630).
 *
 * TEST INFRASTRUCTURE ONLY. It exists to check the CUDA library against the
 * paper. Only the tests, __graft_entry__.smoke() and bench.py's CPU-baseline
 * leg may load it; the library never links, calls or includes anything here,
 * and nothing here includes the library's sources or headers.
 *
 * Every routine follows one passage of the paper, in the paper's order and
 * notation, with no blocking, fusion or reordering beyond what it states:
 *
 *   oracle_pair_list        Sec. III.C Step II: |C_i - C_j| < R_pair (strict),
 *                           minimum image; C_ij = (C_i + C_j)/2 as the
 *                           midpoint of the minimum-image segment, snapped to
 *                           the nearest grid point (NINT, Sec. III.C Step III).
 *   oracle_proto_subdomain  Algorithm 2: the PE ball |o| <= R_PE and the ME
 *                           shell R_PE < |o| <= R_ME around C_0, concatenated
 *                           PE-first (Eqs. rbar and g0).
 *   oracle_real_ylm         Real orthonormal spherical harmonics (textbook
 *                           associated-Legendre recurrence) for Eqs. me/mepole.
 *   oracle_pair_solve       Steps III-V for one pair: gather through the
 *                           translated indices (Eq. l2g), rho_ij = phi_i phi_j,
 *                           multipole moments Q_lm (Eq. mepole), the far-field
 *                           potential on the shell (Eq. me), the reduced PE
 *                           system with boundary charge (Eq. pe_mat_red) built
 *                           from the n = 3 central-difference Laplacian
 *                           (Eq. d2_1), textbook conjugate gradient, and the
 *                           pair energy integral over the PE ball (Eq. exx_omega).
 *   oracle_exx_pairs        Step V over a pair list: E_xx = -sum over ordered
 *                           pairs (self x1, i<j x2) and the force scatter
 *                           D^i += v_ij phi_j, D^j += v_ij phi_i on the ME ball
 *                           (Eqs. Dxx_mlwf, Dxx_mlwf_omega); the _radii form
 *                           takes per-pair radii.
 *   oracle_pair_radius,     Per-pair radii from the orbitals' Gaussian
 *   oracle_pair_list_radii     envelopes (spread-dependent subdomains, the
 *                           outlook of Sec. IV.A; reading listed below).
 *   oracle_laplacian_box,   The same 19-point stencil on a plain box (interior
 *   oracle_laplacian_periodic  points) and on a periodic box, for the pins.
 *   oracle_cg_periodic,     The same CG on a periodic box and on a given ball
 *   oracle_ball_cg             right-hand side, for the pins.
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - radii are in grid points and the balls are integer tests on |o|^2;
 *   - the multipole origin is the snapped grid point g_ij, so rbar = o * delta;
 *   - Q_lm is summed over the PE ball only;
 *   - MOD is the non-negative periodic remainder;
 *   - CG stops when ||r||_2 <= tol * ||b||_2, b including the boundary charge;
 *   - D^i = sum_j v_ij phi_j literally (no a_x, no factor 2 or 4);
 *   - per-pair radii: the eps-support of the Gaussian product envelope seen
 *     from the pair centre, eps = 1e-14, clamped to [r_min, r_max], and
 *     R_ME = R_PE + max(3, ceil(R_PE/3)).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (see build.py).
 * Floating-point contraction is off so that the pair list (where doubles
 * decide integers) is the plain IEEE sequence written below.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846264338327950288

/* Eq. d2_1 with n = 3: central-difference weights w_0 .. w_3 (w_q = w_-q). */
static const double W[4] = {-49.0 / 18.0, 3.0 / 2.0, -3.0 / 20.0, 1.0 / 90.0};

int oracle_version(void) { return 3; }

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Step II: pair list and pair centres                                      */
/* ------------------------------------------------------------------------ */

/* minimum-image displacement along one axis; a tie at exactly L/2 maps to -L/2 */
static double minimg(double x, double L) { return x - L * floor(x / L + 0.5); }

/* non-negative remainder (grid wrap of Eq. l2g) */
static int pmod(long a, int n) {
    long r = a % n;
    return (int)(r < 0 ? r + n : r);
}

/* NINT: nearest integer, halves away from zero (Fortran NINT). */
static long nint(double x) { return (long)round(x); }

/*
 * Pairs i <= j (i-major, j ascending) with |minimg(C_j - C_i)| < r_pair.
 * For each pair: the pair centre C_ij = C_i + d/2 (the midpoint of the
 * minimum-image segment) and g_ij = MOD(NINT(C_ij,a / delta_a), N_a).
 * Returns the number of pairs, or -1 if it exceeds cap.
 */
int oracle_pair_list(int n, const double *centers, const double *cell, const int *grid,
                     double r_pair, int cap, int *pi, int *pj, int *gij) {
    int count = 0;
    double delta[3];
    for (int a = 0; a < 3; ++a) delta[a] = cell[a] / (double)grid[a];
    double r2cut = r_pair * r_pair;
    for (int i = 0; i < n; ++i) {
        for (int j = i; j < n; ++j) {
            double d[3];
            for (int a = 0; a < 3; ++a) d[a] = minimg(centers[3 * j + a] - centers[3 * i + a], cell[a]);
            double d2 = d[0] * d[0] + d[1] * d[1];
            d2 = d2 + d[2] * d[2];
            if (!(d2 < r2cut)) continue;
            if (count >= cap) return -1;
            pi[count] = i;
            pj[count] = j;
            for (int a = 0; a < 3; ++a) {
                double c = centers[3 * i + a] + 0.5 * d[a];
                gij[3 * count + a] = pmod(nint(c / delta[a]), grid[a]);
            }
            ++count;
        }
    }
    return count;
}

/*
 * Per-pair radii for spread-dependent subdomains (the "beta-version" outlook of
 * Sec. IV.A, with Omega = {|phi| > eps}, Sec. II.C). For Gaussian envelopes the
 * product decays as exp(-mu d^2) exp(-(a_i + a_j) s^2) about the weighted centre
 * cbar = C_i + a_j/(a_i + a_j) d, mu = a_i a_j/(a_i + a_j). Its eps-support radius is
 * s_eps = sqrt(max(0, (ln(1/eps) - mu |d|^2)/(a_i + a_j))), seen from the pair
 * centre C_ij = C_i + d/2 at distance |a_j/(a_i + a_j) - 1/2| |d| from cbar:
 *   R_PE = clamp(ceil((s_eps + |cbar - C_ij|)/delta), r_min, r_max),
 *   R_ME = R_PE + max(3, ceil(R_PE/3)).
 * ln_inv_eps is ln(1/eps); delta the largest grid spacing.
 */
int oracle_pair_radius(double ai, double aj, double d2, double delta, double ln_inv_eps, int r_min, int r_max,
                       int *r_me) {
    double beta = ai + aj;
    double mu = ai * aj / beta;
    double t = (ln_inv_eps - mu * d2) / beta;
    double s = t > 0.0 ? sqrt(t) : 0.0;
    double w = fabs(aj / beta - 0.5) * sqrt(d2);
    double rf = ceil((s + w) / delta);
    int r = rf < (double)r_min ? r_min : (rf > (double)r_max ? r_max : (int)rf);
    if (r_me) *r_me = r + ((r + 2) / 3 > 3 ? (r + 2) / 3 : 3);
    return r;
}

/* Pair list as oracle_pair_list plus the per-pair radii of oracle_pair_radius. */
int oracle_pair_list_radii(int n, const double *centers, const double *cell, const int *grid, double r_pair,
                           const double *alphas, double ln_inv_eps, int r_min, int r_max, int cap, int *pi,
                           int *pj, int *gij, int *rpe, int *rme) {
    int cnt = oracle_pair_list(n, centers, cell, grid, r_pair, cap, pi, pj, gij);
    if (cnt < 0) return cnt;
    double delta = 0.0;
    for (int a = 0; a < 3; ++a) {
        double da = cell[a] / (double)grid[a];
        if (da > delta) delta = da;
    }
    for (int p = 0; p < cnt; ++p) {
        int i = pi[p], j = pj[p];
        double d[3];
        for (int a = 0; a < 3; ++a) d[a] = minimg(centers[3 * j + a] - centers[3 * i + a], cell[a]);
        double d2 = d[0] * d[0] + d[1] * d[1];
        d2 = d2 + d[2] * d[2];
        rpe[p] = oracle_pair_radius(alphas[i], alphas[j], d2, delta, ln_inv_eps, r_min, r_max, rme + p);
    }
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2: proto-subdomains                                            */
/* ------------------------------------------------------------------------ */

/*
 * Loop over the grid points around C_0 (offsets o in [-R_ME, R_ME]^3,
 * lexicographic); |o| <= R_PE goes to the PE list, R_PE < |o| <= R_ME to the
 * shell list. off receives 3*N_ME integers, PE points first (Eqs. rbar, g0).
 * If off is NULL only the counts are returned.
 */
int oracle_proto_subdomain(int r_pe, int r_me, int *off, int *n_pe_out, int *n_me_out) {
    int qpe = 0, qsh = 0;
    long rpe2 = (long)r_pe * r_pe, rme2 = (long)r_me * r_me;
    for (int x = -r_me; x <= r_me; ++x)
        for (int y = -r_me; y <= r_me; ++y)
            for (int z = -r_me; z <= r_me; ++z) {
                long s = (long)x * x + (long)y * y + (long)z * z;
                if (s <= rpe2) ++qpe;
                else if (s <= rme2) ++qsh;
            }
    if (off) {
        int a = 0, b = qpe;
        for (int x = -r_me; x <= r_me; ++x)
            for (int y = -r_me; y <= r_me; ++y)
                for (int z = -r_me; z <= r_me; ++z) {
                    long s = (long)x * x + (long)y * y + (long)z * z;
                    if (s <= rpe2) {
                        off[3 * a] = x; off[3 * a + 1] = y; off[3 * a + 2] = z; ++a;
                    } else if (s <= rme2) {
                        off[3 * b] = x; off[3 * b + 1] = y; off[3 * b + 2] = z; ++b;
                    }
                }
    }
    if (n_pe_out) *n_pe_out = qpe;
    if (n_me_out) *n_me_out = qpe + qsh;
    return qpe + qsh;
}

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics (Eqs. me, mepole)                               */
/* ------------------------------------------------------------------------ */

/*
 * Real orthonormal Y_lm at the direction of (x, y, z), for 0 <= l <= lmax,
 * stored at index l*l + l + m, m = -l..l:
 *   Y_l0  = K_l0 P_l^0(cos t)
 *   Y_lm  = sqrt(2) K_lm P_l^m(cos t) cos(m phi)   (m > 0)
 *   Y_l-m = sqrt(2) K_lm P_l^m(cos t) sin(m phi)   (m > 0)
 *   K_lm  = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!)
 * with P_l^m from the standard recurrences (no Condon-Shortley phase; any
 * orthonormal real set gives the same potential). At the origin the direction
 * is taken as +z; only l = 0 matters there because r^l = 0 for l > 0.
 */
void oracle_real_ylm(int lmax, double x, double y, double z, double *out) {
    double r = sqrt(x * x + y * y + z * z);
    double ct = 1.0, st = 0.0, phi = 0.0;
    if (r > 0.0) {
        ct = z / r;
        double rho = sqrt(x * x + y * y);
        st = rho / r;
        phi = atan2(y, x);
    }
    double P[16][16];
    memset(P, 0, sizeof(P));
    for (int m = 0; m <= lmax; ++m) {
        /* P_m^m = (2m-1)!! sin^m */
        double pmm = 1.0;
        for (int k = 1; k <= m; ++k) pmm *= (2.0 * k - 1.0) * st;
        P[m][m] = pmm;
        if (m + 1 <= lmax) P[m + 1][m] = ct * (2.0 * m + 1.0) * pmm;
        for (int l = m + 2; l <= lmax; ++l)
            P[l][m] = ((2.0 * l - 1.0) * ct * P[l - 1][m] - (l + m - 1.0) * P[l - 2][m]) / (double)(l - m);
    }
    for (int l = 0; l <= lmax; ++l) {
        for (int m = 0; m <= l; ++m) {
            double ratio = 1.0; /* (l-m)!/(l+m)! */
            for (int k = l - m + 1; k <= l + m; ++k) ratio /= (double)k;
            double K = sqrt((2.0 * l + 1.0) / (4.0 * ORACLE_PI) * ratio);
            if (m == 0) {
                out[l * l + l] = K * P[l][0];
            } else {
                out[l * l + l + m] = sqrt(2.0) * K * P[l][m] * cos(m * phi);
                out[l * l + l - m] = sqrt(2.0) * K * P[l][m] * sin(m * phi);
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Eq. d2_1: the 19-point Laplacian on plain and periodic boxes (pins)      */
/* ------------------------------------------------------------------------ */

/* f and out are dims[0] x dims[1] x dims[2], C order; interior points only
 * (at least 3 from every face); other points of out are set to 0. */
void oracle_laplacian_box(const double *f, const int *dims, const double *delta, double *out) {
    long s[3] = {(long)dims[1] * dims[2], dims[2], 1};
    long total = (long)dims[0] * dims[1] * dims[2];
    for (long t = 0; t < total; ++t) out[t] = 0.0;
    for (int x = 3; x < dims[0] - 3; ++x)
        for (int y = 3; y < dims[1] - 3; ++y)
            for (int z = 3; z < dims[2] - 3; ++z) {
                long c = x * s[0] + y * s[1] + z;
                double acc = 0.0;
                for (int a = 0; a < 3; ++a) {
                    double d2 = 0.0;
                    for (int q = -3; q <= 3; ++q) d2 += W[q < 0 ? -q : q] * f[c + q * s[a]];
                    acc += d2 / (delta[a] * delta[a]);
                }
                out[c] = acc;
            }
}

void oracle_laplacian_periodic(const double *f, const int *dims, const double *delta, double *out) {
    for (int x = 0; x < dims[0]; ++x)
        for (int y = 0; y < dims[1]; ++y)
            for (int z = 0; z < dims[2]; ++z) {
                int p[3] = {x, y, z};
                double acc = 0.0;
                for (int a = 0; a < 3; ++a) {
                    double d2 = 0.0;
                    for (int q = -3; q <= 3; ++q) {
                        int u[3] = {p[0], p[1], p[2]};
                        u[a] = pmod((long)u[a] + q, dims[a]);
                        d2 += W[q < 0 ? -q : q] * f[((long)u[0] * dims[1] + u[1]) * dims[2] + u[2]];
                    }
                    acc += d2 / (delta[a] * delta[a]);
                }
                out[((long)x * dims[1] + y) * dims[2] + z] = acc;
            }
}

/* ------------------------------------------------------------------------ */
/* Textbook conjugate gradient (Step IV)                                    */
/* ------------------------------------------------------------------------ */

typedef void (*apply_fn)(const double *p, double *Ap, const void *ctx);

static double dot(long n, const double *a, const double *b) {
    double s = 0.0;
    for (long k = 0; k < n; ++k) s += a[k] * b[k];
    return s;
}

/*
 * Solves A x = b from the given x (x0). Stops when ||r|| <= tol ||b|| or after
 * maxit iterations. *it_report receives the first iteration count at which
 * ||r|| <= tol_report ||b|| held (-1 if never). Returns the iteration count.
 */
static int cg(long n, apply_fn apply, const void *ctx, const double *b, double *x, double tol,
              int maxit, double tol_report, int *it_report, double *final_rel) {
    double *r = malloc(sizeof(double) * n), *p = malloc(sizeof(double) * n), *Ap = malloc(sizeof(double) * n);
    apply(x, Ap, ctx);
    for (long k = 0; k < n; ++k) { r[k] = b[k] - Ap[k]; p[k] = r[k]; }
    double bnorm = sqrt(dot(n, b, b));
    double rr = dot(n, r, r);
    int it = 0, rep = -1;
    if (bnorm == 0.0) {
        for (long k = 0; k < n; ++k) x[k] = 0.0;
        rr = 0.0;
        rep = 0;
    } else {
        if (sqrt(rr) <= tol_report * bnorm) rep = 0;
        while (sqrt(rr) > tol * bnorm && it < maxit) {
            apply(p, Ap, ctx);
            double alpha = rr / dot(n, p, Ap);
            for (long k = 0; k < n; ++k) { x[k] += alpha * p[k]; r[k] -= alpha * Ap[k]; }
            double rr_new = dot(n, r, r);
            ++it;
            if (rep < 0 && sqrt(rr_new) <= tol_report * bnorm) rep = it;
            double beta = rr_new / rr;
            rr = rr_new;
            for (long k = 0; k < n; ++k) p[k] = r[k] + beta * p[k];
        }
    }
    if (it_report) *it_report = rep;
    if (final_rel) *final_rel = bnorm > 0.0 ? sqrt(rr) / bnorm : 0.0;
    free(r); free(p); free(Ap);
    return it;
}

/* periodic box: A = -(19-point Laplacian) with wrap */
typedef struct { int dims[3]; double delta[3]; } periodic_ctx;

static void apply_periodic(const double *p, double *Ap, const void *vctx) {
    const periodic_ctx *c = (const periodic_ctx *)vctx;
    oracle_laplacian_periodic(p, c->dims, c->delta, Ap);
    long total = (long)c->dims[0] * c->dims[1] * c->dims[2];
    for (long k = 0; k < total; ++k) Ap[k] = -Ap[k];
}

/* Solves -lap v = b on a periodic box from v = 0 (b must sum to zero). */
int oracle_cg_periodic(const double *b, const int *dims, const double *delta, double *v, double tol,
                       int maxit) {
    periodic_ctx c;
    for (int a = 0; a < 3; ++a) { c.dims[a] = dims[a]; c.delta[a] = delta[a]; }
    long total = (long)dims[0] * dims[1] * dims[2];
    for (long k = 0; k < total; ++k) v[k] = 0.0;
    return cg(total, apply_periodic, &c, b, v, tol, maxit, tol, NULL, NULL);
}

/* ------------------------------------------------------------------------ */
/* Ball geometry: the PE operator of Eq. pe_mat_red                         */
/* ------------------------------------------------------------------------ */

typedef struct {
    int r_pe, r_me, side, n_pe, n_me;
    int *off;  /* 3 * n_me offsets, PE points first */
    int *map;  /* side^3 cube -> compact index (0..n_me-1) or -1 */
    double delta[3];
} ball_t;

static int ball_make(ball_t *B, int r_pe, int r_me, const double *delta) {
    B->r_pe = r_pe; B->r_me = r_me; B->side = 2 * r_me + 1;
    for (int a = 0; a < 3; ++a) B->delta[a] = delta[a];
    oracle_proto_subdomain(r_pe, r_me, NULL, &B->n_pe, &B->n_me);
    B->off = malloc(sizeof(int) * 3 * (size_t)B->n_me);
    long cube = (long)B->side * B->side * B->side;
    B->map = malloc(sizeof(int) * cube);
    if (!B->off || !B->map) return -1;
    oracle_proto_subdomain(r_pe, r_me, B->off, NULL, NULL);
    for (long t = 0; t < cube; ++t) B->map[t] = -1;
    for (int q = 0; q < B->n_me; ++q) {
        long t = ((long)(B->off[3 * q] + r_me) * B->side + (B->off[3 * q + 1] + r_me)) * B->side +
                 (B->off[3 * q + 2] + r_me);
        B->map[t] = q;
    }
    return 0;
}

static void ball_free(ball_t *B) { free(B->off); free(B->map); }

/* compact index of offset (x, y, z), or -1 outside the ME ball */
static int ball_index(const ball_t *B, int x, int y, int z) {
    int R = B->r_me;
    if (x < -R || x > R || y < -R || y > R || z < -R || z > R) return -1;
    return B->map[((long)(x + R) * B->side + (y + R)) * B->side + (z + R)];
}

/* A p = -lap_PE p: the stencil restricted to the PE ball (p = 0 outside it). */
static void apply_ball(const double *p, double *Ap, const void *vctx) {
    const ball_t *B = (const ball_t *)vctx;
    for (int k = 0; k < B->n_pe; ++k) {
        int o[3] = {B->off[3 * k], B->off[3 * k + 1], B->off[3 * k + 2]};
        double acc = 0.0;
        for (int a = 0; a < 3; ++a) {
            double d2 = W[0] * p[k];
            for (int q = 1; q <= 3; ++q) {
                for (int sgn = -1; sgn <= 1; sgn += 2) {
                    int u[3] = {o[0], o[1], o[2]};
                    u[a] += sgn * q;
                    int t = ball_index(B, u[0], u[1], u[2]);
                    if (t >= 0 && t < B->n_pe) d2 += W[q] * p[t];
                }
            }
            acc += d2 / (B->delta[a] * B->delta[a]);
        }
        Ap[k] = -acc;
    }
}

/* Solves A x = b on the PE ball (n_pe unknowns) from x = x0 (given in x). */
int oracle_ball_cg(int r_pe, int r_me, const double *delta, const double *b, double *x, double tol,
                   int maxit) {
    ball_t B;
    if (ball_make(&B, r_pe, r_me, delta)) return -1;
    int it = cg(B.n_pe, apply_ball, &B, b, x, tol, maxit, tol, NULL, NULL);
    ball_free(&B);
    return it;
}

/* Applies A = -lap_PE to p on the PE ball (for step-level parity). */
int oracle_ball_apply(int r_pe, int r_me, const double *delta, const double *p, double *Ap) {
    ball_t B;
    if (ball_make(&B, r_pe, r_me, delta)) return -1;
    apply_ball(p, Ap, &B);
    ball_free(&B);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Steps III-V for one pair                                                 */
/* ------------------------------------------------------------------------ */

typedef struct {
    int grid[3];
    double cell[3], delta[3], dV;
    int lmax;
    double tol, tol_report;
    int maxit;
} geom_t;

static void geom_make(geom_t *G, const double *cell, const int *grid, int lmax, double tol,
                      double tol_report, int maxit) {
    for (int a = 0; a < 3; ++a) {
        G->cell[a] = cell[a]; G->grid[a] = grid[a]; G->delta[a] = cell[a] / (double)grid[a];
    }
    G->dV = G->delta[0] * G->delta[1] * G->delta[2];
    G->lmax = lmax; G->tol = tol; G->tol_report = tol_report; G->maxit = maxit;
}

/* global index of ball point q for the pair centred at g (Eq. l2g) */
static long ball_global(const geom_t *G, const ball_t *B, const int *g, int q) {
    int u[3];
    for (int a = 0; a < 3; ++a) u[a] = pmod((long)g[a] + B->off[3 * q + a], G->grid[a]);
    return ((long)u[0] * G->grid[1] + u[1]) * G->grid[2] + u[2];
}

/*
 * One pair. phi_i, phi_j are full grids. Outputs (any may be NULL):
 *   rho[n_me]  phi_i phi_j on the whole ME ball (the method uses the PE part)
 *   Q[(lmax+1)^2]  multipole moments (Eq. mepole), index l*l+l+m
 *   v[n_me]    the potential: CG solution on the PE ball, Eq. me on the shell
 *   b[n_pe]    right-hand side of Eq. pe_mat_red written as A v = b
 *   iters[2]   CG iterations to tol, and the first count reaching tol_report
 * Returns E_ij = sum over the PE ball of rho v dV (Eq. exx_omega).
 */
static double pair_solve(const geom_t *G, const ball_t *B, const double *phi_i, const double *phi_j,
                         const int *g, double *rho, double *Q, double *v, double *b, int *iters,
                         const double *x0) {
    int n_pe = B->n_pe, n_me = B->n_me, L = G->lmax;
    int nlm = (L + 1) * (L + 1);
    double *rho_l = malloc(sizeof(double) * n_me);
    double *v_l = malloc(sizeof(double) * n_me);
    double *b_l = malloc(sizeof(double) * n_pe);
    double Ql[256];
    double ylm[256];

    /* Step III: gather phi on the translated subdomain, rho_ij = phi_i phi_j */
    for (int q = 0; q < n_me; ++q) {
        long gi = ball_global(G, B, g, q);
        rho_l[q] = phi_i[gi] * phi_j[gi];
    }

    /* Eq. mepole: Q_lm = sum_{PE ball} Y_lm(rbar) |rbar|^l rho dV, origin at g_ij */
    for (int t = 0; t < nlm; ++t) Ql[t] = 0.0;
    for (int q = 0; q < n_pe; ++q) {
        double x = B->off[3 * q] * G->delta[0], y = B->off[3 * q + 1] * G->delta[1],
               z = B->off[3 * q + 2] * G->delta[2];
        double r = sqrt(x * x + y * y + z * z);
        oracle_real_ylm(L, x, y, z, ylm);
        double rl = 1.0;
        for (int l = 0; l <= L; ++l) {
            for (int m = -l; m <= l; ++m) Ql[l * l + l + m] += ylm[l * l + l + m] * rl * rho_l[q] * G->dV;
            rl *= r;
        }
    }

    /* Eq. me on the shell: v = 4 pi sum_lm Q_lm Y_lm / ((2l+1) r^(l+1)) */
    for (int q = 0; q < n_pe; ++q) v_l[q] = 0.0;
    for (int q = n_pe; q < n_me; ++q) {
        double x = B->off[3 * q] * G->delta[0], y = B->off[3 * q + 1] * G->delta[1],
               z = B->off[3 * q + 2] * G->delta[2];
        double r = sqrt(x * x + y * y + z * z);
        oracle_real_ylm(L, x, y, z, ylm);
        double acc = 0.0, rpow = r; /* r^(l+1) */
        for (int l = 0; l <= L; ++l) {
            double s = 0.0;
            for (int m = -l; m <= l; ++m) s += Ql[l * l + l + m] * ylm[l * l + l + m];
            acc += 4.0 * ORACLE_PI * s / ((2.0 * l + 1.0) * rpow);
            rpow *= r;
        }
        v_l[q] = acc;
    }

    /* Eq. pe_mat_red as A v = b: b = 4 pi rho + (lap - lap_PE) v_shell, i.e.
     * the stencil legs of each PE point that land in the shell */
    for (int k = 0; k < n_pe; ++k) {
        int o[3] = {B->off[3 * k], B->off[3 * k + 1], B->off[3 * k + 2]};
        double legs = 0.0;
        for (int a = 0; a < 3; ++a) {
            double d2 = 0.0;
            for (int q = 1; q <= 3; ++q)
                for (int sgn = -1; sgn <= 1; sgn += 2) {
                    int u[3] = {o[0], o[1], o[2]};
                    u[a] += sgn * q;
                    int t = ball_index(B, u[0], u[1], u[2]);
                    if (t >= n_pe) d2 += W[q] * v_l[t];
                }
            legs += d2 / (G->delta[a] * G->delta[a]);
        }
        b_l[k] = 4.0 * ORACLE_PI * rho_l[k] + legs;
    }

    /* Step IV: conjugate gradient on the PE ball */
    if (x0) for (int k = 0; k < n_pe; ++k) v_l[k] = x0[k];
    int rep = -1;
    int it = cg(n_pe, apply_ball, B, b_l, v_l, G->tol, G->maxit, G->tol_report, &rep, NULL);

    /* Step V: E_ij over the PE ball */
    double e = 0.0;
    for (int k = 0; k < n_pe; ++k) e += rho_l[k] * v_l[k];
    e *= G->dV;

    if (rho) memcpy(rho, rho_l, sizeof(double) * n_me);
    if (Q) memcpy(Q, Ql, sizeof(double) * nlm);
    if (v) memcpy(v, v_l, sizeof(double) * n_me);
    if (b) memcpy(b, b_l, sizeof(double) * n_pe);
    if (iters) { iters[0] = it; iters[1] = rep; }
    free(rho_l); free(v_l); free(b_l);
    return e;
}

/*
 * Public single-pair entry (step-level parity and pins). orbitals is the full
 * (n, N0, N1, N2) array; the pair is (i, j) with grid centre gij.
 * x0 (n_pe) is an optional initial guess on the PE ball.
 */
double oracle_pair_solve(const double *cell, const int *grid, const double *orbitals, int i, int j,
                         const int *gij, int r_pe, int r_me, int lmax, double tol, double tol_report,
                         int maxit, const double *x0, double *rho, double *Q, double *v, double *b,
                         int *iters) {
    geom_t G;
    geom_make(&G, cell, grid, lmax, tol, tol_report, maxit);
    ball_t B;
    if (ball_make(&B, r_pe, r_me, G.delta)) return NAN;
    long ng = (long)grid[0] * grid[1] * grid[2];
    double e = pair_solve(&G, &B, orbitals + (long)i * ng, orbitals + (long)j * ng, gij, rho, Q, v,
                          b, iters, x0);
    ball_free(&B);
    return e;
}

/*
 * Step V over a pair list. For each pair p: E_pair[p] = E_ij; iters[2p],
 * iters[2p+1] as in pair_solve. If D is not NULL (n x N0 x N1 x N2, zeroed
 * here), D^i += v phi_j and, for i != j, D^j += v phi_i on the ME ball,
 * accumulated pair by pair in list order (deterministic). If dmask is not
 * NULL only orbitals with dmask[i] != 0 receive contributions, and pairs
 * touching no such orbital are still solved for their energy only if
 * solve_all != 0 (otherwise their E_pair is NaN and they are skipped).
 * Returns E_xx = -(sum_i E_ii + 2 sum_{i<j} E_ij) over the solved pairs.
 */
/*
 * As oracle_exx_pairs, with per-pair radii rpe[p], rme[p] when they are given
 * (NULL: r_pe, r_me for every pair). Balls are built once per distinct radius.
 */
double oracle_exx_pairs_radii(const double *cell, const int *grid, const double *orbitals, int n_orb,
                              int npair, const int *pi, const int *pj, const int *gij, const int *rpe,
                              const int *rme, int r_pe, int r_me, int lmax, double tol, double tol_report,
                              int maxit, double *E_pair, int *iters, double *D, const int *dmask,
                              int solve_all) {
    geom_t G;
    geom_make(&G, cell, grid, lmax, tol, tol_report, maxit);
    /* one ball per distinct (R_PE, R_ME); radii stay below 64 grid points */
    ball_t *balls = calloc(64 * 64, sizeof(ball_t));
    int max_nme = 0;
    for (int p = -1; p < npair; ++p) {
        int a = p < 0 ? r_pe : rpe ? rpe[p] : r_pe, b = p < 0 ? r_me : rme ? rme[p] : r_me;
        if (a < 0 || a >= 64 || b < 0 || b >= 64) { free(balls); return NAN; }
        ball_t *Bp = &balls[a * 64 + b];
        if (!Bp->off) {
            if (ball_make(Bp, a, b, G.delta)) { free(balls); return NAN; }
        }
        if (Bp->n_me > max_nme) max_nme = Bp->n_me;
    }
    long ng = (long)grid[0] * grid[1] * grid[2];
    if (D) memset(D, 0, sizeof(double) * (size_t)n_orb * ng);

    int chunk = 4 * oracle_num_threads();
    if (chunk < 1) chunk = 1;
    double *vbuf = D ? malloc(sizeof(double) * (size_t)chunk * max_nme) : NULL;
    for (int p0 = 0; p0 < npair; p0 += chunk) {
        int p1 = p0 + chunk < npair ? p0 + chunk : npair;
#pragma omp parallel for schedule(dynamic, 1)
        for (int p = p0; p < p1; ++p) {
            int i = pi[p], j = pj[p];
            int want = solve_all || !dmask || dmask[i] || dmask[j];
            if (!want) { E_pair[p] = NAN; if (iters) { iters[2 * p] = -1; iters[2 * p + 1] = -1; } continue; }
            const ball_t *Bp = &balls[(rpe ? rpe[p] : r_pe) * 64 + (rme ? rme[p] : r_me)];
            double *v = vbuf ? vbuf + (size_t)(p - p0) * max_nme : NULL;
            E_pair[p] = pair_solve(&G, Bp, orbitals + (long)i * ng, orbitals + (long)j * ng, gij + 3 * p,
                                   NULL, NULL, v, NULL, iters ? iters + 2 * p : NULL, NULL);
        }
        if (!D) continue;
        /* Eqs. Dxx_mlwf / Dxx_mlwf_omega: scatter in list order */
        for (int p = p0; p < p1; ++p) {
            if (isnan(E_pair[p])) continue;
            int i = pi[p], j = pj[p];
            const ball_t *Bp = &balls[(rpe ? rpe[p] : r_pe) * 64 + (rme ? rme[p] : r_me)];
            const double *v = vbuf + (size_t)(p - p0) * max_nme;
            const double *phi_i = orbitals + (long)i * ng, *phi_j = orbitals + (long)j * ng;
            double *Di = D + (long)i * ng, *Dj = D + (long)j * ng;
            int mi = !dmask || dmask[i], mj = !dmask || dmask[j];
            for (int q = 0; q < Bp->n_me; ++q) {
                long gq = ball_global(&G, Bp, gij + 3 * p, q);
                if (mi) Di[gq] += v[q] * phi_j[gq];
                if (i != j && mj) Dj[gq] += v[q] * phi_i[gq];
            }
        }
    }
    free(vbuf);
    for (int t = 0; t < 64 * 64; ++t)
        if (balls[t].off) ball_free(&balls[t]);
    free(balls);

    double e = 0.0;
    for (int p = 0; p < npair; ++p) {
        if (isnan(E_pair[p])) continue;
        e += (pi[p] == pj[p] ? 1.0 : 2.0) * E_pair[p];
    }
    return -e;
}

double oracle_exx_pairs(const double *cell, const int *grid, const double *orbitals, int n_orb,
                        int npair, const int *pi, const int *pj, const int *gij, int r_pe, int r_me,
                        int lmax, double tol, double tol_report, int maxit, double *E_pair,
                        int *iters, double *D, const int *dmask, int solve_all) {
    return oracle_exx_pairs_radii(cell, grid, orbitals, n_orb, npair, pi, pj, gij, NULL, NULL, r_pe, r_me, lmax,
                                  tol, tol_report, maxit, E_pair, iters, D, dmask, solve_all);
}
