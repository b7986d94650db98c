/*
 * vlbm_oracle.c -- TEST INFRASTRUCTURE, not part of the product.
 *
 * Plain FP64 CPU restatement of the blended D2Q5 vectorial LBM (arXiv
 * 2411.15001). Every step of the scheme is its own loop over an array with a
 * two-cell ghost frame, in the order the paper derives them; nothing is fused,
 * tiled or reordered. Only tests, the smoke check and the CPU-baseline leg of
 * the benchmark call this file. See vlbm_oracle.h for the state layout.
 *
 * Readings taken where the paper is silent or garbled (also listed in the design
 * notes of the repository):
 *  - LMP bounds: the case formulas of Sec. 3.3.1 as printed (bounds of cell i for
 *    u^(1)_{i+1/2}, of cell i+1 for u^(2)_{i+1/2}), which follow the convex
 *    decomposition eq. (convex_decomposition_blending).
 *  - PP density bound: an x-face uses Delta F^rho of the same face, a y-face
 *    Delta G^rho of the same face (the printed subscripts are mixed up).
 *  - Pressure bound: the quadratic forms of matrices A and B as printed. The
 *    denominator of phi is printed with Delta F^E where 2 Delta F^E (that is,
 *    2 dF.w, the form of A) is meant; the closed-form eigenvalues use A.
 *  - Ties: Delta F^rho = 0 gives theta_rho = 1; a zero spectral radius gives no
 *    pressure constraint; u* outside G (rho* <= 0 or gamma_0 >= 0) gives
 *    theta_p = 0; a negative discriminant is clamped to 0; theta is clamped to [0,1].
 *  - Boundaries: periodic wrap; zero gradient copies u and u_1..u_4 of the boundary
 *    cell into both ghost layers; a reflective wall mirrors the cells, negates the
 *    normal momentum, and swaps the populations moving towards / away from it.
 *    Corners apply the x rule first, then the y rule.
 *  - Dirichlet parts (Sec. 4.7, 4.8 set the distributions of boundary cells to the
 *    Maxwellians of prescribed states): a ghost cell holds the prescribed state
 *    at its centre at the step's start time, with populations M_k of that state
 *    at the step's kinetic speed; lambda^n also covers the prescribed states.
 */
#include "vlbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define G 2                         /* ghost layers */
#define NPLANE 20

static int g_threads = 1;

void orc_set_threads(int n) { g_threads = n > 0 ? n : 1; }
int orc_get_threads(void) { return g_threads; }

static int state_in_G(const double u[4]) {
    return u[0] > 0.0 && u[3] - 0.5 * (u[1] * u[1] + u[2] * u[2]) / u[0] > 0.0;
}

static int has_dirichlet(const orc_cfg *c) {
    for (int s = 0; s < 4; ++s)
        if (c->bc[s] == ORC_BC_DIRICHLET || c->bc_hi[s] == ORC_BC_DIRICHLET) return 1;
    return 0;
}

int orc_check_cfg(const orc_cfg *c) {
    if (!c || c->nx < 2 || c->ny < 2) return -1;
    for (int s = 0; s < 4; ++s) {
        const int n = s < 2 ? c->ny : c->nx;   /* cells along side s */
        if (c->bc[s] < 0 || c->bc[s] > 3 || c->bc_hi[s] < 0 || c->bc_hi[s] > 3) return -1;
        if (c->split[s] == 0) {
            if (c->bc_hi[s] != c->bc[s]) return -1;
        } else if (c->split[s] < 2 || c->split[s] > n - 2) {
            return -1;
        }
        if ((c->bc[s] == ORC_BC_PERIODIC || c->bc_hi[s] == ORC_BC_PERIODIC) &&
            (c->bc[s] != c->bc_hi[s] || c->split[s] != 0))
            return -1;
    }
    if ((c->bc[0] == ORC_BC_PERIODIC) != (c->bc[1] == ORC_BC_PERIODIC)) return -1;
    if ((c->bc[2] == ORC_BC_PERIODIC) != (c->bc[3] == ORC_BC_PERIODIC)) return -1;
    if (c->limiter < 0 || c->limiter > 4 || c->sponge < 0) return -1;
    if (!(c->alpha >= 0.0 && c->alpha < 1.0) || !(c->gamma > 1.0)) return -1;
    if (has_dirichlet(c)) {
        const orc_field *f = c->field;
        if (!f || f->nplanes < 0 || f->nplanes > 2 || !(c->dx > 0.0)) return -1;
        if (!state_in_G(f->in) || !state_in_G(f->out)) return -1;
    }
    return 0;
}

/* ---------------------------------------------------------------- physics */

/* Euler x-flux f(u) = (m1, m1 v1 + p, m2 v1, (E + p) v1), ideal gas (Sec. 1). */
void orc_flux_x(double gamma, const double u[4], double f[4]) {
    double rho = u[0], v1 = u[1] / rho, v2 = u[2] / rho;
    double p = (gamma - 1.0) * (u[3] - 0.5 * rho * (v1 * v1 + v2 * v2));
    f[0] = u[1];
    f[1] = u[1] * v1 + p;
    f[2] = u[2] * v1;
    f[3] = (u[3] + p) * v1;
}

/* Euler y-flux g(u) = (m2, m1 v2, m2 v2 + p, (E + p) v2). */
void orc_flux_y(double gamma, const double u[4], double g[4]) {
    double rho = u[0], v1 = u[1] / rho, v2 = u[2] / rho;
    double p = (gamma - 1.0) * (u[3] - 0.5 * rho * (v1 * v1 + v2 * v2));
    g[0] = u[2];
    g[1] = u[1] * v2;
    g[2] = u[2] * v2 + p;
    g[3] = (u[3] + p) * v2;
}

/* D2Q5 Maxwellians of Example "Five-wave (D2Q5) model":
 * M_1,2 = (1-alpha)/4 u +- f/(2a), M_3,4 = (1-alpha)/4 u +- g/(2a), M_5 = alpha u. */
void orc_maxwellians(double gamma, double alpha, double a, const double u[4], double M[5][4]) {
    double f[4], g[4];
    orc_flux_x(gamma, u, f);
    orc_flux_y(gamma, u, g);
    double w = (1.0 - alpha) / 4.0;
    for (int c = 0; c < 4; ++c) {
        M[0][c] = w * u[c] + f[c] / (2.0 * a);
        M[1][c] = w * u[c] - f[c] / (2.0 * a);
        M[2][c] = w * u[c] + g[c] / (2.0 * a);
        M[3][c] = w * u[c] - g[c] / (2.0 * a);
        M[4][c] = alpha * u[c];
    }
}

/* |v| + sqrt(gamma p / rho) of one state; NaN outside G. */
static double cell_speed(double gamma, double rho, double m1, double m2, double E) {
    double v1 = m1 / rho, v2 = m2 / rho;
    double p = (gamma - 1.0) * (E - 0.5 * rho * (v1 * v1 + v2 * v2));
    if (!(rho > 0.0) || !(p >= 0.0)) return NAN;
    return sqrt(v1 * v1 + v2 * v2) + sqrt(gamma * p / rho);
}

/* lambda^n of the numerical section: max of sqrt(v1^2+v2^2) + sqrt(gamma p / rho)
 * over the cells, and over the Dirichlet field's two states if the boundary has a
 * Dirichlet part (reading: the prescribed states are cells of the flow too). */
double orc_max_speed(const orc_cfg *c, const double *s) {
    size_t N = (size_t)c->nx * c->ny;
    double lam = 0.0;
    for (size_t k = 0; k < N; ++k) {
        double sp = cell_speed(c->gamma, s[k], s[N + k], s[2 * N + k], s[3 * N + k]);
        if (!(sp == sp)) return NAN;
        if (sp > lam) lam = sp;
    }
    if (has_dirichlet(c) && c->field) {
        const double *st[2] = {c->field->in, c->field->out};
        for (int k = 0; k < 2; ++k) {
            double sp = cell_speed(c->gamma, st[k][0], st[k][1], st[k][2], st[k][3]);
            if (!(sp == sp)) return NAN;
            if (sp > lam) lam = sp;
        }
    }
    return lam;
}

void orc_init_populations(const orc_cfg *c, double a, double *s) {
    size_t N = (size_t)c->nx * c->ny;
    for (size_t k = 0; k < N; ++k) {
        double u[4] = {s[k], s[N + k], s[2 * N + k], s[3 * N + k]};
        double M[5][4];
        orc_maxwellians(c->gamma, c->alpha, a, u, M);
        for (int q = 1; q <= 4; ++q)
            for (int cc = 0; cc < 4; ++cc) s[(size_t)(4 * q + cc) * N + k] = M[q - 1][cc];
    }
}

/* ---------------------------------------------------------------- limiters */

/* PP density bound of Sec. 3.3.3: theta < kappa rho* / |dF^rho|, made strict by eps. */
double orc_theta_rho_pp(double kappa, double eps, double rs, double dfr) {
    if (dfr == 0.0) return 1.0;
    double t = kappa * rs / fabs(dfr) - eps;
    return t > 0.0 ? t : 0.0;
}

/* LMP density bound of Sec. 3.3.1, the three printed cases. (mu_l, nu_l) are the
 * bounds of the cell left of (below) the face, (mu_r, nu_r) those of the cell right
 * of (above) it. */
double orc_theta_rho_lmp(double kappa, double rs, double dfr,
                         double mu_l, double nu_l, double mu_r, double nu_r) {
    if (dfr == 0.0) return 1.0;
    if (dfr > 0.0) {
        double a1 = nu_r - rs, a2 = rs - mu_l;
        return kappa * (a1 < a2 ? a1 : a2) / dfr;
    }
    double b1 = rs - mu_r, b2 = nu_l - rs;
    return -kappa * (b1 < b2 ? b1 : b2) / dfr;
}

/* Closed-form spectral radius of B^{-1/2} A B^{-1/2} (Sec. 3.4):
 * max(|dF^rho| / rho*, (|gamma_1| + sqrt(Delta)) / (-2 gamma_0)).
 * Returns a negative number when u* is not in G (rho* <= 0 or gamma_0 >= 0). */
double orc_gql_radius(const double us[4], const double df[4]) {
    double rs = us[0], m1 = us[1], m2 = us[2], Es = us[3];
    double dr = df[0], dm1 = df[1], dm2 = df[2], dE = df[3];
    double g0 = m1 * m1 + m2 * m2 - 2.0 * rs * Es;
    if (!(rs > 0.0) || !(g0 < 0.0)) return -1.0;
    double g1 = 2.0 * (dr * Es + dE * rs - dm1 * m1 - dm2 * m2);
    double cq = dm1 * dm1 + dm2 * dm2 - 2.0 * dr * dE;
    double disc = g1 * g1 - 4.0 * g0 * cq;
    if (disc < 0.0) disc = 0.0;
    double r1 = fabs(dr) / rs;
    double r2 = (fabs(g1) + sqrt(disc)) / (-2.0 * g0);
    return r1 > r2 ? r1 : r2;
}

/* Internal-energy bound of Sec. 3.4: theta_p = max(0, kappa / radius - eps). */
double orc_theta_p(double kappa, double eps, const double us[4], const double df[4]) {
    double r = orc_gql_radius(us, df);
    if (r < 0.0) return 0.0;
    if (r == 0.0) return 1.0;
    double t = kappa / r - eps;
    return t > 0.0 ? t : 0.0;
}

/* ---------------------------------------------------------------- ghost frame */

typedef struct {
    int nx, ny, ex, ey;   /* interior and extended sizes */
    double *p[NPLANE];    /* ext planes, cell (I, J) at J*ex + I, I = i + G */
} ext_t;

static int src_index(int i, int n, int bc) {
    if (i >= 0 && i < n) return i;
    if (bc == ORC_BC_PERIODIC) return i < 0 ? i + n : i - n;
    if (bc == ORC_BC_ZEROGRAD) return i < 0 ? 0 : n - 1;
    return i < 0 ? -1 - i : 2 * n - 1 - i;        /* reflective mirror */
}

/* Type of side s (0 west, 1 east, 2 south, 3 north) at index k along it. */
static int side_type(const orc_cfg *c, int s, int k) {
    return k < c->split[s] ? c->bc[s] : c->bc_hi[s];
}

/* The Dirichlet field's state at the centre of cell (i, j) at time t. */
static const double *field_state(const orc_cfg *c, double t, int i, int j) {
    const orc_field *f = c->field;
    double x = c->x0 + (i + 0.5) * c->dx, y = c->y0 + (j + 0.5) * c->dx;
    for (int k = 0; k < f->nplanes; ++k)
        if (!(f->nx[k] * x + f->ny[k] * y >= f->c0[k] + f->c1[k] * t)) return f->out;
    return f->in;
}

/* Copy the 20 values of ext cell (si, sj) into ext cell (di, dj), applying the
 * mirror transform across an x-wall (axis 0) or a y-wall (axis 1) if asked. */
static void copy_cell(ext_t *e, int di, int dj, int si, int sj, int mirror_axis) {
    double v[NPLANE];
    for (int q = 0; q < NPLANE; ++q) v[q] = e->p[q][(size_t)sj * e->ex + si];
    if (mirror_axis == 0) {
        /* normal momentum m1 changes sign in u and every population; u_1 <-> u_2 */
        double t[4];
        for (int c = 0; c < 4; ++c) { t[c] = v[4 + c]; v[4 + c] = v[8 + c]; v[8 + c] = t[c]; }
        for (int q = 0; q < 5; ++q) v[4 * q + 1] = -v[4 * q + 1];
    } else if (mirror_axis == 1) {
        double t[4];
        for (int c = 0; c < 4; ++c) { t[c] = v[12 + c]; v[12 + c] = v[16 + c]; v[16 + c] = t[c]; }
        for (int q = 0; q < 5; ++q) v[4 * q + 2] = -v[4 * q + 2];
    }
    for (int q = 0; q < NPLANE; ++q) e->p[q][(size_t)dj * e->ex + di] = v[q];
}

static int ext_alloc(ext_t *e, int nx, int ny) {
    e->nx = nx; e->ny = ny; e->ex = nx + 2 * G; e->ey = ny + 2 * G;
    size_t n = (size_t)e->ex * e->ey;
    double *blk = (double *)calloc(n * NPLANE, sizeof(double));
    if (!blk) return -1;
    for (int q = 0; q < NPLANE; ++q) e->p[q] = blk + (size_t)q * n;
    return 0;
}

static void ext_free(ext_t *e) { free(e->p[0]); }

/* Ghost cell (i, j) of a Dirichlet part: the field's state and its Maxwellians
 * (populations at equilibrium) at kinetic speed a. */
static void set_dirichlet(const orc_cfg *c, double a, double t, ext_t *e, int i, int j) {
    const double *u = field_state(c, t, i, j);
    double M[5][4];
    orc_maxwellians(c->gamma, c->alpha, a, u, M);
    size_t id = (size_t)(j + G) * e->ex + (i + G);
    for (int cc = 0; cc < 4; ++cc) {
        e->p[cc][id] = u[cc];
        for (int k = 0; k < 4; ++k) e->p[4 * (k + 1) + cc][id] = M[k][cc];
    }
}

/* One ghost cell (i, j) of side s, index k along it: its type's rule. */
static void fill_ghost(const orc_cfg *c, double a, double t, ext_t *e, int s, int i, int j, int k) {
    const int type = side_type(c, s, k);
    if (type == ORC_BC_DIRICHLET) {
        set_dirichlet(c, a, t, e, i, j);
    } else if (s < 2) {
        copy_cell(e, i + G, j + G, src_index(i, c->nx, type) + G, j + G, type == ORC_BC_REFLECT ? 0 : -1);
    } else {
        copy_cell(e, i + G, j + G, i + G, src_index(j, c->ny, type) + G, type == ORC_BC_REFLECT ? 1 : -1);
    }
}

/* Interior copy, then x ghosts of interior rows, then y ghosts of all columns
 * (corners take the y rule applied to the x ghosts). */
static void fill_ext(const orc_cfg *c, double a, double t, const double *in, ext_t *e) {
    int nx = c->nx, ny = c->ny;
    size_t N = (size_t)nx * ny;
    for (int q = 0; q < NPLANE; ++q)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                e->p[q][(size_t)(j + G) * e->ex + (i + G)] = in[q * N + (size_t)j * nx + i];
    for (int j = 0; j < ny; ++j)
        for (int k = 1; k <= G; ++k) {
            fill_ghost(c, a, t, e, 0, -k, j, j);
            fill_ghost(c, a, t, e, 1, nx - 1 + k, j, j);
        }
    for (int i = -G; i < nx + G; ++i)
        for (int k = 1; k <= G; ++k) {
            fill_ghost(c, a, t, e, 2, i, -k, i);
            fill_ghost(c, a, t, e, 3, i, ny - 1 + k, i);
        }
}

int orc_fill_ghosts(const orc_cfg *c, double a, double t, const double *in, double *ext) {
    if (orc_check_cfg(c) || !(a > 0.0)) return -1;
    ext_t e;
    if (ext_alloc(&e, c->nx, c->ny)) return -1;
    fill_ext(c, a, t, in, &e);
    size_t n = (size_t)e.ex * e.ey;
    for (int q = 0; q < NPLANE; ++q) memcpy(ext + (size_t)q * n, e.p[q], n * sizeof(double));
    ext_free(&e);
    return 0;
}

/* ---------------------------------------------------------------- one step */

/* Per-face and per-cell work arrays of one step, all on the extended grid.
 * x-face between ext cells (I, J) and (I+1, J) is stored at J*ex + I;
 * y-face between (I, J) and (I, J+1) at J*ex + I. */
typedef struct {
    double *M[4][4];          /* M_k(u) component c for k = 1..4 at M[k-1][c] */
    double *us_x[4], *df_x[4], *us_y[4], *df_y[4];
    double *mu, *nu;
    double *thr_x, *thr_y, *thp_x, *thp_y, *th_x, *th_y;
    double *blk;
} work_t;

static int work_alloc(work_t *w, size_t n) {
    int count = 16 + 16 + 2 + 6;
    w->blk = (double *)calloc(n * count, sizeof(double));
    if (!w->blk) return -1;
    double *p = w->blk;
    for (int k = 0; k < 4; ++k) for (int c = 0; c < 4; ++c) { w->M[k][c] = p; p += n; }
    for (int c = 0; c < 4; ++c) { w->us_x[c] = p; p += n; }
    for (int c = 0; c < 4; ++c) { w->df_x[c] = p; p += n; }
    for (int c = 0; c < 4; ++c) { w->us_y[c] = p; p += n; }
    for (int c = 0; c < 4; ++c) { w->df_y[c] = p; p += n; }
    w->mu = p; p += n; w->nu = p; p += n;
    w->thr_x = p; p += n; w->thr_y = p; p += n;
    w->thp_x = p; p += n; w->thp_y = p; p += n;
    w->th_x = p; p += n; w->th_y = p; p += n;
    return 0;
}

/* Cell (i, j) (ghost cells included) lies in the sponge layer of Sec. 4.2: within
 * c->sponge cells of a zero-gradient side (a side that is zero-gradient along its
 * whole length). */
static int in_sponge(const orc_cfg *c, int i, int j) {
    const int s = c->sponge;
    if (s <= 0) return 0;
    int zg[4];
    for (int k = 0; k < 4; ++k) zg[k] = c->bc[k] == ORC_BC_ZEROGRAD && c->bc_hi[k] == ORC_BC_ZEROGRAD;
    return (zg[0] && i < s) || (zg[1] && i >= c->nx - s) || (zg[2] && j < s) || (zg[3] && j >= c->ny - s);
}

/* Steps a3-a8 of the scheme on the extended grid: equilibria, face states u* and
 * dF, density bounds, theta. Shared by the kinetic and the flux-form updates. */
static void compute_theta(const orc_cfg *c, double a, const ext_t *e, work_t *w) {
    const int ex = e->ex, ey = e->ey;
    const double kappa = a * (1.0 - c->alpha) / 2.0;       /* Sec. 3.2, after eq. (convex_decomposition_blending) */

    /* a3: Maxwellians of every extended cell */
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int J = 0; J < ey; ++J)
        for (int I = 0; I < ex; ++I) {
            size_t id = (size_t)J * ex + I;
            double u[4] = {e->p[0][id], e->p[1][id], e->p[2][id], e->p[3][id]};
            double M[5][4];
            orc_maxwellians(c->gamma, c->alpha, a, u, M);
            for (int k = 0; k < 4; ++k) for (int cc = 0; cc < 4; ++cc) w->M[k][cc][id] = M[k][cc];
        }

    /* a4: intermediate states (eq. D2Q5_convexproof_3 with 2 beta lambda = 2 kappa)
     * and second-order corrections (eq. 2nd-order_flux) on every face. dF is
     * evaluated as a [(M_1 - u_1)_L - (M_2 - u_2)_R]: on a mirror face both brackets
     * are the same numbers, so dF^rho is exactly 0 there, as it is in exact
     * arithmetic (the LMP bound of Sec. 3.3.1 jumps at dF^rho = 0). */
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int J = 0; J < ey; ++J)
        for (int I = 0; I < ex; ++I) {
            size_t L = (size_t)J * ex + I;
            double uL[4] = {e->p[0][L], e->p[1][L], e->p[2][L], e->p[3][L]}, fL[4], gL[4];
            orc_flux_x(c->gamma, uL, fL);
            orc_flux_y(c->gamma, uL, gL);
            if (I + 1 < ex) {
                size_t R = L + 1;
                double uR[4] = {e->p[0][R], e->p[1][R], e->p[2][R], e->p[3][R]}, fR[4];
                orc_flux_x(c->gamma, uR, fR);
                for (int cc = 0; cc < 4; ++cc) {
                    w->us_x[cc][L] = 0.5 * (uL[cc] + uR[cc]) - (fR[cc] - fL[cc]) / (2.0 * kappa);
                    w->df_x[cc][L] = a * ((w->M[0][cc][L] - e->p[4 + cc][L])
                                          - (w->M[1][cc][R] - e->p[8 + cc][R]));
                }
            }
            if (J + 1 < ey) {
                size_t R = L + ex;
                double uR[4] = {e->p[0][R], e->p[1][R], e->p[2][R], e->p[3][R]}, gR[4];
                orc_flux_y(c->gamma, uR, gR);
                for (int cc = 0; cc < 4; ++cc) {
                    w->us_y[cc][L] = 0.5 * (uL[cc] + uR[cc]) - (gR[cc] - gL[cc]) / (2.0 * kappa);
                    w->df_y[cc][L] = a * ((w->M[2][cc][L] - e->p[12 + cc][L])
                                          - (w->M[3][cc][R] - e->p[16 + cc][R]));
                }
            }
        }

    /* a5: local density bounds (eq. LMP_minmax; relaxed by 0.999 / 1.001 for RLMP) */
    if (c->limiter == ORC_LIM_LMP || c->limiter == ORC_LIM_RLMP) {
#pragma omp parallel for num_threads(g_threads) schedule(static)
        for (int J = 1; J < ey - 1; ++J)
            for (int I = 1; I < ex - 1; ++I) {
                size_t id = (size_t)J * ex + I;
                double v[5] = {e->p[0][id], w->us_x[0][id - 1], w->us_x[0][id],
                               w->us_y[0][id - ex], w->us_y[0][id]};
                double lo = v[0], hi = v[0];
                for (int k = 1; k < 5; ++k) { if (v[k] < lo) lo = v[k]; if (v[k] > hi) hi = v[k]; }
                if (c->limiter == ORC_LIM_RLMP) { lo *= 0.999; hi *= 1.001; }
                w->mu[id] = lo;
                w->nu[id] = hi;
            }
    }

    /* a6-a8: theta_rho, theta_p and theta = min(1, theta_rho, theta_p) on the faces
     * that touch an interior cell; theta = 0 on the faces of sponge-layer cells */
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int J = G - 1; J < ey - G + 1; ++J)
        for (int I = G - 1; I < ex - G + 1; ++I) {
            size_t L = (size_t)J * ex + I;
            for (int dir = 0; dir < 2; ++dir) {
                size_t R = dir == 0 ? L + 1 : L + ex;
                double *const *us = dir == 0 ? w->us_x : w->us_y;
                double *const *df = dir == 0 ? w->df_x : w->df_y;
                double usv[4] = {us[0][L], us[1][L], us[2][L], us[3][L]};
                double dfv[4] = {df[0][L], df[1][L], df[2][L], df[3][L]};
                double thr = 1.0, thp = 1.0, th;
                if (c->limiter == ORC_LIM_FIRST) {
                    th = 0.0;
                } else if (c->limiter == ORC_LIM_SECOND) {
                    th = 1.0;
                } else {
                    if (c->limiter == ORC_LIM_PP)
                        thr = orc_theta_rho_pp(kappa, c->eps, usv[0], dfv[0]);
                    else
                        thr = orc_theta_rho_lmp(kappa, usv[0], dfv[0], w->mu[L], w->nu[L],
                                                w->mu[R], w->nu[R]);
                    thp = orc_theta_p(kappa, c->eps, usv, dfv);
                    th = 1.0;
                    if (thr < th) th = thr;
                    if (thp < th) th = thp;
                    if (th < 0.0) th = 0.0;
                }
                const int iL = I - G, jL = J - G;
                if (in_sponge(c, iL, jL) || in_sponge(c, dir == 0 ? iL + 1 : iL, dir == 0 ? jL : jL + 1))
                    th = 0.0;
                if (dir == 0) { w->thr_x[L] = thr; w->thp_x[L] = thp; w->th_x[L] = th; }
                else          { w->thr_y[L] = thr; w->thp_y[L] = thp; w->th_y[L] = th; }
            }
        }
}

static void export_debug(const orc_cfg *c, const ext_t *e, const work_t *w, orc_debug *d) {
    if (!d) return;
    int nx = c->nx, ny = c->ny, ex = e->ex;
    for (int j = 0; j < ny; ++j)
        for (int i = -1; i < nx; ++i) {
            size_t f = (size_t)j * (nx + 1) + (i + 1);
            size_t L = (size_t)(j + G) * ex + (i + G);
            if (d->theta_x) d->theta_x[f] = w->th_x[L];
            if (d->theta_rho_x) d->theta_rho_x[f] = w->thr_x[L];
            if (d->theta_p_x) d->theta_p_x[f] = w->thp_x[L];
            for (int cc = 0; cc < 4; ++cc) {
                if (d->ustar_x) d->ustar_x[4 * f + cc] = w->us_x[cc][L];
                if (d->dflux_x) d->dflux_x[4 * f + cc] = w->df_x[cc][L];
            }
        }
    for (int j = -1; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t f = (size_t)(j + 1) * nx + i;
            size_t L = (size_t)(j + G) * ex + (i + G);
            if (d->theta_y) d->theta_y[f] = w->th_y[L];
            if (d->theta_rho_y) d->theta_rho_y[f] = w->thr_y[L];
            if (d->theta_p_y) d->theta_p_y[f] = w->thp_y[L];
            for (int cc = 0; cc < 4; ++cc) {
                if (d->ustar_y) d->ustar_y[4 * f + cc] = w->us_y[cc][L];
                if (d->dflux_y) d->dflux_y[4 * f + cc] = w->df_y[cc][L];
            }
        }
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t L = (size_t)(j + G) * ex + (i + G);
            if (d->mu) d->mu[(size_t)j * nx + i] = w->mu[L];
            if (d->nu) d->nu[(size_t)j * nx + i] = w->nu[L];
        }
}

/* a9, kinetic form: eq. (blending_u1) pulls u_1..u_4 from the upwind neighbour;
 * eq. (blending_u) updates u with the local terms of the eliminated u_5. */
int orc_step(const orc_cfg *c, double a, double t, const double *in, double *out, orc_debug *dbg) {
    if (orc_check_cfg(c) || !(a > 0.0)) return -1;
    ext_t e;
    work_t w;
    if (ext_alloc(&e, c->nx, c->ny)) return -1;
    if (work_alloc(&w, (size_t)e.ex * e.ey)) { ext_free(&e); return -1; }
    fill_ext(c, a, t, in, &e);
    compute_theta(c, a, &e, &w);
    export_debug(c, &e, &w, dbg);

    const int nx = c->nx, ny = c->ny, ex = e.ex;
    const size_t N = (size_t)nx * ny;
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t C = (size_t)(j + G) * ex + (i + G);
            size_t W = C - 1, E = C + 1, S = C - ex, Nn = C + ex;
            double t_w = w.th_x[W], t_e = w.th_x[C], t_s = w.th_y[S], t_n = w.th_y[C];
            size_t o = (size_t)j * nx + i;
            for (int cc = 0; cc < 4; ++cc) {
                double u1 = w.M[0][cc][W] + t_w * (w.M[0][cc][W] - e.p[4 + cc][W]);
                double u2 = w.M[1][cc][E] + t_e * (w.M[1][cc][E] - e.p[8 + cc][E]);
                double u3 = w.M[2][cc][S] + t_s * (w.M[2][cc][S] - e.p[12 + cc][S]);
                double u4 = w.M[3][cc][Nn] + t_n * (w.M[3][cc][Nn] - e.p[16 + cc][Nn]);
                double u = u1 + u2 + u3 + u4 + c->alpha * e.p[cc][C]
                           - t_w * (w.M[1][cc][C] - e.p[8 + cc][C])
                           - t_e * (w.M[0][cc][C] - e.p[4 + cc][C])
                           - t_s * (w.M[3][cc][C] - e.p[16 + cc][C])
                           - t_n * (w.M[2][cc][C] - e.p[12 + cc][C]);
                out[(size_t)cc * N + o] = u;
                out[(size_t)(4 + cc) * N + o] = u1;
                out[(size_t)(8 + cc) * N + o] = u2;
                out[(size_t)(12 + cc) * N + o] = u3;
                out[(size_t)(16 + cc) * N + o] = u4;
            }
        }
    free(w.blk);
    ext_free(&e);
    return 0;
}

/* a9, flux form of Sec. 3.2: u^{n+1} = u - (1/a)[F_{i+1/2} - F_{i-1/2} + G_{j+1/2} - G_{j-1/2}]
 * with F = F^(1) + theta dF (eq. 1st-order_flux), and the blended moments
 * v_1, v_2, w_1, w_2 mapped back to u_1..u_4 by the first four rows of Q^{-1}. */
int orc_step_fv(const orc_cfg *c, double a, double t, const double *in, double *out) {
    if (orc_check_cfg(c) || !(a > 0.0)) return -1;
    ext_t e;
    work_t w;
    if (ext_alloc(&e, c->nx, c->ny)) return -1;
    if (work_alloc(&w, (size_t)e.ex * e.ey)) { ext_free(&e); return -1; }
    fill_ext(c, a, t, in, &e);
    compute_theta(c, a, &e, &w);

    const int nx = c->nx, ny = c->ny, ex = e.ex;
    const size_t N = (size_t)nx * ny;
    const double lf = a * (1.0 - c->alpha) / 4.0;
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t C = (size_t)(j + G) * ex + (i + G);
            size_t W = C - 1, E = C + 1, S = C - ex, Nn = C + ex;
            double uc[4], uw[4], ue[4], us[4], un[4];
            double fc[4], fw[4], fe[4], gc[4], gs[4], gn[4];
            for (int cc = 0; cc < 4; ++cc) {
                uc[cc] = e.p[cc][C]; uw[cc] = e.p[cc][W]; ue[cc] = e.p[cc][E];
                us[cc] = e.p[cc][S]; un[cc] = e.p[cc][Nn];
            }
            orc_flux_x(c->gamma, uc, fc); orc_flux_x(c->gamma, uw, fw); orc_flux_x(c->gamma, ue, fe);
            orc_flux_y(c->gamma, uc, gc); orc_flux_y(c->gamma, us, gs); orc_flux_y(c->gamma, un, gn);
            size_t o = (size_t)j * nx + i;
            for (int cc = 0; cc < 4; ++cc) {
                double Fe = 0.5 * (fc[cc] + fe[cc]) - lf * (ue[cc] - uc[cc]) + w.th_x[C] * w.df_x[cc][C];
                double Fw = 0.5 * (fw[cc] + fc[cc]) - lf * (uc[cc] - uw[cc]) + w.th_x[W] * w.df_x[cc][W];
                double Gn = 0.5 * (gc[cc] + gn[cc]) - lf * (un[cc] - uc[cc]) + w.th_y[C] * w.df_y[cc][C];
                double Gs = 0.5 * (gs[cc] + gc[cc]) - lf * (uc[cc] - us[cc]) + w.th_y[S] * w.df_y[cc][S];
                double unew = uc[cc] - (Fe - Fw + Gn - Gs) / a;

                double m1w = w.M[0][cc][W], m2e = w.M[1][cc][E], m3s = w.M[2][cc][S], m4n = w.M[3][cc][Nn];
                double c1 = w.th_x[W] * (m1w - e.p[4 + cc][W]);
                double c2 = w.th_x[C] * (m2e - e.p[8 + cc][E]);
                double c3 = w.th_y[S] * (m3s - e.p[12 + cc][S]);
                double c4 = w.th_y[C] * (m4n - e.p[16 + cc][Nn]);
                double v1 = m1w - m2e + c1 - c2;
                double v2 = m3s - m4n + c3 - c4;
                double w1 = m1w + m2e + c1 + c2;
                double w2 = m3s + m4n + c3 + c4;
                out[(size_t)cc * N + o] = unew;
                out[(size_t)(4 + cc) * N + o] = 0.5 * v1 + 0.5 * w1;
                out[(size_t)(8 + cc) * N + o] = -0.5 * v1 + 0.5 * w1;
                out[(size_t)(12 + cc) * N + o] = 0.5 * v2 + 0.5 * w2;
                out[(size_t)(16 + cc) * N + o] = -0.5 * v2 + 0.5 * w2;
            }
        }
    free(w.blk);
    ext_free(&e);
    return 0;
}
