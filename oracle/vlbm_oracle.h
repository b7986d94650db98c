/*
 * vlbm_oracle.h -- TEST INFRASTRUCTURE, not part of the product.
 *
 * A plain, slow FP64 CPU restatement of the blended D2Q5 vectorial lattice
 * Boltzmann scheme of Wissocq, Liu & Abgrall, "A positive- and bound-preserving
 * vectorial lattice Boltzmann method in two dimensions" (arXiv 2411.15001).
 * It exists only to check the CUDA library: the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark are its only callers. It shares no code,
 * header, table or constant with the CUDA path.
 *
 * State layout: 20 planes of nx*ny doubles, plane q at offset q*nx*ny, cell
 * (i, j) at j*nx + i (x fastest). Planes 0..3 are the conserved variables
 * u = (rho, m1, m2, E); planes 4k..4k+3 (k = 1..4) are the population u_k of the
 * D2Q5 velocity set e_1 = (a,0), e_2 = (-a,0), e_3 = (0,a), e_4 = (0,-a)
 * (Example "Five-wave (D2Q5) model", Sec. 2). u_5 is never stored: the update of
 * eq. (blending_u) only needs u and u_1..u_4.
 *
 * Parity is pinned for every function below by tests under tests/ (the Table 1
 * numbers of Sec. 4.1, closed forms, invariants and brute force). The one
 * unpinned reading is the relaxed-LMP L-infinity column of Table 1: at N = 20
 * this method gives 5.78185e-3 where 5.21913e-3 is printed, while its L1 and L2
 * columns match to six digits.
 */
#ifndef VLBM_ORACLE_H
#define VLBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BC_PERIODIC = 0, ORC_BC_ZEROGRAD = 1, ORC_BC_REFLECT = 2, ORC_BC_DIRICHLET = 3 };

/* Prescribed boundary field of the Dirichlet parts of the boundary (the double
 * Mach reflection of Sec. 4.7 and the jets of Sec. 4.8 set the distributions of
 * boundary cells to the Maxwellians of given states). At time t a Dirichlet ghost
 * cell with centre (x, y) holds the conserved state `in` if
 * nx[k] x + ny[k] y >= c0[k] + c1[k] t for every k < nplanes, else `out`; its
 * populations are M_1..M_4 of that state at the step's kinetic speed. */
typedef struct {
    double in[4], out[4];     /* conserved (rho, m1, m2, E), both inside G */
    int nplanes;              /* 0..2 half-planes */
    double nx[2], ny[2], c0[2], c1[2];
} orc_field;
enum { ORC_LIM_FIRST = 0, ORC_LIM_SECOND = 1, ORC_LIM_PP = 2, ORC_LIM_LMP = 3, ORC_LIM_RLMP = 4 };

typedef struct {
    int nx, ny;
    int bc[4];        /* west, east, south, north */
    int limiter;      /* ORC_LIM_*: theta = 0, theta = 1, or the convex limiters of Sec. 3.3-3.4 */
    double gamma;     /* ideal-gas heat capacity ratio */
    double alpha;     /* D2Q5 rest weight, 1/2 <= alpha < 1 (Prop. convex preservation) */
    double eps;       /* epsilon subtracted in the PP and pressure bounds (1e-16 in Sec. 3.3.3) */
    int sponge;       /* Sec. 4.2: theta = 0 on every face of the cells within `sponge` cells
                         of a zero-gradient side (0 = none) */
    /* A side may switch type once along its length (a partial wall, Sec. 4.7): the
     * ghost cells of side s whose index along the side (column i for south/north,
     * row j for west/east, ghost indices included) is below split[s] take type
     * bc[s], the others bc_hi[s]. split[s] = 0 with bc_hi[s] = bc[s] is a uniform
     * side; otherwise 2 <= split[s] <= n - 2, so that both ends of the side, with
     * the corner ghosts beyond them, are uniform. A periodic side does not switch. */
    int bc_hi[4];
    int split[4];
    double x0, y0, dx;        /* cell (i, j) has centre (x0 + (i + 1/2) dx, y0 + (j + 1/2) dx) */
    const orc_field *field;   /* required when some part of a side is ORC_BC_DIRICHLET */
} orc_cfg;

/* Optional per-face / per-cell outputs of one step. Any pointer may be NULL.
 * x-face i+1/2 (i = -1..nx-1) of row j is at j*(nx+1) + (i+1);
 * y-face j+1/2 (j = -1..ny-1) of column i is at (j+1)*nx + i;
 * 4-vectors (ustar, dflux) store component c at 4*face + c. */
typedef struct {
    double *theta_x, *theta_y;          /* final theta = min(1, theta_rho, theta_p) */
    double *theta_rho_x, *theta_rho_y;  /* density bound (PP / LMP / RLMP) */
    double *theta_p_x, *theta_p_y;      /* internal-energy bound (Sec. 3.4) */
    double *ustar_x, *ustar_y;          /* intermediate states u* (eq. D2Q5_convexproof_3) */
    double *dflux_x, *dflux_y;          /* Delta F, Delta G (eq. 2nd-order_flux) */
    double *mu, *nu;                    /* per-cell density bounds, nx*ny */
} orc_debug;

int    orc_check_cfg(const orc_cfg *c);
void   orc_set_threads(int n);
int    orc_get_threads(void);

/* Euler fluxes f(u), g(u) and the five D2Q5 Maxwellians M_k(u) (k = 1..5 at M[k-1]). */
void   orc_flux_x(double gamma, const double u[4], double f[4]);
void   orc_flux_y(double gamma, const double u[4], double g[4]);
void   orc_maxwellians(double gamma, double alpha, double a, const double u[4], double M[5][4]);

/* lambda = max over cells of |v| + sqrt(gamma p / rho) (Sec. 4 preamble); NaN if a
 * cell is outside the admissible set G. With a Dirichlet part on the boundary the
 * max also covers the field's two states, so that the kinetic speed satisfies
 * Bouchut's condition on the boundary faces too. */
double orc_max_speed(const orc_cfg *c, const double *state);

/* Populations u_k = M_k(u) (k = 1..4) from the conserved planes (Sec. 4 preamble). */
void   orc_init_populations(const orc_cfg *c, double a, double *state);

/* The two per-face limiter bounds of Sec. 3.3 and 3.4. */
double orc_theta_rho_pp(double kappa, double eps, double rho_star, double dflux_rho);
double orc_theta_rho_lmp(double kappa, double rho_star, double dflux_rho,
                         double mu_l, double nu_l, double mu_r, double nu_r);
double orc_theta_p(double kappa, double eps, const double ustar[4], const double dflux[4]);
/* spectral radius of B^{-1/2} A B^{-1/2} for the pair (ustar, dflux), closed form */
double orc_gql_radius(const double ustar[4], const double dflux[4]);

/* One time step from time t with kinetic speed a (Delta t = dx / a), kinetic form:
 * eq. (blending_u1) for u_1..u_4 and eq. (blending_u) for u. t only places the
 * Dirichlet field. Returns 0, or -1 on a bad configuration. in and out must not
 * alias. */
int    orc_step(const orc_cfg *c, double a, double t, const double *in, double *out, orc_debug *dbg);

/* The same step through the flux form and the moments of Sec. 3.2: u by the
 * blended finite-volume update with F = F^(1) + theta dF, populations from the
 * blended moments v_1, v_2, w_1, w_2 by Q^{-1} (eq. moments_matrix). */
int    orc_step_fv(const orc_cfg *c, double a, double t, const double *in, double *out);

/* The extended state of the ghost fill alone (x ghosts of interior rows, then y
 * ghosts of every column): 20 planes of (nx + 4) x (ny + 4) doubles, cell (i, j)
 * (ghosts included, i, j >= -2) at (j + 2) (nx + 4) + i + 2. */
int    orc_fill_ghosts(const orc_cfg *c, double a, double t, const double *in, double *ext);

#ifdef __cplusplus
}
#endif
#endif
