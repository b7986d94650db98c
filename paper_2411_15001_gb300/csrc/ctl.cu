// ctl.cu -- kernels on the device control block alone (reset, final time,
// checkpoint header) and their launchers.
#include "common.cuh"

#include <math.h>

namespace vlbm {

static bool state_in_G(const double u[4]) {
    for (int q = 0; q < 4; ++q)
        if (!(u[q] == u[q]) || u[q] == HUGE_VAL || u[q] == -HUGE_VAL) return false;
    return u[0] > 0.0 && u[3] - 0.5 * (u[1] * u[1] + u[2] * u[2]) / u[0] > 0.0;
}

const char *make_bound(const vlbm_grid &g, const vlbm_boundary *b, Bound *out) {
    Bound B;
    memset(&B, 0, sizeof B);
    for (int s = 0; s < 4; ++s) {
        const int n = s < 2 ? g.ny : g.nx;   // cells along side s
        B.lo[s] = g.bc[s];
        B.hi[s] = b ? b->bc_hi[s] : g.bc[s];
        B.split[s] = b ? b->split[s] : 0;
        if (B.lo[s] < VLBM_BC_PERIODIC || B.lo[s] > VLBM_BC_DIRICHLET || B.hi[s] < VLBM_BC_PERIODIC ||
            B.hi[s] > VLBM_BC_DIRICHLET)
            return "boundary type out of range";
        if (B.split[s] == 0 ? B.hi[s] != B.lo[s] : (B.split[s] < 2 || B.split[s] > n - 2))
            return "split: 0 with bc_hi = bc, or 2 <= split <= n - 2 along the side";
        if ((B.lo[s] == VLBM_BC_PERIODIC || B.hi[s] == VLBM_BC_PERIODIC) && B.split[s] != 0)
            return "a periodic side cannot switch type";
        if (B.lo[s] == VLBM_BC_DIRICHLET || B.hi[s] == VLBM_BC_DIRICHLET) B.has_dir = 1;
    }
    if ((B.lo[0] == VLBM_BC_PERIODIC) != (B.lo[1] == VLBM_BC_PERIODIC) ||
        (B.lo[2] == VLBM_BC_PERIODIC) != (B.lo[3] == VLBM_BC_PERIODIC))
        return "a periodic side must face a periodic side";
    if (B.has_dir) {
        if (!b) return "VLBM_BC_DIRICHLET needs opts->boundary for its field";
        const vlbm_field &f = b->field;
        if (f.nplanes < 0 || f.nplanes > 2) return "field: nplanes must be 0, 1 or 2";
        if (!state_in_G(f.in) || !state_in_G(f.out)) return "field: both states must be finite and in G";
        B.nplanes = f.nplanes;
        for (int k = 0; k < 2; ++k) {
            B.pnx[k] = f.nx[k];
            B.pny[k] = f.ny[k];
            B.c0[k] = f.c0[k];
            B.c1[k] = f.c1[k];
        }
        for (int q = 0; q < 4; ++q) {
            B.in[q] = f.in[q];
            B.out[q] = f.out[q];
        }
    }
    if (b) {
        B.x0 = b->x0;
        B.y0 = b->y0;
    }
    B.dx = g.dx;
    B.ctl = nullptr;
    *out = B;
    return nullptr;
}

__global__ void k_ctl_reset(DevCtl *C, double dx, double alpha, double a_fixed, double eps,
                            double gamma) {
    C->n = 0;
    C->t = 0.0;
    C->a = C->dt = C->a_free = 0.0;
    C->t_end = 0.0;
    C->last = 0;
    C->done = 0;
    C->status = 0;
    C->invalid_init = 0;
    C->first_bad_step = -1;
    C->wait_probe_ns = 0u;
    reset_slots(C);
    C->lambda = 0.0;
    C->min_rho = 0.0;
    C->bad_last = C->nonfinite_last = 0;
    for (int c = 0; c < 4; ++c) C->sum_last[c] = 0.0;
    C->dx = dx;
    C->alpha = alpha;
    C->a_fixed = a_fixed;
    C->eps = eps;
    C->gamma = gamma;
    C->lam_bc = 0.0;
}

// Final time for vlbm_step_to (t_end > 0) or none (t_end <= 0).
__global__ void k_set_tend(DevCtl *C, double t_end) {
    C->t_end = t_end > 0.0 ? t_end : 0.0;
    if (!C->status && !C->invalid_init) C->done = 0;
    plan_next(C, C->t, C->a_free);
}

__global__ void k_load_header(DevCtl *C, const unsigned char *src) {
    const double *h = (const double *)src;
    const long long *hl = (const long long *)src;
    C->n = hl[0];
    C->t = h[1];
    C->a = h[2];
    C->dt = h[3];
    C->a_free = h[4];
    C->t_end = h[5];
    C->last = (int)(hl[6] & 1);
    C->done = (int)((hl[6] >> 1) & 1);
    C->status = (int)hl[7];
    C->invalid_init = 0;
    C->first_bad_step = -1;
    reset_slots(C);
    set_consts(C);
}

cudaError_t launch_ctl_reset(DevCtl *ctl, double dx, double alpha, double a_fixed, double eps,
                             double gamma, cudaStream_t s) {
    k_ctl_reset<<<1, 1, 0, s>>>(ctl, dx, alpha, a_fixed, eps, gamma);
    return cudaGetLastError();
}

cudaError_t launch_set_tend(DevCtl *ctl, double t_end, cudaStream_t s) {
    k_set_tend<<<1, 1, 0, s>>>(ctl, t_end);
    return cudaGetLastError();
}

cudaError_t launch_load_header(DevCtl *ctl, const void *src, cudaStream_t s) {
    k_load_header<<<1, 1, 0, s>>>(ctl, (const unsigned char *)src);
    return cudaGetLastError();
}

// Launch shapes shared by the stream launchers and the graph builder.
void simple_launch_shape(int nx, int ny, dim3 *grid, dim3 *block) {
    *block = dim3(32, 8);
    *grid = dim3((nx + 31) / 32, (ny + 7) / 8);
}

void ghosts_launch_shape(int nx, int ny, dim3 *grid, dim3 *block) {
    const long long total = 4ll * (nx + 4) + 4ll * ny;
    *block = dim3(128);
    *grid = dim3((unsigned)((total + 127) / 128));
}

}  // namespace vlbm
