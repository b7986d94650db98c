// ctl.cu -- kernels on the device control block alone (reset, final time,
// checkpoint header) and their launchers.
#include "common.cuh"

namespace vlbm {

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
