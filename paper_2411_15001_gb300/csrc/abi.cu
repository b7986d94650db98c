// abi.cu -- the extern "C" entry points of include/vlbm.h: argument checks,
// workspace carving, and stream-ordered launches of the step kernels.
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "state.h"

using namespace vlbm;
using namespace vlbm::api;



static thread_local char g_err[256];

namespace vlbm {
namespace api {
int fail(vlbm_state *s, int code, const char *fmt, ...) {
    char *dst = s ? s->err : g_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 256, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(vlbm_state *s, cudaError_t e, const char *what) {
    return fail(s, VLBM_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}
}  // namespace api
}  // namespace vlbm

namespace vlbm {
Layout make_layout(int nx, int ny, int elem) {
    Layout L;
    L.nx = nx;
    L.ny = ny;
    L.elem = elem;
    L.pitch = ((nx + 2 * kOX + 7) / 8) * 8;
    L.rows = ny + 2 * kOY;
    L.buf_bytes = (((size_t)L.rows * kNGroup * L.pitch * 4 * elem + 255) / 256) * 256;
    L.ctl_offset = 2 * L.buf_bytes;
    L.desc_offset = L.ctl_offset + ((sizeof(DevCtl) + 255) / 256) * 256;
    // descriptor block: InstDesc (512 B), BatchCtl (256 B), item table (bands of at
    // least the smallest height)
    L.total = L.desc_offset + 512 + 256 + ((max_items(nx, ny) * sizeof(WorkItem) + 255) / 256) * 256;
    return L;
}
}  // namespace vlbm

static bool grid_ok(const vlbm_grid *g) {
    if (!g || g->nx < 4 || g->ny < 4 || !(g->dx > 0.0)) return false;
    if ((long long)g->nx * g->ny > (1ll << 31)) return false;
    for (int k = 0; k < 4; ++k)
        if (g->bc[k] < VLBM_BC_PERIODIC || g->bc[k] > VLBM_BC_DIRICHLET) return false;
    if ((g->bc[0] == VLBM_BC_PERIODIC) != (g->bc[1] == VLBM_BC_PERIODIC)) return false;
    if ((g->bc[2] == VLBM_BC_PERIODIC) != (g->bc[3] == VLBM_BC_PERIODIC)) return false;
    return true;
}

static int elem_of(int32_t precision) {
    return precision == VLBM_FP64 ? 8 : precision == VLBM_FP32 ? 4 : 0;
}


static cudaError_t step_kernel_only(vlbm_state *s) {
    if (use_fused(s) && s->probe_armed) {
        if (s->precision == VLBM_FP64)
            return launch_step_fused_probe<double>(batch_args_of<double>(s), s->limiter, s->fused_grid, s->stream);
        return launch_step_fused_probe<float>(batch_args_of<float>(s), s->limiter, s->fused_grid, s->stream);
    }
    if (use_fused(s)) {
        if (s->precision == VLBM_FP64)
            return launch_step_fused<double>(batch_args_of<double>(s), s->limiter, s->fused_grid, s->stream);
        return launch_step_fused<float>(batch_args_of<float>(s), s->limiter, s->fused_grid, s->stream);
    }
    if (s->precision == VLBM_FP64) return launch_step_simple<double>(args_of<double>(s), s->stream);
    return launch_step_simple<float>(args_of<float>(s), s->stream);
}

// Before a step of a grid with a prescribed part: its ghosts at the step's t^n and
// a^n (the step kernels write every other ghost of the new state themselves).
static cudaError_t dirichlet_pass(vlbm_state *s) {
    if (!s->bd.has_dir) return cudaSuccess;
    if (s->precision == VLBM_FP64) return launch_dirichlet_ghosts<double>(args_of<double>(s), s->stream);
    return launch_dirichlet_ghosts<float>(args_of<float>(s), s->stream);
}

// Descriptor of this grid for the row-marching kernel, built on the host.
template <typename T>
static void build_desc(vlbm_state *s) {
    InstDesc<T> d;
    memset(&d, 0, sizeof d);
    d.tmap = s->tmap;
    d.buf0 = (T *)s->ws;
    d.buf1 = (T *)((char *)s->ws + s->L.buf_bytes);
    d.pitch = s->L.pitch;
    d.nx = s->grid.nx;
    d.ny = s->grid.ny;
    uniform_types(s->bd, d.bc);
    d.bd = s->bd;
    d.nitems = s->nitems;
    d.ctl = s->ctl;
    d.sponge = s->sponge;
    static_assert(sizeof(InstDesc<T>) <= 512, "descriptor block");
    s->desc_host.assign((unsigned char *)&d, (unsigned char *)&d + sizeof d);
}

// Upload the descriptor, the item table and a zero work counter (stream-ordered;
// the host copies live in the state).
static cudaError_t upload_desc(vlbm_state *s) {
    if (!use_fused(s)) return cudaSuccess;
    char *base = (char *)s->ws + s->L.desc_offset;
    cudaError_t e = cudaMemcpyAsync(base, s->desc_host.data(), s->desc_host.size(), cudaMemcpyHostToDevice,
                                    s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + 512, 0, sizeof(BatchCtl), s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + 768, s->items_host.data(), s->items_host.size() * sizeof(WorkItem),
                            cudaMemcpyHostToDevice, s->stream);
    return e;
}

// One time step: the prescribed ghosts of the state it reads (if any), then the
// collide + limit + stream kernel, which also writes the new state's ghost frame.
// With profiling on, an event pair brackets the step kernel.
cudaError_t vlbm::api::step_once(vlbm_state *s) {
    cudaError_t r;
    if (s->profiling) {
        if (s->ev_used + 2 > s->ev.size()) {
            for (int k = 0; k < 2; ++k) {
                cudaEvent_t e;
                r = cudaEventCreate(&e);
                if (r != cudaSuccess) return r;
                s->ev.push_back(e);
            }
        }
        r = dirichlet_pass(s);
        if (r == cudaSuccess) r = cudaEventRecord(s->ev[s->ev_used], s->stream);
        if (r == cudaSuccess) r = step_kernel_only(s);
        if (r == cudaSuccess) r = cudaEventRecord(s->ev[s->ev_used + 1], s->stream);
        s->ev_used += 2;
    } else {
        r = dirichlet_pass(s);
        if (r == cudaSuccess) r = step_kernel_only(s);
    }
    return r;
}

namespace vlbm {
// TMA descriptor of the two state buffers of a grid seen as one 4D tensor
// [2 buffers][ny + 4 rows][5 groups][4 pitch values] (a group row -- every column's
// four components -- is one contiguous dimension); a box is 64 columns (256 values) of
// all five groups of one row, so a strip row of 128 columns is two boxes. The box's
// innermost extent is 1 KB (FP32): a box with 16-byte innermost rows (one cell's group)
// was measured 4 % slower on the 4096^2 step. The innermost coordinate, 4 x the column,
// is always a multiple of 16 bytes, so a box may start at any column.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

bool encode_state_tmap(CUtensorMap *out, void *base, const Layout &L) {
    static EncodeTiledFn encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            return false;
        }
        encode = (EncodeTiledFn)fn;
    }
    const cuuint64_t dims[4] = {(cuuint64_t)4 * L.pitch, (cuuint64_t)kNGroup, (cuuint64_t)L.rows, 2u};
    const cuuint64_t strides[3] = {(cuuint64_t)4 * L.pitch * L.elem, (cuuint64_t)kNGroup * 4 * L.pitch * L.elem,
                                   (cuuint64_t)L.buf_bytes};
    const cuuint32_t box[4] = {(cuuint32_t)(4 * kFusedBox / 2), (cuuint32_t)kNGroup, 1u, 1u};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    CUresult r = encode(out, L.elem == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                        base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}
}  // namespace vlbm

// A graph of kGraphSteps steps: kernel nodes with the same arguments as the
// stream launches (the step kernel reads its buffers' parity from the control
// block, so every step's node is identical).
template <typename T>
static cudaError_t build_graph(vlbm_state *s) {
    cudaError_t e = cudaGraphCreate(&s->graph, 0);
    if (e != cudaSuccess) return e;
    cudaKernelNodeParams kp;
    memset(&kp, 0, sizeof kp);
    const bool fused = use_fused(s);
    FusedBatchArgs<T> B = batch_args_of<T>(s);
    StepArgs<T> A = args_of<T>(s);
    void *pf[] = {&B};
    void *pa[] = {&A};
    cudaKernelNodeParams kg;
    memset(&kg, 0, sizeof kg);
    const bool dir = s->bd.has_dir;   // prescribed ghosts before each step
    if (dir) {
        kg.func = const_cast<void *>(dirichlet_ghosts_kernel_fn<T>());
        ghosts_launch_shape(s->grid.nx, s->grid.ny, &kg.gridDim, &kg.blockDim);
        kg.kernelParams = pa;
    }
    if (fused) {
        size_t smem = 0;
        kp.func = const_cast<void *>(fused_kernel_fn<T>(s->limiter, &smem));
        kp.gridDim = dim3(s->fused_grid);
        kp.blockDim = dim3(kFusedBox);
        kp.sharedMemBytes = (unsigned)smem;
        kp.kernelParams = pf;
    } else {
        kp.func = const_cast<void *>(simple_kernel_fn<T>(s->limiter));
        simple_launch_shape(s->grid.nx, s->grid.ny, &kp.gridDim, &kp.blockDim);
        kp.kernelParams = pa;
    }
    cudaGraphNode_t prev = nullptr;
    for (int k = 0; k < kGraphSteps && e == cudaSuccess; ++k) {
        cudaGraphNode_t node;
        if (dir) {
            e = cudaGraphAddKernelNode(&node, s->graph, prev ? &prev : nullptr, prev ? 1 : 0, &kg);
            prev = node;
            if (e != cudaSuccess) break;
        }
        e = cudaGraphAddKernelNode(&node, s->graph, prev ? &prev : nullptr, prev ? 1 : 0, &kp);
        prev = node;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&s->gexec, s->graph, 0);
    if (e != cudaSuccess) {
        if (s->gexec) cudaGraphExecDestroy(s->gexec);
        cudaGraphDestroy(s->graph);
        s->gexec = nullptr;
        s->graph = nullptr;
    }
    return e;
}

// n steps: whole groups of kGraphSteps replayed from the graph (not while the
// per-launch kernel timing is on), the rest as single launches.
cudaError_t vlbm::api::step_many(vlbm_state *s, int64_t n) {
    if (!s->profiling && !s->probe_armed && n >= kGraphSteps) {
        cudaError_t e = cudaSuccess;
        if (!s->gexec)
            e = s->precision == VLBM_FP64 ? build_graph<double>(s) : build_graph<float>(s);
        if (e != cudaSuccess) return e;
        for (; n >= kGraphSteps; n -= kGraphSteps) {
            e = cudaGraphLaunch(s->gexec, s->stream);
            if (e != cudaSuccess) return e;
        }
    }
    for (; n > 0; --n) {
        cudaError_t e = step_once(s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static bool make_tmap(vlbm_state *s) { return encode_state_tmap(&s->tmap, s->ws, s->L); }

int vlbm::api::read_ctl(vlbm_state *s, DevCtl *h) {
    cudaError_t e = cudaMemcpyAsync(h, s->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "reading the device control block");
    return VLBM_OK;
}

extern "C" {

size_t vlbm_workspace_bytes(const vlbm_grid *grid, int32_t precision) {
    const int elem = elem_of(precision);
    if (!grid_ok(grid) || !elem) return 0;
    return make_layout(grid->nx, grid->ny, elem).total;
}

int vlbm_init(const vlbm_grid *grid, double gamma, double lambda, int32_t limiter,
              int32_t precision, const vlbm_opts *opts, void *d_workspace, size_t workspace_bytes,
              void *stream, vlbm_state **out) {
    if (!out) return fail(nullptr, VLBM_E_INVAL, "out is NULL");
    *out = nullptr;
    if (!grid_ok(grid))
        return fail(nullptr, VLBM_E_INVAL, "grid: need nx, ny >= 4, dx > 0, bc in 0..3, periodic sides paired");
    if (!(gamma > 1.0)) return fail(nullptr, VLBM_E_INVAL, "gamma must be > 1");
    if (limiter < VLBM_LIM_FIRST_ORDER || limiter > VLBM_LIM_RLMP)
        return fail(nullptr, VLBM_E_INVAL, "limiter out of range");
    const int elem = elem_of(precision);
    if (!elem) return fail(nullptr, VLBM_E_INVAL, "precision out of range");
    vlbm_opts o = {0.5, 1e-16, VLBM_KERNEL_AUTO, 0};
    if (opts) o = *opts;
    if (!(o.alpha >= 0.5 && o.alpha < 1.0)) return fail(nullptr, VLBM_E_INVAL, "alpha must be in [1/2, 1)");
    if (!(o.eps >= 0.0 && o.eps < 1e-3)) return fail(nullptr, VLBM_E_INVAL, "eps must be in [0, 1e-3)");
    if (o.kernel < VLBM_KERNEL_AUTO || o.kernel > VLBM_KERNEL_FUSED)
        return fail(nullptr, VLBM_E_INVAL, "kernel out of range");
    Bound bd;
    if (const char *why = make_bound(*grid, o.boundary, &bd)) return fail(nullptr, VLBM_E_INVAL, "boundary: %s", why);
    if (!sponge_ok(o.sponge, *grid))
        return fail(nullptr, VLBM_E_INVAL, "sponge must be in [0, n / 2] along every axis with a zero-gradient side");
    if (!(lambda == lambda)) return fail(nullptr, VLBM_E_INVAL, "lambda is NaN");
    const Layout L = make_layout(grid->nx, grid->ny, elem);
    if (!d_workspace || ((uintptr_t)d_workspace & 255))
        return fail(nullptr, VLBM_E_NOMEM, "workspace NULL or not 256-byte aligned");
    if (workspace_bytes < L.total)
        return fail(nullptr, VLBM_E_NOMEM, "workspace has %zu bytes, needs %zu", workspace_bytes, L.total);
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(nullptr, VLBM_E_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
    }
    cudaPointerAttributes pa;
    e = cudaPointerGetAttributes(&pa, d_workspace);
    if (e != cudaSuccess || (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        return fail(nullptr, VLBM_E_INVAL, "workspace is not device memory");
    }
    vlbm_state *s = new (std::nothrow) vlbm_state();
    if (!s) return fail(nullptr, VLBM_E_NOMEM, "host allocation failed");
    s->grid = *grid;
    s->precision = precision;
    s->limiter = limiter;
    s->kernel = o.kernel;
    s->gamma = gamma;
    s->lambda = lambda;
    s->alpha = o.alpha;
    s->eps = o.eps;
    s->sponge = o.sponge;
    s->bd = bd;
    s->a_fixed = lambda > 0.0 ? 2.0 * lambda / (1.0 - o.alpha) : 0.0;
    s->L = L;
    s->ws = d_workspace;
    s->stream = (cudaStream_t)stream;
    s->ctl = (DevCtl *)((char *)d_workspace + L.ctl_offset);
    s->bd.ctl = s->ctl;
    s->device = pa.device;
    {
        DeviceGuard g(s->device);
        s->have_tmap = make_tmap(s);
        if (s->have_tmap) {
            int sms = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
            const int per_sm = precision == VLBM_FP64 ? fused_occupancy<double>(limiter)
                                                      : fused_occupancy<float>(limiter);
            const long long ctas = (long long)per_sm * (sms > 0 ? sms : 1);
            // guided bands of at most kFusedMaxChunk rows
            long long work = (long long)strip_count(grid->nx) * grid->ny;
            s->items_host.resize(max_items(grid->nx, grid->ny));
            s->nitems = append_items(s->items_host.data(), 0, grid->nx, grid->ny, kFusedMaxChunk, true, work, ctas);
            s->items_host.resize(s->nitems);
            s->fused_grid = (int)(ctas < s->nitems ? ctas : s->nitems);
            if (precision == VLBM_FP64) build_desc<double>(s);
            else build_desc<float>(s);
        }
        if (o.kernel == VLBM_KERNEL_FUSED && !s->have_tmap) {
            delete s;
            return fail(nullptr, VLBM_E_UNSUPPORTED, "TMA descriptor unavailable for the fused kernel");
        }
    }
    *out = s;
    return VLBM_OK;
}

int vlbm_set_conserved(vlbm_state *s, const void *d_rho, const void *d_mom, const void *d_E) {
    if (!s) return fail(nullptr, VLBM_E_INVAL, "state is NULL");
    if (!d_rho || !d_mom || !d_E) return fail(s, VLBM_E_INVAL, "input plane pointer is NULL");
    return vlbm::api::set_conserved(s, d_rho, d_mom, d_E);
}

}  // extern "C"

int vlbm::api::set_conserved(vlbm_state *s, const void *d_rho, const void *d_mom, const void *d_E) {
    DeviceGuard g(s->device);
    s->roll_scratch = nullptr;
    cudaError_t e = launch_ctl_reset(s->ctl, s->grid.dx, s->alpha, s->a_fixed, s->eps, s->gamma, s->stream);
    if (e == cudaSuccess) e = upload_desc(s);
    if (e == cudaSuccess) {
        if (s->precision == VLBM_FP64)
            e = launch_init<double>(args_of<double>(s), (const double *)d_rho, (const double *)d_mom,
                                    (const double *)d_E, s->stream);
        else
            e = launch_init<float>(args_of<float>(s), (const float *)d_rho, (const float *)d_mom,
                                   (const float *)d_E, s->stream);
    }
    if (e != cudaSuccess) return cuda_fail(s, e, "initialisation launch");
    DevCtl h;
    int rc = read_ctl(s, &h);
    if (rc) return rc;
    s->loaded = true;
    s->tend_active = false;
    s->at_init = true;
    s->probe_armed = false;
    if (h.invalid_init)
        return fail(s, VLBM_E_INVAL, "initial state has cells outside G or not finite");
    return VLBM_OK;
}

extern "C" {

int vlbm_step(vlbm_state *s, int64_t nsteps) {
    if (!s) return fail(nullptr, VLBM_E_INVAL, "state is NULL");
    if (!s->loaded) return fail(s, VLBM_E_INVAL, "no state loaded (call vlbm_set_conserved)");
    if (nsteps < 0) return fail(s, VLBM_E_INVAL, "nsteps < 0");
    DeviceGuard g(s->device);
    if (s->tend_active) {
        cudaError_t e = launch_set_tend(s->ctl, 0.0, s->stream);
        if (e != cudaSuccess) return cuda_fail(s, e, "clearing the final time");
        s->tend_active = false;
    }
    if (nsteps > 0) {
        s->at_init = false;
        s->roll_scratch = nullptr;
    }
    cudaError_t e = step_many(s, nsteps);
    if (e != cudaSuccess) return cuda_fail(s, e, "step launch");
    return VLBM_OK;
}

int vlbm_step_to(vlbm_state *s, double t_end, int64_t max_steps) {
    if (!s) return fail(nullptr, VLBM_E_INVAL, "state is NULL");
    if (!s->loaded) return fail(s, VLBM_E_INVAL, "no state loaded (call vlbm_set_conserved)");
    if (!(t_end > 0.0) || max_steps < 0) return fail(s, VLBM_E_INVAL, "need t_end > 0 and max_steps >= 0");
    DeviceGuard g(s->device);
    cudaError_t e = launch_set_tend(s->ctl, t_end, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "arming the final time");
    s->tend_active = true;
    s->at_init = false;
    s->roll_scratch = nullptr;
    int64_t done_steps = 0, chunk = 64;
    while (done_steps < max_steps) {
        const int64_t k = chunk < max_steps - done_steps ? chunk : max_steps - done_steps;
        e = step_many(s, k);
        if (e != cudaSuccess) return cuda_fail(s, e, "step launch");
        done_steps += k;
        DevCtl h;
        int rc = read_ctl(s, &h);
        if (rc) return rc;
        if (h.done) return h.status;
        if (chunk < 4096) chunk *= 2;
    }
    return VLBM_OK;
}

int vlbm_moments(const vlbm_state *s, void *d_rho, void *d_mom, void *d_E) {
    if (!s) return fail(nullptr, VLBM_E_INVAL, "state is NULL");
    vlbm_state *m = const_cast<vlbm_state *>(s);
    if (!s->loaded) return fail(m, VLBM_E_INVAL, "no state loaded");
    DeviceGuard g(s->device);
    cudaError_t e;
    if (s->precision == VLBM_FP64)
        e = launch_moments<double>(args_of<double>(s), (double *)d_rho, (double *)d_mom, (double *)d_E, s->stream);
    else
        e = launch_moments<float>(args_of<float>(s), (float *)d_rho, (float *)d_mom, (float *)d_E, s->stream);
    if (e != cudaSuccess) return cuda_fail(m, e, "moments launch");
    return VLBM_OK;
}

static int decode_ctl(const DevCtl &h, vlbm_monitor_t *out) {
    out->n = h.n;
    out->t = h.t;
    out->a = h.a;
    out->dt = h.dt;
    out->lambda = h.lambda;
    out->bad_cells = h.bad_last;
    out->nonfinite_cells = h.nonfinite_last;
    out->first_bad_step = h.first_bad_step;
    out->min_rho = h.min_rho;
    out->min_internal_energy = h.min_rhoe;
    for (int c = 0; c < 4; ++c) out->sum[c] = h.sum_last[c];
    out->theta_p_fp64_faces = h.fp64_last;
    out->done = h.done;
    out->status = h.status;
    return h.status;
}

int vlbm_monitors(vlbm_state *s, vlbm_monitor_t *out) {
    if (!s || !out) return fail(s, VLBM_E_INVAL, "state or out is NULL");
    if (!s->loaded) return fail(s, VLBM_E_INVAL, "no state loaded");
    DeviceGuard g(s->device);
    DevCtl h;
    int rc = read_ctl(s, &h);
    if (rc) return rc;
    return decode_ctl(h, out);
}

size_t vlbm_monitors_raw_bytes(void) { return sizeof(DevCtl); }

int vlbm_monitors_async(vlbm_state *s, void *h_dst) {
    if (!s || !h_dst) return fail(s, VLBM_E_INVAL, "state or destination is NULL");
    if (!s->loaded) return fail(s, VLBM_E_INVAL, "no state loaded");
    DeviceGuard g(s->device);
    const cudaError_t e = cudaMemcpyAsync(h_dst, s->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "copying the device control block");
    return VLBM_OK;
}

int vlbm_monitors_decode(const void *h_src, vlbm_monitor_t *out) {
    if (!h_src || !out) return fail(nullptr, VLBM_E_INVAL, "source or out is NULL");
    DevCtl h;
    memcpy(&h, h_src, sizeof h);
    return decode_ctl(h, out);
}

int vlbm_sync(vlbm_state *s) {
    if (!s) return fail(nullptr, VLBM_E_INVAL, "state is NULL");
    if (!s->loaded) return fail(s, VLBM_E_INVAL, "no state loaded");
    DeviceGuard g(s->device);
    DevCtl h;
    int rc = read_ctl(s, &h);
    return rc ? rc : h.status;
}

int vlbm_time(vlbm_state *s, double *t, int64_t *n) {
    if (!s) return fail(nullptr, VLBM_E_INVAL, "state is NULL");
    if (!s->loaded) return fail(s, VLBM_E_INVAL, "no state loaded");
    DeviceGuard g(s->device);
    DevCtl h;
    int rc = read_ctl(s, &h);
    if (rc) return rc;
    if (t) *t = h.t;
    if (n) *n = h.n;
    return h.status;
}

size_t vlbm_checkpoint_bytes(const vlbm_state *s) {
    if (!s) return 0;
    return 64 + (size_t)kNPlane * s->grid.nx * s->grid.ny * s->L.elem;
}

int vlbm_save(const vlbm_state *s, void *d_dst) {
    if (!s) return fail(nullptr, VLBM_E_INVAL, "state is NULL");
    vlbm_state *m = const_cast<vlbm_state *>(s);
    if (!d_dst || ((uintptr_t)d_dst & 15)) return fail(m, VLBM_E_INVAL, "destination NULL or not 16-byte aligned");
    if (!s->loaded) return fail(m, VLBM_E_INVAL, "no state loaded");
    DeviceGuard g(s->device);
    cudaError_t e = s->precision == VLBM_FP64 ? launch_save<double>(args_of<double>(s), d_dst, s->stream)
                                              : launch_save<float>(args_of<float>(s), d_dst, s->stream);
    if (e != cudaSuccess) return cuda_fail(m, e, "save launch");
    return VLBM_OK;
}

int vlbm_load(vlbm_state *s, const void *d_src) {
    if (!s) return fail(nullptr, VLBM_E_INVAL, "state is NULL");
    if (!d_src || ((uintptr_t)d_src & 15)) return fail(s, VLBM_E_INVAL, "source NULL or not 16-byte aligned");
    DeviceGuard g(s->device);
    cudaError_t e = launch_ctl_reset(s->ctl, s->grid.dx, s->alpha, s->a_fixed, s->eps, s->gamma, s->stream);
    if (e == cudaSuccess) e = upload_desc(s);
    if (e == cudaSuccess)
        e = s->precision == VLBM_FP64 ? launch_load<double>(args_of<double>(s), d_src, s->stream)
                                      : launch_load<float>(args_of<float>(s), d_src, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "load launch");
    s->loaded = true;
    s->probe_armed = false;
    s->tend_active = true;  // the restored header may carry a final time
    s->at_init = false;
    s->roll_scratch = nullptr;
    return VLBM_OK;
}

int vlbm_profile(vlbm_state *s, int32_t enable) {
    if (!s) return fail(nullptr, VLBM_E_INVAL, "state is NULL");
    s->profiling = enable != 0;
    if (s->profiling) s->ev_used = 0;
    return VLBM_OK;
}

int vlbm_profile_read(vlbm_state *s, double *kernel_ms, int64_t *launches) {
    if (!s) return fail(nullptr, VLBM_E_INVAL, "state is NULL");
    DeviceGuard g(s->device);
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "profile read");
    double total = 0.0;
    for (size_t k = 0; k + 1 < s->ev_used; k += 2) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, s->ev[k], s->ev[k + 1]);
        if (e != cudaSuccess) return cuda_fail(s, e, "event elapsed time");
        total += ms;
    }
    if (kernel_ms) *kernel_ms = total;
    if (launches) *launches = (int64_t)(s->ev_used / 2);
    return VLBM_OK;
}

void vlbm_destroy(vlbm_state *s) {
    if (!s) return;
    if (s->gexec) cudaGraphExecDestroy(s->gexec);
    if (s->graph) cudaGraphDestroy(s->graph);
    for (cudaEvent_t e : s->ev) cudaEventDestroy(e);
    if (s->aux_ready) {
        DeviceGuard g(s->device);
        for (int i = 0; i < kAuxEvents; ++i) cudaEventDestroy(s->aux_ev[i]);
        cudaStreamDestroy(s->aux_stream);
    }
    delete s;
}

const char *vlbm_strerror(int code) {
    switch (code) {
        case VLBM_OK: return "ok";
        case VLBM_E_INVAL: return "invalid argument";
        case VLBM_E_CUDA: return "CUDA error";
        case VLBM_E_POSITIVITY: return "a cell left the admissible set";
        case VLBM_E_NONFINITE: return "a cell became non-finite";
        case VLBM_E_TIMEOUT: return "a device wait timed out";
        case VLBM_E_UNSUPPORTED: return "unsupported request";
        case VLBM_E_NOMEM: return "workspace too small or misaligned";
        default: return "unknown error code";
    }
}

int vlbm_last_error_detail(const vlbm_state *s, char *buf, size_t n) {
    const char *src = s ? s->err : g_err;
    const size_t len = strlen(src);
    if (buf && n) {
        const size_t k = len < n - 1 ? len : n - 1;
        memcpy(buf, src, k);
        buf[k] = '\0';
    }
    return (int)len;
}

}  // extern "C"

