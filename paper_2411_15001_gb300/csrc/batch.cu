// batch.cu -- the vlbm_batch_* entry points: many independent grids of uneven
// sizes advanced together by the row-marching kernel, one launch per time step
// over the work items of all grids, the steps replayed from a CUDA graph; and the
// autotuner that picks the work decomposition.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/vlbm.h"
#include "vlbm_internal.h"

using namespace vlbm;

namespace {
constexpr int kGraphSteps = 64;        // kernel nodes per graph replay

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// Control blocks and descriptors sit in arrays that the kernel indexes by grid,
// so their strides are the sizes of the types (256-byte multiples).
constexpr size_t kCtlStride = (sizeof(DevCtl) + 255) / 256 * 256;
constexpr size_t kDescStride = sizeof(InstDesc<double>);
static_assert(sizeof(InstDesc<float>) == sizeof(InstDesc<double>), "one descriptor stride for both precisions");
static_assert(kDescStride % 256 == 0, "descriptor stride");
}  // namespace

struct vlbm_batch {
    int n = 0, precision = 0, limiter = 0, device = 0;
    double gamma = 1.4, alpha = 0.5, eps = 1e-16;
    int sponge = 0;
    std::vector<vlbm_grid> grids;
    std::vector<Bound> bds;   // per grid: split sides and the prescribed field (opts->boundary)
    std::vector<Layout> L;
    std::vector<size_t> buf_off;       // per grid: offset of its two state buffers
    std::vector<CUtensorMap> tmaps;
    std::vector<char> loaded;
    size_t ctl_off = 0, desc_off = 0, bctl_off = 0, items_off = 0, items_cap = 0, total = 0;
    void *ws = nullptr;
    cudaStream_t stream = nullptr;
    int sms = 1;
    // work decomposition (tunable)
    int chunk = kFusedMaxChunk, ctas_per_sm = 3, order = VLBM_ORDER_GUIDED;   // until set or autotuned
    int nitems = 0;
    std::vector<unsigned char> desc_host;
    std::vector<WorkItem> items_host;
    bool desc_dirty = true;
    // graph of kGraphSteps launches
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    char err[256] = {0};
};

static thread_local char g_batch_err[256];   // messages of calls without a batch object

static int bfail(vlbm_batch *b, int code, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
static int bfail(vlbm_batch *b, int code, const char *fmt, ...) {
    char *dst = b ? b->err : g_batch_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 256, fmt, ap);
    va_end(ap);
    return code;
}

static bool grid_ok(const vlbm_grid &g) {
    if (g.nx < 4 || g.ny < 4 || !(g.dx > 0.0)) return false;
    for (int k = 0; k < 4; ++k)
        if (g.bc[k] < VLBM_BC_PERIODIC || g.bc[k] > VLBM_BC_DIRICHLET) return false;
    if ((g.bc[0] == VLBM_BC_PERIODIC) != (g.bc[1] == VLBM_BC_PERIODIC)) return false;
    if ((g.bc[2] == VLBM_BC_PERIODIC) != (g.bc[3] == VLBM_BC_PERIODIC)) return false;
    return true;
}

// Workspace layout: the grids' state buffers, then n control blocks, n descriptors
// (arrays indexed by grid), the work counter and the item table (sized for bands
// of the smallest height, max_items).
static size_t plan_layout(vlbm_batch *b, int n, const vlbm_grid *grids, int elem) {
    b->L.resize(n);
    b->buf_off.resize(n);
    size_t off = 0, items = 0;
    for (int i = 0; i < n; ++i) {
        b->L[i] = make_layout(grids[i].nx, grids[i].ny, elem);
        b->buf_off[i] = off;
        off += up256(2 * b->L[i].buf_bytes);
        items += max_items(grids[i].nx, grids[i].ny);
    }
    b->ctl_off = off;
    off += (size_t)n * kCtlStride;
    b->desc_off = off;
    off += (size_t)n * kDescStride;
    b->bctl_off = off;
    off += 256;
    b->items_off = off;
    b->items_cap = items;
    off += up256(items * sizeof(WorkItem));
    return off;
}

template <typename T>
static StepArgs<T> inst_args(const vlbm_batch *b, int i) {
    StepArgs<T> A;
    A.buf0 = (T *)((char *)b->ws + b->buf_off[i]);
    A.buf1 = (T *)((char *)b->ws + b->buf_off[i] + b->L[i].buf_bytes);
    A.pitch = b->L[i].pitch;
    A.nx = b->grids[i].nx;
    A.ny = b->grids[i].ny;
    uniform_types(b->bds[i], A.bc);
    A.limiter = b->limiter;
    A.gamma = b->gamma;
    A.alpha = b->alpha;
    A.eps = b->eps;
    A.ctl = (DevCtl *)((char *)b->ws + b->ctl_off + (size_t)i * kCtlStride);
    A.sponge = b->sponge;
    A.bd = b->bds[i];
    A.bd.ctl = A.ctl;
    return A;
}

// Descriptors and the item table for the current chunk / order: grids in
// longest-first order (LPT, GUIDED) or in index order; a grid's items
// strip-fastest, in bands of `chunk` rows, or under GUIDED in bands of decreasing
// height (at most `chunk`) sized from the work left in all grids.
template <typename T>
static void build_items(vlbm_batch *b) {
    std::vector<int> ord(b->n);
    std::iota(ord.begin(), ord.end(), 0);
    if (b->order == VLBM_ORDER_LPT || b->order == VLBM_ORDER_GUIDED)
        std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
            return (long long)b->grids[x].nx * b->grids[x].ny > (long long)b->grids[y].nx * b->grids[y].ny;
        });
    b->desc_host.assign((size_t)b->n * kDescStride, 0);
    b->items_host.resize(b->items_cap);
    const bool guided = b->order == VLBM_ORDER_GUIDED;
    long long work = 0;
    for (int i = 0; i < b->n; ++i)
        work += (long long)strip_count(b->grids[i].nx) * b->grids[i].ny;
    const long long ctas = (long long)b->ctas_per_sm * b->sms;
    size_t used = 0;
    for (int i : ord) {
        InstDesc<T> d;
        memset(&d, 0, sizeof d);
        d.tmap = b->tmaps[i];
        const StepArgs<T> A = inst_args<T>(b, i);
        d.buf0 = A.buf0;
        d.buf1 = A.buf1;
        d.pitch = A.pitch;
        d.nx = A.nx;
        d.ny = A.ny;
        for (int k = 0; k < 4; ++k) d.bc[k] = A.bc[k];
        d.bd = A.bd;
        d.nitems = append_items(b->items_host.data() + used, i, A.nx, A.ny, b->chunk, guided, work, ctas);
        used += d.nitems;
        d.ctl = A.ctl;
        d.sponge = A.sponge;
        memcpy(&b->desc_host[(size_t)i * kDescStride], &d, sizeof d);
    }
    b->items_host.resize(used);
    b->nitems = (int)used;
    b->desc_dirty = true;
}

static cudaError_t upload(vlbm_batch *b) {
    if (!b->desc_dirty) return cudaSuccess;
    char *base = (char *)b->ws;
    cudaError_t e = cudaMemcpyAsync(base + b->desc_off, b->desc_host.data(), b->desc_host.size(),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + b->items_off, b->items_host.data(), b->items_host.size() * sizeof(WorkItem),
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + b->bctl_off, 0, sizeof(BatchCtl), b->stream);
    // the host copies must outlive the copies: wait for them
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess) b->desc_dirty = false;
    return e;
}

template <typename T>
static FusedBatchArgs<T> batch_args(const vlbm_batch *b) {
    FusedBatchArgs<T> B;
    char *base = (char *)b->ws;
    B.insts = (const InstDesc<T> *)(base + b->desc_off);
    B.items = (const WorkItem *)(base + b->items_off);
    B.nitems = b->nitems;
    B.bctl = (BatchCtl *)(base + b->bctl_off);
    B.gamma = b->gamma;
    B.alpha = b->alpha;
    B.eps = b->eps;
    return B;
}

static int grid_ctas(const vlbm_batch *b) {
    const long long c = (long long)b->ctas_per_sm * b->sms;
    return (int)(c < b->nitems ? c : (b->nitems > 0 ? b->nitems : 1));
}

static void drop_graph(vlbm_batch *b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
}

template <typename T>
static cudaError_t launch_steps(vlbm_batch *b, int64_t nsteps) {
    cudaError_t e = upload(b);
    if (e != cudaSuccess) return e;
    FusedBatchArgs<T> B = batch_args<T>(b);
    const int ctas = grid_ctas(b);
    // grids with a prescribed part get their Dirichlet ghosts before every step
    std::vector<StepArgs<T>> dir;
    for (int i = 0; i < b->n; ++i)
        if (b->bds[i].has_dir) dir.push_back(inst_args<T>(b, i));
    std::vector<void *> dparams(dir.size());
    for (size_t q = 0; q < dir.size(); ++q) dparams[q] = &dir[q];
    if (nsteps >= kGraphSteps && !b->gexec) {
        size_t smem = 0;
        const void *fn = fused_kernel_fn<T>(b->limiter, &smem);
        e = cudaGraphCreate(&b->graph, 0);
        if (e != cudaSuccess) return e;
        void *params[] = {&B};
        cudaKernelNodeParams kp;
        memset(&kp, 0, sizeof kp);
        kp.func = const_cast<void *>(fn);
        kp.gridDim = dim3(ctas);
        kp.blockDim = dim3(kFusedBox);
        kp.sharedMemBytes = (unsigned)smem;
        kp.kernelParams = params;
        cudaGraphNode_t prev = nullptr;
        for (int k = 0; k < kGraphSteps && e == cudaSuccess; ++k) {
            cudaGraphNode_t node;
            for (size_t q = 0; q < dir.size() && e == cudaSuccess; ++q) {
                cudaKernelNodeParams kd;
                memset(&kd, 0, sizeof kd);
                kd.func = const_cast<void *>(dirichlet_ghosts_kernel_fn<T>());
                ghosts_launch_shape(dir[q].nx, dir[q].ny, &kd.gridDim, &kd.blockDim);
                kd.kernelParams = &dparams[q];
                e = cudaGraphAddKernelNode(&node, b->graph, prev ? &prev : nullptr, prev ? 1 : 0, &kd);
                prev = node;
            }
            if (e != cudaSuccess) break;
            e = cudaGraphAddKernelNode(&node, b->graph, prev ? &prev : nullptr, prev ? 1 : 0, &kp);
            prev = node;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, b->graph, 0);
        if (e != cudaSuccess) {
            drop_graph(b);
            return e;
        }
    }
    int64_t left = nsteps;
    while (left >= kGraphSteps && b->gexec) {
        e = cudaGraphLaunch(b->gexec, b->stream);
        if (e != cudaSuccess) return e;
        left -= kGraphSteps;
    }
    for (; left > 0; --left) {
        for (size_t q = 0; q < dir.size() && e == cudaSuccess; ++q) e = launch_dirichlet_ghosts<T>(dir[q], b->stream);
        if (e == cudaSuccess) e = launch_step_fused<T>(B, b->limiter, ctas, b->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static cudaError_t steps(vlbm_batch *b, int64_t nsteps) {
    return b->precision == VLBM_FP64 ? launch_steps<double>(b, nsteps) : launch_steps<float>(b, nsteps);
}

static void rebuild(vlbm_batch *b) {
    if (b->precision == VLBM_FP64) build_items<double>(b);
    else build_items<float>(b);
    drop_graph(b);
}

struct BDeviceGuard {
    int prev = -1;
    explicit BDeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    }
    ~BDeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

extern "C" {

size_t vlbm_batch_workspace_bytes(int32_t n, const vlbm_grid *grids, int32_t precision) {
    if (n <= 0 || !grids || (precision != VLBM_FP32 && precision != VLBM_FP64)) return 0;
    for (int i = 0; i < n; ++i)
        if (!grid_ok(grids[i])) return 0;
    vlbm_batch tmp;
    return plan_layout(&tmp, n, grids, precision == VLBM_FP64 ? 8 : 4);
}

int vlbm_batch_init(int32_t n, const vlbm_grid *grids, double gamma, int32_t limiter, int32_t precision,
                    const vlbm_opts *opts, void *d_workspace, size_t workspace_bytes, void *stream,
                    vlbm_batch **out) {
    if (!out) return bfail(nullptr, VLBM_E_INVAL, "out is NULL");
    *out = nullptr;
    if (n <= 0 || !grids) return bfail(nullptr, VLBM_E_INVAL, "need n > 0 grids");
    for (int i = 0; i < n; ++i)
        if (!grid_ok(grids[i])) return bfail(nullptr, VLBM_E_INVAL, "grid %d invalid", i);
    if (!(gamma > 1.0) || limiter < VLBM_LIM_FIRST_ORDER || limiter > VLBM_LIM_RLMP ||
        (precision != VLBM_FP32 && precision != VLBM_FP64))
        return bfail(nullptr, VLBM_E_INVAL, "gamma, limiter or precision out of range");
    vlbm_opts o = {0.5, 1e-16, VLBM_KERNEL_AUTO, 0};
    if (opts) o = *opts;
    if (!(o.alpha >= 0.5 && o.alpha < 1.0) || !(o.eps >= 0.0 && o.eps < 1e-3))
        return bfail(nullptr, VLBM_E_INVAL, "alpha or eps out of range");
    std::vector<Bound> bds(n);
    for (int i = 0; i < n; ++i)
        if (const char *why = make_bound(grids[i], o.boundary, &bds[i]))
            return bfail(nullptr, VLBM_E_INVAL, "boundary of grid %d: %s", i, why);
    for (int i = 0; i < n; ++i)
        if (!sponge_ok(o.sponge, grids[i]))
            return bfail(nullptr, VLBM_E_INVAL, "sponge of grid %d: at most n / 2 along an axis with a "
                                                "zero-gradient side", i);
    if (!d_workspace || ((uintptr_t)d_workspace & 255))
        return bfail(nullptr, VLBM_E_NOMEM, "workspace NULL or not 256-byte aligned");
    vlbm_batch *b = new (std::nothrow) vlbm_batch();
    if (!b) return bfail(nullptr, VLBM_E_NOMEM, "host allocation failed");
    b->total = plan_layout(b, n, grids, precision == VLBM_FP64 ? 8 : 4);
    if (workspace_bytes < b->total) {
        const size_t need = b->total;
        delete b;
        return bfail(nullptr, VLBM_E_NOMEM, "workspace has %zu bytes, needs %zu", workspace_bytes, need);
    }
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, d_workspace) != cudaSuccess ||
        (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        delete b;
        return bfail(nullptr, VLBM_E_INVAL, "workspace is not device memory");
    }
    b->n = n;
    b->precision = precision;
    b->limiter = limiter;
    b->gamma = gamma;
    b->alpha = o.alpha;
    b->eps = o.eps;
    b->sponge = o.sponge;
    b->grids.assign(grids, grids + n);
    b->bds = bds;
    b->ws = d_workspace;
    b->stream = (cudaStream_t)stream;
    b->device = pa.device;
    b->loaded.assign(n, 0);
    BDeviceGuard g(b->device);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    b->ctas_per_sm = precision == VLBM_FP64 ? fused_occupancy<double>(limiter) : fused_occupancy<float>(limiter);
    b->tmaps.resize(n);
    for (int i = 0; i < n; ++i) {
        if (!encode_state_tmap(&b->tmaps[i], (char *)d_workspace + b->buf_off[i], b->L[i])) {
            delete b;
            return bfail(nullptr, VLBM_E_UNSUPPORTED, "TMA descriptor for grid %d unavailable", i);
        }
    }
    rebuild(b);
    *out = b;
    return VLBM_OK;
}

int vlbm_batch_set_conserved(vlbm_batch *b, int32_t i, const void *d_rho, const void *d_mom, const void *d_E) {
    if (!b || i < 0 || i >= b->n || !d_rho || !d_mom || !d_E) return bfail(b, VLBM_E_INVAL, "bad argument");
    BDeviceGuard g(b->device);
    cudaError_t e;
    DevCtl *ctl = (DevCtl *)((char *)b->ws + b->ctl_off + (size_t)i * kCtlStride);
    e = launch_ctl_reset(ctl, b->grids[i].dx, b->alpha, 0.0, b->eps, b->gamma, b->stream);
    if (e == cudaSuccess) {
        if (b->precision == VLBM_FP64)
            e = launch_init<double>(inst_args<double>(b, i), (const double *)d_rho, (const double *)d_mom,
                                    (const double *)d_E, b->stream);
        else
            e = launch_init<float>(inst_args<float>(b, i), (const float *)d_rho, (const float *)d_mom,
                                   (const float *)d_E, b->stream);
    }
    DevCtl h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, ctl, sizeof h, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, VLBM_E_CUDA, "initialisation of grid %d: %s", i, cudaGetErrorString(e));
    b->loaded[i] = 1;
    if (h.invalid_init) return bfail(b, VLBM_E_INVAL, "grid %d: initial state outside G or not finite", i);
    return VLBM_OK;
}

int vlbm_batch_step(vlbm_batch *b, int64_t nsteps) {
    if (!b || nsteps < 0) return bfail(b, VLBM_E_INVAL, "bad argument");
    for (int i = 0; i < b->n; ++i)
        if (!b->loaded[i]) return bfail(b, VLBM_E_INVAL, "grid %d has no state", i);
    BDeviceGuard g(b->device);
    cudaError_t e = steps(b, nsteps);
    if (e != cudaSuccess) return bfail(b, VLBM_E_CUDA, "batch step: %s", cudaGetErrorString(e));
    return VLBM_OK;
}

int vlbm_batch_moments(const vlbm_batch *b, int32_t i, void *d_rho, void *d_mom, void *d_E) {
    vlbm_batch *m = const_cast<vlbm_batch *>(b);
    if (!b || i < 0 || i >= b->n) return bfail(m, VLBM_E_INVAL, "bad argument");
    BDeviceGuard g(b->device);
    cudaError_t e = b->precision == VLBM_FP64
                        ? launch_moments<double>(inst_args<double>(b, i), (double *)d_rho, (double *)d_mom,
                                                 (double *)d_E, b->stream)
                        : launch_moments<float>(inst_args<float>(b, i), (float *)d_rho, (float *)d_mom,
                                                (float *)d_E, b->stream);
    if (e != cudaSuccess) return bfail(m, VLBM_E_CUDA, "moments: %s", cudaGetErrorString(e));
    return VLBM_OK;
}

int vlbm_batch_save(const vlbm_batch *b, int32_t i, void *d_dst) {
    vlbm_batch *m = const_cast<vlbm_batch *>(b);
    if (!b || i < 0 || i >= b->n || !d_dst || ((uintptr_t)d_dst & 15)) return bfail(m, VLBM_E_INVAL, "bad argument");
    BDeviceGuard g(b->device);
    cudaError_t e = b->precision == VLBM_FP64 ? launch_save<double>(inst_args<double>(b, i), d_dst, b->stream)
                                              : launch_save<float>(inst_args<float>(b, i), d_dst, b->stream);
    if (e != cudaSuccess) return bfail(m, VLBM_E_CUDA, "save: %s", cudaGetErrorString(e));
    return VLBM_OK;
}

int vlbm_batch_monitors(vlbm_batch *b, int32_t i, vlbm_monitor_t *out) {
    if (!b || i < 0 || i >= b->n || !out) return bfail(b, VLBM_E_INVAL, "bad argument");
    BDeviceGuard g(b->device);
    DevCtl h;
    const DevCtl *ctl = (const DevCtl *)((char *)b->ws + b->ctl_off + (size_t)i * kCtlStride);
    cudaError_t e = cudaMemcpyAsync(&h, ctl, sizeof h, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, VLBM_E_CUDA, "monitors: %s", cudaGetErrorString(e));
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

int vlbm_batch_get_tuning(const vlbm_batch *b, vlbm_batch_tuning *t) {
    if (!b || !t) return VLBM_E_INVAL;
    t->chunk = b->chunk;
    t->ctas_per_sm = b->ctas_per_sm;
    t->order = b->order;
    t->items = b->nitems;
    t->ctas = grid_ctas(b);
    return VLBM_OK;
}

int vlbm_batch_set_tuning(vlbm_batch *b, const vlbm_batch_tuning *t) {
    if (!b || !t) return bfail(b, VLBM_E_INVAL, "bad argument");
    if (t->chunk < kFusedMinChunk || t->chunk > 1024 || t->ctas_per_sm < 1 || t->ctas_per_sm > 4 ||
        (t->order != VLBM_ORDER_LPT && t->order != VLBM_ORDER_INDEX && t->order != VLBM_ORDER_GUIDED))
        return bfail(b, VLBM_E_INVAL, "tuning out of range");
    const int maxc = b->precision == VLBM_FP64 ? fused_occupancy<double>(b->limiter)
                                               : fused_occupancy<float>(b->limiter);
    b->chunk = t->chunk;
    b->ctas_per_sm = t->ctas_per_sm < maxc ? t->ctas_per_sm : maxc;
    b->order = t->order;
    rebuild(b);
    return VLBM_OK;
}

int vlbm_batch_autotune(vlbm_batch *b, int32_t trial_steps, vlbm_batch_tuning *best, double *best_ms_per_step) {
    if (!b || trial_steps < 1) return bfail(b, VLBM_E_INVAL, "bad argument");
    for (int i = 0; i < b->n; ++i)
        if (!b->loaded[i]) return bfail(b, VLBM_E_INVAL, "grid %d has no state", i);
    BDeviceGuard g(b->device);
    const int maxc = b->precision == VLBM_FP64 ? fused_occupancy<double>(b->limiter)
                                               : fused_occupancy<float>(b->limiter);
    const int chunks[] = {32, 128, 512, 1024};
    const int orders[] = {VLBM_ORDER_LPT, VLBM_ORDER_INDEX, VLBM_ORDER_GUIDED};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return bfail(b, VLBM_E_CUDA, "event creation failed");
    vlbm_batch_tuning bt = {b->chunk, b->ctas_per_sm, b->order, 0, 0};
    double bms = 1e300;
    int rc = VLBM_OK;
    for (int ch : chunks)
        for (int cps = 1; cps <= maxc && rc == VLBM_OK; ++cps)
            for (int od : orders) {
                b->chunk = ch;
                b->ctas_per_sm = cps;
                b->order = od;
                rebuild(b);
                cudaError_t e = steps(b, 1);   // warm-up of this decomposition
                if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
                if (e == cudaSuccess) e = steps(b, trial_steps);
                if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) {
                    rc = bfail(b, VLBM_E_CUDA, "autotune: %s", cudaGetErrorString(e));
                    break;
                }
                if (ms / trial_steps < bms) {
                    bms = ms / trial_steps;
                    bt.chunk = ch;
                    bt.ctas_per_sm = cps;
                    bt.order = od;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->chunk = bt.chunk;
    b->ctas_per_sm = bt.ctas_per_sm;
    b->order = bt.order;
    rebuild(b);
    bt.items = b->nitems;
    bt.ctas = grid_ctas(b);
    if (best) *best = bt;
    if (best_ms_per_step) *best_ms_per_step = bms;
    return rc;
}

void vlbm_batch_destroy(vlbm_batch *b) {
    if (!b) return;
    drop_graph(b);
    delete b;
}

const char *vlbm_batch_last_error(const vlbm_batch *b) { return b ? b->err : g_batch_err; }

}  // extern "C"
