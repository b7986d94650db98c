// state.h -- the host object behind vlbm_state* and the helpers that the entry
// points of abi.cu (single grid) and adjoint.cu (rollout and adjoint) share.
#pragma once

#include <stdint.h>

#include <vector>

#include "../../include/vlbm.h"
#include "vlbm_internal.h"

constexpr int kAuxEvents = 5;   // events of the reverse sweep's two streams

struct vlbm_state {
    vlbm_grid grid;
    int precision, limiter, kernel;
    double gamma, lambda, alpha, eps, a_fixed;
    int sponge;
    vlbm::Bound bd;     // split sides and the prescribed field (ctl set)
    vlbm::Layout L;
    void *ws;
    cudaStream_t stream;
    vlbm::DevCtl *ctl;
    int device;
    CUtensorMap tmap;   // 4D view [2 buffers][rows][5 groups][4 pitch] of both state buffers
    bool have_tmap;
    int nitems, fused_grid;
    std::vector<unsigned char> desc_host;   // InstDesc<T> of this grid
    std::vector<vlbm::WorkItem> items_host;  // work items in launch order (guided bands)
    bool profiling;
    bool probe_armed;   // vlbm_test_wait_probe: launch the probe instantiation, no graphs
    std::vector<cudaEvent_t> ev;   // event pairs of timed launches
    size_t ev_used;
    bool loaded;        // set_conserved or load has run
    bool tend_active;   // a final time is armed on the device
    bool at_init;       // the state is u_k = M_k(u_0) at n = 0, as set_conserved leaves it
    // CUDA graph of kGraphSteps consecutive steps (built on first use)
    cudaGraph_t graph;
    cudaGraphExec_t gexec;
    // checkpoints written by the last vlbm_rollout (consumed by vlbm_adjoint)
    const void *roll_scratch;
    int64_t roll_steps;
    int32_t roll_every;
    int adj_mode;       // VLBM_ADJOINT_HOLD_A or VLBM_ADJOINT_DIFF_A
    // the reverse sweep's second stream (recomputation) and its events, made on first use
    bool aux_ready;
    cudaStream_t aux_stream;
    cudaEvent_t aux_ev[kAuxEvents];
    char err[256];
};

namespace vlbm {
namespace api {

// Record a message for vlbm_last_error_detail (per state, or per thread when
// s is NULL) and return code.
int fail(vlbm_state *s, int code, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
int cuda_fail(vlbm_state *s, cudaError_t e, const char *what);

// Keep the caller's current device; run the call on the state's device.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

template <typename T>
inline StepArgs<T> args_of(const vlbm_state *s) {
    StepArgs<T> A;
    A.buf0 = (T *)s->ws;
    A.buf1 = (T *)((char *)s->ws + s->L.buf_bytes);
    A.pitch = s->L.pitch;
    A.nx = s->grid.nx;
    A.ny = s->grid.ny;
    uniform_types(s->bd, A.bc);
    A.limiter = s->limiter;
    A.gamma = s->gamma;
    A.alpha = s->alpha;
    A.eps = s->eps;
    A.ctl = s->ctl;
    A.sponge = s->sponge;
    A.bd = s->bd;
    return A;
}

// VLBM_KERNEL_AUTO. FP32: below this many cells a grid has too few row-marching
// work items to fill the GPU and the one-thread-per-cell kernel is faster (PP on a
// GB300, a vortex with density bumps: 11.8 vs 20.4 us per step at 256^2, 27.3 vs
// 35.4 us at 512^2, about even at 640^2, 93 vs 67 us at 1024^2). FP64: every face's
// theta_p solve makes the step FP64-pipe bound, where the one-thread-per-cell
// kernel's many warps per SM win on small grids (0.63 vs 0.77 ms at 512^2, 2.39 vs
// 2.55 ms at 1024^2) and the row-marching kernel on large ones (9.53 vs 8.00 ms at
// 2048^2).
constexpr long long kAutoFusedMinCells = 1ll << 19;
constexpr long long kAutoFusedMinCellsFp64 = 1ll << 22;

inline bool use_fused(const vlbm_state *s) {
    if (!s->have_tmap || s->kernel == VLBM_KERNEL_SIMPLE) return false;
    if (s->kernel == VLBM_KERNEL_FUSED) return true;
    const long long cells = (long long)s->grid.nx * s->grid.ny;
    return cells >= (s->precision == VLBM_FP32 ? kAutoFusedMinCells : kAutoFusedMinCellsFp64);
}

// Arguments of the row-marching kernel for this grid (descriptor block of the workspace).
template <typename T>
inline FusedBatchArgs<T> batch_args_of(const vlbm_state *s) {
    FusedBatchArgs<T> B;
    char *base = (char *)s->ws + s->L.desc_offset;
    B.insts = (const InstDesc<T> *)base;
    B.bctl = (BatchCtl *)(base + 512);
    B.items = (const WorkItem *)(base + 768);
    B.nitems = s->nitems;
    B.gamma = s->gamma;
    B.alpha = s->alpha;
    B.eps = s->eps;
    return B;
}

cudaError_t step_once(vlbm_state *s);           // one step of the state's configured kernel
cudaError_t step_many(vlbm_state *s, int64_t n); // n steps, whole groups of kGraphSteps from a graph
constexpr int kGraphSteps = 64;
int read_ctl(vlbm_state *s, DevCtl *h);         // synchronous copy of the control block
int set_conserved(vlbm_state *s, const void *rho, const void *mom, const void *E);

}  // namespace api
}  // namespace vlbm
