// adjoint.cu -- forward rollout with checkpoints and the reverse sweep that
// gives the gradient of a loss of the final conserved fields with respect to
// the initial ones (include/vlbm.h, "adjoint" section).
//
// Rollout: the state's own step kernel advances n = 0 .. N-1; the state and its
// control block are copied to checkpoint c before step c k.
// Reverse sweep, one segment [s, e] = [c k, min(c k + k, N) - 1] at a time, last
// segment first: the checkpoint is restored into slot 1 of segment buffer c % 2 and
// the same step kernel recomputes the states s+1 .. e into slots 2 .. e-s+1
// (reading slot j, writing slot j+1, with the control block in scratch); then the
// adjoint kernel maps the cotangent of s^{m+1} to that of s^m for m = e .. s. The
// recomputation of segment c - 1 runs on a second stream while the adjoint steps of
// segment c run on the state's stream.
// Finally the transpose of the initialisation u_k^0 = M_k(u_0) folds the
// population cotangents into the conserved planes.
// a^n is held as the forward run produced it: a constant when the state was made
// with a fixed lambda, else the step constants are recorded per step during the
// recomputation. In VLBM_ADJOINT_DIFF_A mode (dynamic a only) the sweep also
// carries dL/da^n of every step, and hands it to the state s^n through
// a^n = 2 lambda^n / (1 - alpha), lambda^n = max over cells: the gradient of the
// cell speed at the (first) cell where the max is taken.
#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "adjoint.cuh"
#include "state.h"

using namespace vlbm;
using namespace vlbm::api;

namespace vlbm {

template <typename T, bool DA, bool EXT>
static cudaError_t launch_adjoint_step_da(const AdjArgs<T> &A, int limiter, cudaStream_t s) {
    const int wx = A.nx + (EXT ? 2 : 0), wy = A.ny + (EXT ? 2 : 0);   // with a boundary: the first ghost layer too
    const dim3 blk(32, 8), grd((wx + 31) / 32, (wy + 7) / 8);
    switch (limiter) {
        case VLBM_LIM_FIRST_ORDER: k_adjoint_step<T, VLBM_LIM_FIRST_ORDER, DA, EXT><<<grd, blk, 0, s>>>(A); break;
        case VLBM_LIM_NONE: k_adjoint_step<T, VLBM_LIM_NONE, DA, EXT><<<grd, blk, 0, s>>>(A); break;
        case VLBM_LIM_PP: k_adjoint_step<T, VLBM_LIM_PP, DA, EXT><<<grd, blk, 0, s>>>(A); break;
        case VLBM_LIM_LMP:
        case VLBM_LIM_RLMP:
            {   // passes 1, 2, then the gather (and the outer ring)
                // faces of cells 0 .. n - 1 (periodic) or -1 .. n - 1 (boundary); bounds and
                // the gather over the cells of the step (with the first ghost layer)
                const dim3 gf((A.nx + (EXT ? 1 : 0) + 31) / 32, (A.ny + (EXT ? 1 : 0) + 7) / 8);
                cudaError_t e;
                if (EXT) {   // every plane: the bounds pass adds into faces pass 1 does not write
                    const size_t NL = (size_t)(A.nx + 4) * (A.ny + 4);
                    e = cudaMemsetAsync(A.lmp, 0, kLPlanes * NL * sizeof(T), s);
                } else {
                    const size_t N = (size_t)A.nx * A.ny;
                    e = cudaMemsetAsync(A.lmp + kLmub * N, 0, 3 * N * sizeof(T), s);
                }
                if (e != cudaSuccess) return e;
                if (limiter == VLBM_LIM_LMP) {
                    k_adj_lmp_faces<T, VLBM_LIM_LMP, EXT, DA><<<gf, blk, 0, s>>>(A);
                    k_adj_lmp_bounds<T, VLBM_LIM_LMP, EXT><<<grd, blk, 0, s>>>(A);
                    k_adjoint_step<T, VLBM_LIM_LMP, DA, EXT><<<grd, blk, 0, s>>>(A);
                } else {
                    k_adj_lmp_faces<T, VLBM_LIM_RLMP, EXT, DA><<<gf, blk, 0, s>>>(A);
                    k_adj_lmp_bounds<T, VLBM_LIM_RLMP, EXT><<<grd, blk, 0, s>>>(A);
                    k_adjoint_step<T, VLBM_LIM_RLMP, DA, EXT><<<grd, blk, 0, s>>>(A);
                }
                if (EXT) {
                    const int ring = 2 * (A.nx + 4) + 2 * (A.ny + 2);
                    k_adj_lmp_ring<T><<<(ring + 255) / 256, 256, 0, s>>>(A);
                }
                break;
            }
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_adjoint_step(const AdjArgs<T> &A, int limiter, cudaStream_t s) {
    if (A.ext)
        return A.abar ? launch_adjoint_step_da<T, true, true>(A, limiter, s)
                      : launch_adjoint_step_da<T, false, true>(A, limiter, s);
    return A.abar ? launch_adjoint_step_da<T, true, false>(A, limiter, s)
                  : launch_adjoint_step_da<T, false, false>(A, limiter, s);
}

template <typename T>
static cudaError_t launch_adjoint_init(const T *init_state, const Layout &L, const StepConsts<T> *kc, const T *cot,
                                       T *grad, double *abar, cudaStream_t s) {
    const dim3 blk(32, 8), grd((L.nx + 31) / 32, (L.ny + 7) / 8);
    k_adjoint_init<T><<<grd, blk, 0, s>>>(init_state, L.pitch, L.nx, L.ny, kc, cot, grad, abar);
    return cudaGetLastError();
}

// Transpose of the ghost fill on the padded cotangent (np ghost layers), then its
// interior into cot.
// With abar (a differentiated a^n), the prescribed ghosts' dL/da^n is added at the
// step's constants k and time t.
template <typename T>
static cudaError_t fold_ghosts(T *pad, int np, const vlbm_state *s, T *cot, cudaStream_t st, const StepConsts<T> *k,
                               const double *t, double *abar) {
    int bc[4];
    uniform_types(s->bd, bc);
    const int nx = s->grid.nx, ny = s->grid.ny;
    k_adjoint_fold_y<T><<<(nx + 2 * np + 127) / 128, 128, 0, st>>>(pad, nx, ny, np, s->bd, bc[2], bc[3], k, t, abar);
    k_adjoint_fold_x<T><<<(ny + 127) / 128, 128, 0, st>>>(pad, nx, ny, np, s->bd, bc[0], bc[1], k, t, abar);
    const dim3 blk(32, 8), grd((nx + 31) / 32, (ny + 7) / 8);
    k_adjoint_unpad<T><<<grd, blk, 0, st>>>(pad, nx, ny, np, cot);
    return cudaGetLastError();
}

// Slots of the dL/da hand-over (256 bytes of the scratch).
struct ARed {
    double abar;
    unsigned long long key;
    unsigned int idx;
};

// dL/da^n accumulated in the slots goes to the conserved values of cot (a grouped
// cotangent of the sweep, or the caller's four planes) at the cell where lambda(st)
// is largest; the slots are reset for the next step.
template <typename T>
static cudaError_t hand_over_abar(const T *st, const Layout &L, double gamma, double alpha, ARed *red, T *cot,
                                  bool grouped, const double *lam_bc, cudaStream_t s) {
    const dim3 blk(32, 8), grd((L.nx + 31) / 32, (L.ny + 7) / 8);
    k_lambda_max<T><<<grd, blk, 0, s>>>(st, L.pitch, L.nx, L.ny, (T)gamma, &red->key);
    k_lambda_argmax<T><<<grd, blk, 0, s>>>(st, L.pitch, L.nx, L.ny, (T)gamma, &red->key, &red->idx);
    k_lambda_apply<T><<<1, 1, 0, s>>>(st, L.pitch, L.nx, gamma, alpha, &red->abar, &red->key, &red->idx, cot,
                                      (long long)L.nx * L.ny, grouped ? 1 : 0, lam_bc);
    return cudaGetLastError();
}

// The constants of the precision T inside a control block.
template <typename T> const StepConsts<T> *ctl_consts(const DevCtl *C);
template <> const StepConsts<float> *ctl_consts<float>(const DevCtl *C) { return &C->kf; }
template <> const StepConsts<double> *ctl_consts<double>(const DevCtl *C) { return &C->kd; }

}  // namespace vlbm

namespace {

constexpr size_t kCtlBytes = ((sizeof(DevCtl) + 255) / 256) * 256;
constexpr size_t kConstSlot = 128;   // one StepConsts<T> of the constants history, then t^n
constexpr size_t kSlotTime = 120;    // offset of t^n (double) in a slot
static_assert(sizeof(StepConsts<double>) <= kSlotTime && sizeof(StepConsts<float>) <= kSlotTime, "slot");

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

// Carving of the caller's scratch block (all offsets 256-byte aligned).
struct Plan {
    int64_t nckpt;        // checkpoints at steps 0, k, 2k, ...
    size_t ckpt_stride;   // state buffer + control block
    // Two segment buffers: the recomputation of one segment overlaps the adjoint
    // steps of the segment after it (see reverse). Each holds
    size_t seg_off[2];    // k + 1 state slots (slot 0 is only ever a TMA window start),
    size_t segctl_off[2]; // the control block of the recomputation,
    size_t desc_off[2];   // 2 k InstDesc of the row-marching kernel (by parity of n),
    size_t khist_off[2];  // the step constants (a^n) and the time t^n of each step.
    size_t cot_off;       // two cotangent buffers of nx x ny cells (grouped, kidx)
    size_t cot_bytes;
    size_t red_off;       // the dL/da hand-over slots
    size_t pad_off;       // a cotangent padded by the ghost layers the adjoint covers (grids with a boundary)
    size_t lmp_off;       // LMP / RLMP: the face and bound planes of the three-pass adjoint
    size_t total;
};

Plan plan_of(const vlbm_state *s, int64_t nsteps, int32_t every) {
    Plan p;
    const size_t buf = s->L.buf_bytes;
    p.nckpt = nsteps > 0 ? (nsteps + every - 1) / every : 1;
    p.ckpt_stride = round256(buf) + kCtlBytes;
    size_t off = (size_t)p.nckpt * p.ckpt_stride;
    for (int q = 0; q < 2; ++q) {
        p.seg_off[q] = off;
        off += (size_t)(every + 1) * round256(buf);
        p.segctl_off[q] = off;
        off += kCtlBytes;
        p.desc_off[q] = off;
        off += (size_t)2 * every * 512;
        p.khist_off[q] = off;
        off += round256((size_t)every * kConstSlot);
    }
    p.cot_bytes = round256((size_t)kNPlane * s->grid.nx * s->grid.ny * s->L.elem);
    p.cot_off = off;
    off += 2 * p.cot_bytes;
    p.red_off = off;
    off += 256;
    const bool lmp = s->limiter == VLBM_LIM_LMP || s->limiter == VLBM_LIM_RLMP;
    const int np = lmp ? 2 : 1;   // the LMP bounds reach the second ghost layer
    p.pad_off = off;
    off += round256((size_t)kNPlane * (s->grid.nx + 2 * np) * (s->grid.ny + 2 * np) * s->L.elem);
    p.lmp_off = off;
    if (lmp) off += round256((size_t)kLPlanes * (s->grid.nx + 4) * (s->grid.ny + 4) * s->L.elem);
    p.total = off;
    return p;
}

char *slot_ptr(char *scratch, const Plan &p, const vlbm_state *s, int q, int64_t j) {
    return scratch + p.seg_off[q] + (size_t)j * round256(s->L.buf_bytes);
}

int check_scratch(vlbm_state *s, void *scratch, size_t bytes, const Plan &p) {
    if (!scratch || ((uintptr_t)scratch & 255)) return fail(s, VLBM_E_NOMEM, "scratch NULL or not 256-byte aligned");
    if (bytes < p.total) return fail(s, VLBM_E_NOMEM, "scratch has %zu bytes, needs %zu", bytes, p.total);
    cudaPointerAttributes pa;
    cudaError_t e = cudaPointerGetAttributes(&pa, scratch);
    if (e != cudaSuccess || (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        return fail(s, VLBM_E_INVAL, "scratch is not device memory");
    }
    return VLBM_OK;
}

// Descriptors of the row-marching kernel for the recomputation: step j of a
// segment reads slot j + 1 and writes slot j + 2. The kernel reads planes
// 20 (n & 1) .. 20 (n & 1) + 19 of its TMA window, so the window starts
// (n & 1) slots before the slot it reads.
template <typename T>
bool build_recompute_descs(vlbm_state *s, char *scratch, const Plan &p, int32_t every, int q,
                           std::vector<unsigned char> &host) {
    host.assign((size_t)2 * every * 512, 0);
    InstDesc<T> base;
    memcpy(&base, s->desc_host.data(), sizeof base);
    for (int par = 0; par < 2; ++par) {
        for (int j = 0; j + 1 < every; ++j) {   // the last state of a segment is not stepped
            InstDesc<T> d = base;
            char *in = slot_ptr(scratch, p, s, q, j + 1);
            if (!encode_state_tmap(&d.tmap, in - (size_t)par * round256(s->L.buf_bytes), s->L)) return false;
            d.buf0 = d.buf1 = (T *)slot_ptr(scratch, p, s, q, j + 2);
            d.ctl = (DevCtl *)(scratch + p.segctl_off[q]);
            memcpy(host.data() + ((size_t)par * every + j) * 512, &d, sizeof d);
        }
    }
    return true;
}

// One recomputation step m = s0 + j of a segment.
// The prescribed ghosts of slot j + 1 (the state s^m, m = s0 + j) at the control
// block's t and a, for the recomputation step and for the adjoint step that read
// that state.
template <typename T>
cudaError_t dirichlet_slot(vlbm_state *s, char *scratch, const Plan &p, int q, int64_t m, int64_t j,
                           cudaStream_t st) {
    if (!s->bd.has_dir) return cudaSuccess;
    StepArgs<T> A = args_of<T>(s);
    T *in = (T *)slot_ptr(scratch, p, s, q, j + 1), *out = (T *)slot_ptr(scratch, p, s, q, j + 2);
    A.buf0 = (m & 1) ? out : in;
    A.buf1 = (m & 1) ? in : out;
    A.ctl = (DevCtl *)(scratch + p.segctl_off[q]);
    A.bd.ctl = A.ctl;
    return launch_dirichlet_ghosts<T>(A, st);
}

template <typename T>
cudaError_t recompute_step(vlbm_state *s, char *scratch, const Plan &p, int32_t every, int q, int64_t m, int64_t j,
                           cudaStream_t st) {
    cudaError_t e0 = dirichlet_slot<T>(s, scratch, p, q, m, j, st);
    if (e0 != cudaSuccess) return e0;
    if (use_fused(s)) {
        FusedBatchArgs<T> B = batch_args_of<T>(s);
        B.insts = (const InstDesc<T> *)(scratch + p.desc_off[q] + ((size_t)(m & 1) * every + j) * 512);
        return launch_step_fused<T>(B, s->limiter, s->fused_grid, st);
    }
    StepArgs<T> A = args_of<T>(s);
    T *in = (T *)slot_ptr(scratch, p, s, q, j + 1), *out = (T *)slot_ptr(scratch, p, s, q, j + 2);
    A.buf0 = (m & 1) ? out : in;
    A.buf1 = (m & 1) ? in : out;
    A.ctl = (DevCtl *)(scratch + p.segctl_off[q]);
    A.bd.ctl = A.ctl;
    return launch_step_simple<T>(A, st);   // writes the new state's ghost frame too
}

int rollout(vlbm_state *s, int64_t nsteps, int32_t every, char *scratch, const Plan &p) {
    const size_t buf = s->L.buf_bytes;
    for (int64_t n = 0; n <= nsteps; ++n) {
        if (n % every == 0 && (n < nsteps || nsteps == 0)) {
            char *ck = scratch + (size_t)(n / every) * p.ckpt_stride;
            const char *cur = (const char *)s->ws + ((n & 1) ? buf : 0);
            cudaError_t e = cudaMemcpyAsync(ck, cur, buf, cudaMemcpyDeviceToDevice, s->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(ck + round256(buf), s->ctl, sizeof(DevCtl), cudaMemcpyDeviceToDevice, s->stream);
            if (e != cudaSuccess) return cuda_fail(s, e, "checkpoint copy");
        }
        if (n == nsteps) break;
        cudaError_t e = step_once(s);
        if (e != cudaSuccess) return cuda_fail(s, e, "step launch");
    }
    s->at_init = false;
    s->roll_scratch = scratch;
    s->roll_steps = nsteps;
    s->roll_every = every;
    return VLBM_OK;
}

// The second stream of the reverse sweep and its events (made on first use, on the
// state's device; destroyed with the state).
static cudaError_t aux_stream(vlbm_state *s) {
    if (s->aux_ready) return cudaSuccess;
    cudaError_t e = cudaStreamCreateWithFlags(&s->aux_stream, cudaStreamNonBlocking);
    for (int i = 0; e == cudaSuccess && i < kAuxEvents; ++i)
        e = cudaEventCreateWithFlags(&s->aux_ev[i], cudaEventDisableTiming);
    if (e == cudaSuccess) s->aux_ready = true;
    return e;
}

// Recomputation of segment c (steps s0 .. e0) into segment buffer q on stream st:
// the checkpoint into slot 1, then the step kernel for steps s0 .. e0 - 1, with the
// constants (and times) of every step recorded for the adjoint steps.
template <typename T>
cudaError_t recompute_segment(vlbm_state *s, char *scratch, const Plan &p, int64_t nsteps, int32_t every, int64_t c,
                              int q, cudaStream_t st) {
    const size_t buf = s->L.buf_bytes;
    const bool fixed_a = s->a_fixed > 0.0;
    const bool diff_a = !fixed_a && s->adj_mode == VLBM_ADJOINT_DIFF_A;
    DevCtl *segctl = (DevCtl *)(scratch + p.segctl_off[q]);
    char *khist = scratch + p.khist_off[q];
    const int64_t s0 = c * every;
    const int64_t e0 = (s0 + every < nsteps ? s0 + every : nsteps) - 1;
    const char *ck = scratch + (size_t)c * p.ckpt_stride;
    cudaError_t e = cudaMemcpyAsync(slot_ptr(scratch, p, s, q, 1), ck, buf, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(segctl, ck + round256(buf), sizeof(DevCtl), cudaMemcpyDeviceToDevice, st);
    for (int64_t m = s0; e == cudaSuccess && m <= e0; ++m) {
        if (!fixed_a)
            e = cudaMemcpyAsync(khist + (m - s0) * kConstSlot, ctl_consts<T>(segctl), sizeof(StepConsts<T>),
                                cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess && diff_a)
            e = cudaMemcpyAsync(khist + (m - s0) * kConstSlot + kSlotTime, &segctl->t, sizeof(double),
                                cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess && m < e0) e = recompute_step<T>(s, scratch, p, every, q, m, m - s0, st);
    }
    if (e == cudaSuccess) e = dirichlet_slot<T>(s, scratch, p, q, e0, e0 - s0, st);   // the segment's last state
    return e;
}

// Reverse sweep, last segment first. The recomputation of segment c - 1 (on the
// second stream, into the other segment buffer) overlaps the adjoint steps of
// segment c (on the state's stream): at small grids neither fills the GPU. Events
// order each segment's adjoint steps after its recomputation, and the
// recomputation into a buffer after the adjoint steps that last read it.
template <typename T>
int reverse(vlbm_state *s, int64_t nsteps, int32_t every, char *scratch, const Plan &p, const void *dLduN,
            void *dLdu0) {
    const bool fixed_a = s->a_fixed > 0.0;
    const bool diff_a = !fixed_a && s->adj_mode == VLBM_ADJOINT_DIFF_A;
    ARed *red = (ARed *)(scratch + p.red_off);
    T *cot[2] = {(T *)(scratch + p.cot_off), (T *)(scratch + p.cot_off + p.cot_bytes)};
    {
        const dim3 blk(32, 8), grd((s->grid.nx + 31) / 32, (s->grid.ny + 7) / 8);
        k_adjoint_seed<T><<<grd, blk, 0, s->stream>>>((const T *)dLduN, s->grid.nx, s->grid.ny, cot[0]);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && diff_a) {
        e = cudaMemsetAsync(red, 0, sizeof(ARed), s->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(&red->idx, 0xff, sizeof(unsigned int), s->stream);
    }
    if (e != cudaSuccess) return cuda_fail(s, e, "cotangent seed");
    std::vector<unsigned char> descs[2];
    if (use_fused(s)) {
        for (int q = 0; q < 2; ++q) {
            if (!build_recompute_descs<T>(s, scratch, p, every, q, descs[q]))
                return fail(s, VLBM_E_CUDA, "TMA descriptor of a recomputation slot");
            e = cudaMemcpyAsync(scratch + p.desc_off[q], descs[q].data(), descs[q].size(), cudaMemcpyHostToDevice,
                                s->stream);
            if (e != cudaSuccess) return cuda_fail(s, e, "descriptor upload");
        }
    }
    e = aux_stream(s);
    if (e != cudaSuccess) return cuda_fail(s, e, "second stream of the reverse sweep");
    cudaStream_t aux = s->aux_stream;
    cudaEvent_t ev_fork = s->aux_ev[0], ev_rec[2] = {s->aux_ev[1], s->aux_ev[2]},
                ev_adj[2] = {s->aux_ev[3], s->aux_ev[4]};
    bool adj_used[2] = {false, false};   // an adjoint step has read buffer q (ev_adj[q] recorded)
    int cur = 0;
    AdjArgs<T> A;
    A.pitch = s->L.pitch;
    A.nx = s->grid.nx;
    A.ny = s->grid.ny;
    A.abar = diff_a ? &red->abar : nullptr;
    bool periodic = true;
    for (int q = 0; q < 4; ++q) periodic = periodic && s->grid.bc[q] == VLBM_BC_PERIODIC;
    A.ext = periodic ? 0 : 1;
    A.pad = (s->limiter == VLBM_LIM_LMP || s->limiter == VLBM_LIM_RLMP) ? 2 : 1;
    uniform_types(s->bd, A.bc);
    A.sponge = s->sponge;
    A.lmp = (T *)(scratch + p.lmp_off);
    T *pad = (T *)(scratch + p.pad_off);
    const int64_t clast = nsteps > 0 ? p.nckpt - 1 : -1;
    // the second stream starts after everything the state's stream holds so far
    e = cudaEventRecord(ev_fork, s->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, ev_fork, 0);
    if (e == cudaSuccess && clast >= 0) {
        e = recompute_segment<T>(s, scratch, p, nsteps, every, clast, (int)(clast & 1), aux);
        if (e == cudaSuccess) e = cudaEventRecord(ev_rec[clast & 1], aux);
    }
    for (int64_t c = clast; e == cudaSuccess && c >= 0; --c) {
        const int q = (int)(c & 1);
        DevCtl *segctl = (DevCtl *)(scratch + p.segctl_off[q]);
        char *khist = scratch + p.khist_off[q];
        const int64_t s0 = c * every;
        const int64_t e0 = (s0 + every < nsteps ? s0 + every : nsteps) - 1;
        e = cudaStreamWaitEvent(s->stream, ev_rec[q], 0);
        if (e == cudaSuccess && c > 0) {   // segment c - 1 into the other buffer, once its readers are done
            const int qn = q ^ 1;
            if (adj_used[qn]) e = cudaStreamWaitEvent(aux, ev_adj[qn], 0);
            if (e == cudaSuccess) e = recompute_segment<T>(s, scratch, p, nsteps, every, c - 1, qn, aux);
            if (e == cudaSuccess) e = cudaEventRecord(ev_rec[qn], aux);
        }
        if (e != cudaSuccess) break;
        for (int64_t m = e0; m >= s0; --m) {
            A.fwd = (const T *)slot_ptr(scratch, p, s, q, m - s0 + 1);
            A.cot_in = cot[cur];
            A.cot_out = A.ext ? pad : cot[cur ^ 1];
            A.k = fixed_a ? ctl_consts<T>(segctl) : (const StepConsts<T> *)(khist + (m - s0) * kConstSlot);
            e = launch_adjoint_step<T>(A, s->limiter, s->stream);
            if (e == cudaSuccess && A.ext)
                e = fold_ghosts<T>(pad, A.pad, s, cot[cur ^ 1], s->stream, A.k,
                                   (const double *)(khist + (m - s0) * kConstSlot + kSlotTime), A.abar);
            if (e != cudaSuccess) break;
            cur ^= 1;
            if (diff_a && m > 0) {   // a^m came from lambda of s^m (a^0 waits for the init map)
                e = hand_over_abar<T>(A.fwd, s->L, s->gamma, s->alpha, red, cot[cur], true, &segctl->lam_bc,
                                      s->stream);
                if (e != cudaSuccess) break;
            }
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev_adj[q], s->stream);
        adj_used[q] = true;
    }
    // join: whatever the second stream still holds comes before the state's next work
    cudaError_t ej = cudaEventRecord(ev_fork, aux);
    if (ej == cudaSuccess) ej = cudaStreamWaitEvent(s->stream, ev_fork, 0);
    if (e == cudaSuccess) e = ej;
    if (e != cudaSuccess) return cuda_fail(s, e, "reverse sweep");
    const size_t buf = s->L.buf_bytes;
    const char *ck0 = scratch;
    DevCtl *segctl0 = (DevCtl *)(scratch + p.segctl_off[0]);
    e = launch_adjoint_init<T>((const T *)ck0, s->L, ctl_consts<T>((const DevCtl *)(ck0 + round256(buf))), cot[cur],
                               (T *)dLdu0, diff_a ? &red->abar : nullptr, s->stream);
    if (e == cudaSuccess && diff_a)
        e = hand_over_abar<T>((const T *)ck0, s->L, s->gamma, s->alpha, red, (T *)dLdu0, false, &segctl0->lam_bc,
                              s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "initialisation adjoint launch");
    return VLBM_OK;
}

}  // namespace


extern "C" {

size_t vlbm_adjoint_scratch_bytes(const vlbm_state *s, int64_t nsteps, int32_t ckpt_every) {
    if (!s || nsteps < 0 || ckpt_every < 1) return 0;
    return plan_of(s, nsteps, ckpt_every).total;
}

int vlbm_rollout(vlbm_state *s, int64_t nsteps, int32_t ckpt_every, void *d_scratch, size_t scratch_bytes) {
    if (!s) return fail(nullptr, VLBM_E_INVAL, "state is NULL");
    if (nsteps < 0 || ckpt_every < 1) return fail(s, VLBM_E_INVAL, "need nsteps >= 0 and ckpt_every >= 1");
    if (!s->loaded || !s->at_init)
        return fail(s, VLBM_E_INVAL, "rollout starts from the state vlbm_set_conserved leaves (n = 0)");
    DeviceGuard g(s->device);
    const Plan p = plan_of(s, nsteps, ckpt_every);
    int rc = check_scratch(s, d_scratch, scratch_bytes, p);
    if (rc) return rc;
    return rollout(s, nsteps, ckpt_every, (char *)d_scratch, p);
}

int vlbm_adjoint_set_mode(vlbm_state *s, int32_t mode) {
    if (!s) return fail(nullptr, VLBM_E_INVAL, "state is NULL");
    if (mode != VLBM_ADJOINT_HOLD_A && mode != VLBM_ADJOINT_DIFF_A) return fail(s, VLBM_E_INVAL, "mode out of range");
    s->adj_mode = mode;
    return VLBM_OK;
}

int vlbm_adjoint(vlbm_state *s, const void *d_u0, int64_t nsteps, int32_t ckpt_every, const void *d_dLduN,
                 void *d_dLdu0, void *d_scratch, size_t scratch_bytes) {
    if (!s) return fail(nullptr, VLBM_E_INVAL, "state is NULL");
    if (nsteps < 0 || ckpt_every < 1) return fail(s, VLBM_E_INVAL, "need nsteps >= 0 and ckpt_every >= 1");
    if (!d_dLduN || !d_dLdu0) return fail(s, VLBM_E_INVAL, "cotangent pointer is NULL");
    DeviceGuard g(s->device);
    const Plan p = plan_of(s, nsteps, ckpt_every);
    int rc = check_scratch(s, d_scratch, scratch_bytes, p);
    if (rc) return rc;
    char *scratch = (char *)d_scratch;
    if (d_u0) {
        const long long N = (long long)s->grid.nx * s->grid.ny;
        const char *u0 = (const char *)d_u0;
        const size_t pb = (size_t)N * s->L.elem;
        rc = set_conserved(s, u0, u0 + pb, u0 + 3 * pb);
        if (rc) return rc;
        rc = rollout(s, nsteps, ckpt_every, scratch, p);
        if (rc) return rc;
    } else if (s->roll_scratch != d_scratch || s->roll_steps != nsteps || s->roll_every != ckpt_every) {
        return fail(s, VLBM_E_INVAL, "no rollout with these steps, interval and scratch precedes this call");
    }
    return s->precision == VLBM_FP64 ? reverse<double>(s, nsteps, ckpt_every, scratch, p, d_dLduN, d_dLdu0)
                                     : reverse<float>(s, nsteps, ckpt_every, scratch, p, d_dLduN, d_dLdu0);
}

}  // extern "C"
