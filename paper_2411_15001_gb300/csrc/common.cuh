// common.cuh -- reductions, the end-of-step finaliser, ghost frame, initial
// state, moments and checkpoints. Shared by all step kernels.
#pragma once

#include "physics.cuh"
#include "vlbm_internal.h"
#include "../../include/vlbm.h"

namespace vlbm {

// Offset of value 0 of cell (i, j) in a state buffer, and of value q relative to it
// (layout: sidx in vlbm_internal.h).
template <typename T>
__device__ __forceinline__ long long cidx(const StepArgs<T> &A, int i, int j) {
    return sidx(A.pitch, 0, i, j);
}
template <typename T>
__device__ __forceinline__ long long qoff(const StepArgs<T> &A, int q) {
    return (long long)(q >> 2) * 4 * A.pitch + (q & 3);
}

// The four values of one group of a cell (state layout in vlbm_internal.h): one vector
// access (16 bytes in FP32, two of 16 bytes in FP64); `p` is 16-byte aligned.
template <typename T>
__device__ __forceinline__ void ld_group(const T *p, T v[4]) {
    if constexpr (is_f64<T>::value) {
        const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    } else {
        const float4 a = *reinterpret_cast<const float4 *>(p);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    }
}
template <typename T>
__device__ __forceinline__ void st_group(T *p, T a, T b, T c, T d) {
    if constexpr (is_f64<T>::value) {
        reinterpret_cast<double2 *>(p)[0] = make_double2(a, b);
        reinterpret_cast<double2 *>(p)[1] = make_double2(c, d);
    } else {
        *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
    }
}

// NaN-propagating max / min.
template <typename T> __device__ __forceinline__ T pmax(T a, T b) { return (b > a || b != b) ? b : a; }
template <typename T> __device__ __forceinline__ T pmin(T a, T b) { return (b < a || b != b) ? b : a; }

// Error-free sum of two floats (Knuth's TwoSum) and a double-float accumulator:
// the FP32 path keeps its conservation sums as (hi, lo) float pairs (about 48
// significant bits) and converts to double once per CTA, because FP64
// instructions run at a small fraction of the FP32 rate on this GPU.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

struct DFloat {
    float hi, lo;
    __device__ __forceinline__ void add(float bh, float bl) {
        float s, e;
        two_sum(hi, bh, s, e);
        e = __fadd_rn(e, __fadd_rn(lo, bl));
        hi = __fadd_rn(s, e);
        lo = __fsub_rn(e, __fsub_rn(hi, s));
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Per-thread conservation sums. FP32: Kahan-compensated float accumulators
// (the compensation keeps about twice the float precision over a column of a
// few hundred cells); the warp and CTA reductions carry (hi, lo) pairs with
// TwoSum, and one double per CTA goes to the FP64 atomics.
template <typename T> struct SumAcc;
template <> struct SumAcc<float> {
    float s[4], c[4];
    __device__ __forceinline__ void zero() { for (int q = 0; q < 4; ++q) s[q] = c[q] = 0.f; }
    __device__ __forceinline__ void add_cell(const float u[4]) {
        for (int q = 0; q < 4; ++q) {
            const float y = __fsub_rn(u[q], c[q]);
            const float t = __fadd_rn(s[q], y);
            c[q] = __fsub_rn(__fsub_rn(t, s[q]), y);
            s[q] = t;
        }
    }
    __device__ __forceinline__ void shfl_add(int off) {
        for (int q = 0; q < 4; ++q) {
            DFloat a{s[q], -c[q]};
            a.add(__shfl_xor_sync(0xffffffffu, s[q], off), -__shfl_xor_sync(0xffffffffu, c[q], off));
            s[q] = a.hi;
            c[q] = -a.lo;
        }
    }
    __device__ __forceinline__ double value(int q) const { return (double)s[q] - (double)c[q]; }
};
template <> struct SumAcc<double> {
    double s[4];
    __device__ __forceinline__ void zero() { for (int q = 0; q < 4; ++q) s[q] = 0.0; }
    __device__ __forceinline__ void add_cell(const double u[4]) { for (int q = 0; q < 4; ++q) s[q] += u[q]; }
    __device__ __forceinline__ void shfl_add(int off) {
        for (int q = 0; q < 4; ++q) s[q] += __shfl_xor_sync(0xffffffffu, s[q], off);
    }
    __device__ __forceinline__ double value(int q) const { return s[q]; }
};

template <typename T>
__device__ __forceinline__ bool all_finite(const T u[4]) {
    return isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]) && isfinite(u[3]);
}

// Per-thread monitor of the cells a thread wrote: max lambda, min rho, sums,
// the counts of cells outside G / non-finite, and of faces whose theta_p needed
// the FP64 solve.
template <typename T>
struct Monitor {
    T lam, minrho, minrhoe;
    SumAcc<T> sum;
    unsigned int bad, nonfin, fp64;
    __device__ __forceinline__ void init() {
        lam = T(0);
        minrho = T(INFINITY);
        minrhoe = T(INFINITY);
        sum.zero();
        bad = nonfin = fp64 = 0u;
    }
    __device__ __forceinline__ void add_cell(const T u[4], T gamma, T gm1) {
        // internal energy in the state's precision (reported; admissibility below
        // is decided by the exact test)
        T rhoe;
        const T sp = cell_speed_rhoe(u, gamma, gm1, rhoe);   // NaN or inf if any component is
        lam = pmax(lam, sp);
        minrho = pmin(minrho, u[0]);
        minrhoe = pmin(minrhoe, rhoe);
        sum.add_cell(u);
        // no finite speed: a non-finite value, or finite values outside G (p < 0 gives a
        // NaN sound speed); a finite speed can still belong to a state outside G (rho < 0)
        if (!(sp <= T(3.0e38))) {
            if (all_finite(u)) ++bad;
            else ++nonfin;
        } else if (!in_G(u)) {
            ++bad;
        }
    }
    __device__ __forceinline__ void warp_reduce() {
        for (int off = 16; off > 0; off >>= 1) {
            lam = pmax(lam, __shfl_xor_sync(0xffffffffu, lam, off));
            minrho = pmin(minrho, __shfl_xor_sync(0xffffffffu, minrho, off));
            minrhoe = pmin(minrhoe, __shfl_xor_sync(0xffffffffu, minrhoe, off));
            sum.shfl_add(off);
            bad += __shfl_xor_sync(0xffffffffu, bad, off);
            nonfin += __shfl_xor_sync(0xffffffffu, nonfin, off);
            fp64 += __shfl_xor_sync(0xffffffffu, fp64, off);
        }
    }
};

// Publish one CTA's monitor into the step's reduction slots. Must be called by
// every thread of the CTA (uses shared memory and __syncthreads).
template <typename T>
__device__ void block_publish(Monitor<T> &m, DevCtl *C) {
    __shared__ Monitor<T> part[32];
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    const int lane = tid & 31, warp = tid >> 5, nwarp = (nthr + 31) >> 5;
    m.warp_reduce();
    if (lane == 0) part[warp] = m;
    __syncthreads();
    if (warp == 0) {
        if (lane < nwarp) m = part[lane];
        else m.init();
        m.warp_reduce();
        if (lane == 0) {
            atomicMax(&C->lam_key, ordered_key((double)m.lam));
            atomicMin(&C->minrho_key, ordered_key((double)m.minrho));
            atomicMin(&C->minrhoe_key, ordered_key((double)m.minrhoe));
            for (int c = 0; c < 4; ++c) atomicAdd(&C->sum[c], m.sum.value(c));
            if (m.bad) atomicAdd(&C->bad, (unsigned long long)m.bad);
            if (m.nonfin) atomicAdd(&C->nonfinite, (unsigned long long)m.nonfin);
            if (m.fp64) atomicAdd(&C->fp64_faces, (unsigned long long)m.fp64);
        }
    }
}

__device__ __forceinline__ void reset_slots(DevCtl *C) {
    C->lam_key = 0ull;
    C->minrho_key = ~0ull;
    C->minrhoe_key = ~0ull;
    C->bad = 0ull;
    C->nonfinite = 0ull;
    C->fp64_faces = 0ull;
    for (int c = 0; c < 4; ++c) C->sum[c] = 0.0;
    C->blocks_done = 0u;
}

// Free-running kinetic speed a = 2 lambda / (1 - alpha) (= 4 lambda at alpha = 1/2,
// the critical Bouchut speed of Sec. 4), or the fixed one.
__device__ __forceinline__ double next_speed(const DevCtl *C, double lam) {
    return C->a_fixed > 0.0 ? C->a_fixed : 2.0 * lam / (1.0 - C->alpha);
}

// The constants of the step about to run with kinetic speed C->a, in both
// precisions (FP64 divisions once per step instead of once per CTA or cell).
__device__ __forceinline__ void set_consts(DevCtl *C) {
    C->kf = make_consts<float>(C->a, C->alpha, C->gamma, C->eps);
    C->kd = make_consts<double>(C->a, C->alpha, C->gamma, C->eps);
}

template <typename T> __device__ __forceinline__ StepConsts<T> consts_of(const DevCtl *C);
template <> __device__ __forceinline__ StepConsts<float> consts_of<float>(const DevCtl *C) { return C->kf; }
template <> __device__ __forceinline__ StepConsts<double> consts_of<double>(const DevCtl *C) { return C->kd; }

// Step control for the next step: Delta t = dx / a, shortened to land on t_end.
__device__ __forceinline__ void plan_next(DevCtl *C, double t, double a_free) {
    double a = a_free, dt = C->dx / a_free;
    int last = 0;
    if (C->t_end > 0.0 && !C->done) {
        if (t >= C->t_end) {
            C->done = 1;
        } else if (t + dt >= C->t_end) {
            dt = C->t_end - t;
            a = C->dx / dt;
            last = 1;
        }
    }
    C->a = a;
    C->dt = dt;
    C->last = last;
    set_consts(C);
}

// Called by one thread of the last CTA to finish a step: the grid-wide max of
// lambda over the new state sets a^{n+1} (Sec. 4 preamble), time advances by
// the step's Delta t, monitors are published, sticky errors recorded.
__device__ inline void finalize_step(DevCtl *C) {
    volatile DevCtl *V = C;
    const double lam_cells = key_to_double(V->lam_key);
    const double lam = C->lam_bc > lam_cells ? C->lam_bc : lam_cells;   // NaN stays NaN
    const double minrho = key_to_double(V->minrho_key);
    const double minrhoe = key_to_double(V->minrhoe_key);
    const unsigned long long bad = V->bad, nonfin = V->nonfinite;
    C->fp64_last = (long long)V->fp64_faces;
    double s[4];
    for (int c = 0; c < 4; ++c) s[c] = V->sum[c];
    const long long n1 = C->n + 1;
    const double t1 = C->t + C->dt;
    C->lambda = lam;
    C->min_rho = minrho;
    C->min_rhoe = minrhoe;
    C->bad_last = (long long)bad;
    C->nonfinite_last = (long long)nonfin;
    for (int c = 0; c < 4; ++c) C->sum_last[c] = s[c];
    if ((bad || nonfin) && C->first_bad_step < 0) C->first_bad_step = n1;
    // a cell outside G is the positivity failure, even when the same step also made
    // values non-finite; without a finite lambda no further step can be planned
    if (bad && !C->status) C->status = VLBM_E_POSITIVITY;
    if (nonfin || !isfinite(lam)) {
        if (!C->status) C->status = VLBM_E_NONFINITE;
        C->done = 1;
    }
    if (C->last || C->status == VLBM_E_TIMEOUT) C->done = 1;
    double a_free = next_speed(C, lam);
    if (!(a_free > 0.0) || !isfinite(a_free)) {
        C->done = 1;
        if (!C->status) C->status = VLBM_E_NONFINITE;
        a_free = C->a;
    }
    C->n = n1;
    C->t = t1;
    C->a_free = a_free;
    plan_next(C, t1, a_free);
    reset_slots(C);
    __threadfence();
}

// Last-CTA detection: returns true in every thread of the CTA that finished last.
__device__ __forceinline__ bool last_block(DevCtl *C, unsigned int nblocks) {
    __shared__ unsigned int ticket;
    __threadfence();
    __syncthreads();
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    if (tid == 0) ticket = atomicAdd(&C->blocks_done, 1u);
    __syncthreads();
    return ticket == nblocks - 1;
}

// ----------------------------------------------------------------- ghost frame

// Source of ghost index i along an axis of n cells with the side's rule;
// *mirror is set for a reflective wall (Sec. 4.8: symmetry wall).
__device__ __forceinline__ int ghost_source(int i, int n, int bc_lo, int bc_hi, bool *mirror) {
    *mirror = false;
    if (i >= 0 && i < n) return i;
    const int bc = i < 0 ? bc_lo : bc_hi;
    if (bc == VLBM_BC_PERIODIC) return i < 0 ? i + n : i - n;
    if (bc == VLBM_BC_TRANSMISSIVE) return i < 0 ? 0 : n - 1;
    *mirror = true;
    return i < 0 ? -1 - i : 2 * n - 1 - i;
}

// Source of ghost index i (outside [0, n)) under side type `type` (not Dirichlet).
__device__ __forceinline__ int ghost_source_typed(int i, int n, int type, bool *mirror) {
    *mirror = type == VLBM_BC_REFLECTIVE;
    if (type == VLBM_BC_PERIODIC) return i < 0 ? i + n : i - n;
    if (type == VLBM_BC_TRANSMISSIVE) return i < 0 ? 0 : n - 1;
    return i < 0 ? -1 - i : 2 * n - 1 - i;
}

// The prescribed field at the centre of cell (i, j) at time t (vlbm_field): both
// sides of each half-plane test rounded after every operation, products first,
// in double whatever the state's precision.
template <typename T>
__device__ __forceinline__ void field_state(const Bound &B, int i, int j, double t, T u[4]) {
    const double x = __dadd_rn(B.x0, __dmul_rn((double)i + 0.5, B.dx));
    const double y = __dadd_rn(B.y0, __dmul_rn((double)j + 0.5, B.dx));
    bool inside = true;
    for (int k = 0; k < B.nplanes; ++k)
        if (!(__dadd_rn(__dmul_rn(B.pnx[k], x), __dmul_rn(B.pny[k], y)) >= __dadd_rn(B.c0[k], __dmul_rn(B.c1[k], t))))
            inside = false;
#pragma unroll
    for (int q = 0; q < 4; ++q) u[q] = (T)(inside ? B.in[q] : B.out[q]);
}

template <typename T>
struct GhostState {
    T u[4];
    int hit;   // the cell holds a prescribed state (populations at equilibrium)
};

// Ghost cell (i, j) as the boundary prescribes it: a Dirichlet part of a side
// (the field at the cell's centre), or a corner that takes the y rule of a
// Dirichlet x ghost (its copy or mirror image). hit = 0 for every other cell.
// The x rule applies first, then the y rule, as for the other ghost cells.
template <typename T>
__device__ __noinline__ GhostState<T> dirichlet_ghost(const Bound *B, int nx, int ny, int i, int j) {
    GhostState<T> g;
    g.hit = 0;
    const bool gx = i < 0 || i >= nx, gy = j < 0 || j >= ny;
    int sj = j;
    bool flip = false;
    if (gy) {
        const int ty = side_type(*B, j < 0 ? 2 : 3, i);
        if (ty != VLBM_BC_DIRICHLET) {
            if (!gx) return g;
            sj = ghost_source_typed(j, ny, ty, &flip);
            if (side_type(*B, i < 0 ? 0 : 1, sj) != VLBM_BC_DIRICHLET) return g;
        }
    } else {
        if (!gx || side_type(*B, i < 0 ? 0 : 1, j) != VLBM_BC_DIRICHLET) return g;
    }
    field_state(*B, i, sj, B->ctl->t, g.u);
    if (flip) g.u[2] = -g.u[2];
    g.hit = 1;
    return g;
}

// Ghost index of thread t of a ghost pass: the 2 x (nx + 4) cells of the top and
// bottom layers first, then the 2 x ny of the left and right ones.
template <typename T>
__device__ __forceinline__ bool ghost_of_thread(const StepArgs<T> &A, long long t, int *gi, int *gj) {
    const int nx = A.nx, ny = A.ny;
    const long long rowpart = 4ll * (nx + 4);
    if (t >= rowpart + 4ll * ny) return false;
    if (t < rowpart) {
        const int r = (int)(t / (nx + 4));
        *gi = (int)(t % (nx + 4)) - 2;
        *gj = r < 2 ? r - 2 : ny + (r - 2);
    } else {
        const long long q = t - rowpart;
        const int c = (int)(q / ny);
        *gj = (int)(q % ny);
        *gi = c < 2 ? c - 2 : nx + (c - 2);
    }
    return true;
}

// If the boundary prescribes ghost (gi, gj), write its state and Maxwellians at the
// kinetic speed of the control block's next step into buf; true if it did.
template <typename T>
__device__ __forceinline__ bool write_dirichlet_ghost(const StepArgs<T> &A, T *buf, int gi, int gj) {
    const GhostState<T> gs = dirichlet_ghost<T>(&A.bd, A.nx, A.ny, gi, gj);
    if (!gs.hit) return false;
    const StepConsts<T> k = consts_of<T>(A.ctl);
    T f[4], g[4], M1[4], M2[4], M3[4], M4[4];
    euler_fluxes(gs.u, k.gm1, f, g);
    maxwell_pm(gs.u, f, k, M1, M2);
    maxwell_pm(gs.u, g, k, M3, M4);
    const long long dst = cidx(A, gi, gj);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        buf[dst + qoff(A, q)] = gs.u[q];
        buf[dst + qoff(A, (4 + q))] = M1[q];
        buf[dst + qoff(A, (8 + q))] = M2[q];
        buf[dst + qoff(A, (12 + q))] = M3[q];
        buf[dst + qoff(A, (16 + q))] = M4[q];
    }
    return true;
}

// The prescribed ghosts alone, in buffer (n & 1), before a step of the row-marching
// kernel (which writes every other ghost as an image of the cells it updates).
template <typename T>
__global__ void k_dirichlet_ghosts(StepArgs<T> A) {
    int gi, gj;
    if (!ghost_of_thread(A, (long long)blockIdx.x * blockDim.x + threadIdx.x, &gi, &gj)) return;
    write_dirichlet_ghost(A, (A.ctl->n & 1) ? A.buf1 : A.buf0, gi, gj);
}

// The fields of a grid's descriptor that the step kernels' cell loops use, held in
// registers (the descriptor itself lives in global memory).
struct Geo {
    int pitch, nx, ny;
    int bc[4];
    int sponge;
};

// Write the ghost images of interior cell (c, O) into `out`: its periodic
// copies, zero-gradient copies or mirror images on the other side of every
// boundary it sits next to (the inverse of the ghost_source map). Prescribed
// (Dirichlet) parts get no images: the step that reads them evaluates the field.
// A side that switches type does so at least two cells from its ends, so the
// types at (c, O) hold for the corner images too.
template <typename T>
__device__ __forceinline__ void write_ghost_images(const Geo &D, T *out, int c, int O,
                                                   const T nv[kNPlane], const Bound *bd) {
    const int tW = D.bc[0] >= 0 ? D.bc[0] : side_type(*bd, 0, O);
    const int tE = D.bc[1] >= 0 ? D.bc[1] : side_type(*bd, 1, O);
    const int tS = D.bc[2] >= 0 ? D.bc[2] : side_type(*bd, 2, c);
    const int tN = D.bc[3] >= 0 ? D.bc[3] : side_type(*bd, 3, c);
    int gx[3], gy[3];
    bool mxs[3], mys[3];
    int ngx = 1, ngy = 1;
    gx[0] = c;
    mxs[0] = false;
    gy[0] = O;
    mys[0] = false;
    const int nx = D.nx, ny = D.ny;
    if (tW == VLBM_BC_PERIODIC) {
        if (c >= nx - 2) { gx[ngx] = c - nx; mxs[ngx++] = false; }
        if (c <= 1) { gx[ngx] = c + nx; mxs[ngx++] = false; }
    } else {
        if (c == 0 && tW == VLBM_BC_TRANSMISSIVE) {
            gx[ngx] = -1; mxs[ngx++] = false;
            gx[ngx] = -2; mxs[ngx++] = false;
        }
        if (c <= 1 && tW == VLBM_BC_REFLECTIVE) { gx[ngx] = -1 - c; mxs[ngx++] = true; }
        if (c == nx - 1 && tE == VLBM_BC_TRANSMISSIVE) {
            gx[ngx] = nx; mxs[ngx++] = false;
            gx[ngx] = nx + 1; mxs[ngx++] = false;
        }
        if (c >= nx - 2 && tE == VLBM_BC_REFLECTIVE) { gx[ngx] = 2 * nx - 1 - c; mxs[ngx++] = true; }
    }
    if (tS == VLBM_BC_PERIODIC) {
        if (O >= ny - 2) { gy[ngy] = O - ny; mys[ngy++] = false; }
        if (O <= 1) { gy[ngy] = O + ny; mys[ngy++] = false; }
    } else {
        if (O == 0 && tS == VLBM_BC_TRANSMISSIVE) {
            gy[ngy] = -1; mys[ngy++] = false;
            gy[ngy] = -2; mys[ngy++] = false;
        }
        if (O <= 1 && tS == VLBM_BC_REFLECTIVE) { gy[ngy] = -1 - O; mys[ngy++] = true; }
        if (O == ny - 1 && tN == VLBM_BC_TRANSMISSIVE) {
            gy[ngy] = ny; mys[ngy++] = false;
            gy[ngy] = ny + 1; mys[ngy++] = false;
        }
        if (O >= ny - 2 && tN == VLBM_BC_REFLECTIVE) { gy[ngy] = 2 * ny - 1 - O; mys[ngy++] = true; }
    }
    for (int a = 0; a < ngx; ++a)
        for (int e = 0; e < ngy; ++e) {
            if (a == 0 && e == 0) continue;
            T *base = out + sidx(D.pitch, 0, gx[a], gy[e]);
#pragma unroll
            for (int g = 0; g < kNGroup; ++g) {
                // u_1 <-> u_2 across an x-wall, u_3 <-> u_4 across a y-wall; the normal
                // momentum of every group negated
                const int gs = (g == 1 || g == 2) ? 3 - g : ((g == 3 || g == 4) ? 7 - g : g);
                const bool sw = (g == 1 || g == 2) ? mxs[a] : ((g == 3 || g == 4) ? mys[e] : false);
                T v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = sw ? nv[4 * gs + q] : nv[4 * g + q];
                if (mxs[a]) v[1] = -v[1];
                if (mys[e]) v[2] = -v[2];
                T *gp = base + (long long)g * 4 * D.pitch;   // scalar stores: the images are rare, and a
#pragma unroll                                                 // vector store would pin its values to aligned registers
                for (int q = 0; q < 4; ++q) gp[q] = v[q];
            }
        }
}


// Fill the two ghost layers of buffer (n & 1): periodic wrap, zero-gradient copy
// of u and u_1..u_4, or the mirror image (normal momentum negated in u and all
// populations, u_1 <-> u_2 across an x-wall, u_3 <-> u_4 across a y-wall); a
// prescribed state with its Maxwellians at the next step's kinetic speed.
// Corners take the x rule, then the y rule.
template <typename T>
__global__ void k_ghosts(StepArgs<T> A) {
    const int nx = A.nx, ny = A.ny;
    int gi, gj;
    if (!ghost_of_thread(A, (long long)blockIdx.x * blockDim.x + threadIdx.x, &gi, &gj)) return;
    T *buf = (A.ctl->n & 1) ? A.buf1 : A.buf0;
    if (A.bd.has_dir && write_dirichlet_ghost(A, buf, gi, gj)) return;
    // source cell: the y rule (type at column gi) applied to the x rule (type at the
    // source row); uniform sides skip the look-up
    bool mx = false, my = false;
    int sj = gj, si = gi;
    if (gj < 0 || gj >= ny) {
        const int s = gj < 0 ? 2 : 3;
        sj = ghost_source_typed(gj, ny, A.bc[s] >= 0 ? A.bc[s] : side_type(A.bd, s, gi), &my);
    }
    if (gi < 0 || gi >= nx) {
        const int s = gi < 0 ? 0 : 1;
        si = ghost_source_typed(gi, nx, A.bc[s] >= 0 ? A.bc[s] : side_type(A.bd, s, sj), &mx);
    }
    const long long src = cidx(A, si, sj), dst = cidx(A, gi, gj);
    T v[kNPlane];
#pragma unroll
    for (int q = 0; q < kNPlane; ++q) v[q] = buf[src + qoff(A, q)];
    if (mx) {
#pragma unroll
        for (int c = 0; c < 4; ++c) { const T x = v[4 + c]; v[4 + c] = v[8 + c]; v[8 + c] = x; }
#pragma unroll
        for (int k = 0; k < 5; ++k) v[4 * k + 1] = -v[4 * k + 1];
    }
    if (my) {
#pragma unroll
        for (int c = 0; c < 4; ++c) { const T x = v[12 + c]; v[12 + c] = v[16 + c]; v[16 + c] = x; }
#pragma unroll
        for (int k = 0; k < 5; ++k) v[4 * k + 2] = -v[4 * k + 2];
    }
#pragma unroll
    for (int q = 0; q < kNPlane; ++q) buf[dst + qoff(A, q)] = v[q];
}

// ----------------------------------------------------------------- initial state

// Conserved planes of u_0 into buffer 0, with lambda^0 and admissibility.
template <typename T>
__global__ void k_init_load(StepArgs<T> A, const T *__restrict__ rho, const T *__restrict__ mom,
                            const T *__restrict__ E) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    DevCtl *C = A.ctl;
    Monitor<T> m;
    m.init();
    const T gamma = T(A.gamma), gm1 = T(A.gamma - 1.0);
    if (i < A.nx && j < A.ny) {
        const long long k = (long long)j * A.nx + i, N = (long long)A.nx * A.ny;
        T u[4] = {rho[k], mom[k], mom[N + k], E[k]};
        const long long d = cidx(A, i, j);
#pragma unroll
        for (int c = 0; c < 4; ++c) A.buf0[d + qoff(A, c)] = u[c];
        m.add_cell(u, gamma, gm1);
    }
    block_publish(m, C);
    if (last_block(C, gridDim.x * gridDim.y)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            volatile DevCtl *V = C;
            // lambda^0 also covers the prescribed boundary states (as every later lambda^n)
            double lam_bc = 0.0;
            if (A.bd.has_dir) {
                T st[4];
                for (int q = 0; q < 4; ++q) st[q] = (T)A.bd.in[q];
                lam_bc = (double)cell_speed(st, gamma, gm1);
                for (int q = 0; q < 4; ++q) st[q] = (T)A.bd.out[q];
                const double l2 = (double)cell_speed(st, gamma, gm1);
                if (l2 > lam_bc) lam_bc = l2;
            }
            C->lam_bc = lam_bc;
            const double lam_cells = key_to_double(V->lam_key);
            const double lam = lam_bc > lam_cells ? lam_bc : lam_cells;
            const unsigned long long bad = V->bad + V->nonfinite;
            C->invalid_init = bad ? 1 : 0;
            C->lambda = lam;
            C->min_rho = key_to_double(V->minrho_key);
            C->min_rhoe = key_to_double(V->minrhoe_key);
            for (int c = 0; c < 4; ++c) C->sum_last[c] = V->sum[c];
            double a_free = next_speed(C, lam);
            if (!(a_free > 0.0) || !isfinite(a_free)) {
                C->invalid_init = 1;
                a_free = 1.0;
            }
            C->n = 0;
            C->t = 0.0;
            C->a_free = a_free;
            C->done = C->invalid_init;
            C->status = C->invalid_init ? VLBM_E_INVAL : 0;
            plan_next(C, 0.0, a_free);
            reset_slots(C);
            __threadfence();
        }
    }
}

// Populations at equilibrium, u_k^0 = M_k(u_0) (Sec. 4 preamble), with a^0.
template <typename T>
__global__ void k_init_pops(StepArgs<T> A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= A.nx || j >= A.ny) return;
    const StepConsts<T> k = consts_of<T>(A.ctl);
    const long long d = cidx(A, i, j);
    T u[4], f[4], g[4], M1[4], M2[4], M3[4], M4[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) u[c] = A.buf0[d + qoff(A, c)];
    euler_fluxes(u, k.gm1, f, g);
    maxwell_pm(u, f, k, M1, M2);
    maxwell_pm(u, g, k, M3, M4);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        A.buf0[d + qoff(A, (4 + c))] = M1[c];
        A.buf0[d + qoff(A, (8 + c))] = M2[c];
        A.buf0[d + qoff(A, (12 + c))] = M3[c];
        A.buf0[d + qoff(A, (16 + c))] = M4[c];
    }
}

// ----------------------------------------------------------------- outputs

template <typename T>
__global__ void k_moments(StepArgs<T> A, T *rho, T *mom, T *E) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= A.nx || j >= A.ny) return;
    const T *buf = (A.ctl->n & 1) ? A.buf1 : A.buf0;
    const long long d = cidx(A, i, j), k = (long long)j * A.nx + i, N = (long long)A.nx * A.ny;
    if (rho) rho[k] = buf[d + qoff(A, 0)];
    if (mom) {
        mom[k] = buf[d + qoff(A, 1)];
        mom[N + k] = buf[d + qoff(A, 2)];
    }
    if (E) E[k] = buf[d + qoff(A, 3)];
}

// Checkpoint: 64-byte header {n, t, a, dt, a_free, t_end, last|done<<1, status},
// then the 20 planes of the current state, compact.
template <typename T>
__global__ void k_save(StepArgs<T> A, unsigned char *dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const DevCtl *C = A.ctl;
    if (i == 0 && j == 0) {
        double *h = (double *)dst;
        long long *hl = (long long *)dst;
        hl[0] = C->n;
        h[1] = C->t;
        h[2] = C->a;
        h[3] = C->dt;
        h[4] = C->a_free;
        h[5] = C->t_end;
        hl[6] = (long long)C->last | ((long long)C->done << 1);
        hl[7] = (long long)C->status;
    }
    if (i >= A.nx || j >= A.ny) return;
    const T *buf = (C->n & 1) ? A.buf1 : A.buf0;
    T *out = (T *)(dst + 64);
    const long long d = cidx(A, i, j), k = (long long)j * A.nx + i, N = (long long)A.nx * A.ny;
#pragma unroll
    for (int q = 0; q < kNPlane; ++q) out[q * N + k] = buf[d + qoff(A, q)];
}

// Restore: the state goes into buffer (n & 1) of the stored n, so that the
// step sequence (and its ping-pong parity) is exactly the uninterrupted one.
template <typename T>
__global__ void k_load(StepArgs<T> A, const unsigned char *src) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const long long n = ((const long long *)src)[0];
    if (i < A.nx && j < A.ny) {
        T *buf = (n & 1) ? A.buf1 : A.buf0;
        const T *in = (const T *)(src + 64);
        const long long d = cidx(A, i, j), k = (long long)j * A.nx + i, N = (long long)A.nx * A.ny;
#pragma unroll
        for (int q = 0; q < kNPlane; ++q) buf[d + qoff(A, q)] = in[q * N + k];
    }
}

}  // namespace vlbm
