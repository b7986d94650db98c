// vlbm_internal.h -- device-side data layout and launch interfaces shared by the
// translation units of libvlbm (not part of the public ABI; see include/vlbm.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#include "../../include/vlbm.h"

namespace vlbm {

// State buffer layout: padded rows, each holding the five groups of four values of
// its cells -- the conserved u, then the populations u_1..u_4 (u_5 is never stored),
// each group's four components (rho, m1, m2, E) contiguous -- group after group:
//   value q of cell (i, j), -2 <= i < nx+2, -2 <= j < ny+2, lives at
//   (((j + kOY) * kNGroup + q / 4) * pitch + (i + kOX)) * 4 + q % 4.
// A cell's group is one 16-byte (FP32) or 32-byte (FP64) vector, so a warp moves 32
// consecutive cells' group as one contiguous, sector-aligned 512 (1024) bytes, and a
// thread loads or stores a whole group with one vector access. Padded columns 0, 1
// and nx+2, nx+3 hold the two ghost layers of the x sides, rows 0, 1 and ny+2, ny+3
// those of the y sides; pitch (cells) is a multiple of 8.
constexpr int kOX = 2;
constexpr int kOY = 2;
constexpr int kNPlane = 20;   // u (4) and u_1..u_4 (4 each); u_5 is never stored
constexpr int kNGroup = 5;    // groups of four values per cell

__host__ __device__ __forceinline__ long long sidx(int pitch, int q, int i, int j) {
    return (((long long)(j + kOY) * kNGroup + (q >> 2)) * pitch + (i + kOX)) * 4 + (q & 3);
}

struct Layout {
    int nx, ny;
    int pitch;          // cells per padded row of one group (nx + 2 kOX, a multiple of 8)
    int rows;           // ny + 4
    int elem;           // bytes per element (4 or 8)
    size_t buf_bytes;   // bytes of one 20-value state buffer
    size_t ctl_offset;  // byte offset of the control block in the workspace
    size_t desc_offset; // byte offset of the row-marching kernel's descriptor block
    size_t total;       // workspace bytes
};

Layout make_layout(int nx, int ny, int elem);

// Order-preserving key of a double for atomicMin/atomicMax on unsigned 64-bit
// integers (NaN with the sign bit clear sorts above +inf).
__host__ __device__ inline unsigned long long ordered_key(double x) {
#ifdef __CUDA_ARCH__
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
#else
    unsigned long long b;
    memcpy(&b, &x, sizeof b);
#endif
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__host__ __device__ inline double key_to_double(unsigned long long k) {
    unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double x;
    memcpy(&x, &b, sizeof x);
    return x;
#endif
}

// Constants of one step, derived from the kinetic speed a^n (Sec. 2 and Sec. 3.2).
template <typename T>
struct StepConsts {
    T a, two_a, inv2a;        // a, 2a, 1/(2a)
    T kappa, two_kappa, inv2k;  // kappa = a (1 - alpha) / 2, 2 kappa, 1/(2 kappa)
    T w, alpha;               // (1 - alpha)/4 and alpha
    T gamma, gm1;             // gamma, gamma - 1
    T eps;                    // epsilon of the PP and pressure bounds
    float eps_margin;         // 2 eps as float, the FP32 screen's allowance for epsilon
    float T1;                 // FP32 screen: an upper bound of (1 + 2 eps) / kappa, raised by 64 u
    float inv_kappa;          // 1 / kappa
    double kappa64, eps64;    // FP64 copies for the internal-energy solve
};

// Device control block: time-step state written by the last CTA of each step
// (the grid-wide lambda^n dependency of Sec. 4 is resolved at the kernel
// boundary), the per-step reduction slots, and the published monitors.
struct DevCtl {
    // step state
    long long n;           // steps taken; the current state is buffer n & 1
    double t;              // simulated time
    double a;              // kinetic speed of the next step
    double dt;             // time step of the next step
    double a_free;         // kinetic speed before any shortening to reach t_end
    double t_end;          // > 0: stop at this time (last step clipped)
    int last;              // the next step is the clipped final one
    int done;              // no further step may run
    int status;            // sticky VLBM_E_* (0 = OK)
    int invalid_init;      // cells of u_0 outside G at the last initialisation
    long long first_bad_step;
    // reduction slots of the step in flight (reset by the finaliser)
    unsigned long long lam_key;      // ordered key of max lambda
    unsigned long long minrho_key;   // ordered key of min rho
    unsigned long long minrhoe_key;  // ordered key of min internal energy E - |m|^2 / (2 rho)
    unsigned long long bad;          // cells outside G
    unsigned long long nonfinite;    // non-finite cells
    unsigned long long fp64_faces;   // faces whose theta_p needed the FP64 solve
    double sum[4];
    unsigned int blocks_done;
    unsigned int wait_probe_ns;  // testing hook (vlbm_test_wait_probe): how long every CTA of the probe
                                 // instantiation of the row-marching kernel waits on a barrier nothing completes
    // published monitors of the current state
    double lambda;
    double min_rho;
    double min_rhoe;       // min internal energy per volume of the current state
    long long bad_last;
    long long nonfinite_last;
    long long fp64_last;
    double sum_last[4];
    // constants
    double dx, alpha, a_fixed, eps, gamma;
    double lam_bc;         // cell speed of the prescribed boundary states (0: none), in lambda^n
    // the next step's constants (derived from a), set whenever a is
    StepConsts<float> kf;
    StepConsts<double> kd;
};

static_assert(sizeof(DevCtl) == 480, "bench.py reads the control block size");

// Boundary beyond one uniform rule per side (vlbm_boundary): side s switches from
// type lo[s] to hi[s] at index split[s] along it (0: uniform), and the prescribed
// field of the VLBM_BC_DIRICHLET parts. Built on the host, read by the kernels on
// their rare boundary paths only.
struct Bound {
    int lo[4], hi[4], split[4];
    int has_dir;                       // some part of a side is VLBM_BC_DIRICHLET
    int nplanes;
    double x0, y0, dx;
    double pnx[2], pny[2], c0[2], c1[2];
    double in[4], out[4];              // conserved states of the field
    const DevCtl *ctl;                 // the grid's control block (the field reads t)
};

// Type of side s at index k along it (column for south / north, row for west / east).
__host__ __device__ inline int side_type(const Bound &B, int s, int k) {
    return k < B.split[s] ? B.lo[s] : B.hi[s];
}

// Validate grid.bc with the optional vlbm_boundary and build the Bound of a grid
// (ctl left NULL). Returns NULL, or a static message naming what is wrong.
const char *make_bound(const vlbm_grid &g, const vlbm_boundary *b, Bound *out);

// The uniform type of each side, -1 where the side switches type: what the hot
// paths test (zero-gradient sides for the sponge, the ghost images' fast path).
inline void uniform_types(const Bound &B, int bc[4]) {
    for (int s = 0; s < 4; ++s) bc[s] = B.split[s] == 0 ? B.lo[s] : -1;
}

// One grid as the row-marching kernel sees it (device memory, 64-byte aligned).
template <typename T>
struct alignas(256) InstDesc {
    CUtensorMap tmap;     // 4D view [2 buffers][ny + 4 rows][5 groups][4 pitch] of both state buffers
    T *buf0, *buf1;
    int pitch, nx, ny;
    int bc[4];
    int nitems;           // this grid's work items in the launch
    DevCtl *ctl;
    int sponge;           // width of the theta = 0 layer at zero-gradient sides (Sec. 4.2)
    Bound bd;             // split sides and the prescribed field
};

static_assert(offsetof(InstDesc<float>, tmap) == 0 && offsetof(InstDesc<double>, tmap) == 0,
              "the row-marching kernel finds the descriptor from its tensor map");

// A sponge width fits a grid when it is >= 0 and at most half the cells along every
// axis that has a zero-gradient side (the layer exists only next to such sides).
inline bool sponge_ok(int w, const vlbm_grid &g) {
    if (w < 0) return false;
    const bool tx = g.bc[0] == VLBM_BC_TRANSMISSIVE || g.bc[1] == VLBM_BC_TRANSMISSIVE;
    const bool ty = g.bc[2] == VLBM_BC_TRANSMISSIVE || g.bc[3] == VLBM_BC_TRANSMISSIVE;
    return !(tx && 2 * w > g.nx) && !(ty && 2 * w > g.ny);
}

// Sponge layer of Sec. 4.2: theta = 0 on every face of a cell that lies within
// `w` cells of a zero-gradient side (ghost cells included); w = 0 disables it.
struct Sponge {
    int w, nx, ny;
    bool tw, te, ts, tn;   // west, east, south, north side is zero-gradient
    __host__ __device__ Sponge(int w_, int nx_, int ny_, const int bc[4])
        : w(w_), nx(nx_), ny(ny_), tw(bc[0] == VLBM_BC_TRANSMISSIVE), te(bc[1] == VLBM_BC_TRANSMISSIVE),
          ts(bc[2] == VLBM_BC_TRANSMISSIVE), tn(bc[3] == VLBM_BC_TRANSMISSIVE) {}
    __host__ __device__ bool cell(int i, int j) const {
        return (tw && i < w) || (te && i >= nx - w) || (ts && j < w) || (tn && j >= ny - w);
    }
};

// Work counter of one row-marching launch; reset by the last CTA to leave.
struct BatchCtl {
    unsigned int work, ctas_done;
};

// One work item of the row-marching kernel: rows [y0, y1) of the strip of output
// columns [x0, x0 + w) of grid `inst` (xw = x0 | w << 24; w <= kFusedOut).
struct alignas(16) WorkItem {
    int inst, xw, y0, y1;
};

template <typename T>
struct FusedBatchArgs {
    const InstDesc<T> *insts;
    const WorkItem *items;  // in the order the CTAs take them
    int nitems;
    BatchCtl *bctl;
    double gamma, alpha, eps;
};

template <typename T>
struct StepArgs {
    T *buf0, *buf1;     // the two state buffers
    int pitch;          // cells per padded row of one group
    int nx, ny;
    int bc[4];          // west, east, south, north: the uniform type, -1 where a side switches
    int limiter;
    double gamma;
    double alpha;
    double eps;
    DevCtl *ctl;
    int sponge;         // width of the theta = 0 layer at zero-gradient sides (Sec. 4.2)
    Bound bd;           // split sides and the prescribed field
};

// Host launchers (stream-ordered; return cudaError_t of the launch).
cudaError_t launch_ctl_reset(DevCtl *ctl, double dx, double alpha, double a_fixed, double eps,
                             double gamma, cudaStream_t s);
template <typename T> cudaError_t launch_init(const StepArgs<T> &a, const T *rho, const T *mom,
                                              const T *E, cudaStream_t s);
template <typename T> cudaError_t launch_ghosts(const StepArgs<T> &a, cudaStream_t s);
// The prescribed (Dirichlet) ghosts alone, before a row-marching step (shape as the ghost pass).
template <typename T> cudaError_t launch_dirichlet_ghosts(const StepArgs<T> &a, cudaStream_t s);
template <typename T> const void *dirichlet_ghosts_kernel_fn();
template <typename T> cudaError_t launch_step_simple(const StepArgs<T> &a, cudaStream_t s);
// Row-marching kernel over the work items of one or more grids, `grid` persistent CTAs.
template <typename T> cudaError_t launch_step_fused(const FusedBatchArgs<T> &a, int limiter, int grid,
                                                   cudaStream_t s);
// The instantiation with the wait probe of vlbm_test_wait_probe (same launch shape).
template <typename T> cudaError_t launch_step_fused_probe(const FusedBatchArgs<T> &a, int limiter, int grid,
                                                         cudaStream_t s);
template <typename T> int fused_occupancy(int limiter);   // CTAs per SM of the fused kernel
// Kernel function and dynamic shared memory of the fused kernel, for graph nodes.
template <typename T> const void *fused_kernel_fn(int limiter, size_t *smem);
// Kernel functions and launch shapes of the one-thread-per-cell step and of the
// ghost-frame passes (for CUDA graph kernel nodes).
template <typename T> const void *simple_kernel_fn(int limiter);
void simple_launch_shape(int nx, int ny, dim3 *grid, dim3 *block);
void ghosts_launch_shape(int nx, int ny, dim3 *grid, dim3 *block);
bool encode_state_tmap(CUtensorMap *out, void *base, const Layout &L);
constexpr int kFusedBox = 128;                             // TMA box width (columns) = threads per CTA
constexpr int kFusedHalo = 2;                              // box columns on either side of a strip
constexpr int kFusedOut = kFusedBox - 2 * kFusedHalo;      // most output columns of a strip (124)
constexpr int kFusedMinChunk = 4;                          // rows per work item, bounds
constexpr int kFusedMaxChunk = 128;

// Strips of a grid of nx columns: as few as hold kFusedOut columns each, of even widths
// as equal as possible (the last takes an odd remainder), so that every strip starts on
// an even column (a 32-byte sector of FP32 groups) and no strip is nearly empty.
inline int strip_count(int nx) { return (nx + kFusedOut - 1) / kFusedOut; }
inline void strip_of(int nx, int s, int *x0, int *w) {
    const int ns = strip_count(nx), pairs = nx / 2, base = pairs / ns, extra = pairs % ns;
    *x0 = 2 * (s * base + (s < extra ? s : extra));
    *w = s == ns - 1 ? nx - *x0 : 2 * (base + (s < extra ? 1 : 0));
}

// Work items of one grid appended to `out`, strip-fastest within each band of
// rows. Uniform order: bands of `hmax` rows. Guided order (guided self-scheduling,
// Polychronopoulos & Kuck 1987): each band is as high as the work left -- strip-rows
// of this grid and of the grids after it, `work_left`, which the call decreases --
// divided by the CTA count (rounded up), within [kFusedMinChunk, hmax]: the first
// items are tall (few repeated halo rows), the last ones short (a CTA taking one
// near the end of the step finishes soon after the others), and a grid too small to
// give every CTA a tall band is cut into about one band per CTA. Measured on the
// 4096^2 blast (3 CTAs x 152 SMs): 6.6 % faster than the best uniform height; work
// left / (2 x CTAs) was within 2.5 % of it; a minimum height of 4 rows instead of
// 16 gains 0.7 % there and 1.8 x on a 256^2 grid (one wave of short bands instead
// of a few CTAs marching 16 rows each).
inline int append_items(WorkItem *out, int inst, int nx, int ny, int hmax, bool guided,
                        long long &work_left, long long ctas) {
    const int strips = strip_count(nx);
    int n = 0;
    for (int y = 0; y < ny;) {
        long long h = hmax;
        if (guided) {
            const long long c = ctas > 0 ? ctas : 1;
            h = (work_left + c - 1) / c;
            if (h < kFusedMinChunk) h = kFusedMinChunk;
            if (h > hmax) h = hmax;
        }
        if (h > ny - y) h = ny - y;
        for (int s = 0; s < strips; ++s) {
            int x0, w;
            strip_of(nx, s, &x0, &w);
            if (out) out[n] = WorkItem{inst, x0 | (w << 24), y, y + (int)h};
            ++n;
        }
        work_left -= (long long)strips * h;
        y += (int)h;
    }
    return n;
}
// Upper bound of append_items' count for any order with hmax >= kFusedMinChunk.
inline size_t max_items(int nx, int ny) {
    const size_t strips = strip_count(nx);
    return strips * ((ny + kFusedMinChunk - 1) / kFusedMinChunk + 1);
}
template <typename T> cudaError_t launch_moments(const StepArgs<T> &a, T *rho, T *mom, T *E,
                                                 cudaStream_t s);
template <typename T> cudaError_t launch_save(const StepArgs<T> &a, void *dst, cudaStream_t s);
template <typename T> cudaError_t launch_load(const StepArgs<T> &a, const void *src, cudaStream_t s);
cudaError_t launch_set_tend(DevCtl *ctl, double t_end, cudaStream_t s);
cudaError_t launch_load_header(DevCtl *ctl, const void *src, cudaStream_t s);

}  // namespace vlbm
