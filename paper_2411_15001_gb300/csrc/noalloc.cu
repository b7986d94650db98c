// noalloc.cu -- vlbm_step_noalloc: one time step that needs no workspace.
//
// For callers that cannot allocate device memory at all: a plugin inside a host
// application whose memory pool already owns the whole device, a real-time loop
// that may not take the implicit device synchronisation of cudaMalloc, a
// sandbox whose allocator is closed to it. They already hold the state they
// step (20 compact planes in, 20 compact planes out); the only scratch the step
// needs -- one reduction record per CTA for the monitors and the next kinetic
// speed -- lives in a file-scope __device__ array of fixed size that every GPU
// loading this library keeps until the process exits.
//
// The kernel is the one-thread-per-cell step (cell_step of step_simple.cuh),
// reading the compact input through a loader that applies the boundary rules
// on the fly instead of a ghost frame. A second one-CTA kernel reduces the
// per-CTA records in a fixed order.
#include <mutex>

#include "common.cuh"
#include "step_simple.cuh"

namespace vlbm {

namespace {

constexpr int kNaBX = 32, kNaBY = 8;          // 256 threads, one cell each
constexpr int kNoAllocMaxBlocks = 8192;       // reduction records in the scratch array

struct NoAllocPartial {
    double lam, minrho;
    double sum[4];
    unsigned int bad, nonfin, fp64, pad;
};

struct NoAllocResult {
    double lam, minrho;
    double sum[4];
    long long bad, nonfin, fp64;
};

constexpr size_t kNoAllocScratchBytes =
    ((kNoAllocMaxBlocks * sizeof(NoAllocPartial) + sizeof(NoAllocResult) + 255) / 256) * 256;

// The scratch: per-CTA records, then the reduced result. Every call overwrites
// what it reads, so nothing has to start at zero.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Compact 20-plane input (plane q at q * nx * ny, cell (i, j) at j * nx + i);
// ghost cells are mapped to their source cell with the side's boundary rule,
// exactly as the ghost frame of the workspace path holds them.
template <typename T>
struct CompactLoad {
    const T *__restrict__ in;
    int nx, ny;
    int bc[4];
    long long N;
    __device__ __forceinline__ T v(int q, int i, int j) const {
        bool mx, my;
        const int si = ghost_source(i, nx, bc[0], bc[1], &mx);
        const int sj = ghost_source(j, ny, bc[2], bc[3], &my);
        int qq = q;
        if (mx && q >= 4 && q < 12) qq = q < 8 ? q + 4 : q - 4;      // u_1 <-> u_2
        if (my && q >= 12) qq = q < 16 ? q + 4 : q - 4;              // u_3 <-> u_4
        T val = in[qq * N + (long long)sj * nx + si];
        const int comp = q & 3;
        if ((mx && comp == 1) || (my && comp == 2)) val = -val;      // normal momentum
        return val;
    }
    __device__ __forceinline__ void u4(int q0, int i, int j, T out[4]) const {
#pragma unroll
        for (int c = 0; c < 4; ++c) out[c] = v(q0 + c, i, j);
    }
};

template <typename T, int LIM>
__global__ void __launch_bounds__(kNaBX *kNaBY)
    k_step_noalloc(CompactLoad<T> L, T *__restrict__ out, const StepConsts<T> k, int sponge,
                   NoAllocPartial *part) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    Monitor<T> mon;
    mon.init();
    if (i < L.nx && j < L.ny) {
        T nv[kNPlane];
        cell_step<T, LIM>(L, i, j, k, Sponge(sponge, L.nx, L.ny, L.bc), nv, mon.fp64);
        const long long d = (long long)j * L.nx + i;
#pragma unroll
        for (int q = 0; q < kNPlane; ++q) out[q * L.N + d] = nv[q];
        mon.add_cell(nv, k.gamma, k.gm1);
    }
    __shared__ Monitor<T> sh[kNaBX * kNaBY / 32];
    const int tid = threadIdx.x + blockDim.x * threadIdx.y, lane = tid & 31, warp = tid >> 5;
    mon.warp_reduce();
    if (lane == 0) sh[warp] = mon;
    __syncthreads();
    if (warp == 0) {
        if (lane < kNaBX * kNaBY / 32) mon = sh[lane];
        else mon.init();
        mon.warp_reduce();
        if (lane == 0) {
            NoAllocPartial &p = part[blockIdx.x + gridDim.x * blockIdx.y];
            p.lam = (double)mon.lam;
            p.minrho = (double)mon.minrho;
            for (int c = 0; c < 4; ++c) p.sum[c] = mon.sum.value(c);
            p.bad = mon.bad;
            p.nonfin = mon.nonfin;
            p.fp64 = mon.fp64;
        }
    }
}

// One CTA: fixed-order reduction of the per-CTA records (the same result on
// every run).
__global__ void k_noalloc_reduce(const NoAllocPartial *part, int n, NoAllocResult *res) {
    __shared__ NoAllocResult sh[256];
    NoAllocResult r;
    r.lam = 0.0;
    r.minrho = INFINITY;
    for (int c = 0; c < 4; ++c) r.sum[c] = 0.0;
    r.bad = r.nonfin = r.fp64 = 0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
        const NoAllocPartial &p = part[b];
        r.lam = pmax(r.lam, p.lam);
        r.minrho = pmin(r.minrho, p.minrho);
        for (int c = 0; c < 4; ++c) r.sum[c] += p.sum[c];
        r.bad += p.bad;
        r.nonfin += p.nonfin;
        r.fp64 += p.fp64;
    }
    sh[threadIdx.x] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int t = 1; t < (int)blockDim.x; ++t) {
            const NoAllocResult &o = sh[t];
            r.lam = pmax(r.lam, o.lam);
            r.minrho = pmin(r.minrho, o.minrho);
            for (int c = 0; c < 4; ++c) r.sum[c] += o.sum[c];
            r.bad += o.bad;
            r.nonfin += o.nonfin;
            r.fp64 += o.fp64;
        }
        *res = r;
    }
}

template <typename T>
cudaError_t launch_noalloc(const vlbm_grid *g, int limiter, const void *in, void *out, double a,
                           double alpha, double gamma, double eps, int sponge, unsigned char *scratch,
                           cudaStream_t s) {
    CompactLoad<T> L;
    L.in = (const T *)in;
    L.nx = g->nx;
    L.ny = g->ny;
    for (int q = 0; q < 4; ++q) L.bc[q] = g->bc[q];
    L.N = (long long)g->nx * g->ny;
    const dim3 blk(kNaBX, kNaBY), grd((g->nx + kNaBX - 1) / kNaBX, (g->ny + kNaBY - 1) / kNaBY);
    NoAllocPartial *part = (NoAllocPartial *)scratch;
    NoAllocResult *res = (NoAllocResult *)(scratch + kNoAllocMaxBlocks * sizeof(NoAllocPartial));
    T *o = (T *)out;
    const StepConsts<T> k = make_consts<T>(a, alpha, gamma, eps);
    switch (limiter) {
        case VLBM_LIM_FIRST_ORDER: k_step_noalloc<T, VLBM_LIM_FIRST_ORDER><<<grd, blk, 0, s>>>(L, o, k, sponge, part); break;
        case VLBM_LIM_NONE: k_step_noalloc<T, VLBM_LIM_NONE><<<grd, blk, 0, s>>>(L, o, k, sponge, part); break;
        case VLBM_LIM_PP: k_step_noalloc<T, VLBM_LIM_PP><<<grd, blk, 0, s>>>(L, o, k, sponge, part); break;
        case VLBM_LIM_LMP: k_step_noalloc<T, VLBM_LIM_LMP><<<grd, blk, 0, s>>>(L, o, k, sponge, part); break;
        default: k_step_noalloc<T, VLBM_LIM_RLMP><<<grd, blk, 0, s>>>(L, o, k, sponge, part); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_noalloc_reduce<<<1, 256, 0, s>>>(part, (int)(grd.x * grd.y), res);
    return cudaGetLastError();
}

// Device address of the scratch array, looked up once per device with that
// device current (the host-side symbol is only a stand-in, not a device address).
std::mutex g_scratch_mutex;
unsigned char *g_scratch_ptr[64];

cudaError_t scratch_for_device(int dev, unsigned char **out) {
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (unsigned char *)p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

}  // namespace vlbm

using namespace vlbm;

extern "C" int vlbm_step_noalloc(const vlbm_grid *grid, double gamma, double a, int32_t limiter,
                                 int32_t precision, const vlbm_opts *opts, const void *d_in, void *d_out,
                                 vlbm_step_result *result, void *stream) {
    if (!grid || grid->nx < 4 || grid->ny < 4 || !(grid->dx > 0.0)) return VLBM_E_INVAL;
    // a prescribed field needs the time, which this call does not keep
    if (opts && opts->boundary) return VLBM_E_UNSUPPORTED;
    for (int q = 0; q < 4; ++q) {
        if (grid->bc[q] == VLBM_BC_DIRICHLET) return VLBM_E_UNSUPPORTED;
        if (grid->bc[q] < VLBM_BC_PERIODIC || grid->bc[q] > VLBM_BC_REFLECTIVE) return VLBM_E_INVAL;
    }
    if ((grid->bc[0] == VLBM_BC_PERIODIC) != (grid->bc[1] == VLBM_BC_PERIODIC) ||
        (grid->bc[2] == VLBM_BC_PERIODIC) != (grid->bc[3] == VLBM_BC_PERIODIC))
        return VLBM_E_INVAL;
    if (!(gamma > 1.0) || !(a > 0.0) || !(a < 1e300)) return VLBM_E_INVAL;
    if (limiter < VLBM_LIM_FIRST_ORDER || limiter > VLBM_LIM_RLMP) return VLBM_E_INVAL;
    if (precision != VLBM_FP32 && precision != VLBM_FP64) return VLBM_E_INVAL;
    double alpha = 0.5, eps = 1e-16;
    int sponge = 0;
    if (opts) {
        alpha = opts->alpha;
        eps = opts->eps;
        sponge = opts->sponge;
    }
    if (!(alpha >= 0.5 && alpha < 1.0) || !(eps >= 0.0 && eps < 1e-3)) return VLBM_E_INVAL;
    if (!sponge_ok(sponge, *grid)) return VLBM_E_INVAL;
    if (!d_in || !d_out || d_in == d_out || !result) return VLBM_E_INVAL;
    const long long blocks =
        (long long)((grid->nx + kNaBX - 1) / kNaBX) * ((grid->ny + kNaBY - 1) / kNaBY);
    if (blocks > kNoAllocMaxBlocks) return VLBM_E_INVAL;   // > 8192 CTAs of 32 x 8 cells
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return VLBM_E_CUDA;
    }
    unsigned char *scratch = nullptr;
    cudaError_t e = scratch_for_device(dev, &scratch);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return VLBM_E_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    e = precision == VLBM_FP64
            ? launch_noalloc<double>(grid, limiter, d_in, d_out, a, alpha, gamma, eps, sponge, scratch, s)
            : launch_noalloc<float>(grid, limiter, d_in, d_out, a, alpha, gamma, eps, sponge, scratch, s);
    if (e != cudaSuccess) return VLBM_E_CUDA;
    NoAllocResult r;
    e = cudaMemcpyAsync(&r, scratch + kNoAllocMaxBlocks * sizeof(NoAllocPartial), sizeof r,
                        cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return VLBM_E_CUDA;
    result->lambda = r.lam;
    result->a_next = 2.0 * r.lam / (1.0 - alpha);
    result->min_rho = r.minrho;
    for (int c = 0; c < 4; ++c) result->sum[c] = r.sum[c];
    result->bad_cells = r.bad;
    result->nonfinite_cells = r.nonfin;
    result->theta_p_fp64_faces = r.fp64;
    if (r.bad) return VLBM_E_POSITIVITY;   // cells outside G (their lambda is NaN)
    if (r.nonfin || !(r.lam <= 1e300)) return VLBM_E_NONFINITE;
    return VLBM_OK;
}
