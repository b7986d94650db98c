// kernels_impl.cuh -- host launchers for one storage type VLBM_T (included by
// kernels_f32.cu and kernels_f64.cu so that the two precisions compile in parallel).
#include "common.cuh"
#include "step_fused.cuh"
#include "step_simple.cuh"

namespace vlbm {

namespace {
constexpr int kBX = 32, kBY = 8;
inline dim3 cell_grid(int nx, int ny) { return dim3((nx + kBX - 1) / kBX, (ny + kBY - 1) / kBY); }
}  // namespace

template <>
cudaError_t launch_ghosts<VLBM_T>(const StepArgs<VLBM_T> &A, cudaStream_t s) {
    dim3 grd, blk;
    ghosts_launch_shape(A.nx, A.ny, &grd, &blk);
    k_ghosts<VLBM_T><<<grd, blk, 0, s>>>(A);
    return cudaGetLastError();
}

template <>
cudaError_t launch_dirichlet_ghosts<VLBM_T>(const StepArgs<VLBM_T> &A, cudaStream_t s) {
    dim3 grd, blk;
    ghosts_launch_shape(A.nx, A.ny, &grd, &blk);
    k_dirichlet_ghosts<VLBM_T><<<grd, blk, 0, s>>>(A);
    return cudaGetLastError();
}

template <>
const void *dirichlet_ghosts_kernel_fn<VLBM_T>() {
    return (const void *)k_dirichlet_ghosts<VLBM_T>;
}

template <>
cudaError_t launch_init<VLBM_T>(const StepArgs<VLBM_T> &A, const VLBM_T *rho, const VLBM_T *mom,
                                const VLBM_T *E, cudaStream_t s) {
    const dim3 blk(kBX, kBY), grd = cell_grid(A.nx, A.ny);
    k_init_load<VLBM_T><<<grd, blk, 0, s>>>(A, rho, mom, E);
    k_init_pops<VLBM_T><<<grd, blk, 0, s>>>(A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_ghosts<VLBM_T>(A, s);
}

template <>
cudaError_t launch_step_simple<VLBM_T>(const StepArgs<VLBM_T> &A, cudaStream_t s) {
    dim3 grd, blk;
    simple_launch_shape(A.nx, A.ny, &grd, &blk);
    switch (A.limiter) {
        case VLBM_LIM_FIRST_ORDER: k_step_simple<VLBM_T, VLBM_LIM_FIRST_ORDER><<<grd, blk, 0, s>>>(A); break;
        case VLBM_LIM_NONE: k_step_simple<VLBM_T, VLBM_LIM_NONE><<<grd, blk, 0, s>>>(A); break;
        case VLBM_LIM_PP: k_step_simple<VLBM_T, VLBM_LIM_PP><<<grd, blk, 0, s>>>(A); break;
        case VLBM_LIM_LMP: k_step_simple<VLBM_T, VLBM_LIM_LMP><<<grd, blk, 0, s>>>(A); break;
        case VLBM_LIM_RLMP: k_step_simple<VLBM_T, VLBM_LIM_RLMP><<<grd, blk, 0, s>>>(A); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <>
const void *simple_kernel_fn<VLBM_T>(int limiter) {
    switch (limiter) {
        case VLBM_LIM_FIRST_ORDER: return (const void *)k_step_simple<VLBM_T, VLBM_LIM_FIRST_ORDER>;
        case VLBM_LIM_NONE: return (const void *)k_step_simple<VLBM_T, VLBM_LIM_NONE>;
        case VLBM_LIM_PP: return (const void *)k_step_simple<VLBM_T, VLBM_LIM_PP>;
        case VLBM_LIM_LMP: return (const void *)k_step_simple<VLBM_T, VLBM_LIM_LMP>;
        default: return (const void *)k_step_simple<VLBM_T, VLBM_LIM_RLMP>;
    }
}

namespace {
template <int LIM, bool PROBE = false>
cudaError_t fused_one(const FusedBatchArgs<VLBM_T> &B, int grid, cudaStream_t s) {
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    const size_t smem = sizeof(FusedSmem<VLBM_T, fused_lag(LIM)>);
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_step_fused<VLBM_T, LIM, PROBE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    k_step_fused<VLBM_T, LIM, PROBE><<<grid, kFB, smem, s>>>(B);
    return cudaGetLastError();
}

template <int LIM>
int fused_blocks_per_sm() {
    int nb = 0;
    const size_t smem = sizeof(FusedSmem<VLBM_T, fused_lag(LIM)>);
    cudaFuncSetAttribute(k_step_fused<VLBM_T, LIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_fused<VLBM_T, LIM>, kFB, smem) != cudaSuccess)
        nb = 1;
    return nb > 0 ? nb : 1;
}
}  // namespace

template <>
int fused_occupancy<VLBM_T>(int limiter) {
    switch (limiter) {
        case VLBM_LIM_FIRST_ORDER: return fused_blocks_per_sm<VLBM_LIM_FIRST_ORDER>();
        case VLBM_LIM_NONE: return fused_blocks_per_sm<VLBM_LIM_NONE>();
        case VLBM_LIM_PP: return fused_blocks_per_sm<VLBM_LIM_PP>();
        case VLBM_LIM_LMP: return fused_blocks_per_sm<VLBM_LIM_LMP>();
        default: return fused_blocks_per_sm<VLBM_LIM_RLMP>();
    }
}

template <>
const void *fused_kernel_fn<VLBM_T>(int limiter, size_t *smem) {
    *smem = fused_lag(limiter) == 2 ? sizeof(FusedSmem<VLBM_T, 2>) : sizeof(FusedSmem<VLBM_T, 1>);
    fused_blocks_per_sm<VLBM_LIM_PP>();   // sets the dynamic shared memory attributes
    switch (limiter) {
        case VLBM_LIM_FIRST_ORDER: fused_blocks_per_sm<VLBM_LIM_FIRST_ORDER>(); return (const void *)k_step_fused<VLBM_T, VLBM_LIM_FIRST_ORDER>;
        case VLBM_LIM_NONE: fused_blocks_per_sm<VLBM_LIM_NONE>(); return (const void *)k_step_fused<VLBM_T, VLBM_LIM_NONE>;
        case VLBM_LIM_PP: return (const void *)k_step_fused<VLBM_T, VLBM_LIM_PP>;
        case VLBM_LIM_LMP: fused_blocks_per_sm<VLBM_LIM_LMP>(); return (const void *)k_step_fused<VLBM_T, VLBM_LIM_LMP>;
        default: fused_blocks_per_sm<VLBM_LIM_RLMP>(); return (const void *)k_step_fused<VLBM_T, VLBM_LIM_RLMP>;
    }
}

template <>
cudaError_t launch_step_fused_probe<VLBM_T>(const FusedBatchArgs<VLBM_T> &B, int limiter, int grid,
                                            cudaStream_t s) {
    switch (limiter) {
        case VLBM_LIM_FIRST_ORDER: return fused_one<VLBM_LIM_FIRST_ORDER, true>(B, grid, s);
        case VLBM_LIM_NONE: return fused_one<VLBM_LIM_NONE, true>(B, grid, s);
        case VLBM_LIM_PP: return fused_one<VLBM_LIM_PP, true>(B, grid, s);
        case VLBM_LIM_LMP: return fused_one<VLBM_LIM_LMP, true>(B, grid, s);
        case VLBM_LIM_RLMP: return fused_one<VLBM_LIM_RLMP, true>(B, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_step_fused<VLBM_T>(const FusedBatchArgs<VLBM_T> &B, int limiter, int grid,
                                      cudaStream_t s) {
    switch (limiter) {
        case VLBM_LIM_FIRST_ORDER: return fused_one<VLBM_LIM_FIRST_ORDER>(B, grid, s);
        case VLBM_LIM_NONE: return fused_one<VLBM_LIM_NONE>(B, grid, s);
        case VLBM_LIM_PP: return fused_one<VLBM_LIM_PP>(B, grid, s);
        case VLBM_LIM_LMP: return fused_one<VLBM_LIM_LMP>(B, grid, s);
        case VLBM_LIM_RLMP: return fused_one<VLBM_LIM_RLMP>(B, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_moments<VLBM_T>(const StepArgs<VLBM_T> &A, VLBM_T *rho, VLBM_T *mom, VLBM_T *E,
                                   cudaStream_t s) {
    k_moments<VLBM_T><<<cell_grid(A.nx, A.ny), dim3(kBX, kBY), 0, s>>>(A, rho, mom, E);
    return cudaGetLastError();
}

template <>
cudaError_t launch_save<VLBM_T>(const StepArgs<VLBM_T> &A, void *dst, cudaStream_t s) {
    k_save<VLBM_T><<<cell_grid(A.nx, A.ny), dim3(kBX, kBY), 0, s>>>(A, (unsigned char *)dst);
    return cudaGetLastError();
}

template <>
cudaError_t launch_load<VLBM_T>(const StepArgs<VLBM_T> &A, const void *src, cudaStream_t s) {
    cudaError_t e0 = launch_load_header(A.ctl, src, s);
    if (e0 != cudaSuccess) return e0;
    k_load<VLBM_T><<<cell_grid(A.nx, A.ny), dim3(kBX, kBY), 0, s>>>(A, (const unsigned char *)src);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_ghosts<VLBM_T>(A, s);
}

}  // namespace vlbm
