// testing.cu -- the test hooks of include/vlbm_testing.h: the FP32 theta of
// caller-supplied faces, and the arming of the row-marching kernel's wait probe.
#include "common.cuh"
#include "state.h"

#include "../../include/vlbm_testing.h"

using namespace vlbm;
using namespace vlbm::api;

namespace {

// One thread per face: combine_theta<float>, the function the FP32 step kernels call.
__global__ void k_test_theta_faces(long long n, StepConsts<float> k, const float *__restrict__ faces,
                                   float *__restrict__ theta, int *__restrict__ stage) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float *f = faces + 9 * i;
    float us[4], df[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        us[q] = f[q];
        df[q] = f[4 + q];
    }
    unsigned int n64 = 0;
    int st = kStageNone;
    theta[i] = combine_theta(f[8], us, df, k, n64, &st);
    stage[i] = st;
}

__global__ void k_set_wait_probe(DevCtl *C, unsigned int limit_ns) { C->wait_probe_ns = limit_ns; }

}  // namespace

extern "C" {

int vlbm_test_theta_faces(int64_t n, double a, double alpha, double eps, const void *d_faces, void *d_theta,
                          void *d_stage, void *stream) {
    if (n < 0) return fail(nullptr, VLBM_E_INVAL, "n < 0");
    if (n == 0) return VLBM_OK;
    if (!d_faces || !d_theta || !d_stage) return fail(nullptr, VLBM_E_INVAL, "a device pointer is NULL");
    if (!(a > 0.0) || !(alpha >= 0.5 && alpha < 1.0) || !(eps >= 0.0 && eps < 1e-3))
        return fail(nullptr, VLBM_E_INVAL, "need a > 0, 1/2 <= alpha < 1, 0 <= eps < 1e-3");
    const StepConsts<float> k = make_consts<float>(a, alpha, 1.4, eps);
    const int blk = 256;
    const long long grd = (n + blk - 1) / blk;
    if (grd > 0x7fffffffll) return fail(nullptr, VLBM_E_INVAL, "n too large for one launch");
    k_test_theta_faces<<<(unsigned)grd, blk, 0, (cudaStream_t)stream>>>(
        (long long)n, k, (const float *)d_faces, (float *)d_theta, (int *)d_stage);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "theta face launch");
    return VLBM_OK;
}

int vlbm_test_wait_probe(vlbm_state *s, uint32_t limit_ns) {
    if (!s) return fail(nullptr, VLBM_E_INVAL, "state is NULL");
    if (!s->loaded) return fail(s, VLBM_E_INVAL, "no state loaded");
    DeviceGuard g(s->device);
    k_set_wait_probe<<<1, 1, 0, s->stream>>>(s->ctl, limit_ns);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(s, e, "wait probe launch");
    s->probe_armed = limit_ns > 0;
    return VLBM_OK;
}

}  // extern "C"
