/*
 * vlbm_testing.h -- test hooks of libvlbm (include/vlbm.h): entry points that run
 * one stage of the step kernels on inputs the caller chooses, or make a bounded
 * device wait run out on purpose, so that tests can check those parts directly.
 * None of them is needed to run the scheme. Return codes, device pointers and
 * streams follow the conventions of vlbm.h; the hooks allocate nothing.
 */
#ifndef VLBM_TESTING_H
#define VLBM_TESTING_H

#include "vlbm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Stages of the FP32 theta of a face (the d_stage output below). */
#define VLBM_THETA_STAGE_NONE 0      /* min(1, theta_rho) <= 0: theta_p not evaluated */
#define VLBM_THETA_STAGE_SCREEN 1    /* the float endpoint screen proved theta_p >= min(1, theta_rho) */
#define VLBM_THETA_STAGE_INTERVAL 2  /* a tight float interval of the spectral radius */
#define VLBM_THETA_STAGE_FP64 3      /* the double-precision interval stage */

/* theta = min(1, theta_rho, theta_p) of n faces, computed by the same device
 * function as the FP32 step kernels (Sec. 3.2; theta_p of Sec. 3.4, eq. GQL: the
 * closed-form spectral radius varrho of B^-1/2 A B^-1/2, theta_p = max(0, kappa /
 * varrho - eps)), for the step constants of kinetic speed a (kappa = a (1 - alpha)
 * / 2) and epsilon eps, as the end-of-step finaliser would form them.
 *   d_faces: device array of n records of 9 floats: u* (rho, m1, m2, E), dF (rho,
 *     m1, m2, E) of the face, then theta_rho (the density bound; 1 for PP in FP32,
 *     whose density bound theta_p carries).
 *   d_theta (out): n floats; d_stage (out): n int32 VLBM_THETA_STAGE_* codes.
 * Enqueued on `stream` (a cudaStream_t) on the current device; asynchronous.
 * Errors: VLBM_E_INVAL (n < 0, a NULL pointer, a <= 0, alpha outside [1/2, 1),
 * eps outside [0, 1e-3)), VLBM_E_CUDA (launch). */
VLBM_API int vlbm_test_theta_faces(int64_t n, double a, double alpha, double eps, const void *d_faces,
                                   void *d_theta, void *d_stage, void *stream);

/* Arm the wait probe of the row-marching kernel for the state's next steps: while it
 * is armed, vlbm_step and vlbm_step_to launch the kernel's probe instantiation (the
 * same source with one addition, and one launch per step, no graph replay), in
 * which every CTA first waits, bounded by limit_ns nanoseconds, on an mbarrier that
 * no copy and no thread completes. The wait runs out, and the CTA takes the kernel's
 * timeout path: it has issued no load, processes no work item, records
 * VLBM_E_TIMEOUT (reported by the next synchronising call) and leaves the work
 * counter reset for the next launch; the state does not advance. limit_ns = 0
 * disarms the probe, as do vlbm_set_conserved and vlbm_load. Only the row-marching
 * kernel (VLBM_KERNEL_FUSED) waits on barriers. Asynchronous on the state's stream.
 * Errors: VLBM_E_INVAL (s NULL or nothing loaded), VLBM_E_CUDA. */
VLBM_API int vlbm_test_wait_probe(vlbm_state *s, uint32_t limit_ns);

#ifdef __cplusplus
}
#endif
#endif
