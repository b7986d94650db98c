// step_fused.cuh -- one blended collide + limit + stream step as a single
// row-marching pass: every cell's 20 values are read from HBM once and written
// once.
//
// Decomposition. The grid is cut into strips of kFOut = 124 output columns.
// A CTA of kFB = 128 threads (one padded column each, two halo columns on
// either side) marches up a strip; persistent CTAs split the strips' rows
// evenly. Rows arrive by TMA (one 3D box of 128 columns x 20 planes per row)
// into a 3-slot ring completed on mbarriers, so up to three rows are in flight
// per CTA while earlier rows are computed.
//
// Per row R (output row O = R - 2, the radius-2 LMP stencil of eq. LMP_minmax):
//  P1  fluxes, Maxwellians and non-equilibrium parts d_k of row R; the values
//      x-neighbours need (u, f, d_1, d_2) go to a 4-row shared ring, the ones
//      only the own column needs (u, g, d_3, d_4) stay in a 4-row register
//      history; rho* of the y-face R - 1/2.
//  P2  density bounds mu, nu of row R - 1 (LMP/RLMP).
//  P3  theta of the x-faces of row R - 1 and of the y-face R - 3/2 (Sec.
//      3.3-3.4); then u*, dF of the x-faces of row R and the y-face R - 1/2.
//  P4  collide + stream of row O (eq. blending_u1 / blending_u), stores, monitors.
// Three __syncthreads per row; every quantity is computed once.
#pragma once

#include "common.cuh"
#include "tma.cuh"

namespace vlbm {

constexpr int kFB = 128;       // threads per CTA = TMA box width (columns)
constexpr int kFOut = 124;     // output columns per strip
constexpr int kRawSlots = 3;   // TMA row ring
constexpr int kXSlots = 4;     // shared ring of per-row neighbour data

template <typename T>
struct FusedSmem {
    T raw[kRawSlots][kNPlane][kFB];
    T X[kXSlots][16][kFB];     // u (0..3), f (4..7), d_1 (8..11), d_2 (12..15)
    T rsx[2][kFB];             // rho* of x-face (b, b+1)
    T mu[2][kFB], nu[2][kFB];  // density bounds
    T thx[2][kFB];             // theta of x-face (b, b+1)
    unsigned long long bar[kRawSlots];
    int abort;
};

template <typename T>
struct Hist {
    T u[4], g[4], d3[4], d4[4];
};

template <typename T, int LIM>
struct FusedCtx {
    FusedSmem<T> &S;
    const CUtensorMap *tmap;
    const StepArgs<T> &A;
    const StepConsts<T> &k;
    T *__restrict__ out;
    Monitor<T> &mon;
    int b, zin;
    uint32_t nissued, nconsumed;
    // current item
    int xb, xpad, c, y0, y1, R1;
    // carried face state
    T xs_us[4], xs_df[4];   // x-face (c+1/2) of row R-1
    T ys_us[4], ys_df[4];   // y-face between rows R-2 and R-1
    T rsy_prev;             // rho* of that y-face
    T mu2, nu2;             // bounds of row R-2 (own column)
    T thy_prev;             // theta of the y-face between rows R-3 and R-2

    __device__ __forceinline__ void issue(int row) {
        const int slot = nissued % kRawSlots;
        mbar_expect_tx(&S.bar[slot], (uint32_t)(kNPlane * kFB * sizeof(T)));
        tma_load_3d(&S.raw[slot][0][0], tmap, &S.bar[slot], xpad, row + kOY, zin);
        ++nissued;
    }

    __device__ __forceinline__ void reset_state() {
#pragma unroll
        for (int q = 0; q < 4; ++q) xs_us[q] = xs_df[q] = ys_us[q] = ys_df[q] = T(0);
        rsy_prev = mu2 = nu2 = thy_prev = T(0);
    }

    // One row iteration; H0 receives row R, H1..H3 hold rows R-1..R-3.
    // Returns false if a wait timed out (the CTA then stops).
    __device__ __forceinline__ bool row(int R, Hist<T> &H0, const Hist<T> &H1, const Hist<T> &H2,
                                        const Hist<T> &H3) {
        // ---------------------------------------------------------------- P1
        const int slot = nconsumed % kRawSlots;
        const uint32_t par = (nconsumed / kRawSlots) & 1u;
        ++nconsumed;
        if (!mbar_wait_bounded(&S.bar[slot], par)) S.abort = 1;
        T u[4], f[4], g[4], M1[4], M2[4], M3[4], M4[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) u[q] = S.raw[slot][q][b];
        euler_fluxes(u, k.gm1, f, g);
        maxwell_pm(u, f, k, M1, M2);
        maxwell_pm(u, g, k, M3, M4);
        const int xs = R & 3;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const T d1 = RN<T>::sub(M1[q], S.raw[slot][4 + q][b]);
            const T d2 = RN<T>::sub(M2[q], S.raw[slot][8 + q][b]);
            H0.d3[q] = RN<T>::sub(M3[q], S.raw[slot][12 + q][b]);
            H0.d4[q] = RN<T>::sub(M4[q], S.raw[slot][16 + q][b]);
            H0.u[q] = u[q];
            H0.g[q] = g[q];
            S.X[xs][q][b] = u[q];
            S.X[xs][4 + q][b] = f[q];
            S.X[xs][8 + q][b] = d1;
            S.X[xs][12 + q][b] = d2;
        }
        const T rsy_new = face_star(H1.u[0], H1.g[0], u[0], g[0], k);  // y-face R - 1/2
        __syncthreads();                                                  // S1
        if (S.abort) return false;
        if (b == 0 && R + kRawSlots <= R1) issue(R + kRawSlots);

        const int bl = b > 0 ? b - 1 : 0, br = b < kFB - 1 ? b + 1 : b;
        // ---------------------------------------------------------------- P2
        T mu1 = T(0), nu1 = T(0);
        if (LIM == VLBM_LIM_LMP || LIM == VLBM_LIM_RLMP) {
            const int rp = (R - 1) & 1;
            const T v0 = H1.u[0], v1 = S.rsx[rp][bl], v2 = S.rsx[rp][b];
            mu1 = fmin(fmin(fmin(v0, v1), fmin(v2, rsy_prev)), rsy_new);
            nu1 = fmax(fmax(fmax(v0, v1), fmax(v2, rsy_prev)), rsy_new);
            if (LIM == VLBM_LIM_RLMP) {  // Sec. 3.3.2
                mu1 = RN<T>::mul(mu1, T(0.999));
                nu1 = RN<T>::mul(nu1, T(1.001));
            }
            S.mu[rp][b] = mu1;
            S.nu[rp][b] = nu1;
            __syncthreads();                                              // S2
        }
        // ---------------------------------------------------------------- P3
        T tx, ty;
        if (LIM == VLBM_LIM_FIRST_ORDER) {
            tx = ty = T(0);
        } else if (LIM == VLBM_LIM_NONE) {
            tx = ty = T(1);
        } else {
            T trx, try_;
            if (LIM == VLBM_LIM_PP) {
                trx = theta_rho_pp(xs_us[0], xs_df[0], k);
                try_ = theta_rho_pp(ys_us[0], ys_df[0], k);
            } else {
                const int rp = (R - 1) & 1;
                trx = theta_rho_lmp(xs_us[0], xs_df[0], S.mu[rp][b], S.nu[rp][b], S.mu[rp][br],
                                    S.nu[rp][br], k);
                try_ = theta_rho_lmp(ys_us[0], ys_df[0], mu2, nu2, mu1, nu1, k);
            }
            unsigned int nx64 = 0, ny64 = 0;
            tx = combine_theta(trx, xs_us, xs_df, k, nx64);
            ty = combine_theta(try_, ys_us, ys_df, k, ny64);
            // faces counted once: an x-face by the cell west of it, a y-face by the one south of it
            const bool col_own = b >= 2 && b < 2 + kFOut && c < A.nx;
            if (col_own && R - 1 >= y0 && R - 1 < y1) mon.fp64 += nx64;
            if (col_own && R - 2 >= y0 && R - 2 < y1) mon.fp64 += ny64;
        }
        S.thx[(R - 1) & 1][b] = tx;
        mu2 = mu1;
        nu2 = nu1;
        // new x-face (b, b+1) of row R and y-face R - 1/2
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            xs_us[q] = face_star(S.X[xs][q][b], S.X[xs][4 + q][b], S.X[xs][q][br], S.X[xs][4 + q][br], k);
            xs_df[q] = face_dflux(S.X[xs][8 + q][b], S.X[xs][12 + q][br], k);
            ys_us[q] = q == 0 ? rsy_new : face_star(H1.u[q], H1.g[q], H0.u[q], H0.g[q], k);
            ys_df[q] = face_dflux(H1.d3[q], H0.d4[q], k);
        }
        S.rsx[R & 1][b] = xs_us[0];
        rsy_prev = rsy_new;
        __syncthreads();                                                  // S3
        // ---------------------------------------------------------------- P4
        const int O = R - 2;
        const int xo = O & 3, tp = O & 1;
        const T tw = S.thx[tp][bl], te = S.thx[tp][b];
        const T ts = thy_prev, tn = ty;
        T un[4], p1[4], p2[4], p3[4], p4[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const T M1W = maxwell_plus(S.X[xo][q][bl], S.X[xo][4 + q][bl], k);
            const T M2E = maxwell_minus(S.X[xo][q][br], S.X[xo][4 + q][br], k);
            const T M3S = maxwell_plus(H3.u[q], H3.g[q], k);
            const T M4N = maxwell_minus(H1.u[q], H1.g[q], k);
            p1[q] = blend_pop(M1W, S.X[xo][8 + q][bl], tw);
            p2[q] = blend_pop(M2E, S.X[xo][12 + q][br], te);
            p3[q] = blend_pop(M3S, H3.d3[q], ts);
            p4[q] = blend_pop(M4N, H1.d4[q], tn);
            un[q] = blend_u(p1[q], p2[q], p3[q], p4[q], H2.u[q], tw, S.X[xo][12 + q][b], te,
                            S.X[xo][8 + q][b], ts, H2.d4[q], tn, H2.d3[q], k);
        }
        thy_prev = ty;
        if (O >= y0 && O < y1 && b >= 2 && b < 2 + kFOut && c < A.nx) {
            const long long d = (long long)(O + kOY) * A.pitch + (c + kOX);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                out[q * A.plane + d] = un[q];
                out[(4 + q) * A.plane + d] = p1[q];
                out[(8 + q) * A.plane + d] = p2[q];
                out[(12 + q) * A.plane + d] = p3[q];
                out[(16 + q) * A.plane + d] = p4[q];
            }
            mon.add_cell(un, k.gamma, k.gm1);
        }
        return true;
    }

    // Wait (bounded) for this CTA's loads still in flight before it exits.
    __device__ void drain() {
        if (b == 0) {
            while (nconsumed < nissued) {
                const int slot = nconsumed % kRawSlots;
                mbar_wait_bounded(&S.bar[slot], (nconsumed / kRawSlots) & 1u, 500000000ull);
                ++nconsumed;
            }
        }
    }
};

template <typename T, int LIM>
__global__ void __launch_bounds__(kFB, sizeof(T) == 4 ? 3 : 1)
    k_step_fused(const __grid_constant__ CUtensorMap tmap, StepArgs<T> A, int strips) {
    DevCtl *C = A.ctl;
    if (C->done) return;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    FusedSmem<T> &S = *reinterpret_cast<FusedSmem<T> *>(smem_raw);
    const long long n = C->n;
    const StepConsts<T> k = make_consts<T>(C->a, A.alpha, A.gamma, A.eps);
    Monitor<T> mon;
    mon.init();
    FusedCtx<T, LIM> X{S, &tmap, A, k, (n & 1) ? A.buf0 : A.buf1, mon};
    X.b = threadIdx.x;
    X.zin = (n & 1) ? kNPlane : 0;
    X.nissued = X.nconsumed = 0;
    // TMA destinations must be 128-byte aligned; dynamic shared memory follows
    // the static block of the reductions, so check rather than assume.
    if (smem_addr(&S.raw[0][0][0]) & 127u) {
        if (X.b == 0) atomicCAS(&C->status, 0, VLBM_E_UNSUPPORTED);
        return;
    }
    if (X.b == 0) {
        for (int s = 0; s < kRawSlots; ++s) mbar_init(&S.bar[s], 1);
        S.abort = 0;
        fence_mbar_init();
    }
    __syncthreads();
    const int ny = A.ny;
    const long long total = (long long)strips * ny;
    const long long L0 = total * blockIdx.x / gridDim.x, L1 = total * (blockIdx.x + 1) / gridDim.x;
    bool ok = true;
    for (long long Lc = L0; Lc < L1 && ok;) {
        const int s = (int)(Lc / ny);
        X.y0 = (int)(Lc % ny);
        X.y1 = (int)(X.y0 + (L1 - Lc) < (long long)ny ? X.y0 + (L1 - Lc) : ny);
        Lc += X.y1 - X.y0;
        X.xb = kFOut * s - 2;
        X.xpad = X.xb + kOX;
        X.c = X.xb + X.b;
        const int R0 = X.y0 - 2;
        X.R1 = X.y1 + 1;
        if (X.b == 0)
            for (int r = R0; r < R0 + kRawSlots && r <= X.R1; ++r) X.issue(r);
        X.reset_state();
        Hist<T> h0, h1, h2, h3;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            h0.u[q] = h1.u[q] = h2.u[q] = h3.u[q] = T(1);
            h0.g[q] = h1.g[q] = h2.g[q] = h3.g[q] = T(0);
            h0.d3[q] = h1.d3[q] = h2.d3[q] = h3.d3[q] = T(0);
            h0.d4[q] = h1.d4[q] = h2.d4[q] = h3.d4[q] = T(0);
        }
        for (int R = R0; R <= X.R1 && ok; R += 4) {
            ok = X.row(R, h0, h1, h2, h3);
            if (ok && R + 1 <= X.R1) ok = X.row(R + 1, h3, h0, h1, h2);
            if (ok && R + 2 <= X.R1) ok = X.row(R + 2, h2, h3, h0, h1);
            if (ok && R + 3 <= X.R1) ok = X.row(R + 3, h1, h2, h3, h0);
        }
    }
    if (!ok) {
        X.drain();
        if (X.b == 0) atomicCAS(&C->status, 0, VLBM_E_TIMEOUT);
    }
    block_publish(mon, C);
    if (last_block(C, gridDim.x)) {
        if (X.b == 0) finalize_step(C);
    }
}

}  // namespace vlbm
