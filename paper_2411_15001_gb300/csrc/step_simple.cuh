// step_simple.cuh -- one blended collide + limit + stream step, one thread per
// cell, gathering its radius-2 stencil straight from global memory (L1/L2).
//
// This is the plain GPU form of the step: every face quantity a cell needs is
// recomputed by that cell's thread. It serves the FP64 path and small grids,
// and is the cross-check of the row-marching fused kernel.
#pragma once

#include "common.cuh"

namespace vlbm {

template <typename T>
struct CellLoad {
    const T *__restrict__ in;
    int pitch;
    __device__ __forceinline__ T v(int q, int i, int j) const { return in[sidx(pitch, q, i, j)]; }
    // values q0 .. q0 + 3 of cell (i, j), q0 a multiple of 4: a whole group, one vector load
    __device__ __forceinline__ void u4(int q0, int i, int j, T out[4]) const {
        ld_group(in + sidx(pitch, q0, i, j), out);
    }
};

// theta of the four faces of cell (i, j), Sec. 3.2-3.4, given the face states.
template <typename T, int LIM, typename Loader>
__device__ __forceinline__ void cell_thetas(const Loader &L, int i, int j, const T uC[4],
                                            const T uW[4], const T uE[4], const T uS[4],
                                            const T uN[4], const T usW[4], const T dfW[4],
                                            const T usE[4], const T dfE[4], const T usS[4],
                                            const T dfS[4], const T usN[4], const T dfN[4],
                                            const StepConsts<T> &k, T th[4], unsigned int &n_fp64) {
    if (LIM == VLBM_LIM_FIRST_ORDER) {
        th[0] = th[1] = th[2] = th[3] = T(0);
        return;
    }
    if (LIM == VLBM_LIM_NONE) {
        th[0] = th[1] = th[2] = th[3] = T(1);
        return;
    }
    T tr[4];
    if (LIM == VLBM_LIM_PP) {
        tr[0] = pp_density_target(usW[0], dfW[0], k);
        tr[1] = pp_density_target(usE[0], dfE[0], k);
        tr[2] = pp_density_target(usS[0], dfS[0], k);
        tr[3] = pp_density_target(usN[0], dfN[0], k);
    } else {
        // density bounds (eq. LMP_minmax) of C and its four neighbours; the extra
        // face densities come from the radius-2 and diagonal cells
        const T rWW = L.v(0, i - 2, j), mWW = L.v(1, i - 2, j);
        const T rEE = L.v(0, i + 2, j), mEE = L.v(1, i + 2, j);
        const T rSS = L.v(0, i, j - 2), nSS = L.v(2, i, j - 2);
        const T rNN = L.v(0, i, j + 2), nNN = L.v(2, i, j + 2);
        const T rSW = L.v(0, i - 1, j - 1), mSW = L.v(1, i - 1, j - 1), nSW = L.v(2, i - 1, j - 1);
        const T rSE = L.v(0, i + 1, j - 1), mSE = L.v(1, i + 1, j - 1), nSE = L.v(2, i + 1, j - 1);
        const T rNW = L.v(0, i - 1, j + 1), mNW = L.v(1, i - 1, j + 1), nNW = L.v(2, i - 1, j + 1);
        const T rNE = L.v(0, i + 1, j + 1), mNE = L.v(1, i + 1, j + 1), nNE = L.v(2, i + 1, j + 1);
        auto mn5 = [](T a, T b, T c, T d, T e) { return fmin(fmin(fmin(a, b), fmin(c, d)), e); };
        auto mx5 = [](T a, T b, T c, T d, T e) { return fmax(fmax(fmax(a, b), fmax(c, d)), e); };
        // cell W = (i-1, j)
        const T w_x = face_star(rWW, mWW, uW[0], uW[1], k);
        const T w_s = face_star(rSW, nSW, uW[0], uW[2], k);
        const T w_n = face_star(uW[0], uW[2], rNW, nNW, k);
        // cell E = (i+1, j)
        const T e_x = face_star(uE[0], uE[1], rEE, mEE, k);
        const T e_s = face_star(rSE, nSE, uE[0], uE[2], k);
        const T e_n = face_star(uE[0], uE[2], rNE, nNE, k);
        // cell S = (i, j-1)
        const T s_w = face_star(rSW, mSW, uS[0], uS[1], k);
        const T s_e = face_star(uS[0], uS[1], rSE, mSE, k);
        const T s_s = face_star(rSS, nSS, uS[0], uS[2], k);
        // cell N = (i, j+1)
        const T n_w = face_star(rNW, mNW, uN[0], uN[1], k);
        const T n_e = face_star(uN[0], uN[1], rNE, mNE, k);
        const T n_n = face_star(uN[0], uN[2], rNN, nNN, k);
        T muC = mn5(uC[0], usW[0], usE[0], usS[0], usN[0]);
        T nuC = mx5(uC[0], usW[0], usE[0], usS[0], usN[0]);
        T muW = mn5(uW[0], w_x, usW[0], w_s, w_n), nuW = mx5(uW[0], w_x, usW[0], w_s, w_n);
        T muE = mn5(uE[0], usE[0], e_x, e_s, e_n), nuE = mx5(uE[0], usE[0], e_x, e_s, e_n);
        T muS = mn5(uS[0], s_w, s_e, s_s, usS[0]), nuS = mx5(uS[0], s_w, s_e, s_s, usS[0]);
        T muN = mn5(uN[0], n_w, n_e, usN[0], n_n), nuN = mx5(uN[0], n_w, n_e, usN[0], n_n);
        if (LIM == VLBM_LIM_RLMP) {  // Sec. 3.3.2
            const T lo = T(0.999), hi = T(1.001);
            muC = RN<T>::mul(muC, lo); muW = RN<T>::mul(muW, lo); muE = RN<T>::mul(muE, lo);
            muS = RN<T>::mul(muS, lo); muN = RN<T>::mul(muN, lo);
            nuC = RN<T>::mul(nuC, hi); nuW = RN<T>::mul(nuW, hi); nuE = RN<T>::mul(nuE, hi);
            nuS = RN<T>::mul(nuS, hi); nuN = RN<T>::mul(nuN, hi);
        }
        tr[0] = theta_rho_lmp(usW[0], dfW[0], muW, nuW, muC, nuC, k);
        tr[1] = theta_rho_lmp(usE[0], dfE[0], muC, nuC, muE, nuE, k);
        tr[2] = theta_rho_lmp(usS[0], dfS[0], muS, nuS, muC, nuC, k);
        tr[3] = theta_rho_lmp(usN[0], dfN[0], muC, nuC, muN, nuN, k);
    }
    unsigned int own = 0, other = 0;   // faces are owned by their west / south cell
    th[0] = combine_theta(tr[0], usW, dfW, k, other);
    th[1] = combine_theta(tr[1], usE, dfE, k, own);
    th[2] = combine_theta(tr[2], usS, dfS, k, other);
    th[3] = combine_theta(tr[3], usN, dfN, k, own);
    n_fp64 += own;
}

// Face state u* and dF (eq. D2Q5_convexproof_3, eq. 2nd-order_flux).
template <typename T>
__device__ __forceinline__ void face_state(const T uL[4], const T fL[4], const T uR[4],
                                           const T fR[4], const T dL[4], const T dR[4],
                                           const StepConsts<T> &k, T us[4], T df[4]) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        us[c] = face_star(uL[c], fL[c], uR[c], fR[c], k);
        df[c] = face_dflux(dL[c], dR[c], k);
    }
}

// One cell of the blended collide + limit + stream step, gathering its radius-2
// stencil through the loader L (L.v(q, i, j) = value q of cell (i, j), ghost cells
// included; L.u4(q0, i, j, out) = values q0 .. q0 + 3). Writes the cell's 20 new values to nv (u, then u_1..u_4).
template <typename T, int LIM, typename Loader>
__device__ __forceinline__ void cell_step(const Loader &L, int i, int j, const StepConsts<T> &k,
                                          const Sponge &sp, T nv[kNPlane], unsigned int &n_fp64) {
    T uC[4], uW[4], uE[4], uS[4], uN[4];
    L.u4(0, i, j, uC);
    L.u4(0, i - 1, j, uW);
    L.u4(0, i + 1, j, uE);
    L.u4(0, i, j - 1, uS);
    L.u4(0, i, j + 1, uN);
    T fC[4], gC[4], fW[4], gW[4], fE[4], gE[4], fS[4], gS[4], fN[4], gN[4];
    euler_fluxes(uC, k.gm1, fC, gC);
    euler_fluxes(uW, k.gm1, fW, gW);
    euler_fluxes(uE, k.gm1, fE, gE);
    euler_fluxes(uS, k.gm1, fS, gS);
    euler_fluxes(uN, k.gm1, fN, gN);
    T M1C[4], M2C[4], M3C[4], M4C[4], M1W[4], M2E[4], M3S[4], M4N[4], dum[4];
    maxwell_pm(uC, fC, k, M1C, M2C);
    maxwell_pm(uC, gC, k, M3C, M4C);
    maxwell_pm(uW, fW, k, M1W, dum);
    maxwell_pm(uE, fE, k, dum, M2E);
    maxwell_pm(uS, gS, k, M3S, dum);
    maxwell_pm(uN, gN, k, dum, M4N);
    // non-equilibrium parts d_k = M_k - u_k of the cells the update reads
    T d1C[4], d2C[4], d3C[4], d4C[4], d1W[4], d2E[4], d3S[4], d4N[4];
    {
        T p1C[4], p2C[4], p3C[4], p4C[4], p1W[4], p2E[4], p3S[4], p4N[4];
        L.u4(4, i, j, p1C);
        L.u4(8, i, j, p2C);
        L.u4(12, i, j, p3C);
        L.u4(16, i, j, p4C);
        L.u4(4, i - 1, j, p1W);
        L.u4(8, i + 1, j, p2E);
        L.u4(12, i, j - 1, p3S);
        L.u4(16, i, j + 1, p4N);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            d1C[c] = RN<T>::sub(M1C[c], p1C[c]);
            d2C[c] = RN<T>::sub(M2C[c], p2C[c]);
            d3C[c] = RN<T>::sub(M3C[c], p3C[c]);
            d4C[c] = RN<T>::sub(M4C[c], p4C[c]);
            d1W[c] = RN<T>::sub(M1W[c], p1W[c]);
            d2E[c] = RN<T>::sub(M2E[c], p2E[c]);
            d3S[c] = RN<T>::sub(M3S[c], p3S[c]);
            d4N[c] = RN<T>::sub(M4N[c], p4N[c]);
        }
    }
    T usW[4], dfW[4], usE[4], dfE[4], usS[4], dfS[4], usN[4], dfN[4];
    face_state(uW, fW, uC, fC, d1W, d2C, k, usW, dfW);   // x-face i-1/2
    face_state(uC, fC, uE, fE, d1C, d2E, k, usE, dfE);   // x-face i+1/2
    face_state(uS, gS, uC, gC, d3S, d4C, k, usS, dfS);   // y-face j-1/2
    face_state(uC, gC, uN, gN, d3C, d4N, k, usN, dfN);   // y-face j+1/2
    T th[4];
    cell_thetas<T, LIM>(L, i, j, uC, uW, uE, uS, uN, usW, dfW, usE, dfE, usS, dfS, usN, dfN, k, th,
                        n_fp64);
    if (sp.w > 0) {   // sponge layer (Sec. 4.2): theta = 0 on the faces of layer cells
        const bool cC = sp.cell(i, j);
        if (cC || sp.cell(i - 1, j)) th[0] = T(0);
        if (cC || sp.cell(i + 1, j)) th[1] = T(0);
        if (cC || sp.cell(i, j - 1)) th[2] = T(0);
        if (cC || sp.cell(i, j + 1)) th[3] = T(0);
    }
    // collide + stream, eq. (blending_u1) and eq. (blending_u)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const T u1 = blend_pop(M1W[c], d1W[c], th[0]);
        const T u2 = blend_pop(M2E[c], d2E[c], th[1]);
        const T u3 = blend_pop(M3S[c], d3S[c], th[2]);
        const T u4 = blend_pop(M4N[c], d4N[c], th[3]);
        nv[c] = blend_u(u1, u2, u3, u4, uC[c], th[0], d2C[c], th[1], d1C[c], th[2], d4C[c], th[3],
                        d3C[c], k);
        nv[4 + c] = u1;
        nv[8 + c] = u2;
        nv[12 + c] = u3;
        nv[16 + c] = u4;
    }
}

template <typename T, int LIM>
__global__ void __launch_bounds__(256) k_step_simple(StepArgs<T> A) {
    DevCtl *C = A.ctl;
    if (C->done) return;
    const long long n = C->n;
    CellLoad<T> L{(n & 1) ? A.buf1 : A.buf0, A.pitch};
    T *__restrict__ out = (n & 1) ? A.buf0 : A.buf1;
    const StepConsts<T> k = consts_of<T>(C);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    Monitor<T> mon;
    mon.init();
    if (i < A.nx && j < A.ny) {
        T nv[kNPlane];
        cell_step<T, LIM>(L, i, j, k, Sponge(A.sponge, A.nx, A.ny, A.bc), nv, mon.fp64);
        T *base = out + cidx(A, i, j);
#pragma unroll
        for (int g = 0; g < kNGroup; ++g)
            st_group(base + qoff(A, 4 * g), nv[4 * g], nv[4 * g + 1], nv[4 * g + 2], nv[4 * g + 3]);
        // the new state's ghost frame: images of the cells next to a side (prescribed
        // ghosts are written before the step that reads them)
        if (i < 2 || i >= A.nx - 2 || j < 2 || j >= A.ny - 2) {
            Geo D;
            D.pitch = A.pitch;
            D.nx = A.nx;
            D.ny = A.ny;
            for (int q = 0; q < 4; ++q) D.bc[q] = A.bc[q];
            D.sponge = A.sponge;
            write_ghost_images(D, out, i, j, nv, &A.bd);
        }
        mon.add_cell(nv, k.gamma, k.gm1);
    }
    block_publish(mon, C);
    if (last_block(C, gridDim.x * gridDim.y)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) finalize_step(C);
    }
}

}  // namespace vlbm
