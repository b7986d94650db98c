// adjoint.cuh -- transpose of one blended collide + limit + stream step.
//
// For cotangents (ubar', pbar_k') of the step's outputs it returns the cotangents
// of its inputs (u, u_1..u_4), holding the kinetic speed a^n fixed and
// differentiating the limiter piecewise on the branch the forward step took
// (theta = 1, theta_rho, theta_p or the clamp at 0). One thread per cell
// gathers every term in which its inputs appear:
//  - the streamed populations u_k'(c') = M_k(c) + theta d_k(c) of the downstream
//    neighbour c' and the local terms -theta d_k(c) of its own u'(c)
//    (eq. blending_u1 / blending_u);
//  - the face states u* and dF of its four faces (eq. D2Q5_convexproof_3,
//    eq. 2nd-order_flux) through the limiter's derivative;
//  - the Maxwellians M_k = (1-alpha)/4 u +- f/(2a) (Example D2Q5) through the
//    Jacobians of the Euler fluxes.
// The forward state is read from a padded buffer with its ghost frame; the
// cotangents are compact planes. On a periodic grid the gather wraps around. With
// a boundary (ext) the step reads ghost cells filled from the state (the ghost
// fill G): the gather then also runs over the first ghost layer, where no output
// exists (zero cotangent), into a buffer padded by one cell, and k_adjoint_fold_*
// apply the transpose of G (y ghosts into their sources, then x ghosts; a mirror
// ghost's map is its own transpose; a prescribed ghost depends on no state).
//
// Optionally (DA) the kernel also accumulates abar = dL/da^n, the cotangent of
// the step's kinetic speed: a enters the Maxwellians (f / 2a), kappa = a (1 -
// alpha) / 2 (u* and both bounds of theta) and dF = a (d_L - d_R). With a^n =
// 2 lambda^n / (1 - alpha) and lambda^n the max over the cells of s^n (Sec. 4
// preamble), k_lambda_* below hand abar on to the cell where the max is taken.
#pragma once

#include "common.cuh"
#include "step_simple.cuh"

namespace vlbm {

template <typename T>
struct AdjArgs {
    const T *fwd;          // forward state s^n (padded, ghost frame filled)
    int pitch, nx, ny;
    const T *cot_in;       // cotangent of s^{n+1}: nx x ny cells (kidx layout below)
    T *cot_out;            // cotangent of s^n: nx x ny cells, or padded (ext)
    const StepConsts<T> *k;  // constants of the step (kinetic speed a^n as the forward run used it)
    double *abar;          // DA: accumulates dL/da^n
    int ext;               // 1: grid with a boundary (cot_out padded by `pad` cells, see above)
    int pad;               // 1, or 2 for LMP / RLMP (their bounds reach the second ghost layer)
    // LMP / RLMP: per-face theta and (u*, dF) cotangents, per-cell bound cotangents,
    // filled by k_adj_lmp_faces / k_adj_lmp_bounds before the gather. Planes of
    // nx ny cells (periodic) or (nx + 4) (ny + 4) (with a boundary: cells -2 .. n + 1):
    // thE, thN, usbE[4], dfbE[4], usbN[4], dfbN[4], mub, nub, rb, and (DA) taE, taN.
    T *lmp;
    int bc[4];             // uniform side types (-1 where a side switches), for the sponge
    int sponge;            // theta = 0 layer of the forward step (Sec. 4.2)
};

// Cotangent buffers hold, like the state, rows of five 4-value groups: value q of
// cell (x, y) of a buffer w cells wide at ((y * 5 + q / 4) * w + x) * 4 + q % 4 (x, y
// from 0; a padded buffer counts its ghost layers in). A cell's group is one 16-byte
// (FP32) or 32-byte (FP64) access, and a warp's cells of one group are contiguous.
__host__ __device__ __forceinline__ long long kidx(int w, int q, long long x, long long y) {
    return ((y * kNGroup + (q >> 2)) * w + x) * 4 + (q & 3);
}

// w^T df/du for the Euler x-flux (dir 0) or y-flux (dir 1) at state u.
template <typename T>
__device__ __forceinline__ void flux_vjp(const T u[4], T gm1, int dir, const T w[4], T r[4]) {
    const T ir = T(1) / u[0];
    const T v1 = u[1] * ir, v2 = u[2] * ir;
    const T q = T(0.5) * (v1 * v1 + v2 * v2);
    const T p = gm1 * (u[3] - u[0] * q);
    const T H = (u[3] + p) * ir;
    if (dir == 0) {
        r[0] = w[1] * (gm1 * q - v1 * v1) - w[2] * v1 * v2 + w[3] * v1 * (gm1 * q - H);
        r[1] = w[0] + w[1] * (T(2) - gm1) * v1 + w[2] * v2 + w[3] * (H - gm1 * v1 * v1);
        r[2] = -w[1] * gm1 * v2 + w[2] * v1 - w[3] * gm1 * v1 * v2;
        r[3] = w[1] * gm1 + w[3] * (T(1) + gm1) * v1;
    } else {
        r[0] = -w[1] * v1 * v2 + w[2] * (gm1 * q - v2 * v2) + w[3] * v2 * (gm1 * q - H);
        r[1] = w[1] * v2 - w[2] * gm1 * v1 - w[3] * gm1 * v1 * v2;
        r[2] = w[0] + w[1] * v1 + w[2] * (T(2) - gm1) * v2 + w[3] * (H - gm1 * v2 * v2);
        r[3] = w[2] * gm1 + w[3] * (T(1) + gm1) * v2;
    }
}

// Gradient of theta = theta_p = kappa / varrho - eps (Sec. 3.4, the internal-energy
// bound active) with respect to (u*, dF).
template <typename T>
__device__ __forceinline__ void thp_grad(const T us[4], const T df[4], const StepConsts<T> &k, T gus[4], T gdf[4]) {
    const T rs = us[0], m1 = us[1], m2 = us[2], Es = us[3];
    const T dr = df[0], dm1 = df[1], dm2 = df[2], dE = df[3];
    const T g0 = m1 * m1 + m2 * m2 - T(2) * rs * Es;
    const T g1 = T(2) * (dr * Es + dE * rs - dm1 * m1 - dm2 * m2);
    const T cq = dm1 * dm1 + dm2 * dm2 - T(2) * dr * dE;
    T disc = g1 * g1 - T(4) * g0 * cq;
    if (disc < T(0)) disc = T(0);
    const T sd = sqrt(disc);
    const T r1 = fabs(dr) / rs;
    const T r2 = (fabs(g1) + sd) / (T(-2) * g0);
    T gr_us[4], gr_df[4];
    if (r1 > r2) {   // the step takes r = r1 > r2 ? r1 : r2
        const T sg = dr > T(0) ? T(1) : (dr < T(0) ? T(-1) : T(0));
        gr_us[0] = -fabs(dr) / (rs * rs);
        gr_us[1] = gr_us[2] = gr_us[3] = T(0);
        gr_df[0] = sg / rs;
        gr_df[1] = gr_df[2] = gr_df[3] = T(0);
    } else {
        const T D = T(-2) * g0;
        const T sg1 = g1 > T(0) ? T(1) : (g1 < T(0) ? T(-1) : T(0));
        // dN = sg1 dg1 + ddisc / (2 sd); dD = -2 dg0; dr2 = (dN - r2 dD) / D
        const T hs = sd > T(0) ? T(0.5) / sd : T(0);
        // gradients of g0, g1, cq
        const T dg0_us[4] = {T(-2) * Es, T(2) * m1, T(2) * m2, T(-2) * rs};
        const T dg1_us[4] = {T(2) * dE, T(-2) * dm1, T(-2) * dm2, T(2) * dr};
        const T dg1_df[4] = {T(2) * Es, T(-2) * m1, T(-2) * m2, T(2) * rs};
        const T dcq_df[4] = {T(-2) * dE, T(2) * dm1, T(2) * dm2, T(-2) * dr};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            // ddisc = 2 g1 dg1 - 4 cq dg0 - 4 g0 dcq
            const T ddisc_us = T(2) * g1 * dg1_us[c] - T(4) * cq * dg0_us[c];
            const T ddisc_df = T(2) * g1 * dg1_df[c] - T(4) * g0 * dcq_df[c];
            const T dN_us = sg1 * dg1_us[c] + hs * ddisc_us;
            const T dN_df = sg1 * dg1_df[c] + hs * ddisc_df;
            gr_us[c] = (dN_us - r2 * (T(-2) * dg0_us[c])) / D;
            gr_df[c] = dN_df / D;
        }
    }
    const T rr = r1 > r2 ? r1 : r2;
    const T f = -k.kappa / (rr * rr);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        gus[c] = f * gr_us[c];
        gdf[c] = f * gr_df[c];
    }
}

// Forward theta of a face (as combine_theta computes it) and its gradient with
// respect to (u*, dF) on the active branch. Density bounds of the PP kind only.
// *active: theta is one of the two bounds (not 1, not clamped), both of the form
// kappa X - eps, so that d theta / d kappa = (theta + eps) / kappa at fixed (u*, dF).
template <typename T, int LIM>
__device__ __forceinline__ T theta_and_grad(const T us[4], const T df[4], const StepConsts<T> &k,
                                            T gus[4], T gdf[4], bool *active) {
    *active = false;
#pragma unroll
    for (int c = 0; c < 4; ++c) gus[c] = gdf[c] = T(0);
    if (LIM == VLBM_LIM_FIRST_ORDER) return T(0);
    if (LIM == VLBM_LIM_NONE) return T(1);
    const T tr = theta_rho_pp(us[0], df[0], k);
    unsigned int dummy = 0;
    const T th = combine_theta(tr, us, df, k, dummy);
    if (!(th > T(0)) || !(th < T(1))) return th;    // clamped: no gradient
    *active = true;
    if (th == tr) {                                  // density bound active (Sec. 3.3.3)
        const T ad = fabs(df[0]);
        gus[0] = k.kappa / ad;
        gdf[0] = -k.kappa * us[0] * (df[0] > T(0) ? T(1) : T(-1)) / (ad * ad);
        return th;
    }
    thp_grad(us, df, k, gus, gdf);
    return th;
}

enum { kLthE = 0, kLthN = 1, kLusbE = 2, kLdfbE = 6, kLusbN = 10, kLdfbN = 14, kLmub = 18, kLnub = 19, kLrb = 20,
       kLtaE = 21, kLtaN = 22, kLPlanes = 23 };   // taE / taN: d theta / d a^n (DA)

// Cells of one LMP plane, and the index of cell (i, j) in it: compact with the
// periodic wrap, or padded by two cells on a grid with a boundary (-1 outside).
template <typename T>
__device__ __forceinline__ long long lmp_cells(const AdjArgs<T> &A) {
    return A.ext ? (long long)(A.nx + 4) * (A.ny + 4) : (long long)A.nx * A.ny;
}
template <typename T>
__device__ __forceinline__ long long lmp_ix(const AdjArgs<T> &A, int i, int j) {
    if (A.ext) {
        if (i < -2 || i > A.nx + 1 || j < -2 || j > A.ny + 1) return -1;
        return (long long)(j + 2) * (A.nx + 4) + (i + 2);
    }
    i = i < 0 ? i + A.nx : (i >= A.nx ? i - A.nx : i);
    j = j < 0 ? j + A.ny : (j >= A.ny ? j - A.ny : j);
    return (long long)j * A.nx + i;
}

// rho* of the x-face (i, i+1) or the y-face (j, j+1) of row / column of cell (i, j)
// (the density component of u*, eq. D2Q5_convexproof_3: the flux of rho is the
// normal momentum), from the padded forward state.
template <typename T>
__device__ __forceinline__ T rho_star_x(const CellLoad<T> &L, int i, int j, const StepConsts<T> &k) {
    return face_star(L.v(0, i, j), L.v(1, i, j), L.v(0, i + 1, j), L.v(1, i + 1, j), k);
}
template <typename T>
__device__ __forceinline__ T rho_star_y(const CellLoad<T> &L, int i, int j, const StepConsts<T> &k) {
    return face_star(L.v(0, i, j), L.v(2, i, j), L.v(0, i, j + 1), L.v(2, i, j + 1), k);
}

// LMP bounds of cell (i, j) (eq. LMP_minmax; RLMP x 0.999 / 1.001): the min / max of
// rho and of rho* on the four faces, in the order rho, west, east, south, north;
// *imin / *imax: the first of them where the min / max is reached.
template <typename T, int LIM>
__device__ __forceinline__ void lmp_bounds(const CellLoad<T> &L, int i, int j, const StepConsts<T> &k, T *mu, T *nu,
                                           int *imin, int *imax) {
    const T v[5] = {L.v(0, i, j), rho_star_x(L, i - 1, j, k), rho_star_x(L, i, j, k), rho_star_y(L, i, j - 1, k),
                    rho_star_y(L, i, j, k)};
    T lo = v[0], hi = v[0];
    int a = 0, b = 0;
#pragma unroll
    for (int q = 1; q < 5; ++q) {
        if (v[q] < lo) { lo = v[q]; a = q; }
        if (v[q] > hi) { hi = v[q]; b = q; }
    }
    *mu = LIM == VLBM_LIM_RLMP ? RN<T>::mul(lo, T(0.999)) : lo;
    *nu = LIM == VLBM_LIM_RLMP ? RN<T>::mul(hi, T(1.001)) : hi;
    *imin = a;
    *imax = b;
}

// d/da^n of the LMP bounds of cell (i, j) at a fixed state: the bound is rho (no
// a-dependence) or rho* of one face, rho* = (rhoL + rhoR)/2 - (mR - mL)/(2 kappa)
// with m the momentum normal to the face and kappa proportional to a, so
// d rho* / da = (mR - mL) / (2 kappa a). imin / imax: the candidates lmp_bounds chose.
template <typename T, int LIM>
__device__ __forceinline__ void lmp_bounds_da(const CellLoad<T> &L, int i, int j, const StepConsts<T> &k, int imin,
                                              int imax, T *dmu, T *dnu) {
    auto drs = [&](int which) -> T {
        const T s = k.inv2k / k.a;
        switch (which) {
            case 1: return (L.v(1, i, j) - L.v(1, i - 1, j)) * s;
            case 2: return (L.v(1, i + 1, j) - L.v(1, i, j)) * s;
            case 3: return (L.v(2, i, j) - L.v(2, i, j - 1)) * s;
            case 4: return (L.v(2, i, j + 1) - L.v(2, i, j)) * s;
            default: return T(0);
        }
    };
    *dmu = LIM == VLBM_LIM_RLMP ? T(0.999) * drs(imin) : drs(imin);
    *dnu = LIM == VLBM_LIM_RLMP ? T(1.001) * drs(imax) : drs(imax);
}

// d theta / da^n of one LMP face at a fixed state, on the branch the step took:
// dus / ddf are d u* / da and d dF / da of the face, d* the bounds' derivatives.
template <typename T, int LIM>
__device__ __forceinline__ T lmp_face_da(const T us[4], const T df[4], T muL, T nuL, T muR, T nuR, T dmuL, T dnuL,
                                         T dmuR, T dnuR, const T dus[4], const T ddf[4], const StepConsts<T> &k) {
    const T tr = theta_rho_lmp(us[0], df[0], muL, nuL, muR, nuR, k);
    unsigned int dummy = 0;
    const T th = combine_theta(tr, us, df, k, dummy);
    if (!(th > T(0)) || !(th < T(1))) return T(0);
    const T ia = T(1) / k.a;
    if (th == tr) {          // theta = s kappa X / dF^rho, kappa proportional to a
        const T dr = df[0], rs = us[0];
        T dX;
        if (dr > T(0)) {
            const T a1 = nuR - rs, a2 = rs - muL;
            dX = a1 < a2 ? dnuR - dus[0] : dus[0] - dmuL;
            return th * ia + k.kappa / dr * dX - th * ddf[0] / dr;
        }
        const T b1 = rs - muR, b2 = nuL - rs;
        dX = b1 < b2 ? dus[0] - dmuR : dnuL - dus[0];
        return th * ia - k.kappa / dr * dX - th * ddf[0] / dr;
    }
    T gus[4], gdf[4];       // theta_p = kappa / varrho - eps
    thp_grad(us, df, k, gus, gdf);
    T d = (th + k.eps) * ia;
#pragma unroll
    for (int c = 0; c < 4; ++c) d += gus[c] * dus[c] + gdf[c] * ddf[c];
    return d;
}

// One face of the LMP adjoint: theta as the step computes it, from the face states
// (us, df) and the bounds of the cells left (L) and right (R) of it; with tb, the
// cotangent of theta, the cotangents of u*, dF go to usb, dfb (4 each) and those of
// the bounds to the cells' mub / nub slots.
template <typename T, int LIM>
__device__ __forceinline__ T lmp_face(const T us[4], const T df[4], T muL, T nuL, T muR, T nuR, T tb,
                                      const StepConsts<T> &k, T usb[4], T dfb[4], T *mubL, T *nubL, T *mubR,
                                      T *nubR) {
#pragma unroll
    for (int c = 0; c < 4; ++c) usb[c] = dfb[c] = T(0);
    const T tr = theta_rho_lmp(us[0], df[0], muL, nuL, muR, nuR, k);
    unsigned int dummy = 0;
    const T th = combine_theta(tr, us, df, k, dummy);
    if (tb == T(0) || !(th > T(0)) || !(th < T(1))) return th;   // no cotangent, or clamped
    if (th == tr) {          // density bound active (Sec. 3.3.1): theta = s kappa X / dF^rho
        const T dr = df[0], rs = us[0];
        const T g = k.kappa / dr;                                   // d theta / dX, with s folded in
        T gX = T(0), *slot = nullptr;   // dX / drho* and the bound X takes its other term from
        T gB = T(0);
        if (dr > T(0)) {
            const T a1 = nuR - rs, a2 = rs - muL;
            if (a1 < a2) { gX = T(-1); gB = T(1); slot = nubR; }      // X = nuR - rho*
            else { gX = T(1); gB = T(-1); slot = mubL; }               // X = rho* - muL
            usb[0] = tb * g * gX;
            atomicAdd(slot, tb * g * gB);
        } else {
            const T b1 = rs - muR, b2 = nuL - rs;
            if (b1 < b2) { gX = T(1); gB = T(-1); slot = mubR; }       // X = rho* - muR
            else { gX = T(-1); gB = T(1); slot = nubL; }               // X = nuL - rho*
            usb[0] = -tb * g * gX;
            atomicAdd(slot, -tb * g * gB);
        }
        dfb[0] = -tb * th / dr;
        return th;
    }
    T gus[4], gdf[4];   // internal-energy bound active
    thp_grad(us, df, k, gus, gdf);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        usb[c] = tb * gus[c];
        dfb[c] = tb * gdf[c];
    }
    return th;
}

// Pass 1 of the LMP / RLMP adjoint: each cell takes its east and north faces. On a
// periodic grid every cell; with a boundary (EXT) cells -1 .. n - 1 in both
// directions (every face next to an interior cell), outputs outside the interior
// having no cotangent; faces of sponge cells have theta = 0 and no cotangent.
template <typename T, int LIM, bool EXT, bool DA>
__global__ void __launch_bounds__(256) k_adj_lmp_faces(AdjArgs<T> A) {
    constexpr int e = EXT ? 1 : 0;
    const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x) - e, j = (int)(blockIdx.y * blockDim.y + threadIdx.y) - e;
    if (i >= A.nx || j >= A.ny) return;
    const StepConsts<T> k = *A.k;
    const CellLoad<T> L{A.fwd, A.pitch};
    const long long NL = lmp_cells(A);
    const long long lC = lmp_ix(A, i, j), lE = lmp_ix(A, i + 1, j), lN = lmp_ix(A, i, j + 1);
    T *P = A.lmp;
    auto cot = [&](int q, int x, int y) -> T {   // output cotangent q of cell (x, y)
        if (EXT) {
            if ((unsigned)x >= (unsigned)A.nx || (unsigned)y >= (unsigned)A.ny) return T(0);
        } else {
            x = x < 0 ? x + A.nx : (x >= A.nx ? x - A.nx : x);
            y = y < 0 ? y + A.ny : (y >= A.ny ? y - A.ny : y);
        }
        return A.cot_in[kidx(A.nx, q, x, y)];
    };
    T uC[4], uE[4], uN[4], fC[4], gC[4], fE[4], gE[4], fN[4], gN[4];
    L.u4(0, i, j, uC);
    L.u4(0, i + 1, j, uE);
    L.u4(0, i, j + 1, uN);
    euler_fluxes(uC, k.gm1, fC, gC);
    euler_fluxes(uE, k.gm1, fE, gE);
    euler_fluxes(uN, k.gm1, fN, gN);
    T usE[4], dfE[4], usN[4], dfN[4], tbE = T(0), tbN = T(0);
    T dusE[4], ddfE[4], dusN[4], ddfN[4];   // DA: d u* / da, d dF / da of the two faces
    T p1C[4], p2E[4], p3C[4], p4N[4];   // population groups, one vector load each
    L.u4(4, i, j, p1C);
    L.u4(8, i + 1, j, p2E);
    L.u4(12, i, j, p3C);
    L.u4(16, i, j + 1, p4N);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const T d1C = RN<T>::sub(maxwell_plus(uC[c], fC[c], k), p1C[c]);
        const T d2E = RN<T>::sub(maxwell_minus(uE[c], fE[c], k), p2E[c]);
        const T d3C = RN<T>::sub(maxwell_plus(uC[c], gC[c], k), p3C[c]);
        const T d4N = RN<T>::sub(maxwell_minus(uN[c], gN[c], k), p4N[c]);
        if (DA) {
            dusE[c] = (fE[c] - fC[c]) * k.inv2k / k.a;
            ddfE[c] = (d1C - d2E) - (fC[c] + fE[c]) * k.inv2a;
            dusN[c] = (gN[c] - gC[c]) * k.inv2k / k.a;
            ddfN[c] = (d3C - d4N) - (gC[c] + gN[c]) * k.inv2a;
        }
        usE[c] = face_star(uC[c], fC[c], uE[c], fE[c], k);
        dfE[c] = face_dflux(d1C, d2E, k);
        usN[c] = face_star(uC[c], gC[c], uN[c], gN[c], k);
        dfN[c] = face_dflux(d3C, d4N, k);
        // cotangent of theta: the pulled populations theta d and the local -theta d of u'
        const T ubC = cot(c, i, j), ubE = cot(c, i + 1, j), ubN = cot(c, i, j + 1);
        tbE += d1C * (cot(4 + c, i + 1, j) + ubE - ubC) + d2E * (cot(8 + c, i, j) + ubC - ubE);
        tbN += d3C * (cot(12 + c, i, j + 1) + ubN - ubC) + d4N * (cot(16 + c, i, j) + ubC - ubN);
    }
    T muC, nuC, muE, nuE, muN, nuN;
    int aC, bC, aE, bE, aN, bN;
    lmp_bounds<T, LIM>(L, i, j, k, &muC, &nuC, &aC, &bC);
    lmp_bounds<T, LIM>(L, i + 1, j, k, &muE, &nuE, &aE, &bE);
    lmp_bounds<T, LIM>(L, i, j + 1, k, &muN, &nuN, &aN, &bN);
    bool spE = false, spN = false;   // sponge faces (Sec. 4.2): theta = 0 whatever the limiter
    if (EXT && A.sponge > 0) {
        const Sponge sp(A.sponge, A.nx, A.ny, A.bc);
        const bool sc = sp.cell(i, j);
        spE = sc || sp.cell(i + 1, j);
        spN = sc || sp.cell(i, j + 1);
    }
    T usb[4], dfb[4];
    T th = lmp_face<T, LIM>(usE, dfE, muC, nuC, muE, nuE, spE ? T(0) : tbE, k, usb, dfb, &P[kLmub * NL + lC],
                            &P[kLnub * NL + lC], &P[kLmub * NL + lE], &P[kLnub * NL + lE]);
    P[kLthE * NL + lC] = spE ? T(0) : th;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        P[(kLusbE + c) * NL + lC] = usb[c];
        P[(kLdfbE + c) * NL + lC] = dfb[c];
    }
    th = lmp_face<T, LIM>(usN, dfN, muC, nuC, muN, nuN, spN ? T(0) : tbN, k, usb, dfb, &P[kLmub * NL + lC],
                          &P[kLnub * NL + lC], &P[kLmub * NL + lN], &P[kLnub * NL + lN]);
    P[kLthN * NL + lC] = spN ? T(0) : th;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        P[(kLusbN + c) * NL + lC] = usb[c];
        P[(kLdfbN + c) * NL + lC] = dfb[c];
    }
    if (DA) {
        T dmC, dnC, dmE, dnE, dmN, dnN;
        lmp_bounds_da<T, LIM>(L, i, j, k, aC, bC, &dmC, &dnC);
        lmp_bounds_da<T, LIM>(L, i + 1, j, k, aE, bE, &dmE, &dnE);
        lmp_bounds_da<T, LIM>(L, i, j + 1, k, aN, bN, &dmN, &dnN);
        P[kLtaE * NL + lC] =
            spE ? T(0) : lmp_face_da<T, LIM>(usE, dfE, muC, nuC, muE, nuE, dmC, dnC, dmE, dnE, dusE, ddfE, k);
        P[kLtaN * NL + lC] =
            spN ? T(0) : lmp_face_da<T, LIM>(usN, dfN, muC, nuC, muN, nuN, dmC, dnC, dmN, dnN, dusN, ddfN, k);
    }
}

// Pass 2: the bound cotangents of each cell go to the value its min / max took:
// its own density (rb) or rho* of one of its faces (the density component of that
// face's u* cotangent). RLMP scales by 0.999 / 1.001. With a boundary (EXT) the
// cells of the first ghost layer too (their bounds enter the boundary faces).
template <typename T, int LIM, bool EXT>
__global__ void __launch_bounds__(256) k_adj_lmp_bounds(AdjArgs<T> A) {
    constexpr int e = EXT ? 1 : 0;
    const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x) - e, j = (int)(blockIdx.y * blockDim.y + threadIdx.y) - e;
    if (i >= A.nx + e || j >= A.ny + e) return;
    const long long NL = lmp_cells(A), cC = lmp_ix(A, i, j);
    T *P = A.lmp;
    const T mb = P[kLmub * NL + cC], nb = P[kLnub * NL + cC];
    if (mb == T(0) && nb == T(0)) return;
    const StepConsts<T> k = *A.k;
    const CellLoad<T> L{A.fwd, A.pitch};
    T mu, nu;
    int a, b;
    lmp_bounds<T, LIM>(L, i, j, k, &mu, &nu, &a, &b);
    const long long cW = lmp_ix(A, i - 1, j), cS = lmp_ix(A, i, j - 1);
    auto give = [&](int which, T v) {
        if (v == T(0)) return;
        T *dst = which == 0 ? &P[kLrb * NL + cC]
               : which == 1 ? &P[kLusbE * NL + cW]
               : which == 2 ? &P[kLusbE * NL + cC]
               : which == 3 ? &P[kLusbN * NL + cS]
                            : &P[kLusbN * NL + cC];
        atomicAdd(dst, v);
    };
    give(a, LIM == VLBM_LIM_RLMP ? mb * T(0.999) : mb);
    give(b, LIM == VLBM_LIM_RLMP ? nb * T(1.001) : nb);
}

template <typename T, int LIM, bool DA, bool EXT>
__device__ __forceinline__ double adjoint_cell(const AdjArgs<T> &A, int i, int j) {
    const StepConsts<T> k = *A.k;
    CellLoad<T> L{A.fwd, A.pitch};
    // ---------------------------------------------------------- forward quantities
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
    T d1C[4], d2C[4], d3C[4], d4C[4], d1W[4], d2E[4], d3S[4], d4N[4];
    {
        T pg[8][4];   // population groups, one vector load each
        L.u4(4, i, j, pg[0]);
        L.u4(8, i, j, pg[1]);
        L.u4(12, i, j, pg[2]);
        L.u4(16, i, j, pg[3]);
        L.u4(4, i - 1, j, pg[4]);
        L.u4(8, i + 1, j, pg[5]);
        L.u4(12, i, j - 1, pg[6]);
        L.u4(16, i, j + 1, pg[7]);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            d1C[c] = RN<T>::sub(maxwell_plus(uC[c], fC[c], k), pg[0][c]);
            d2C[c] = RN<T>::sub(maxwell_minus(uC[c], fC[c], k), pg[1][c]);
            d3C[c] = RN<T>::sub(maxwell_plus(uC[c], gC[c], k), pg[2][c]);
            d4C[c] = RN<T>::sub(maxwell_minus(uC[c], gC[c], k), pg[3][c]);
            d1W[c] = RN<T>::sub(maxwell_plus(uW[c], fW[c], k), pg[4][c]);
            d2E[c] = RN<T>::sub(maxwell_minus(uE[c], fE[c], k), pg[5][c]);
            d3S[c] = RN<T>::sub(maxwell_plus(uS[c], gS[c], k), pg[6][c]);
            d4N[c] = RN<T>::sub(maxwell_minus(uN[c], gN[c], k), pg[7][c]);
        }
    }
    T us[4][4], df[4][4];   // faces W, E, S, N
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        us[0][c] = face_star(uW[c], fW[c], uC[c], fC[c], k);
        df[0][c] = face_dflux(d1W[c], d2C[c], k);
        us[1][c] = face_star(uC[c], fC[c], uE[c], fE[c], k);
        df[1][c] = face_dflux(d1C[c], d2E[c], k);
        us[2][c] = face_star(uS[c], gS[c], uC[c], gC[c], k);
        df[2][c] = face_dflux(d3S[c], d4C[c], k);
        us[3][c] = face_star(uC[c], gC[c], uN[c], gN[c], k);
        df[3][c] = face_dflux(d3C[c], d4N[c], k);
    }
    constexpr bool kLmp = LIM == VLBM_LIM_LMP || LIM == VLBM_LIM_RLMP;
    T th[4], gus[4][4], gdf[4][4];
    bool act[4];
    if constexpr (!kLmp) {
#pragma unroll
        for (int f = 0; f < 4; ++f) th[f] = theta_and_grad<T, LIM>(us[f], df[f], k, gus[f], gdf[f], &act[f]);
    }
    // theta = 0 on the faces of sponge cells, whatever the limiter (a sponge needs a
    // zero-gradient side: never on a periodic grid, whose gather keeps its registers)
    if (EXT && A.sponge > 0) {
        const Sponge sp(A.sponge, A.nx, A.ny, A.bc);
        const bool cc = sp.cell(i, j);
        const bool in[4] = {cc || sp.cell(i - 1, j), cc || sp.cell(i + 1, j), cc || sp.cell(i, j - 1),
                            cc || sp.cell(i, j + 1)};
#pragma unroll
        for (int f = 0; f < 4; ++f)
            if (in[f]) {
                th[f] = T(0);
                act[f] = false;
#pragma unroll
                for (int c = 0; c < 4; ++c) gus[f][c] = gdf[f][c] = T(0);
            }
    }
    // ---------------------------------------------------------- cotangents
    // of the outputs of cell (x, y), a group of four at a time: wrapped on a periodic
    // grid, 0 outside the interior on a grid with a boundary
    int xW = i - 1, xE = i + 1, yS = j - 1, yN = j + 1;
    if constexpr (!EXT) {
        xW = i > 0 ? xW : A.nx - 1;
        xE = i < A.nx - 1 ? xE : 0;
        yS = j > 0 ? yS : A.ny - 1;
        yN = j < A.ny - 1 ? yN : 0;
    }
    auto grp = [&](int g, int x, int y, T v[4]) {
        if constexpr (EXT) {
            if ((unsigned)x >= (unsigned)A.nx || (unsigned)y >= (unsigned)A.ny) {
                v[0] = v[1] = v[2] = v[3] = T(0);
                return;
            }
        }
        ld_group(A.cot_in + kidx(A.nx, 4 * g, x, y), v);
    };
    long long lC = 0, lW = 0, lS = 0, NL = 0;   // the cell and its west / south neighbours in the LMP planes
    if constexpr (kLmp) {   // theta of the four faces as pass 1 found it
        NL = lmp_cells(A);
        lC = lmp_ix(A, i, j);
        lW = lmp_ix(A, i - 1, j);
        lS = lmp_ix(A, i, j - 1);
        th[0] = A.lmp[kLthE * NL + lW];
        th[1] = A.lmp[kLthE * NL + lC];
        th[2] = A.lmp[kLthN * NL + lS];
        th[3] = A.lmp[kLthN * NL + lC];
    }
    T ubC[4], ubW[4], ubE[4], ubS[4], ubN[4];
    T qC[4][4], q1E[4], q2W[4], q3N[4], q4S[4];   // population cotangents as stored
    grp(0, i, j, ubC);
    grp(0, xW, j, ubW);
    grp(0, xE, j, ubE);
    grp(0, i, yS, ubS);
    grp(0, i, yN, ubN);
    grp(1, i, j, qC[0]);
    grp(2, i, j, qC[1]);
    grp(3, i, j, qC[2]);
    grp(4, i, j, qC[3]);
    grp(1, xE, j, q1E);
    grp(2, xW, j, q2W);
    grp(3, i, yN, q3N);
    grp(4, i, yS, q4S);
    T P1C[4], P2C[4], P3C[4], P4C[4], P1E[4], P2W[4], P3N[4], P4S[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        // streamed populations carry the cotangent of u' as well (u' sums them)
        P1C[c] = qC[0][c] + ubC[c];
        P2C[c] = qC[1][c] + ubC[c];
        P3C[c] = qC[2][c] + ubC[c];
        P4C[c] = qC[3][c] + ubC[c];
        P1E[c] = q1E[c] + ubE[c];
        P2W[c] = q2W[c] + ubW[c];
        P3N[c] = q3N[c] + ubN[c];
        P4S[c] = q4S[c] + ubS[c];
    }
    // theta cotangents of the four faces
    T tb[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        tb[0] += d1W[c] * (P1C[c] - ubW[c]) + d2C[c] * (P2W[c] - ubC[c]);
        tb[1] += d1C[c] * (P1E[c] - ubC[c]) + d2E[c] * (P2C[c] - ubE[c]);
        tb[2] += d3S[c] * (P3C[c] - ubS[c]) + d4C[c] * (P4S[c] - ubC[c]);
        tb[3] += d3C[c] * (P3N[c] - ubC[c]) + d4N[c] * (P4C[c] - ubN[c]);
    }
    // ---------------------------------------------------------- input cotangents
    T wx[4], wy[4], out[kNPlane];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        T usb_W, usb_E, usb_S, usb_N, dfb_W, dfb_E, dfb_S, dfb_N;
        if constexpr (kLmp) {   // passes 1 and 2 left the face cotangents
            const T *P = A.lmp;
            usb_W = P[(kLusbE + c) * NL + lW];
            usb_E = P[(kLusbE + c) * NL + lC];
            usb_S = P[(kLusbN + c) * NL + lS];
            usb_N = P[(kLusbN + c) * NL + lC];
            dfb_W = P[(kLdfbE + c) * NL + lW];
            dfb_E = P[(kLdfbE + c) * NL + lC];
            dfb_S = P[(kLdfbN + c) * NL + lS];
            dfb_N = P[(kLdfbN + c) * NL + lC];
        } else {
            usb_W = tb[0] * gus[0][c];
            usb_E = tb[1] * gus[1][c];
            usb_S = tb[2] * gus[2][c];
            usb_N = tb[3] * gus[3][c];
            dfb_W = tb[0] * gdf[0][c];
            dfb_E = tb[1] * gdf[1][c];
            dfb_S = tb[2] * gdf[2][c];
            dfb_N = tb[3] * gdf[3][c];
        }
        const T db1 = th[1] * (P1E[c] - ubC[c]) + k.a * dfb_E;
        const T db2 = th[0] * (P2W[c] - ubC[c]) - k.a * dfb_W;
        const T db3 = th[3] * (P3N[c] - ubC[c]) + k.a * dfb_N;
        const T db4 = th[2] * (P4S[c] - ubC[c]) - k.a * dfb_S;
        const T Mb1 = P1E[c] + db1, Mb2 = P2W[c] + db2, Mb3 = P3N[c] + db3, Mb4 = P4S[c] + db4;
        out[4 + c] = -db1;
        out[8 + c] = -db2;
        out[12 + c] = -db3;
        out[16 + c] = -db4;
        out[c] = k.alpha * ubC[c] + k.w * (Mb1 + Mb2 + Mb3 + Mb4) + T(0.5) * (usb_W + usb_E + usb_S + usb_N);
        wx[c] = (Mb1 - Mb2) * k.inv2a + (usb_E - usb_W) * k.inv2k;
        wy[c] = (Mb3 - Mb4) * k.inv2a + (usb_N - usb_S) * k.inv2k;
    }
    T rx[4], ry[4];
    flux_vjp(uC, k.gm1, 0, wx, rx);
    flux_vjp(uC, k.gm1, 1, wy, ry);
#pragma unroll
    for (int c = 0; c < 4; ++c) out[c] += rx[c] + ry[c];
    if constexpr (kLmp) out[0] += A.lmp[kLrb * NL + lC];   // the density where a cell's bound was taken
    {
        const int w = EXT ? A.nx + 2 * A.pad : A.nx, o = EXT ? A.pad : 0;
#pragma unroll
        for (int g = 0; g < kNGroup; ++g)
            st_group(A.cot_out + kidx(w, 4 * g, i + o, j + o), out[4 * g], out[4 * g + 1], out[4 * g + 2],
                     out[4 * g + 3]);
    }
    if constexpr (!DA) {
        return 0.0;
    } else {
        // d/da of the face states: u* = (uL + uR)/2 - (fR - fL)/(2 kappa) with kappa ~ a,
        // dF = a (dL - dR) with dM_{1,3}/da = -F/(2a^2), dM_{2,4}/da = +F/(2a^2)
        const T ia = T(1) / k.a, h = k.inv2a * ia;
        T dth[4];
        if constexpr (kLmp) {   // pass 1 left d theta / da of every face
            dth[0] = A.lmp[kLtaE * NL + lW];
            dth[1] = A.lmp[kLtaE * NL + lC];
            dth[2] = A.lmp[kLtaN * NL + lS];
            dth[3] = A.lmp[kLtaN * NL + lC];
        } else {
#pragma unroll
            for (int f = 0; f < 4; ++f) dth[f] = act[f] ? (th[f] + k.eps) * ia : T(0);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                dth[0] += gus[0][c] * (fC[c] - fW[c]) * k.inv2k * ia + gdf[0][c] * ((d1W[c] - d2C[c]) - (fW[c] + fC[c]) * k.inv2a);
                dth[1] += gus[1][c] * (fE[c] - fC[c]) * k.inv2k * ia + gdf[1][c] * ((d1C[c] - d2E[c]) - (fC[c] + fE[c]) * k.inv2a);
                dth[2] += gus[2][c] * (gC[c] - gS[c]) * k.inv2k * ia + gdf[2][c] * ((d3S[c] - d4C[c]) - (gS[c] + gC[c]) * k.inv2a);
                dth[3] += gus[3][c] * (gN[c] - gC[c]) * k.inv2k * ia + gdf[3][c] * ((d3C[c] - d4N[c]) - (gC[c] + gN[c]) * k.inv2a);
            }
        }
        double ab = 0.0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            // outputs of this cell: the four pulled populations and u'
            const T du1 = -(T(1) + th[0]) * fW[c] * h + d1W[c] * dth[0];
            const T du2 = (T(1) + th[1]) * fE[c] * h + d2E[c] * dth[1];
            const T du3 = -(T(1) + th[2]) * gS[c] * h + d3S[c] * dth[2];
            const T du4 = (T(1) + th[3]) * gN[c] * h + d4N[c] * dth[3];
            const T loc = dth[0] * d2C[c] + th[0] * fC[c] * h + dth[1] * d1C[c] - th[1] * fC[c] * h +
                          dth[2] * d4C[c] + th[2] * gC[c] * h + dth[3] * d3C[c] - th[3] * gC[c] * h;
            ab += (double)(qC[0][c] * du1 + qC[1][c] * du2 + qC[2][c] * du3 + qC[3][c] * du4) +
                  (double)(ubC[c] * (du1 + du2 + du3 + du4 - loc));
        }
        return ab;
    }
}


// LMP / RLMP with a boundary: the cells of the second ghost layer (the outer ring of
// the padded cotangent, 2 (nx + 4) + 2 (ny + 2) cells). Their outputs and the
// faces between them and the first layer carry no theta cotangent, but the bounds
// of a first-layer cell can be taken at rho* of such a face: that u* cotangent
// reaches the ring cell through u* = (uL + uR)/2 -/+ (F(uR) - F(uL)) / (2 kappa).
template <typename T>
__global__ void __launch_bounds__(256) k_adj_lmp_ring(AdjArgs<T> A) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int w = A.nx + 4, h = A.ny + 2;
    if (t >= 2 * w + 2 * h) return;
    int i, j;
    if (t < 2 * w) { i = t % w - 2; j = t < w ? -2 : A.ny + 1; }
    else { const int r = t - 2 * w; j = r % h - 1; i = r < h ? -2 : A.nx + 1; }
    const long long NL = lmp_cells(A);
    auto usb = [&](int plane, int x, int y) -> T {
        const long long c = lmp_ix(A, x, y);
        return c < 0 ? T(0) : A.lmp[plane * NL + c];
    };
    T out[kNPlane];
#pragma unroll
    for (int q = 0; q < kNPlane; ++q) out[q] = T(0);
    T uW[4], uE[4], uS[4], uN[4];
    bool any = false;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uW[c] = usb(kLusbE + c, i - 1, j);
        uE[c] = usb(kLusbE + c, i, j);
        uS[c] = usb(kLusbN + c, i, j - 1);
        uN[c] = usb(kLusbN + c, i, j);
        any = any || uW[c] != T(0) || uE[c] != T(0) || uS[c] != T(0) || uN[c] != T(0);
    }
    if (any) {   // only then is the cell's state read (a ring cell on a corner may hold none)
        const StepConsts<T> k = *A.k;
        const CellLoad<T> L{A.fwd, A.pitch};
        T u[4], wx[4], wy[4], rx[4], ry[4];
        L.u4(0, i, j, u);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            out[c] = T(0.5) * (uW[c] + uE[c] + uS[c] + uN[c]);
            wx[c] = (uE[c] - uW[c]) * k.inv2k;
            wy[c] = (uN[c] - uS[c]) * k.inv2k;
        }
        flux_vjp(u, k.gm1, 0, wx, rx);
        flux_vjp(u, k.gm1, 1, wy, ry);
#pragma unroll
        for (int c = 0; c < 4; ++c) out[c] += rx[c] + ry[c];
    }
#pragma unroll
    for (int g = 0; g < kNGroup; ++g)
        st_group(A.cot_out + kidx(w, 4 * g, i + 2, j + 2), out[4 * g], out[4 * g + 1], out[4 * g + 2], out[4 * g + 3]);
}

// Sum of v over the CTA's warps into *dst (every thread of the CTA calls it).
__device__ __forceinline__ void warp_sum_atomic(double v, double *dst) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(dst, v);
}

template <typename T, int LIM, bool DA, bool EXT>
__global__ void __launch_bounds__(256) k_adjoint_step(AdjArgs<T> A) {
    // with a boundary (EXT) the threads cover the first ghost layer too: cells -1 .. n
    constexpr int e = EXT ? 1 : 0;
    const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x) - e;
    const int j = (int)(blockIdx.y * blockDim.y + threadIdx.y) - e;
    double abar = 0.0;
    if (i < A.nx + e && j < A.ny + e) abar = adjoint_cell<T, LIM, DA, EXT>(A, i, j);
    if constexpr (DA) warp_sum_atomic(abar, A.abar);   // blocks are 32 x 8: whole warps
}

// Cotangent of the initialisation u_k^0 = M_k(u_0) (Sec. 4 preamble) folded into
// the conserved planes: ubar_0 = ubar^0 + sum_k (dM_k/du)^T pbar_k^0, with u_0
// read from the padded initial state and a^0 held fixed.
// With abar (not NULL), also the init map's part of dL/da^0: u_k^0 = M_k(u_0; a^0).
template <typename T>
__global__ void __launch_bounds__(256) k_adjoint_init(const T *init_state, int pitch, int nx,
                                                      int ny, const StepConsts<T> *kc, const T *cot, T *grad,
                                                      double *abar) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    double ab = 0.0;
    if (i < nx && j < ny) {
        const long long N = (long long)nx * ny, c = (long long)j * nx + i;
        const T w = kc->w, inv2a = kc->inv2a, gm1 = kc->gm1;
        const CellLoad<T> L{init_state, pitch};
        T u[4], wx[4], wy[4], rx[4], ry[4], ub[4], p[4][4], gr[4];
        L.u4(0, i, j, u);
        ld_group(cot + kidx(nx, 0, i, j), ub);
#pragma unroll
        for (int g = 0; g < 4; ++g) ld_group(cot + kidx(nx, 4 + 4 * g, i, j), p[g]);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            gr[q] = ub[q] + w * (p[0][q] + p[1][q] + p[2][q] + p[3][q]);
            wx[q] = (p[0][q] - p[1][q]) * inv2a;
            wy[q] = (p[2][q] - p[3][q]) * inv2a;
        }
        flux_vjp(u, gm1, 0, wx, rx);
        flux_vjp(u, gm1, 1, wy, ry);
#pragma unroll
        for (int q = 0; q < 4; ++q) grad[q * N + c] = gr[q] + (rx[q] + ry[q]);
        if (abar) {   // dM_{1,3}/da = -F/(2a^2), dM_{2,4}/da = +F/(2a^2), F = f or g
            T f[4], g[4];
            euler_fluxes(u, gm1, f, g);
            const T h = inv2a / kc->a;
#pragma unroll
            for (int q = 0; q < 4; ++q) ab -= (double)(((p[0][q] - p[1][q]) * f[q] + (p[2][q] - p[3][q]) * g[q]) * h);
        }
    }
    if (abar) warp_sum_atomic(ab, abar);
}

// ------------------------------------------------ lambda^n and its argmax cell

// Pass 1: *key = max over the cells of s (padded) of the ordered key of lambda,
// computed as the forward run's monitors compute it.
template <typename T>
__global__ void __launch_bounds__(256) k_lambda_max(const T *st, int pitch, int nx, int ny, T gamma,
                                                    unsigned long long *key) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    unsigned long long kk = 0ull;
    if (i < nx && j < ny) {
        const CellLoad<T> L{st, pitch};
        T u[4];
        L.u4(0, i, j, u);
        kk = ordered_key((double)cell_speed(u, gamma, gamma - T(1)));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, kk, off);
        kk = o > kk ? o : kk;
    }
    if ((threadIdx.x & 31) == 0 && kk) atomicMax(key, kk);
}

// Pass 2: *idx = the smallest cell index j nx + i whose lambda is the max (the
// subgradient of the max taken at one of its cells).
template <typename T>
__global__ void __launch_bounds__(256) k_lambda_argmax(const T *st, int pitch, int nx, int ny, T gamma,
                                                       const unsigned long long *key, unsigned int *idx) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= nx || j >= ny) return;
    const CellLoad<T> L{st, pitch};
    T u[4];
    L.u4(0, i, j, u);
    if (ordered_key((double)cell_speed(u, gamma, gamma - T(1))) == *key) atomicMin(idx, (unsigned)(j * nx + i));
}

// One thread: cot[q][idx] += abar * 2 / (1 - alpha) * d lambda / d u_q at the argmax
// cell (lambda = |v| + sqrt(gamma p / rho)); then the slots are reset. cot is a
// cotangent buffer of the sweep (grouped, kidx) or the caller's four planes (N cells each).
// When the prescribed boundary states' speed lam_bc exceeds every cell's (the step
// compares them the same way), lambda^n does not depend on the state: nothing is added.
template <typename T>
__global__ void k_lambda_apply(const T *st, int pitch, int nx, double gamma, double alpha,
                               double *abar, unsigned long long *key, unsigned int *idx, T *cot, long long N,
                               int grouped, const double *lam_bc) {
    const unsigned int id = *idx;
    const double ab = *abar;
    const bool bc_wins = *lam_bc > key_to_double(*key);
    *abar = 0.0;
    *key = 0ull;
    *idx = 0xffffffffu;
    if (id == 0xffffffffu || ab == 0.0 || bc_wins) return;
    const int i = (int)(id % (unsigned)nx), j = (int)(id / (unsigned)nx);
    const CellLoad<T> L{st, pitch};
    T ut[4];
    L.u4(0, i, j, ut);
    const double r = ut[0], m1 = ut[1], m2 = ut[2], E = ut[3];
    const double v1 = m1 / r, v2 = m2 / r, s2 = v1 * v1 + v2 * v2, sp = sqrt(s2);
    const double p = (gamma - 1.0) * (E - 0.5 * r * s2);
    const double c = sqrt(gamma * p / r);
    // |v|: d/dm_i = v_i / (|v| rho), d/drho = -|v| / rho (0 at rest: a subgradient)
    double g[4] = {sp > 0.0 ? -sp / r : 0.0, sp > 0.0 ? v1 / (sp * r) : 0.0, sp > 0.0 ? v2 / (sp * r) : 0.0, 0.0};
    // c = sqrt(gamma p / rho): dc = gamma / (2 c rho) (dp - p drho / rho)
    const double kc = gamma / (2.0 * c * r);
    const double dp[4] = {0.5 * (gamma - 1.0) * s2, -(gamma - 1.0) * v1, -(gamma - 1.0) * v2, gamma - 1.0};
    g[0] += kc * (dp[0] - p / r);
    for (int q = 1; q < 4; ++q) g[q] += kc * dp[q];
    const double s = ab * 2.0 / (1.0 - alpha);
    const long long cc = (long long)j * nx + i;
    for (int q = 0; q < 4; ++q) cot[grouped ? kidx(nx, q, i, j) : q * N + cc] += (T)(s * g[q]);
}

}  // namespace vlbm

namespace vlbm {

// Transpose of the ghost fill on a padded cotangent (`pad` ghost layers, (nx + 2 pad) x
// (ny + 2 pad) per plane): the cotangent of each ghost goes to the cell it was filled
// from (ZG copy, periodic copy, or mirror image with its map; a prescribed ghost
// keeps nothing). The y rule was applied last, so it is undone first. One thread
// takes every ghost of a column (y) or row (x) in turn: ghosts that share a source
// (the layers of a zero-gradient side) never add to it at the same time.
template <typename T>
__device__ __forceinline__ void fold_one(T *cot, int w, int pad, int gi, int gj, int si, int sj, bool mx, bool my) {
#pragma unroll
    for (int q = 0; q < kNPlane; ++q) {
        int src = q;   // the mirror map is a symmetric permutation with signs: its own transpose
        if (mx && q >= 4 && q < 12) src = q < 8 ? q + 4 : q - 4;
        if (my && q >= 12) src = q < 16 ? q + 4 : q - 4;
        T v = cot[kidx(w, src, gi + pad, gj + pad)];
        if ((mx && (q & 3) == 1) || (my && (q & 3) == 2)) v = -v;
        cot[kidx(w, q, si + pad, sj + pad)] += v;
    }
}

// dL/da^n of a prescribed ghost: its populations are M_k(u_field; a^n), u_field the
// field at the cell's centre at t^n (piecewise constant in t: no time derivative
// almost everywhere); dM_{1,3}/da = -F/(2a^2), dM_{2,4}/da = +F/(2a^2).
template <typename T>
__device__ __forceinline__ double prescribed_abar(const T *cot, int w, int pad, const Bound &bd, int gi, int gj,
                                                  double t, const StepConsts<T> &k) {
    T u[4], f[4], gf[4];
    field_state(bd, gi, gj, t, u);
    euler_fluxes(u, k.gm1, f, gf);
    const T h = k.inv2a / k.a;
    auto at = [&](int q) { return cot[kidx(w, q, gi + pad, gj + pad)]; };
    double ab = 0.0;
#pragma unroll
    for (int c = 0; c < 4; ++c)
        ab += (double)(((at(8 + c) - at(4 + c)) * f[c] + (at(16 + c) - at(12 + c)) * gf[c]) * h);
    return ab;
}

template <typename T>
__global__ void k_adjoint_fold_y(T *cot, int nx, int ny, int pad, Bound bd, int bc2, int bc3,
                                 const StepConsts<T> *k, const double *t, double *abar) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;   // one thread per column -pad .. nx + pad - 1
    const int w = nx + 2 * pad;
    if (tid >= w) return;
    const int gi = tid - pad;
    double ab = 0.0;
    for (int l = 0; l < 2 * pad; ++l) {
        const int gj = l < pad ? -1 - l : ny + (l - pad);
        const int s = gj < 0 ? 2 : 3;
        const int type = (s == 2 ? bc2 : bc3) >= 0 ? (s == 2 ? bc2 : bc3) : side_type(bd, s, gi);
        if (type == VLBM_BC_DIRICHLET) {
            if (abar) ab += prescribed_abar(cot, w, pad, bd, gi, gj, *t, *k);
            continue;
        }
        bool my;
        const int sj = ghost_source_typed(gj, ny, type, &my);
        fold_one(cot, w, pad, gi, gj, gi, sj, false, my);
    }
    if (abar && ab != 0.0) atomicAdd(abar, ab);
}

template <typename T>
__global__ void k_adjoint_fold_x(T *cot, int nx, int ny, int pad, Bound bd, int bc0, int bc1,
                                 const StepConsts<T> *k, const double *t, double *abar) {
    const int gj = blockIdx.x * blockDim.x + threadIdx.x;   // one thread per interior row
    if (gj >= ny) return;
    const int w = nx + 2 * pad;
    double ab = 0.0;
    for (int l = 0; l < 2 * pad; ++l) {
        const int gi = l < pad ? -1 - l : nx + (l - pad);
        const int s = gi < 0 ? 0 : 1;
        const int type = (s == 0 ? bc0 : bc1) >= 0 ? (s == 0 ? bc0 : bc1) : side_type(bd, s, gj);
        if (type == VLBM_BC_DIRICHLET) {   // (the corners the y fold moved here included)
            if (abar) ab += prescribed_abar(cot, w, pad, bd, gi, gj, *t, *k);
            continue;
        }
        bool mx;
        const int si = ghost_source_typed(gi, nx, type, &mx);
        fold_one(cot, w, pad, gi, gj, si, gj, mx, false);
    }
    if (abar && ab != 0.0) atomicAdd(abar, ab);
}

// Interior of a padded cotangent into an unpadded one.
template <typename T>
__global__ void k_adjoint_unpad(const T *cot_pad, int nx, int ny, int pad, T *cot) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= nx || j >= ny) return;
    const int w = nx + 2 * pad;
#pragma unroll
    for (int g = 0; g < kNGroup; ++g) {
        T v[4];
        ld_group(cot_pad + kidx(w, 4 * g, i + pad, j + pad), v);
        st_group(cot + kidx(nx, 4 * g, i, j), v[0], v[1], v[2], v[3]);
    }
}

// The sweep's first cotangent: dL/du^N (the caller's four planes) in group 0 of every
// cell, zero population cotangents.
template <typename T>
__global__ void k_adjoint_seed(const T *dLduN, int nx, int ny, T *cot) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= nx || j >= ny) return;
    const long long N = (long long)nx * ny, c = (long long)j * nx + i;
    st_group(cot + kidx(nx, 0, i, j), dLduN[c], dLduN[N + c], dLduN[2 * N + c], dLduN[3 * N + c]);
#pragma unroll
    for (int g = 1; g < kNGroup; ++g) st_group(cot + kidx(nx, 4 * g, i, j), T(0), T(0), T(0), T(0));
}

}  // namespace vlbm
