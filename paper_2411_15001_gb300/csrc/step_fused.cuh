// step_fused.cuh -- one blended collide + limit + stream step as a single
// row-marching pass: every cell's 20 values are read from HBM once and written
// once, together with the ghost images of the boundary cells.
//
// Work. A grid is cut into strips of at most kFusedOut = 124 output columns (even
// widths, strip_of) and bands of rows; a work item is one (instance, strip, band),
// listed by the host in the order CTAs take them (tall bands first under guided
// scheduling). Persistent CTAs of kFB = 128 threads (one column each: two halo
// columns on either side of the strip, the radius of the LMP stencil) take items
// from a global counter, so items that cost more (faces whose
// theta_p needs the FP64 solve cluster on shocks) do not hold up the step. One
// launch can advance many independent grids (a batch); each grid has its own
// kinetic speed, control block and completion count, and the CTA that finishes a
// grid's last item runs that grid's end-of-step reduction.
//
// Rows arrive by TMA (two boxes of 64 columns x 5 groups of 4 values per row, see the
// state layout in vlbm_internal.h) into a 3-slot ring completed on mbarriers. Per row R
// (output row O = R - lag: lag 1 for PP and the fixed thetas, lag 2 for LMP / RLMP,
// whose bounds have the radius-2 stencil of eq. LMP_minmax):
//  P1  fluxes, Maxwellians, non-equilibrium parts d_k of row R; what x-neighbours
//      need (u, f, d_1, d_2) goes to a shared ring of lag + 2 rows, what only the own
//      column needs (g, d_3, d_4; its u is read back from the ring) to a register
//      history; rho* of y-face R - 1/2.
//  P2  density bounds of row R - 1 (LMP/RLMP).
//  P3  PP and the fixed thetas: u*, dF and theta of the x-face of row R and of y-face
//      R - 1/2 (Sec. 3.3-3.4). LMP / RLMP: theta of the x-faces of row R - 1 and of
//      y-face R - 3/2, their face states formed again there.
// Barriers: S1 after P1 (the ring row R and the previous row's theta are
// complete); the bounds a thread needs of its right neighbour (LMP / RLMP) it forms
// itself from the shared rows.
//  P4  collide + stream of row O (eq. blending_u1 / blending_u), stores, ghost
//      images, monitors.
// Strips start on even columns, so no 32-byte sector of a group row is written
// partially by two CTAs; a cell's group goes out as one vector store.
#pragma once

#include "common.cuh"
#include "tma.cuh"

namespace vlbm {

constexpr int kFB = kFusedBox;     // threads per CTA = TMA box width (columns)
constexpr int kFHalo = kFusedHalo; // box columns left (and right) of the strip
constexpr int kRawSlots = 3;   // TMA row ring

// The output row of row iteration R is R - lag: 1 for PP and the fixed thetas, 2
// for LMP / RLMP (the bounds of a cell need the row above it).
__host__ __device__ constexpr int fused_lag(int limiter) {
    return limiter == VLBM_LIM_LMP || limiter == VLBM_LIM_RLMP ? 2 : 1;
}

template <typename T, int LAG>
struct FusedSmem {
    static constexpr int kX = LAG + 2;          // rows R - LAG .. R in use, one being refilled
    T raw[kRawSlots][2][kNGroup][kFB / 2][4];   // [slot][half of the strip][group][column][component]
    T X[kX][16][kFB];          // u (0..3), f (4..7), d_1 (8..11), d_2 (12..15)
    T rsx[LAG == 2 ? 2 : 1][kFB];   // LMP / RLMP: rho* of x-face (b, b+1), by row R & 1
    T thx[2][kFB];             // theta of x-face (b, b+1): PP by row R & 1, LMP / RLMP by (R - 1) & 1
    unsigned long long bar[kRawSlots];
    int item;
    int abort;
};

// Register history of the own column; u is kept only for the row just loaded (rows
// before it read theirs back from the shared ring).
template <typename T>
struct Hist {
    T u[4], g[4], d3[4], d4[4];
};

template <typename T, int LIM>
struct FusedCtx {
    static constexpr int kLag = fused_lag(LIM);
    static constexpr int kX = kLag + 2;
    FusedSmem<T, kLag> &S;
    const CUtensorMap *tmap;
    const Geo &D;
    const StepConsts<T> &k;
    T *__restrict__ out;
    Monitor<T> &mon;
    int b, zin;
    uint32_t &nissued, &nconsumed;
    int xb, xpad, c, y0, y1, R1, wout;   // strip: box origin, padded origin, own column, rows, width
    // PP and the fixed thetas form the faces of row R (x-face c+1/2, y-face R-1/2) in
    // row R and limit them there, so row R - 1 is complete (output lag 1; one theta of
    // a y-face crosses rows). LMP / RLMP need the density bounds of both cells of a
    // face, complete one row later, so they limit the faces of row R-1 in row R,
    // recomputing the face states there (output lag 2).
    static constexpr bool kRecompute = LIM == VLBM_LIM_LMP || LIM == VLBM_LIM_RLMP;
    T xs_us[4], xs_df[4];   // LMP / RLMP: x-face (c+1/2) of row R-1
    T ys_us[4], ys_df[4];   // LMP / RLMP: y-face between rows R-2 and R-1
    T rsy_prev;             // rho* of the y-face between rows R-2 and R-1
    T mu2, nu2;             // bounds of row R-2 (own column)
    T thy_prev;             // LMP / RLMP: theta of the y-face between rows R-3 and R-2
    T ty1;                  // PP: theta of the y-face (R-2, R-1)
    Hist<T> h1, h2;         // rows R-1, R-2 of the own column (h2: LMP / RLMP; their u unused)
    T p3n[4];               // u_3 of the next output row after the step (pulled from the one below)

    // Slot of row R (>= -2) in the shared ring X.
    static __device__ __forceinline__ int xslot(int R) { return (R + 2 * kX) % kX; }

    // The grid's descriptor (the tensor map is its first member).
    __device__ __forceinline__ const InstDesc<T> *desc() const {
        return reinterpret_cast<const InstDesc<T> *>(tmap);
    }

    __device__ __forceinline__ void issue(int row) {
        const int slot = nissued % kRawSlots;
        mbar_expect_tx(&S.bar[slot], (uint32_t)(kNPlane * kFB * sizeof(T)));
        tma_load_4d(&S.raw[slot][0][0][0][0], tmap, &S.bar[slot], 4 * xpad, 0, row + kOY, zin);
        tma_load_4d(&S.raw[slot][1][0][0][0], tmap, &S.bar[slot], 4 * (xpad + kFB / 2), 0, row + kOY, zin);
        ++nissued;
    }

    // The history before row R0 (the item's first): a neutral row. The own column's u of
    // earlier rows is read back from the shared ring (the same values P1 stored there),
    // so the ring slot of row R0 - 1 gets u = 1 in the own column.
    __device__ __forceinline__ void reset_state(int R0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            xs_us[q] = xs_df[q] = ys_us[q] = ys_df[q] = T(0);
            S.X[xslot(R0 - 1)][q][b] = T(1);
            h1.g[q] = h2.g[q] = T(0);
            h1.d3[q] = h2.d3[q] = T(0);
            h1.d4[q] = h2.d4[q] = T(0);
            p3n[q] = T(0);
        }
        rsy_prev = mu2 = nu2 = thy_prev = ty1 = T(0);
    }

    // P1 of row R (see the file comment); returns rho* of the y-face R - 1/2. f and d1
    // receive the own column's x-flux and d_1 (also in the shared ring) for next_faces.
    __device__ __forceinline__ T p1(int R, Hist<T> &h0, T f[4], T d1[4]) {
        const int slot = nconsumed % kRawSlots;
        const uint32_t par = (nconsumed / kRawSlots) & 1u;
        ++nconsumed;
        if (!mbar_wait_bounded(&S.bar[slot], par)) S.abort = 1;
        T u[4], g[4], M1[4], M2[4], M3[4], M4[4], pv[4];
        ld_group(&S.raw[slot][b >> 6][0][b & 63][0], u);
        euler_fluxes(u, k.gm1, f, g);
        maxwell_pm(u, f, k, M1, M2);
        maxwell_pm(u, g, k, M3, M4);
        const int xs = xslot(R);
        // each population group is read right where its non-equilibrium part is formed
        ld_group(&S.raw[slot][b >> 6][1][b & 63][0], pv);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            S.X[xs][q][b] = u[q];
            S.X[xs][4 + q][b] = f[q];
            d1[q] = RN<T>::sub(M1[q], pv[q]);
            S.X[xs][8 + q][b] = d1[q];
        }
        ld_group(&S.raw[slot][b >> 6][2][b & 63][0], pv);
#pragma unroll
        for (int q = 0; q < 4; ++q) S.X[xs][12 + q][b] = RN<T>::sub(M2[q], pv[q]);   // d_2
        ld_group(&S.raw[slot][b >> 6][3][b & 63][0], pv);
#pragma unroll
        for (int q = 0; q < 4; ++q) h0.d3[q] = RN<T>::sub(M3[q], pv[q]);
        ld_group(&S.raw[slot][b >> 6][4][b & 63][0], pv);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            h0.d4[q] = RN<T>::sub(M4[q], pv[q]);
            h0.u[q] = u[q];
            h0.g[q] = g[q];
        }
        return face_star(S.X[xslot(R - 1)][0][b], h1.g[0], u[0], g[0], k);  // y-face R - 1/2
    }

    // Face states of the x-face (b, b+1) of row R and of the y-face R - 1/2 (PP and the
    // fixed thetas); the own column's u, x-flux and d_1 from registers, the right
    // neighbour's from the shared ring.
    __device__ __forceinline__ void row_faces(int R, const Hist<T> &h0, T rsy_new, int br, const T f[4],
                                              const T d1[4], T xus[4], T xdf[4], T yus[4], T ydf[4]) const {
        const int xs = xslot(R);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            xus[q] = face_star(h0.u[q], f[q], S.X[xs][q][br], S.X[xs][4 + q][br], k);
            xdf[q] = face_dflux(d1[q], S.X[xs][12 + q][br], k);
            yus[q] = q == 0 ? rsy_new : face_star(S.X[xslot(R - 1)][q][b], h1.g[q], h0.u[q], h0.g[q], k);
            ydf[q] = face_dflux(h1.d3[q], h0.d4[q], k);
        }
    }

    // PP and the fixed thetas: theta of the x-face (c, c+1) of row R (stored in the
    // shared slot R & 1 for the neighbours) and of the y-face (R - 1, R) of the own
    // column (returned), from their face states, with the sponge layer.
    __device__ __forceinline__ T row_thetas(int R, const T xus[4], const T xdf[4], const T yus[4],
                                            const T ydf[4]) {
        T tx, ty;
        // theta is needed for the x-faces of columns kFHalo-1 .. kFHalo+wout-1 and the
        // y-faces of the strip's own columns, inside the grid. The other threads hold
        // halo padding or (past the last column) TMA fill, on which the FP32 screen
        // would fail and send the face to the FP64 solve: they skip theta.
        const bool live = b >= kFHalo - 1 && b < kFHalo + wout && c < D.nx;
        if (LIM == VLBM_LIM_FIRST_ORDER) {
            tx = ty = T(0);
        } else if (LIM == VLBM_LIM_NONE) {
            tx = ty = T(1);
        } else if (!live) {
            tx = ty = T(0);
        } else {
            unsigned int nx64 = 0, ny64 = 0;
            tx = combine_theta(pp_density_target(xus[0], xdf[0], k), xus, xdf, k, nx64);
            ty = combine_theta(pp_density_target(yus[0], ydf[0], k), yus, ydf, k, ny64);
            // faces counted once: an x-face by the cell west of it, a y-face by the one south of it
            const bool col_own = b >= kFHalo && b < kFHalo + wout && c < D.nx;
            if (col_own && R >= y0 && R < y1) mon.fp64 += nx64;
            if (col_own && R - 1 >= y0 && R - 1 < y1) mon.fp64 += ny64;
        }
        if (D.sponge > 0) {   // sponge layer (Sec. 4.2): theta = 0 on the faces of layer cells
            const Sponge sp(D.sponge, D.nx, D.ny, D.bc);
            const bool c0 = sp.cell(c, R);
            if (c0 || sp.cell(c + 1, R)) tx = T(0);        // x-face (c, c+1) of row R
            if (c0 || sp.cell(c, R - 1)) ty = T(0);        // y-face (R-1, R) of column c
        }
        S.thx[R & 1][b] = tx;
        return ty;
    }

    // LMP density bounds (eq. LMP_minmax): min / max of rho of a cell and rho* of its
    // west, east, south and north faces (exact), RLMP scaled (Sec. 3.3.2).
    __device__ __forceinline__ void minmax5(T v0, T v1, T v2, T v3, T v4, T &mu, T &nu) const {
        mu = fmin(fmin(fmin(v0, v1), fmin(v2, v3)), v4);
        nu = fmax(fmax(fmax(v0, v1), fmax(v2, v3)), v4);
        if (LIM == VLBM_LIM_RLMP) {
            mu = RN<T>::mul(mu, T(0.999));
            nu = RN<T>::mul(nu, T(1.001));
        }
    }

    // Bounds of row R - 1, own column.
    __device__ __forceinline__ void bounds(int R, T rsy_new, int bl, T &mu, T &nu) const {
        const int rp = (R - 1) & 1;
        minmax5(S.X[xslot(R - 1)][0][b], S.rsx[rp][bl], S.rsx[rp][b], rsy_prev, rsy_new, mu, nu);
    }

    // Bounds of row R - 1 of the column to the right (br), from the shared rows R - 2 ..
    // R (rho and the y-momentum, the y-flux of rho) and the x-faces' rho*: the same
    // operations on the same values as that column's own thread, so the same bits,
    // without a barrier to publish them.
    __device__ __forceinline__ void bounds_right(int R, int br, T &mu, T &nu) const {
        const int rp = (R - 1) & 1, x0 = xslot(R - 2), x1 = xslot(R - 1), x2 = xslot(R);
        const T r1 = S.X[x1][0][br], m1 = S.X[x1][2][br];
        const T syp = face_star(S.X[x0][0][br], S.X[x0][2][br], r1, m1, k);
        const T syn = face_star(r1, m1, S.X[x2][0][br], S.X[x2][2][br], k);
        minmax5(r1, S.rsx[rp][b], S.rsx[rp][br], syp, syn, mu, nu);
    }

    // The rows of an item before row y0 + 1: no output row of the item uses their
    // collide (rows below y0 - 1), so they only load the row and form what the next
    // rows read -- the thetas of their faces (PP and the fixed thetas) or rho* of the
    // x-faces and, in row y0, the bounds of row y0 - 1 (LMP / RLMP).
    __device__ __forceinline__ bool row_warm(int R) {
        Hist<T> h0;
        T fo[4], d1o[4];
        const T rsy_new = p1(R, h0, fo, d1o);
        __syncthreads();                                                  // S1
        if (S.abort) return false;
        if (b == 0 && R + kRawSlots <= R1) issue(R + kRawSlots);
        const int bl = b > 0 ? b - 1 : 0, br = b < kFB - 1 ? b + 1 : b;
        if constexpr (kRecompute) {
            bounds(R, rsy_new, bl, mu2, nu2);
            const int xs = xslot(R);
            S.rsx[R & 1][b] = face_star(h0.u[0], S.X[xs][4][b], S.X[xs][0][br], S.X[xs][4][br], k);
            h2 = h1;
        } else {
            T xus[4], xdf[4], yus[4], ydf[4];
            row_faces(R, h0, rsy_new, br, fo, d1o, xus, xdf, yus, ydf);
            ty1 = row_thetas(R, xus, xdf, yus, ydf);
        }
        rsy_prev = rsy_new;
        h1 = h0;
        return true;
    }

    // LMP / RLMP: theta of the x-face (c, c+1) of row R - 1 and of the y-face (R - 2, R - 1)
    // of the own column (P3), with the sponge layer; (mu1, nu1) and (muR, nuR) are the
    // density bounds of row R - 1 of the own column and of the one to the right.
    __device__ __forceinline__ void thetas(int R, int br, T mu1, T nu1, T muR, T nuR, T &tx, T &ty) {
        // theta is needed for the x-faces of columns kFHalo-1 .. kFHalo+wout-1 and the
        // y-faces of the strip's own columns, inside the grid. The other threads hold
        // halo padding or (past the last column) TMA fill, on which the FP32 screen
        // would fail and send the face to the FP64 solve: they skip theta.
        const bool live = b >= kFHalo - 1 && b < kFHalo + wout && c < D.nx;
        if (LIM == VLBM_LIM_FIRST_ORDER) {
            tx = ty = T(0);
        } else if (LIM == VLBM_LIM_NONE) {
            tx = ty = T(1);
        } else if (!live) {
            tx = ty = T(0);
        } else {
            {
                const int xp = xslot(R - 1);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    xs_us[q] = face_star(S.X[xp][q][b], S.X[xp][4 + q][b], S.X[xp][q][br], S.X[xp][4 + q][br], k);
                    xs_df[q] = face_dflux(S.X[xp][8 + q][b], S.X[xp][12 + q][br], k);
                    ys_us[q] = q == 0 ? rsy_prev
                                      : face_star(S.X[xslot(R - 2)][q][b], h2.g[q], S.X[xp][q][b], h1.g[q], k);
                    ys_df[q] = face_dflux(h2.d3[q], h1.d4[q], k);
                }
            }
            const T trx = theta_rho_lmp(xs_us[0], xs_df[0], mu1, nu1, muR, nuR, k);
            const T try_ = theta_rho_lmp(ys_us[0], ys_df[0], mu2, nu2, mu1, nu1, k);
            unsigned int nx64 = 0, ny64 = 0;
            tx = combine_theta(trx, xs_us, xs_df, k, nx64);
            ty = combine_theta(try_, ys_us, ys_df, k, ny64);
            // faces counted once: an x-face by the cell west of it, a y-face by the one south of it
            const bool col_own = b >= kFHalo && b < kFHalo + wout && c < D.nx;
            if (col_own && R - 1 >= y0 && R - 1 < y1) mon.fp64 += nx64;
            if (col_own && R - 2 >= y0 && R - 2 < y1) mon.fp64 += ny64;
        }
        if (D.sponge > 0) {   // sponge layer (Sec. 4.2): theta = 0 on the faces of layer cells
            const Sponge sp(D.sponge, D.nx, D.ny, D.bc);
            const bool c1 = sp.cell(c, R - 1);
            if (c1 || sp.cell(c + 1, R - 1)) tx = T(0);        // x-face (c, c+1) of row R-1
            if (c1 || sp.cell(c, R - 2)) ty = T(0);            // y-face (R-2, R-1) of column c
        }
    }

    // One row iteration; returns false if a wait timed out (the CTA then stops).
    __device__ __forceinline__ bool row(int R) {
        Hist<T> h0;
        T fo[4], d1o[4];
        // ---------------------------------------------------------------- P1
        const T rsy_new = p1(R, h0, fo, d1o);
        const int bl = b > 0 ? b - 1 : 0, br = b < kFB - 1 ? b + 1 : b;
        __syncthreads();                                                  // S1
        if (S.abort) return false;
        if (b == 0 && R + kRawSlots <= R1) issue(R + kRawSlots);
        T tw, te, ts, tn;   // thetas of the west, east, south and north faces of row O
        if constexpr (kRecompute) {
            // -------------------------------------------------------- P2
            T mu1, nu1, muR, nuR, tx, ty;
            bounds(R, rsy_new, bl, mu1, nu1);
            bounds_right(R, br, muR, nuR);
            // -------------------------------------------------------- P3
            thetas(R, br, mu1, nu1, muR, nuR, tx, ty);
            S.thx[(R - 1) & 1][b] = tx;
            mu2 = mu1;
            nu2 = nu1;
            // rho* of the x-face (b, b+1) of row R, for the next row's density bounds
            const int xs = xslot(R);
            S.rsx[R & 1][b] = face_star(h0.u[0], S.X[xs][4][b], S.X[xs][0][br], S.X[xs][4][br], k);
            tw = S.thx[(R - 2) & 1][bl];
            te = S.thx[(R - 2) & 1][b];
            ts = thy_prev;
            tn = ty;
            thy_prev = ty;
        } else {
            // -------------------------------------------------------- P3
            T xus[4], xdf[4], yus[4], ydf[4];
            row_faces(R, h0, rsy_new, br, fo, d1o, xus, xdf, yus, ydf);
            const T ty = row_thetas(R, xus, xdf, yus, ydf);
            tw = S.thx[(R - 1) & 1][bl];
            te = S.thx[(R - 1) & 1][b];
            ts = ty1;
            tn = ty;
            ty1 = ty;
        }
        rsy_prev = rsy_new;
        // No barrier before P4: it reads theta of row O's x-faces (written one row ago)
        // and the ring row O, ordered by this row's S1; every slot this row's P3 writes
        // is read only after the next row's S1, and every slot the next row overwrites
        // is read here before this thread reaches that S1.
        // ---------------------------------------------------------------- P4
        // row O and the row above it: g, d_3, d_4 in the register history (LMP / RLMP:
        // h2, h1; PP and the fixed thetas: h1 and the row just loaded), u in the ring
        const int O = R - kLag;
        const int xo = xslot(O);
        const Hist<T> &hc = kRecompute ? h2 : h1;
        const Hist<T> &hn = kRecompute ? h1 : h0;
        T nv[kNPlane];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const T M1W = maxwell_plus(S.X[xo][q][bl], S.X[xo][4 + q][bl], k);
            const T M2E = maxwell_minus(S.X[xo][q][br], S.X[xo][4 + q][br], k);
            const T M4N = maxwell_minus(kRecompute ? S.X[xslot(R - 1)][q][b] : h0.u[q], hn.g[q], k);
            nv[4 + q] = blend_pop(M1W, S.X[xo][8 + q][bl], tw);
            nv[8 + q] = blend_pop(M2E, S.X[xo][12 + q][br], te);
            nv[12 + q] = p3n[q];
            nv[16 + q] = blend_pop(M4N, hn.d4[q], tn);
            nv[q] = blend_u(nv[4 + q], nv[8 + q], nv[12 + q], nv[16 + q], S.X[xo][q][b], tw, S.X[xo][12 + q][b],
                            te, S.X[xo][8 + q][b], ts, hc.d4[q], tn, hc.d3[q], k);
            // u_3 of row O + 1 after the step, pulled from row O with theta of y-face O + 1/2
            p3n[q] = blend_pop(maxwell_plus(S.X[xo][q][b], hc.g[q], k), hc.d3[q], tn);
        }
        if (O >= y0 && O < y1 && b >= kFHalo && b < kFHalo + wout && c < D.nx) {
            T *base = out + sidx(D.pitch, 0, c, O);
#pragma unroll
            for (int g = 0; g < kNGroup; ++g)
                st_group(base + (long long)g * 4 * D.pitch, nv[4 * g], nv[4 * g + 1], nv[4 * g + 2], nv[4 * g + 3]);
            if (c < 2 || c >= D.nx - 2 || O < 2 || O >= D.ny - 2) write_ghost_images(D, out, c, O, nv, &desc()->bd);
            mon.add_cell(nv, k.gamma, k.gm1);
        }
        // shift the register history
        if constexpr (kRecompute) h2 = h1;
        h1 = h0;
        return true;
    }
};

// Wait (bounded) for this CTA's loads still in flight before it exits.
template <typename SM>
__device__ void drain_loads(SM &S, uint32_t nissued, uint32_t nconsumed) {
    if (threadIdx.x == 0) {
        while (nconsumed < nissued) {
            const int slot = nconsumed % kRawSlots;
            mbar_wait_bounded(&S.bar[slot], (nconsumed / kRawSlots) & 1u, 500000000ull);
            ++nconsumed;
        }
    }
}

// PROBE: the instantiation that vlbm_test_wait_probe selects (the others carry no
// probe code): before any load, every CTA makes a bounded wait on a barrier that no
// copy and no thread completes; it runs out and the CTA takes the timeout path below.
// Registers: three CTAs of 128 threads per SM (shared memory allows no more); PP and the
// fixed thetas held to 144 registers, where they run 1 % faster than at the 154 the
// compiler picks by itself (no spills either way).
template <typename T, int LIM, bool PROBE = false>
__global__ void __launch_bounds__(kFB, sizeof(T) == 4 ? 3 : 1) __maxnreg__(sizeof(T) == 4 && fused_lag(LIM) == 1 ? 144 : 255)
    k_step_fused(FusedBatchArgs<T> B) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    constexpr int kLag = fused_lag(LIM);
    FusedSmem<T, kLag> &S = *reinterpret_cast<FusedSmem<T, kLag> *>(smem_raw);
    const int b = threadIdx.x;
    // TMA destinations must be 128-byte aligned; dynamic shared memory follows
    // the static block of the reductions, so check rather than assume.
    if (smem_addr(&S.raw[0][0][0][0][0]) & 127u) {
        if (b == 0) atomicCAS(&B.insts[0].ctl->status, 0, VLBM_E_UNSUPPORTED);
        return;
    }
    if (b == 0) {
        for (int s = 0; s < kRawSlots; ++s) mbar_init(&S.bar[s], 1);
        S.abort = 0;
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t nissued = 0, nconsumed = 0;
    bool ok = true;
    if constexpr (PROBE) {
        const unsigned int probe = B.insts[0].ctl->wait_probe_ns;
        if (b == 0 && !mbar_wait_bounded(&S.bar[0], 0u, probe > 0u ? probe : 1u)) S.abort = 1;
        __syncthreads();
        ok = S.abort == 0;
    }
    if (ok) for (;;) {
        if (b == 0) S.item = (int)atomicAdd(&B.bctl->work, 1u);
        __syncthreads();
        const int item = S.item;
        __syncthreads();
        if (item >= B.nitems) break;
        const WorkItem it = B.items[item];
        const InstDesc<T> &D = B.insts[it.inst];
        DevCtl *C = D.ctl;
        if (C->done) continue;
        Geo geo;
        geo.pitch = D.pitch;
        geo.nx = D.nx;
        geo.ny = D.ny;
        for (int q = 0; q < 4; ++q) geo.bc[q] = D.bc[q];
        geo.sponge = D.sponge;
        const long long n = C->n;
        const StepConsts<T> k = consts_of<T>(C);
        Monitor<T> mon;
        mon.init();
        FusedCtx<T, LIM> X{S, &D.tmap, geo, k, (n & 1) ? D.buf0 : D.buf1, mon, b, (n & 1) ? 1 : 0,
                           nissued, nconsumed};
        X.y0 = it.y0;
        X.y1 = it.y1;
        X.wout = (int)((unsigned)it.xw >> 24);
        X.xb = (it.xw & 0xffffff) - kFHalo;
        X.xpad = X.xb + kOX;
        X.c = X.xb + b;
        // rows y0 - lag .. y1 + lag - 1 (output rows y0 - 1 .. y1 - 1): LMP / RLMP start
        // at row y0 - 2 (the bounds of row y0 - 1 need rho* of the y-face y0 - 3/2),
        // the others at y0 - 1; rows before y0 + lag - 1 only load and form faces
        const int R0 = X.y0 - kLag;
        X.R1 = X.y1 + kLag - 1;
        if (b == 0)
            for (int r = R0; r < R0 + kRawSlots && r <= X.R1; ++r) X.issue(r);
        X.reset_state(R0);
        int R = R0;
        for (; R < X.y0 + kLag - 1 && ok; ++R) ok = X.row_warm(R);
        for (; R <= X.R1 && ok; ++R) ok = X.row(R);
        if (!ok) break;
        // the item's monitors go to its grid; the CTA finishing the grid's last item
        // ends that grid's step
        block_publish(mon, C);
        if (last_block(C, (unsigned)D.nitems)) {
            if (b == 0) finalize_step(C);
        }
    }
    if (!ok) {
        drain_loads(S, nissued, nconsumed);
        if (b == 0) atomicCAS(&B.insts[0].ctl->status, 0, VLBM_E_TIMEOUT);
        // keep fetching so that the counter reaches the end before the reset below
        for (;;) {
            if (b == 0) S.item = (int)atomicAdd(&B.bctl->work, 1u);
            __syncthreads();
            const int item = S.item;
            __syncthreads();
            if (item >= B.nitems) break;
        }
    }
    // the last CTA to leave resets the work counter for the next launch
    if (b == 0) {
        __threadfence();
        if (atomicAdd(&B.bctl->ctas_done, 1u) == gridDim.x - 1) {
            B.bctl->work = 0u;
            B.bctl->ctas_done = 0u;
            __threadfence();
        }
    }
}

}  // namespace vlbm
