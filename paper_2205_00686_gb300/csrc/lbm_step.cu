// Fused coupled time step: D2Q9 MRT pseudopotential flow lattice (Section 2)
// + D2Q5 MRT temperature lattice with the rho c_v-weighted streaming
// (Section 3.2, Eq. 39), one launch per time step.
//
// Work decomposition.  A CTA of NT threads owns a strip of W = NT - 8 output
// columns and sweeps a segment of rows from bottom to top; thread t handles
// window column X = x0 - 4 + t at every stage.  Each output row needs data
// three rows / columns away (psi at depth 3 -> F_m and u at depth 2 -> div u
// and both collisions at depth 1 -> pull streaming), so the sweep runs four
// stages skewed in rows and keeps each stage's results in small shared-memory
// rings three rows deep:
//
//   phase alpha of iteration k:  A(k)    load f, g, P of row k; rho, T, j, psi
//                                C(k-3)  div u, grad T (Eqs. 49-50), Q, S,
//                                        D2Q5 collision -> g*
//                                D9(k-3) pull-stream f* into row k-3, store
//   phase beta of iteration k:   B(k-1)  F_m (Eq. 9), F_b, u (Eq. 11),
//                                        D2Q9 collision (Eqs. 5, 8) -> f*
//                                D5(k-4) weighted streaming of g* into row
//                                        k-4 (Eq. 39), store
//
// with one __syncthreads() after each phase.  Every population is read from
// HBM once per step (plus a 4-column halo per strip and a 3-row halo per
// segment, served mostly by L2) and written once.  There are no tensor-core
// contractions here: the step is a bandwidth-bound stencil.
//
// The CTAs are persistent and pull (domain, strip, segment) units from an
// atomic counter, so one launch serves one domain or hundreds of domains of
// uneven size; the last CTA to finish advances every domain's device-side
// step counter, clears the next slot of its density-sum ring and resets the
// counter, which makes the launch replayable inside a CUDA graph.  No CTA
// ever waits on another.
#include "lbm_internal.cuh"

namespace lbm {

template <class R, int NT>
struct StepSmem {
    R psi[3][NT];
    R rho[3][NT];
    R T[3][NT];
    R ux[3][NT];
    R uy[3][NT];
    R fs[3][9][NT];    // post-collision f (deviation form)
    R gs[3][5][NT];    // post-collision g (deviation form)
    R own[5][7][NT];   // per column: g_dev[5], rho, P^{n-1} of the row
    double red[NT / 32];
    int unit;
};

__device__ __forceinline__ int slot3(int r) { return (r + 6) % 3; }
__device__ __forceinline__ int slot5(int r) { return (r + 10) % 5; }

template <int PREC, int NT>
__device__ __forceinline__ void process_unit(const Inst& I, const Unit& U,
                                             const Phys<typename Types<PREC>::R>& P,
                                             StepSmem<typename Types<PREC>::R, NT>& S) {
    typedef typename Types<PREC>::R R;
    typedef typename Types<PREC>::TF TF;
    typedef typename Types<PREC>::TG TG;

    const int t = threadIdx.x;
    const int nx = I.nx, ny = I.ny, pitch = I.pitch;
    const bool perx = I.flow[EW] == PERIODIC;
    const bool pery = I.flow[ES] == PERIODIC;
    const long long step = __ldcg(&I.ctl->step);
    const int par = (int)(step & 1);
    const bool first = step == 0;
    const size_t plane = (size_t)ny * pitch;
    const TF* __restrict__ fsrc = (const TF*)I.f[par];
    const TG* __restrict__ gsrc = (const TG*)I.g[par];
    const R* __restrict__ Psrc = (const R*)I.P[par];
    TF* __restrict__ fdst = (TF*)I.f[par ^ 1];
    TG* __restrict__ gdst = (TG*)I.g[par ^ 1];
    R* __restrict__ Pdst = (R*)I.P[par ^ 1];
    const R rho_ref = (R)I.rho_ref;
    const R T_ref = (R)I.T_ref;
    const bool use_mass = P.gravity != R(0);
    const R rho_ave = use_mass ? (R)(__ldcg(&I.ctl->mass[(step + 2) % 3]) * I.inv_n) : R(0);
    const R cot = (R)I.cot_theta;
    const int y0 = U.y0, y1 = U.y1, x0 = U.x0, x1 = U.x1;
    const bool wallS = I.flow[ES] == WALL, wallN = I.flow[EN] == WALL;

    // ---- column bookkeeping (fixed for the unit)
    const int X = x0 - 4 + t;
    const bool colvalid = perx || (X >= 0 && X < nx);
    const int gx = perx ? wrapi(X, nx) : X;
    auto extx = [&](int Xp) { return perx ? Xp : min(max(Xp, 0), nx - 1); };
    auto sidx = [&](int Xp) { return extx(Xp) - x0 + 4; };
    auto gcol = [&](int c) { return perx ? wrapi(x0 - 4 + c, nx) : x0 - 4 + c; };
    const int xl1 = sidx(X - 1), xr1 = sidx(X + 1);
    const int cLL = sidx(extx(X - 1) - 1), cLR = sidx(extx(X - 1) + 1);
    const int cRL = sidx(extx(X + 1) - 1), cRR = sidx(extx(X + 1) + 1);
    const bool inB = colvalid && X >= x0 - 2 && X < x1 + 2;
    const bool inC = colvalid && X >= x0 - 1 && X < x1 + 1;
    const bool inD = X >= x0 && X < x1;
    const bool left_edge = !perx && X == 0;
    const bool right_edge = !perx && X == nx - 1;

    auto rowvalid = [&](int r) { return pery || (r >= 0 && r < ny); };
    auto grow = [&](int r) { return pery ? wrapi(r, ny) : r; };

    // registers carried from A(k-1) to B(k-1)
    R fp[9], rhop = R(1), rhodp = R(0), jxp = R(0), jyp = R(0), Tp = R(0), psip = R(0);
#pragma unroll
    for (int q = 0; q < 9; ++q) fp[q] = R(0);
    double mass_acc = 0.0;
    int errbits = 0;

    for (int k = y0 - 3; k <= y1 + 3; ++k) {
        // ================= phase alpha =================
        const bool doA = k < y1 + 3 && rowvalid(k);
        R fa[9], ga[5], pa = R(0);
#pragma unroll
        for (int q = 0; q < 9; ++q) fa[q] = R(0);
#pragma unroll
        for (int q = 0; q < 5; ++q) ga[q] = R(0);
        if (doA && colvalid) {
            const size_t off = (size_t)grow(k) * pitch + gx;
#pragma unroll
            for (int q = 0; q < 9; ++q) fa[q] = (R)ld_st(fsrc + q * plane + off);
#pragma unroll
            for (int q = 0; q < 5; ++q) ga[q] = (R)ld_st(gsrc + q * plane + off);
            pa = ld_st(Psrc + off);
        }

        // ---- C(k-3): div u, grad T, Q, S and the D2Q5 MRT collision (Eq. 39)
        {
            const int r = k - 3;
            if (r >= y0 - 1 && r < y1 + 1 && rowvalid(r) && inC) {
                const int so = slot5(r);
                R gd[5];
#pragma unroll
                for (int q = 0; q < 5; ++q) gd[q] = S.own[so][q][t];
                const R rho = S.own[so][5][t];
                const R Pp = S.own[so][6][t];
                const R Td = gd[0] + gd[1] + gd[2] + gd[3] + gd[4];
                const R T = Td + T_ref;
                const R m1 = gd[1] - gd[3];
                const R m2 = gd[2] - gd[4];
                const R m3d = gd[1] + gd[2] + gd[3] + gd[4];
                const R m4 = gd[1] - gd[2] + gd[3] - gd[4];
                // Eqs. 49-50: c_s^2 d_x T = -varsigma_1 m_1^(1), m_1^eq = 0
                const R dTx = -P.vs1_cs2h * m1;
                const R dTy = -P.vs1_cs2h * m2;
                const int sc = slot3(r), sd = slot3(r - 1), su = slot3(r + 1);
                const R uxc = S.ux[sc][t], uyc = S.uy[sc][t];
                // neighbour rows: solid -> u = 0, open -> the boundary row
                R uxS0, uxS1, uxS2, uyS0, uyS1, uyS2, uxN0, uxN1, uxN2, uyN0, uyN1, uyN2;
                if (rowvalid(r - 1) || !wallS) {
                    const int s = rowvalid(r - 1) ? sd : sc;
                    uxS0 = S.ux[s][xl1]; uxS1 = S.ux[s][t]; uxS2 = S.ux[s][xr1];
                    uyS0 = S.uy[s][xl1]; uyS1 = S.uy[s][t]; uyS2 = S.uy[s][xr1];
                } else {
                    uxS0 = uxS1 = uxS2 = uyS0 = uyS1 = uyS2 = R(0);
                }
                if (rowvalid(r + 1) || !wallN) {
                    const int s = rowvalid(r + 1) ? su : sc;
                    uxN0 = S.ux[s][xl1]; uxN1 = S.ux[s][t]; uxN2 = S.ux[s][xr1];
                    uyN0 = S.uy[s][xl1]; uyN1 = S.uy[s][t]; uyN2 = S.uy[s][xr1];
                } else {
                    uxN0 = uxN1 = uxN2 = uyN0 = uyN1 = uyN2 = R(0);
                }
                const R uxW = S.ux[sc][xl1], uxE = S.ux[sc][xr1];
                const R uyW = S.uy[sc][xl1], uyE = S.uy[sc][xr1];
                (void)uyW; (void)uyE; (void)uxS1; (void)uxN1;
                // isotropic central difference, (1/c_s^2) sum_i w_i c_i phi(x + c_i)
                const R divu = (uxE - uxW) * R(1.0 / 3.0) +
                               (uxN2 + uxS2 - uxN0 - uxS0) * R(1.0 / 12.0) +
                               (uyN1 - uyS1) * R(1.0 / 3.0) +
                               (uyN2 + uyN0 - uyS2 - uyS0) * R(1.0 / 12.0);
                const R C = rho * P.cv;
                // Q = -[rho c_v u.grad T + T (dp/dT)_rho div u]  (Eq. 20)
                const R Q = -(C * (uxc * dTx + uyc * dTy) + T * eos_dpdT(P, rho, T) * divu);
                const R Pn = Q / C;
                // S = w^ rho c_v (dt/2) d_t^2 T with d_t^2 T ~ P^n - P^{n-1} (Eq. 24)
                const R St = first ? R(0) : C * R(0.5) * (Pn - Pp);
                const R Qs = Q + St;
                // moment-space collision (Eqs. 39, 40, 47), deviation form
                const R m0s = Td + Qs;
                const R m1s = P.one_m_vs1 * m1;
                const R m2s = P.one_m_vs1 * m2;
                const R m3s = m3d - P.vs3 * (m3d - P.w_dot * Td) + P.w_dot * Qs;
                const R m4s = P.one_m_vs4 * m4;
                const R a = R(0.25) * (m3s + m4s), b = R(0.25) * (m3s - m4s);
                S.gs[sc][0][t] = m0s - m3s;
                S.gs[sc][1][t] = a + R(0.5) * m1s;
                S.gs[sc][2][t] = b + R(0.5) * m2s;
                S.gs[sc][3][t] = a - R(0.5) * m1s;
                S.gs[sc][4][t] = b - R(0.5) * m2s;
                if (inD && r >= y0 && r < y1) Pdst[(size_t)grow(r) * pitch + gx] = Pn;
            }
        }

        // ---- D9(k-3): pull streaming of f* (Eq. 6) with wall / open rules
        {
            const int r = k - 3;
            if (r >= y0 && r < y1 && inD) {
                const int sc = slot3(r), sd = slot3(r - 1), su = slot3(r + 1);
                const bool vd = rowvalid(r - 1), vu = rowvalid(r + 1);
                const int rowS = vd ? sd : sc;   // source row for c_y = +1 (open: own row)
                const int rowN = vu ? su : sc;   // source row for c_y = -1
                const bool bS = !vd && wallS, bN = !vu && wallN;
                R fo[9];
                if (P.frozen_flow) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) fo[q] = S.fs[sc][q][t];
                } else {
                    fo[0] = S.fs[sc][0][t];
                    fo[1] = S.fs[sc][1][xl1];
                    fo[3] = S.fs[sc][3][xr1];
                    fo[2] = bS ? S.fs[sc][4][t] : S.fs[rowS][2][t];
                    fo[5] = bS ? S.fs[sc][7][t] : S.fs[rowS][5][xl1];
                    fo[6] = bS ? S.fs[sc][8][t] : S.fs[rowS][6][xr1];
                    fo[4] = bN ? S.fs[sc][2][t] : S.fs[rowN][4][t];
                    fo[7] = bN ? S.fs[sc][5][t] : S.fs[rowN][7][xr1];
                    fo[8] = bN ? S.fs[sc][6][t] : S.fs[rowN][8][xl1];
                }
                const size_t off = (size_t)grow(r) * pitch + gx;
#pragma unroll
                for (int q = 0; q < 9; ++q) st_st(fdst + q * plane + off, (TF)fo[q]);
            }
        }

        // ---- A(k): moments, EOS, psi
        R rho_a = R(1), rhod_a = R(0), jx_a = R(0), jy_a = R(0), T_a = R(0), psi_a = R(0);
        if (doA && colvalid) {
            rhod_a = ((fa[0] + fa[1]) + (fa[2] + fa[3])) + ((fa[4] + fa[5]) + (fa[6] + fa[7])) + fa[8];
            rho_a = rhod_a + rho_ref;
            const R Td = (ga[0] + ga[1]) + (ga[2] + ga[3]) + ga[4];
            T_a = Td + T_ref;
            jx_a = (fa[1] - fa[3]) + (fa[5] - fa[6]) + (fa[8] - fa[7]);
            jy_a = (fa[2] - fa[4]) + (fa[5] + fa[6]) - (fa[7] + fa[8]);
            const R q2 = psi2_of(P, rho_a, T_a);
            if (!(q2 >= R(0))) errbits |= (q2 != q2) ? ERR_NONFINITE : ERR_PSI;
            psi_a = rsq(q2);
            const int s3 = slot3(k), s5 = slot5(k);
            S.psi[s3][t] = psi_a;
            S.rho[s3][t] = rho_a;
            S.T[s3][t] = T_a;
#pragma unroll
            for (int q = 0; q < 5; ++q) S.own[s5][q][t] = ga[q];
            S.own[s5][5][t] = rho_a;
            S.own[s5][6][t] = pa;
            if (use_mass && inD && k >= y0 && k < y1) mass_acc += (double)rho_a;
        }
        __syncthreads();

        // ================= phase beta =================
        // ---- B(k-1): interaction force, velocity, D2Q9 MRT collision
        {
            const int r = k - 1;
            if (r >= y0 - 2 && r < y1 + 2 && rowvalid(r) && inB) {
                const int sc = slot3(r), sd = slot3(r - 1), su = slot3(r + 1);
                const bool vd = rowvalid(r - 1), vu = rowvalid(r + 1);
                R pSW, pS, pSE, pNW, pN, pNE;
                const R pW = S.psi[sc][xl1], pE = S.psi[sc][xr1];
                // Ding-Spelt ghost layer (Section 3.3): rho_ghost = rho(layer 2)
                // + tan(pi/2 - theta) |rho(x+1, layer 1) - rho(x-1, layer 1)|
                auto ghost = [&](int c, int cm, int cp, int s_far, int edge) -> R {
                    const R rg = S.rho[s_far][c] + cot * rabs(S.rho[sc][cp] - S.rho[sc][cm]);
                    const R Tg = I.therm[edge] == T_DIRICHLET ? (R)wall_T(I, edge, gcol(c))
                                                              : S.T[sc][c];
                    const R q2 = psi2_of(P, rg, Tg);
                    if (!(q2 >= R(0))) errbits |= (q2 != q2) ? ERR_NONFINITE : ERR_PSI;
                    return rsq(q2);
                };
                if (vd || !wallS) {
                    const int s = vd ? sd : sc;
                    pSW = S.psi[s][xl1]; pS = S.psi[s][t]; pSE = S.psi[s][xr1];
                } else {
                    pSW = ghost(xl1, cLL, cLR, su, ES);
                    pS = ghost(t, xl1, xr1, su, ES);
                    pSE = ghost(xr1, cRL, cRR, su, ES);
                }
                if (vu || !wallN) {
                    const int s = vu ? su : sc;
                    pNW = S.psi[s][xl1]; pN = S.psi[s][t]; pNE = S.psi[s][xr1];
                } else {
                    pNW = ghost(xl1, cLL, cLR, sd, EN);
                    pN = ghost(t, xl1, xr1, sd, EN);
                    pNE = ghost(xr1, cRL, cRR, sd, EN);
                }
                // Eq. 9 with varpi(1) = 1/3, varpi(2) = 1/12
                const R sx = (pE - pW) * R(1.0 / 3.0) + (pNE + pSE - pNW - pSW) * R(1.0 / 12.0);
                const R sy = (pN - pS) * R(1.0 / 3.0) + (pNE + pNW - pSE - pSW) * R(1.0 / 12.0);
                const R Fmx = P.negG * psip * sx;
                const R Fmy = P.negG * psip * sy;
                const R Fx = Fmx;
                const R Fy = Fmy - P.gravity * (rhop - rho_ave);
                R ux = R(0), uy = R(0);
                if (!P.frozen_flow) {
                    const R ir = R(1) / rhop;
                    ux = (jxp + R(0.5) * Fx) * ir;
                    uy = (jyp + R(0.5) * Fy) * ir;
                }
                S.ux[sc][t] = ux;
                S.uy[sc][t] = uy;
                if (r >= y0 - 1 && r < y1 + 1 && inC) {
                    if (P.frozen_flow) {
#pragma unroll
                        for (int q = 0; q < 9; ++q) S.fs[sc][q][t] = fp[q];
                    } else {
                        const R* f = fp;
                        const R rr = rhop;
                        const R uu = ux * ux + uy * uy;
                        const R s14 = (f[1] + f[2]) + (f[3] + f[4]);
                        const R s58 = (f[5] + f[6]) + (f[7] + f[8]);
                        // non-equilibrium parts m - m^eq of the moments of Eq. 7
                        // (deviation storage shifts m_e by -2 rho_ref, m_eps by rho_ref)
                        const R ne1 = (R(-4) * f[0] - s14 + R(2) * s58) + R(2) * rhodp - R(3) * rr * uu;
                        const R ne2 = (R(4) * f[0] - R(2) * s14 + s58) - rhodp + R(3) * rr * uu;
                        const R ne4 = (R(-2) * f[1] + R(2) * f[3] + f[5] - f[6] - f[7] + f[8]) + rr * ux;
                        const R ne6 = (R(-2) * f[2] + R(2) * f[4] + f[5] + f[6] - f[7] - f[8]) + rr * uy;
                        const R ne7 = (f[1] - f[2] + f[3] - f[4]) - rr * (ux * ux - uy * uy);
                        const R ne8 = (f[5] - f[6] + f[7] - f[8]) - rr * ux * uy;
                        // Li forcing (Eq. 8)
                        const R uF = ux * Fx + uy * Fy;
                        const R Fm2 = (Fmx * Fmx + Fmy * Fmy) / (psip * psip);
                        const R F1 = R(6) * uF + P.sig_e * Fm2;
                        const R F2 = R(-6) * uF - P.sig_eps * Fm2;
                        const R F7 = R(2) * (ux * Fx - uy * Fy);
                        const R F8 = ux * Fy + uy * Fx;
                        // m* - m = -S (m - m^eq) + (I - S/2) F; for j the
                        // change is exactly F because rho u = j + F/2
                        const R d1 = -P.s_e * ne1 + P.hs_e * F1;
                        const R d2 = -P.s_eps * ne2 + P.hs_eps * F2;
                        const R d4 = -P.s_q * ne4 - P.hs_q * Fx;
                        const R d6 = -P.s_q * ne6 - P.hs_q * Fy;
                        const R d7 = -P.s_p * ne7 + P.hs_p * F7;
                        const R d8 = -P.s_p * ne8 + P.hs_p * F8;
                        // f* = f + M^{-1} (m* - m), M^{-1} = M^T diag(1/9, 1/36,
                        // 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4)
                        const R a1 = d1 * R(1.0 / 36.0), a2 = d2 * R(1.0 / 36.0);
                        const R a3 = Fx * R(1.0 / 6.0), a5 = Fy * R(1.0 / 6.0);
                        const R a4 = d4 * R(1.0 / 12.0), a6 = d6 * R(1.0 / 12.0);
                        const R a7 = d7 * R(0.25), a8 = d8 * R(0.25);
                        const R cax = -a1 - R(2) * a2;   // common to the axis directions
                        const R cdg = R(2) * a1 + a2;    // common to the diagonals
                        S.fs[sc][0][t] = f[0] - R(4) * a1 + R(4) * a2;
                        S.fs[sc][1][t] = f[1] + cax + a3 - R(2) * a4 + a7;
                        S.fs[sc][2][t] = f[2] + cax + a5 - R(2) * a6 - a7;
                        S.fs[sc][3][t] = f[3] + cax - a3 + R(2) * a4 + a7;
                        S.fs[sc][4][t] = f[4] + cax - a5 + R(2) * a6 - a7;
                        S.fs[sc][5][t] = f[5] + cdg + a3 + a4 + a5 + a6 + a8;
                        S.fs[sc][6][t] = f[6] + cdg - a3 - a4 + a5 + a6 - a8;
                        S.fs[sc][7][t] = f[7] + cdg - a3 - a4 - a5 - a6 + a8;
                        S.fs[sc][8][t] = f[8] + cdg + a3 + a4 - a5 - a6 - a8;
                    }
                }
            }
        }

        // ---- D5(k-4): rho c_v-weighted streaming of g* (Eq. 39)
        {
            const int r = k - 4;
            if (r >= y0 && r < y1 && inD) {
                const int so = slot5(r);
                const int sc = slot3(r), sd = slot3(r - 1), su = slot3(r + 1);
                R gd[5];
#pragma unroll
                for (int q = 0; q < 5; ++q) gd[q] = S.own[so][q][t];
                R go[5];
                if (P.frozen_thermal) {
#pragma unroll
                    for (int q = 0; q < 5; ++q) go[q] = gd[q];
                } else {
                    const R rho = S.own[so][5][t];
                    // thermal walls: halfway anti-bounce-back (Dirichlet) or
                    // bounce-back (adiabatic) supplies the incoming g*
                    auto wallg = [&](int edge, int opp) -> R {
                        const R out = S.gs[sc][opp][t];
                        if (I.therm[edge] == T_DIRICHLET)
                            return -out + R(2) * P.w5_1 * ((R)wall_T(I, edge, gx) - T_ref);
                        return out;
                    };
                    R A[5];
                    A[0] = S.gs[sc][0][t];
                    A[1] = left_edge ? wallg(EW, 3) : S.gs[sc][1][xl1];
                    A[3] = right_edge ? wallg(EE, 1) : S.gs[sc][3][xr1];
                    A[2] = rowvalid(r - 1) ? S.gs[sd][2][t] : wallg(ES, 4);
                    A[4] = rowvalid(r + 1) ? S.gs[su][4][t] : wallg(EN, 2);
                    const R iC = R(1) / (rho * P.cv);
#pragma unroll
                    for (int q = 0; q < 5; ++q) go[q] = gd[q] + (A[q] - gd[q]) * iC;
                }
                const size_t off = (size_t)grow(r) * pitch + gx;
#pragma unroll
                for (int q = 0; q < 5; ++q) st_st(gdst + q * plane + off, go[q]);
            }
        }
        __syncthreads();

#pragma unroll
        for (int q = 0; q < 9; ++q) fp[q] = fa[q];
        rhop = rho_a;
        rhodp = rhod_a;
        jxp = jx_a;
        jyp = jy_a;
        Tp = T_a;
        psip = psi_a;
    }
    (void)Tp;

    if (errbits) atomicOr(&I.ctl->err, errbits);
    if (use_mass) {
        // block sum of this unit's output densities -> ring slot step % 3
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mass_acc += __shfl_down_sync(0xffffffffu, mass_acc, o);
        if ((t & 31) == 0) S.red[t >> 5] = mass_acc;
        __syncthreads();
        if (t == 0) {
            double s = 0.0;
            for (int w = 0; w < NT / 32; ++w) s += S.red[w];
            atomicAdd(&I.ctl->mass[step % 3], s);
        }
        __syncthreads();
    }
}

template <int PREC, int NT>
__global__ void __launch_bounds__(NT) k_step(StepLaunch L, Phys<typename Types<PREC>::R> P) {
    typedef typename Types<PREC>::R R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    StepSmem<R, NT>& S = *reinterpret_cast<StepSmem<R, NT>*>(smem_raw);
    for (;;) {
        if (threadIdx.x == 0) S.unit = (int)atomicAdd(&L.sched[0], 1u);
        __syncthreads();
        const int u = S.unit;
        __syncthreads();
        if (u >= L.n_units) break;
        const Unit U = L.units[u];
        const Inst I = L.insts[U.inst];
        process_unit<PREC, NT>(I, U, P, S);
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned done = atomicAdd(&L.sched[1], 1u);
        if (done == gridDim.x - 1) {
            // every other CTA has finished: advance the domains' step counters,
            // clear the density-sum slot the next step accumulates into, and
            // reset the work counter for the next launch
            __threadfence();
            for (int i = 0; i < L.n_inst; ++i) {
                Ctl* c = L.insts[i].ctl;
                const long long s = __ldcg(&c->step);
                c->mass[(s + 1) % 3] = 0.0;
                c->step = s + 1;
            }
            L.sched[0] = 0u;
            L.sched[1] = 0u;
            __threadfence();
        }
    }
}

template <int PREC, int NT>
static int launch_one(const StepLaunch& L, cudaStream_t st) {
    typedef typename Types<PREC>::R R;
    const size_t smem = sizeof(StepSmem<R, NT>);
    static bool attr_set = false;
    if (!attr_set) {
        if (cudaFuncSetAttribute(k_step<PREC, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return -1;
        attr_set = true;
    }
    Phys<R> P = make_phys<R>(L.phys);
    k_step<PREC, NT><<<L.grid, NT, smem, st>>>(L, P);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int PREC, int NT>
static int occ_one(int* ctas, size_t* smem_bytes) {
    typedef typename Types<PREC>::R R;
    const size_t smem = sizeof(StepSmem<R, NT>);
    if (cudaFuncSetAttribute(k_step<PREC, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_step<PREC, NT>, NT, smem) !=
        cudaSuccess)
        return -1;
    *smem_bytes = smem;
    return 0;
}

int step_launch(int prec, int threads, const StepLaunch& L, cudaStream_t st) {
    if (threads == 128) {
        if (prec == 0) return launch_one<0, 128>(L, st);
        if (prec == 1) return launch_one<1, 128>(L, st);
        return launch_one<2, 128>(L, st);
    }
    if (prec == 0) return launch_one<0, 256>(L, st);
    if (prec == 1) return launch_one<1, 256>(L, st);
    return launch_one<2, 256>(L, st);
}

int step_occupancy(int prec, int threads, int* ctas, size_t* smem) {
    if (threads == 128) {
        if (prec == 0) return occ_one<0, 128>(ctas, smem);
        if (prec == 1) return occ_one<1, 128>(ctas, smem);
        return occ_one<2, 128>(ctas, smem);
    }
    if (prec == 0) return occ_one<0, 256>(ctas, smem);
    if (prec == 1) return occ_one<1, 256>(ctas, smem);
    return occ_one<2, 256>(ctas, smem);
}

}  // namespace lbm
