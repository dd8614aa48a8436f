/*
 * FP64 CPU oracle for the coupled time step of the thermal lattice Boltzmann
 * model for liquid-vapor phase change (Wang, Huang & He, arXiv 2205.00686).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, by __graft_entry__.smoke() and by
 * the cpu_baseline / --impl reference legs of bench.py.  The product path (the
 * CUDA library) never calls it, and the two share no code.
 *
 * The step is written as plain whole-field loops, one loop per phase, in the
 * order the paper's equations are stated:
 *   1. rho = sum f, T = sum g                               (Eq. 11, Eq. 25)
 *   2. p_EOS(rho,T) (Peng-Robinson, Eq. 10) and psi          (Section 2)
 *      plus the wetting ghost layer of walls                 (Section 3.3)
 *   3. F_m = -G psi(x) sum_i varpi(|c_i|^2) psi(x+c_i) c_i   (Eq. 9)
 *   4. F_n = F_m + F_b, u from rho u = sum c f + F_n/2        (Eq. 11, Section 4.3)
 *   5. div u (isotropic central difference; the paper leaves its form open)
 *   6. grad T from the local first moments                   (Eqs. 49-50)
 *   7. (dp/dT)_rho, Q, P^n = Q/(rho c_v), S                  (Eqs. 20, 23, 24)
 *   8. D2Q9 MRT collision in moment space                    (Eqs. 5, 7, 8)
 *   9. D2Q5 MRT collision in moment space                    (Eqs. 39, 40, 47)
 *  10. D2Q9 streaming + flow boundaries                      (Eq. 6)
 *  11. D2Q5 rho c_v-weighted streaming + thermal boundaries  (Eq. 39)
 *  12. keep P^n for the next step's d_t^2 T
 *
 * Matrix products use the transformation matrices as printed (Eq. 4 with the
 * third row read as the Lallemand-Luo row, Eq. 40), and their inverses are
 * obtained numerically by Gauss-Jordan elimination, not by closed forms.
 *
 * Readings of the paper where it is silent or garbled are listed in the repo's
 * design notes; each is marked "reading:" at the line that takes it.
 *
 * Pins (tests/test_oracle_*.py): equilibrium moments, Eq. 33 sums, matrix
 * inverses, the Peng-Robinson critical point and acentric factor, the
 * (dp/dT)_rho closed form against finite differences, Maxwell coexistence
 * against an independent scipy solution, exact mass conservation, momentum,
 * uniform fixed point, droplet symmetry, the textbook D2Q5 diffusion scheme
 * (frozen flow, rho c_v = 1), the exact Fourier amplification of the blend
 * and its continuum limit lambda k^2/(rho c_v), steady conduction, transient
 * conduction against its Fourier series, flat-interface coexistence, the
 * Laplace law, and the instability of the literal c_v = 0.1 reading.  The
 * coupling terms (tests/test_oracle_coupling.py): compression heating of one
 * step against -T (dp/dT) div u / (rho c_v), a sound wave on the adiabat at
 * the adiabatic sound speed, the S history term keeping it there at every
 * phase, an isobaric temperature wave decaying at lambda k^2 / (rho c_p) and
 * advected at the flow speed, the local gradient of Eqs. 49-50 against the
 * spectral gradient and exactly in steady conduction, and the source moments
 * of Eq. 33.  The flow lattice (tests/test_oracle_transport.py): shear-wave
 * and channel decay at nu k^2 (s_p, halfway bounce-back), the forcing of
 * Eq. 8 against Guo's velocity-space term, the momentum gain F_n, and the
 * Ding-Spelt ghost layer relaxing a droplet to 60 and 120 degrees.  The
 * diagnostics against direct sums (tests/test_oracle_diagnostics.py).
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* D2Q9 velocity set, Eq. 2 (c = 1) */
static const int CX9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
/* D2Q5 velocity set, Eq. 26 */
static const int CX5[5] = {0, 1, 0, -1, 0};
static const int CY5[5] = {0, 0, 1, 0, -1};

/* Eq. 4.  reading: the third row is printed as (4,-2,-2,-2,1,1,1,1,1); the
 * matrix cited (Lallemand & Luo) and the printed m^eq of Eq. 7 both require
 * (4,-2,-2,-2,-2,1,1,1,1), which is used here. */
static const double M9_PRINTED[81] = {
    1, 1, 1, 1, 1, 1, 1, 1, 1,
    -4, -1, -1, -1, -1, 2, 2, 2, 2,
    4, -2, -2, -2, -2, 1, 1, 1, 1,
    0, 1, 0, -1, 0, 1, -1, -1, 1,
    0, -2, 0, 2, 0, 1, -1, -1, 1,
    0, 0, 1, 0, -1, 1, 1, -1, -1,
    0, 0, -2, 0, 2, 1, 1, -1, -1,
    0, 1, -1, 1, -1, 0, 0, 0, 0,
    0, 0, 0, 0, 0, 1, -1, 1, -1};

/* Eq. 40, the non-orthogonal D2Q5 matrix */
static const double M5_PRINTED[25] = {
    1, 1, 1, 1, 1,
    0, 1, 0, -1, 0,
    0, 0, 1, 0, -1,
    0, 1, 1, 1, 1,
    0, 1, -1, 1, -1};

struct orc_sim {
    int nx, ny;
    orc_params p;
    orc_bc bc;
    /* derived */
    double Tc, kpr, sp, vs12, cs2h, cot_theta;
    double w5[5];
    double M[81], Minv[81], Mh[25], Mhinv[25];
    double S[9], Lam[5];
    /* state at time t */
    double *f, *g, *Pprev;
    long step;
    double rho_ave_prev;
    int err;
    /* per-step work arrays */
    double *rho, *T, *psi, *Fmx, *Fmy, *Fx, *Fy, *ux, *uy;
    double *divu, *dTx, *dTy, *Q, *Pn, *Stot;
    double *fs, *gs, *fn, *gn;
    double *gpsi_S, *gpsi_N;
};

/* ---------------------------------------------------------------------- */
/* small dense linear algebra                                               */

/* Gauss-Jordan inverse with partial pivoting of an n x n row-major matrix */
static int gj_inverse(const double* A, double* Ainv, int n) {
    double w[9 * 18];
    int m = 2 * n;
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < m; ++c)
            w[r * m + c] = c < n ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(w[r * m + c]) > fabs(w[piv * m + c])) piv = r;
        if (w[piv * m + c] == 0.0) return ORC_EINVAL;
        if (piv != c)
            for (int k = 0; k < m; ++k) {
                double t = w[c * m + k];
                w[c * m + k] = w[piv * m + k];
                w[piv * m + k] = t;
            }
        double d = w[c * m + c];
        for (int k = 0; k < m; ++k) w[c * m + k] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double e = w[r * m + c];
            if (e != 0.0)
                for (int k = 0; k < m; ++k) w[r * m + k] -= e * w[c * m + k];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) Ainv[r * n + c] = w[r * m + n + c];
    return ORC_OK;
}

static void matvec(const double* A, const double* x, double* y, int n) {
    for (int r = 0; r < n; ++r) {
        double acc = 0.0;
        for (int c = 0; c < n; ++c) acc += A[r * n + c] * x[c];
        y[r] = acc;
    }
}

void orc_matrices(double M[81], double Minv[81], double Mh[25], double Mhinv[25]) {
    memcpy(M, M9_PRINTED, sizeof(M9_PRINTED));
    memcpy(Mh, M5_PRINTED, sizeof(M5_PRINTED));
    gj_inverse(M, Minv, 9);
    gj_inverse(Mh, Mhinv, 5);
}

/* ---------------------------------------------------------------------- */
/* equation of state (Section 2, Eq. 10)                                    */

void orc_set_defaults(orc_params* p) {
    memset(p, 0, sizeof(*p));
    p->a = 3.0 / 49.0;
    p->b = 2.0 / 21.0;
    p->R = 1.0;
    p->omega = 0.344;
    p->G = -1.0;
    p->sigma = 0.0;
    p->nu = 0.1;
    p->s0 = p->s_e = p->s_eps = p->s_j = p->s_q = 1.0;
    p->lambda = 1.0 / 3.0;
    p->cv = 5.0;
    p->w_dot = 2.0 / 3.0;
    p->vs0 = p->vs3 = p->vs4 = 1.0;
    p->gravity = 0.0;
    p->frozen_flow = 0;
    p->frozen_thermal = 0;
}

/* a = 0.45724 R^2 Tc^2 / pc and b = 0.0778 R Tc / pc, so Tc follows from a/b */
double orc_Tc(const orc_params* p) { return 0.0778 * p->a / (0.45724 * p->b * p->R); }

static double pr_k(const orc_params* p) {
    return 0.37464 + 1.54226 * p->omega - 0.26992 * p->omega * p->omega;
}

static double pr_phi(const orc_params* p, double T) {
    double h = 1.0 + pr_k(p) * (1.0 - sqrt(T / orc_Tc(p)));
    return h * h;
}

double orc_p_eos(const orc_params* p, double rho, double T) {
    double a = p->a, b = p->b;
    return rho * p->R * T / (1.0 - b * rho) -
           a * pr_phi(p, T) * rho * rho / (1.0 + 2.0 * b * rho - b * b * rho * rho);
}

/* (dp_EOS/dT) at constant rho: derivative of Eq. 10 with
 * dphi/dT = -k (1 + k(1 - sqrt(T/Tc))) / sqrt(T Tc).  The paper uses this
 * quantity in Q (Eq. 20) without printing it. */
double orc_dpdT(const orc_params* p, double rho, double T) {
    double a = p->a, b = p->b, Tc = orc_Tc(p), k = pr_k(p);
    double h = 1.0 + k * (1.0 - sqrt(T / Tc));
    double dphi = -k * h / sqrt(T * Tc);
    return rho * p->R / (1.0 - b * rho) -
           a * dphi * rho * rho / (1.0 + 2.0 * b * rho - b * b * rho * rho);
}

/* psi^2 = 2 (p_EOS - rho c_s^2) / (G dx^2), c_s^2 = 1/3, dx = 1 */
double orc_psi2(const orc_params* p, double rho, double T) {
    return 2.0 * (orc_p_eos(p, rho, T) - rho / 3.0) / p->G;
}

static double dp_drho(const orc_params* p, double rho, double T) {
    double a = p->a, b = p->b;
    double d = 1.0 + 2.0 * b * rho - b * b * rho * rho;
    double dd = 2.0 * b - 2.0 * b * b * rho;
    double e = 1.0 - b * rho;
    return p->R * T / (e * e) - a * pr_phi(p, T) * (2.0 * rho * d - rho * rho * dd) / (d * d);
}

/* root of p(rho) = ps on [lo, hi] where p is monotone increasing */
static double bisect_p(const orc_params* p, double T, double ps, double lo, double hi) {
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (orc_p_eos(p, mid, T) < ps) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* equal-area integral in the p-v plane, written with v = 1/rho:
 * int_{rho_g}^{rho_l} (p(rho) - ps) / rho^2 drho  (composite Simpson) */
static double maxwell_area(const orc_params* p, double T, double ps, double rg, double rl) {
    const int n = 20000;
    double h = (rl - rg) / n, acc = 0.0;
    for (int i = 0; i <= n; ++i) {
        double r = rg + i * h;
        double v = (orc_p_eos(p, r, T) - ps) / (r * r);
        double wgt = (i == 0 || i == n) ? 1.0 : (i % 2 ? 4.0 : 2.0);
        acc += wgt * v;
    }
    return acc * h / 3.0;
}

/* Maxwell equal-area construction for the flat-interface coexistence
 * densities at temperature T (T < Tc). */
int orc_maxwell(const orc_params* p, double T, double* rho_g, double* rho_l) {
    double rmax = 1.0 / p->b;
    /* spinodals: sign changes of dp/drho on a fine grid, refined by bisection */
    double sp[2];
    int ns = 0;
    const int ngrid = 20000;
    double prev_r = 1e-6, prev_d = dp_drho(p, prev_r, T);
    for (int i = 1; i < ngrid && ns < 2; ++i) {
        double r = 1e-6 + (rmax - 1e-3) * i / ngrid;
        double d = dp_drho(p, r, T);
        if ((d > 0) != (prev_d > 0)) {
            double lo = prev_r, hi = r;
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (lo + hi);
                double dm = dp_drho(p, mid, T);
                if ((dm > 0) == (prev_d > 0)) lo = mid; else hi = mid;
            }
            sp[ns++] = 0.5 * (lo + hi);
        }
        prev_r = r;
        prev_d = d;
    }
    if (ns < 2) return ORC_EINVAL;
    double p_hi = orc_p_eos(p, sp[0], T);  /* local maximum (vapour spinodal) */
    double p_lo = orc_p_eos(p, sp[1], T);  /* local minimum (liquid spinodal) */
    if (p_lo < 1e-12) p_lo = 1e-12;
    double lo = p_lo, hi = p_hi, rg = 0, rl = 0;
    for (int it = 0; it < 100; ++it) {
        double ps = 0.5 * (lo + hi);
        rg = bisect_p(p, T, ps, 1e-12, sp[0]);
        rl = bisect_p(p, T, ps, sp[1], rmax * (1.0 - 1e-12));
        double A = maxwell_area(p, T, ps, rg, rl);
        if (A > 0) lo = ps; else hi = ps;
    }
    *rho_g = rg;
    *rho_l = rl;
    return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* equilibria                                                               */

/* Eq. 3, c_s^2 = 1/3 */
void orc_feq(double rho, double ux, double uy, double f[9]) {
    const double cs2 = 1.0 / 3.0;
    double uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        double cu = CX9[i] * ux + CY9[i] * uy;
        f[i] = W9[i] * rho * (1.0 + cu / cs2 + cu * cu / (2.0 * cs2 * cs2) - uu / (2.0 * cs2));
    }
}

/* Eq. 7 */
void orc_meq(double rho, double ux, double uy, double meq[9]) {
    double uu = ux * ux + uy * uy;
    meq[0] = rho;
    meq[1] = rho * (-2.0 + 3.0 * uu);
    meq[2] = rho * (1.0 - 3.0 * uu);
    meq[3] = rho * ux;
    meq[4] = -rho * ux;
    meq[5] = rho * uy;
    meq[6] = -rho * uy;
    meq[7] = rho * (ux * ux - uy * uy);
    meq[8] = rho * ux * uy;
}

static void d2q5_weights(const orc_params* p, double w[5]) {
    w[0] = 1.0 - p->w_dot;
    for (int i = 1; i < 5; ++i) w[i] = p->w_dot / 4.0;
}

/* Eq. 22 */
void orc_geq(const orc_params* p, double T, double g[5]) {
    double w[5];
    d2q5_weights(p, w);
    for (int i = 0; i < 5; ++i) g[i] = w[i] * T;
}

/* ---------------------------------------------------------------------- */
/* create / destroy                                                         */

static int valid_bc(int nx, int ny, const orc_bc* bc) {
    for (int e = 0; e < 4; ++e) {
        if (bc->flow[e] < 0 || bc->flow[e] > 2) return 0;
        if (bc->therm[e] < 0 || bc->therm[e] > 2) return 0;
        /* a periodic thermal edge needs a periodic flow edge; a periodic flow
         * edge may carry a Dirichlet or adiabatic thermal edge: Section 4.1
         * streams the flow populations periodically and holds T = T_g at the
         * edges by halfway anti-bounce-back */
        if (bc->therm[e] == ORC_T_PERIODIC && bc->flow[e] != ORC_PERIODIC) return 0;
    }
    if ((bc->flow[ORC_W] == ORC_PERIODIC) != (bc->flow[ORC_E] == ORC_PERIODIC)) return 0;
    if ((bc->flow[ORC_S] == ORC_PERIODIC) != (bc->flow[ORC_N] == ORC_PERIODIC)) return 0;
    if ((bc->therm[ORC_W] == ORC_T_PERIODIC) != (bc->therm[ORC_E] == ORC_T_PERIODIC)) return 0;
    if ((bc->therm[ORC_S] == ORC_T_PERIODIC) != (bc->therm[ORC_N] == ORC_T_PERIODIC)) return 0;
    /* walls are horizontal (south / north) only */
    if (bc->flow[ORC_W] == ORC_WALL || bc->flow[ORC_E] == ORC_WALL) return 0;
    if (bc->flow[ORC_W] != ORC_PERIODIC && nx < 2) return 0;
    if (bc->flow[ORC_S] != ORC_PERIODIC && ny < 2) return 0;
    return 1;
}

orc_sim* orc_create(int nx, int ny, const orc_params* p, const orc_bc* bc, int* err) {
    if (err) *err = ORC_OK;
    if (nx < 1 || ny < 1 || !p || !bc || !valid_bc(nx, ny, bc) || p->cv <= 0 ||
        p->w_dot <= 0 || p->w_dot >= 1 || p->nu <= 0 || p->lambda <= 0) {
        if (err) *err = ORC_EINVAL;
        return NULL;
    }
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    if (!s) {
        if (err) *err = ORC_ENOMEM;
        return NULL;
    }
    s->nx = nx;
    s->ny = ny;
    s->p = *p;
    s->bc = *bc;
    s->Tc = orc_Tc(p);
    s->kpr = pr_k(p);
    s->sp = 1.0 / (3.0 * p->nu + 0.5);          /* nu = c_s^2 (1/s_p - 1/2) */
    s->cs2h = p->w_dot / 2.0;                     /* Section 3.2.1 */
    s->vs12 = 1.0 / (p->lambda / s->cs2h + 0.5);  /* lambda = (1/vs - 1/2) cs2h */
    /* Ding-Spelt coefficient tan(pi/2 - theta) */
    s->cot_theta = tan(M_PI / 2.0 - bc->theta_deg * M_PI / 180.0);
    d2q5_weights(p, s->w5);
    orc_matrices(s->M, s->Minv, s->Mh, s->Mhinv);
    /* S = diag(s0, se, seps, sj, sq, sj, sq, sp, sp) (Section 2) */
    double S[9] = {p->s0, p->s_e, p->s_eps, p->s_j, p->s_q, p->s_j, p->s_q, s->sp, s->sp};
    memcpy(s->S, S, sizeof(S));
    double L[5] = {p->vs0, s->vs12, s->vs12, p->vs3, p->vs4};
    memcpy(s->Lam, L, sizeof(L));

    size_t N = (size_t)nx * ny;
    double** arrays[] = {&s->rho, &s->T, &s->psi, &s->Fmx, &s->Fmy, &s->Fx, &s->Fy,
                         &s->ux, &s->uy, &s->divu, &s->dTx, &s->dTy, &s->Q, &s->Pn,
                         &s->Stot, &s->Pprev};
    for (size_t k = 0; k < sizeof(arrays) / sizeof(arrays[0]); ++k) {
        *arrays[k] = (double*)calloc(N, sizeof(double));
        if (!*arrays[k]) goto oom;
    }
    s->f = (double*)calloc(9 * N, sizeof(double));
    s->fs = (double*)calloc(9 * N, sizeof(double));
    s->fn = (double*)calloc(9 * N, sizeof(double));
    s->g = (double*)calloc(5 * N, sizeof(double));
    s->gs = (double*)calloc(5 * N, sizeof(double));
    s->gn = (double*)calloc(5 * N, sizeof(double));
    s->gpsi_S = (double*)calloc(nx, sizeof(double));
    s->gpsi_N = (double*)calloc(nx, sizeof(double));
    if (!s->f || !s->fs || !s->fn || !s->g || !s->gs || !s->gn || !s->gpsi_S || !s->gpsi_N)
        goto oom;
    return s;
oom:
    orc_destroy(s);
    if (err) *err = ORC_ENOMEM;
    return NULL;
}

void orc_destroy(orc_sim* s) {
    if (!s) return;
    double* arrays[] = {s->rho, s->T, s->psi, s->Fmx, s->Fmy, s->Fx, s->Fy, s->ux, s->uy,
                        s->divu, s->dTx, s->dTy, s->Q, s->Pn, s->Stot, s->Pprev, s->f,
                        s->fs, s->fn, s->g, s->gs, s->gn, s->gpsi_S, s->gpsi_N};
    for (size_t k = 0; k < sizeof(arrays) / sizeof(arrays[0]); ++k) free(arrays[k]);
    free(s);
}

/* ---------------------------------------------------------------------- */
/* boundary helpers                                                         */

static int wrap(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

/* x index of a (possibly outside) column: periodic -> wrap, open -> clamp */
static int ext_x(const orc_sim* s, int x) {
    if (x >= 0 && x < s->nx) return x;
    if (s->bc.flow[ORC_W] == ORC_PERIODIC) return wrap(x, s->nx);
    return x < 0 ? 0 : s->nx - 1;
}

/* wall / Dirichlet temperature along an edge (heater segment on the south) */
static double wall_T(const orc_sim* s, int edge, int x) {
    if (edge == ORC_S && x >= s->bc.heater_x0 && x < s->bc.heater_x1) return s->bc.T_heater;
    return s->bc.T_edge[edge];
}

#define AT(arr, x, y) ((arr)[(size_t)(y) * s->nx + (x)])

/* psi at any node within one layer of the domain (Section 3.3 for walls).
 * reading: beyond an open edge psi is copied from the boundary node; at a
 * corner the x rule is applied first, then the y rule. */
static double psi_ext(const orc_sim* s, int x, int y) {
    int xe = ext_x(s, x);
    if (y >= 0 && y < s->ny) return AT(s->psi, xe, y);
    int edge = y < 0 ? ORC_S : ORC_N;
    int kind = s->bc.flow[edge];
    if (kind == ORC_PERIODIC) return AT(s->psi, xe, wrap(y, s->ny));
    if (kind == ORC_OPEN) return AT(s->psi, xe, y < 0 ? 0 : s->ny - 1);
    return edge == ORC_S ? s->gpsi_S[xe] : s->gpsi_N[xe];
}

/* velocity beyond the domain for div u.  reading: solid nodes carry u = 0,
 * open edges copy the boundary row, periodic edges wrap. */
static void u_ext(const orc_sim* s, int x, int y, double* ux, double* uy) {
    int xe = ext_x(s, x);
    if (y >= 0 && y < s->ny) {
        *ux = AT(s->ux, xe, y);
        *uy = AT(s->uy, xe, y);
        return;
    }
    int edge = y < 0 ? ORC_S : ORC_N;
    int kind = s->bc.flow[edge];
    if (kind == ORC_WALL) {
        *ux = 0.0;
        *uy = 0.0;
        return;
    }
    int ye = kind == ORC_PERIODIC ? wrap(y, s->ny) : (y < 0 ? 0 : s->ny - 1);
    *ux = AT(s->ux, xe, ye);
    *uy = AT(s->uy, xe, ye);
}

/* ---------------------------------------------------------------------- */
/* phases 1-4: macroscopic fields of the current state                      */

static void compute_macro(orc_sim* s) {
    const int nx = s->nx, ny = s->ny;
    const size_t N = (size_t)nx * ny;
    const orc_params* p = &s->p;

    /* 1. rho = sum_i f_i (Eq. 11), T = sum_i g_i (Eq. 25) */
#pragma omp parallel for schedule(static)
    for (size_t n = 0; n < N; ++n) {
        double r = 0.0, t = 0.0;
        for (int i = 0; i < 9; ++i) r += s->f[i * N + n];
        for (int i = 0; i < 5; ++i) t += s->g[i * N + n];
        s->rho[n] = r;
        s->T[n] = t;
    }
    /* 2. psi = sqrt(2 (p_EOS - rho c_s^2) / G) */
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (size_t n = 0; n < N; ++n) {
        double q = orc_psi2(p, s->rho[n], s->T[n]);
        if (!(q >= 0.0)) bad = 1;
        s->psi[n] = sqrt(q);
    }
    if (bad) s->err = ORC_EPSI;
    /* wetting ghost layer, Section 3.3: rho_{x,0} = rho_{x,2} + tan(pi/2 -
     * theta) |rho_{x+1,1} - rho_{x-1,1}| where layer 1 is the fluid row next
     * to the wall.  reading: the ghost layer extends the fluid into the wall,
     * so its psi is taken at the temperature of the fluid node next to it
     * (layer 1), for every thermal wall kind; the wall temperature itself
     * enters only the thermal lattice's anti-bounce-back. */
    for (int e = ORC_S; e <= ORC_N; ++e) {
        if (s->bc.flow[e] != ORC_WALL) continue;
        int y1 = e == ORC_S ? 0 : ny - 1;   /* paper's layer 1 */
        int y2 = e == ORC_S ? 1 : ny - 2;   /* paper's layer 2 */
        double* gp = e == ORC_S ? s->gpsi_S : s->gpsi_N;
        for (int x = 0; x < nx; ++x) {
            double rg = AT(s->rho, x, y2) +
                        s->cot_theta * fabs(AT(s->rho, ext_x(s, x + 1), y1) -
                                            AT(s->rho, ext_x(s, x - 1), y1));
            double tg = AT(s->T, x, y1);
            double q = orc_psi2(p, rg, tg);
            if (!(q >= 0.0)) s->err = ORC_EPSI;
            gp[x] = sqrt(q);
        }
    }
    /* 3. F_m = -G psi(x) sum_{i=1..8} varpi(|c_i|^2) psi(x + c_i) c_i (Eq. 9),
     *    varpi(1) = 1/3, varpi(2) = 1/12 */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double sx = 0.0, sy = 0.0;
            for (int i = 1; i < 9; ++i) {
                double wv = (i < 5) ? 1.0 / 3.0 : 1.0 / 12.0;
                double pn = psi_ext(s, x + CX9[i], y + CY9[i]);
                sx += wv * pn * CX9[i];
                sy += wv * pn * CY9[i];
            }
            double pc = AT(s->psi, x, y);
            AT(s->Fmx, x, y) = -p->G * pc * sx;
            AT(s->Fmy, x, y) = -p->G * pc * sy;
        }
    /* 4. F_n = F_m + F_b with F_b = (rho - rho_ave)(0, -g) (Section 4.3),
     *    rho u = sum_i c_i f_i + F_n / 2 (Eq. 11).  reading: rho_ave is the
     *    domain mean of the previous step's density. */
#pragma omp parallel for schedule(static)
    for (size_t n = 0; n < N; ++n) {
        double fx = s->Fmx[n];
        double fy = s->Fmy[n] - (s->rho[n] - s->rho_ave_prev) * p->gravity;
        s->Fx[n] = fx;
        s->Fy[n] = fy;
        if (p->frozen_flow) {
            s->ux[n] = 0.0;
            s->uy[n] = 0.0;
            continue;
        }
        double jx = 0.0, jy = 0.0;
        for (int i = 0; i < 9; ++i) {
            jx += CX9[i] * s->f[i * N + n];
            jy += CY9[i] * s->f[i * N + n];
        }
        s->ux[n] = (jx + 0.5 * fx) / s->rho[n];
        s->uy[n] = (jy + 0.5 * fy) / s->rho[n];
    }
}

/* ---------------------------------------------------------------------- */
/* the coupled step                                                         */

static int one_step(orc_sim* s) {
    const int nx = s->nx, ny = s->ny;
    const size_t N = (size_t)nx * ny;
    const orc_params* p = &s->p;

    compute_macro(s);
    double rho_sum = 0.0;
    for (size_t n = 0; n < N; ++n) rho_sum += s->rho[n];
    double rho_ave_next = rho_sum / (double)N;

    /* 5. div u.  reading: the isotropic central difference
     *    d_a phi = (1/c_s^2) sum_i w_i c_ia phi(x + c_i), D2Q9 weights. */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double d = 0.0;
            for (int i = 1; i < 9; ++i) {
                double vx, vy;
                u_ext(s, x + CX9[i], y + CY9[i], &vx, &vy);
                d += 3.0 * W9[i] * (CX9[i] * vx + CY9[i] * vy);
            }
            AT(s->divu, x, y) = d;
        }
    /* 6. grad T from local moments, Eqs. 49-50: cs2h d_x T = -vs1 m1^(1),
     *    with m1^(1) ~ m1 - m1^eq = m1 (m1^eq = 0, Eq. 47). */
#pragma omp parallel for schedule(static)
    for (size_t n = 0; n < N; ++n) {
        double gl[5], m[5];
        for (int i = 0; i < 5; ++i) gl[i] = s->g[i * N + n];
        matvec(s->Mh, gl, m, 5);
        s->dTx[n] = -s->Lam[1] * m[1] / s->cs2h;
        s->dTy[n] = -s->Lam[2] * m[2] / s->cs2h;
    }
    /* 7. Q = -[rho c_v u.grad T + T (dp/dT)_rho div u] (Eq. 20);
     *    reading: d_t^2 T ~ (P^n - P^{n-1}) with P = Q / (rho c_v), which is
     *    d_t1 T by Eq. 34; the first step takes P^{-1} = P^0 (S = 0).
     *    S_i = w_i rho c_v (dt/2) d_t^2 T (Eq. 24). */
#pragma omp parallel for schedule(static)
    for (size_t n = 0; n < N; ++n) {
        double C = s->rho[n] * p->cv;
        double q = -(C * (s->ux[n] * s->dTx[n] + s->uy[n] * s->dTy[n]) +
                     s->T[n] * orc_dpdT(p, s->rho[n], s->T[n]) * s->divu[n]);
        double Pn = q / C;
        double Pprev = s->step == 0 ? Pn : s->Pprev[n];
        s->Q[n] = q;
        s->Pn[n] = Pn;
        s->Stot[n] = C * 0.5 * (Pn - Pprev);
    }
    /* 8. D2Q9 MRT collision (Eq. 5) with the forcing of Eq. 8 */
    if (!p->frozen_flow) {
#pragma omp parallel for schedule(static)
        for (size_t n = 0; n < N; ++n) {
            double fl[9], m[9], meq[9], F[9], ms[9], fo[9];
            for (int i = 0; i < 9; ++i) fl[i] = s->f[i * N + n];
            matvec(s->M, fl, m, 9);
            double r = s->rho[n], ux = s->ux[n], uy = s->uy[n];
            double Fx = s->Fx[n], Fy = s->Fy[n];
            orc_meq(r, ux, uy, meq);
            double uF = ux * Fx + uy * Fy;
            double Fm2 = s->Fmx[n] * s->Fmx[n] + s->Fmy[n] * s->Fmy[n];
            double ps2 = s->psi[n] * s->psi[n];
            F[0] = 0.0;
            F[1] = 6.0 * uF + p->sigma * Fm2 / (ps2 * (1.0 / s->S[1] - 0.5));
            F[2] = -6.0 * uF - p->sigma * Fm2 / (ps2 * (1.0 / s->S[2] - 0.5));
            F[3] = Fx;
            F[4] = -Fx;
            F[5] = Fy;
            F[6] = -Fy;
            F[7] = 2.0 * (ux * Fx - uy * Fy);
            F[8] = ux * Fy + uy * Fx;
            for (int k = 0; k < 9; ++k)
                ms[k] = m[k] - s->S[k] * (m[k] - meq[k]) + (1.0 - 0.5 * s->S[k]) * F[k];
            matvec(s->Minv, ms, fo, 9);
            for (int i = 0; i < 9; ++i) s->fs[i * N + n] = fo[i];
        }
    }
    /* 9. D2Q5 MRT collision (Eq. 39): m* = m - Lambda (m - m^eq) + Mh (G + S),
     *    m^eq = [T, 0, 0, w_dot T, 0] (Eq. 47), G_i = w_i Q (Eq. 23). */
#pragma omp parallel for schedule(static)
    for (size_t n = 0; n < N; ++n) {
        double gl[5], m[5], src[5], msrc[5], ms[5], go[5];
        for (int i = 0; i < 5; ++i) gl[i] = s->g[i * N + n];
        matvec(s->Mh, gl, m, 5);
        double T = s->T[n];
        double meq[5] = {T, 0.0, 0.0, p->w_dot * T, 0.0};
        for (int i = 0; i < 5; ++i) src[i] = s->w5[i] * s->Q[n] + s->w5[i] * s->Stot[n];
        matvec(s->Mh, src, msrc, 5);
        for (int k = 0; k < 5; ++k) ms[k] = m[k] - s->Lam[k] * (m[k] - meq[k]) + msrc[k];
        matvec(s->Mhinv, ms, go, 5);
        for (int i = 0; i < 5; ++i) s->gs[i * N + n] = go[i];
    }
    /* 10. D2Q9 streaming f_i(x + c_i, t + 1) = f*_i(x, t) (Eq. 6), pull form.
     *     Walls: halfway bounce-back.  reading (open edges): the unknown f_i
     *     is extrapolated with zero gradient from the next interior node. */
    if (!p->frozen_flow) {
        static const int OPP9[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
        for (int i = 0; i < 9; ++i)
#pragma omp parallel for schedule(static)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    int sx = x - CX9[i], sy = y - CY9[i];
                    int xout = sx < 0 || sx >= nx, yout = sy < 0 || sy >= ny;
                    double v;
                    if (yout && s->bc.flow[sy < 0 ? ORC_S : ORC_N] == ORC_WALL) {
                        v = s->fs[OPP9[i] * N + (size_t)y * nx + x];
                    } else {
                        int px = sx, py = sy;
                        if (xout) px = s->bc.flow[ORC_W] == ORC_PERIODIC ? wrap(sx, nx) : x;
                        if (yout) py = s->bc.flow[ORC_S] == ORC_PERIODIC ? wrap(sy, ny) : y;
                        v = s->fs[i * N + (size_t)py * nx + px];
                    }
                    s->fn[i * N + (size_t)y * nx + x] = v;
                }
    }
    /* 11. D2Q5 streaming with the rho c_v blend (Eq. 39):
     *     rho c_v g_i(y, t+1) = g*_i(y - c_i, t) + (rho c_v - 1) g_i(y, t).
     *     reading: rho c_v is taken at the destination node y and time t.
     *     Thermal walls: halfway anti-bounce-back (Dirichlet) or bounce-back
     *     (adiabatic) supplies the incoming post-collision value. */
    {
        static const int OPP5[5] = {0, 3, 4, 1, 2};
        for (int i = 0; i < 5; ++i)
#pragma omp parallel for schedule(static)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    size_t n = (size_t)y * nx + x;
                    int sx = x - CX5[i], sy = y - CY5[i];
                    int edge = -1;
                    if (sx < 0) edge = ORC_W;
                    else if (sx >= nx) edge = ORC_E;
                    else if (sy < 0) edge = ORC_S;
                    else if (sy >= ny) edge = ORC_N;
                    double A;
                    if (edge < 0) {
                        A = s->gs[i * N + (size_t)sy * nx + sx];
                    } else if (s->bc.therm[edge] == ORC_T_PERIODIC) {
                        A = s->gs[i * N + (size_t)wrap(sy, ny) * nx + wrap(sx, nx)];
                    } else if (s->bc.therm[edge] == ORC_T_DIRICHLET) {
                        A = -s->gs[OPP5[i] * N + n] + 2.0 * s->w5[i] * wall_T(s, edge, x);
                    } else {
                        A = s->gs[OPP5[i] * N + n];
                    }
                    double C = s->rho[n] * p->cv;
                    double gold = s->g[i * N + n];
                    s->gn[i * N + n] = gold + (A - gold) / C;
                }
    }
    /* 12. keep P^n; advance */
    if (!p->frozen_flow) {
        double* t = s->f;
        s->f = s->fn;
        s->fn = t;
    }
    if (!p->frozen_thermal) {
        double* t = s->g;
        s->g = s->gn;
        s->gn = t;
    }
    memcpy(s->Pprev, s->Pn, N * sizeof(double));
    s->rho_ave_prev = rho_ave_next;
    s->step += 1;
    if (s->err) return s->err;
    for (size_t n = 0; n < N; ++n)
        if (!isfinite(s->rho[n]) || !isfinite(s->T[n])) {
            s->err = ORC_ENONFINITE;
            return s->err;
        }
    return ORC_OK;
}

int orc_step(orc_sim* s, int n) {
    if (!s || n < 0) return ORC_EINVAL;
    if (s->err) return s->err;
    for (int k = 0; k < n; ++k) {
        int rc = one_step(s);
        if (rc) return rc;
    }
    return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* init, fields, populations                                                */

int orc_init(orc_sim* s, const double* rho, const double* ux, const double* uy,
             const double* T) {
    if (!s || !rho || !ux || !uy || !T) return ORC_EINVAL;
    const size_t N = (size_t)s->nx * s->ny;
    double sum = 0.0;
    for (size_t n = 0; n < N; ++n) {
        double fe[9], ge[5];
        orc_feq(rho[n], ux[n], uy[n], fe);
        orc_geq(&s->p, T[n], ge);
        for (int i = 0; i < 9; ++i) s->f[i * N + n] = fe[i];
        for (int i = 0; i < 5; ++i) s->g[i * N + n] = ge[i];
        s->Pprev[n] = 0.0;
        sum += rho[n];
    }
    s->rho_ave_prev = sum / (double)N;
    s->step = 0;
    s->err = ORC_OK;
    return ORC_OK;
}

int orc_fields(orc_sim* s, double* rho, double* ux, double* uy, double* T) {
    if (!s) return ORC_EINVAL;
    int saved = s->err;
    compute_macro(s);
    const size_t N = (size_t)s->nx * s->ny;
    if (rho) memcpy(rho, s->rho, N * sizeof(double));
    if (ux) memcpy(ux, s->ux, N * sizeof(double));
    if (uy) memcpy(uy, s->uy, N * sizeof(double));
    if (T) memcpy(T, s->T, N * sizeof(double));
    int rc = s->err;
    s->err = saved ? saved : rc;
    return rc;
}

int orc_get_populations(const orc_sim* s, double* f, double* g, double* P) {
    if (!s) return ORC_EINVAL;
    const size_t N = (size_t)s->nx * s->ny;
    if (f) memcpy(f, s->f, 9 * N * sizeof(double));
    if (g) memcpy(g, s->g, 5 * N * sizeof(double));
    if (P) memcpy(P, s->Pprev, N * sizeof(double));
    return ORC_OK;
}

int orc_set_populations(orc_sim* s, const double* f, const double* g, const double* P,
                        long step, double rho_ave_prev) {
    if (!s || !f || !g || !P || step < 0) return ORC_EINVAL;
    const size_t N = (size_t)s->nx * s->ny;
    memcpy(s->f, f, 9 * N * sizeof(double));
    memcpy(s->g, g, 5 * N * sizeof(double));
    memcpy(s->Pprev, P, N * sizeof(double));
    s->step = step;
    s->rho_ave_prev = rho_ave_prev;
    s->err = ORC_OK;
    return ORC_OK;
}

/* test hook: a copy of one per-node quantity as the last step computed it
 * (the phase that produced it is named beside each code in lbm_oracle.h) */
int orc_work(const orc_sim* s, int which, double* out) {
    if (!s || !out) return ORC_EINVAL;
    const size_t N = (size_t)s->nx * s->ny;
    const double* src = NULL;
    size_t n = N;
    switch (which) {
        case ORC_W_RHO: src = s->rho; break;
        case ORC_W_T: src = s->T; break;
        case ORC_W_PSI: src = s->psi; break;
        case ORC_W_FMX: src = s->Fmx; break;
        case ORC_W_FMY: src = s->Fmy; break;
        case ORC_W_FX: src = s->Fx; break;
        case ORC_W_FY: src = s->Fy; break;
        case ORC_W_UX: src = s->ux; break;
        case ORC_W_UY: src = s->uy; break;
        case ORC_W_DIVU: src = s->divu; break;
        case ORC_W_DTX: src = s->dTx; break;
        case ORC_W_DTY: src = s->dTy; break;
        case ORC_W_Q: src = s->Q; break;
        case ORC_W_PN: src = s->Pn; break;
        case ORC_W_S: src = s->Stot; break;
        case ORC_W_FSTAR: src = s->fs; n = 9 * N; break;
        case ORC_W_GSTAR: src = s->gs; n = 5 * N; break;
        case ORC_W_GHOST_PSI_S: src = s->gpsi_S; n = (size_t)s->nx; break;
        case ORC_W_GHOST_PSI_N: src = s->gpsi_N; n = (size_t)s->nx; break;
        default: return ORC_EINVAL;
    }
    memcpy(out, src, n * sizeof(double));
    return ORC_OK;
}

long orc_step_count(const orc_sim* s) { return s ? s->step : -1; }
int orc_last_error(const orc_sim* s) { return s ? s->err : ORC_EINVAL; }

/* ---------------------------------------------------------------------- */
/* diagnostics: mass, energy, droplet / bubble size (Sections 3.3 and 4)    */

int orc_diagnostics(orc_sim* s, double rho_l, double rho_g, int sessile, orc_diag* d) {
    if (!s || !d) return ORC_EINVAL;
    int saved = s->err;
    compute_macro(s);
    s->err = saved;
    const size_t N = (size_t)s->nx * s->ny;
    /* the interface sits at rho = (rho_l + rho_g) / 2 (Section 3.3) */
    double rmid = 0.5 * (rho_l + rho_g);
    memset(d, 0, sizeof(*d));
    for (size_t n = 0; n < N; ++n) {
        double r = s->rho[n], T = s->T[n], ux = s->ux[n], uy = s->uy[n];
        if (!isfinite(r) || !isfinite(T) || !isfinite(ux) || !isfinite(uy)) d->nonfinite += 1;
        d->mass += r;
        d->energy += r * s->p.cv * T;
        if (r > rmid) {
            d->liquid_mass += r;
            d->liquid_area += 1.0;
        }
        double phi = (r - rho_g) / (rho_l - rho_g);
        phi = phi < 0.0 ? 0.0 : (phi > 1.0 ? 1.0 : phi);
        d->liquid_area_smooth += phi;
        double um = sqrt(ux * ux + uy * uy);
        if (um > d->max_u) d->max_u = um;
    }
    /* equivalent diameter of the liquid area: a disc, or a half disc for a
     * droplet sitting on a wall */
    double fac = sessile ? 8.0 / M_PI : 4.0 / M_PI;
    d->diameter = sqrt(fac * d->liquid_area);
    d->diameter_smooth = sqrt(fac * d->liquid_area_smooth);
    d->step = s->step;
    return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* reconfiguration between steps (Section 4.2: the sessile droplet is first */
/* relaxed without evaporation to its contact angle, then the wall heats)   */

int orc_reconfigure(orc_sim* s, const orc_params* p, const orc_bc* bc) {
    if (!s || !p || !bc || !valid_bc(s->nx, s->ny, bc) || p->cv <= 0 || p->nu <= 0 ||
        p->lambda <= 0 || p->w_dot != s->p.w_dot)
        return ORC_EINVAL;
    /* the flow boundary kinds fix the geometry of the problem */
    for (int e = 0; e < 4; ++e)
        if (bc->flow[e] != s->bc.flow[e]) return ORC_EINVAL;
    s->p = *p;
    s->bc = *bc;
    s->Tc = orc_Tc(p);
    s->kpr = pr_k(p);
    s->sp = 1.0 / (3.0 * p->nu + 0.5);
    s->cs2h = p->w_dot / 2.0;
    s->vs12 = 1.0 / (p->lambda / s->cs2h + 0.5);
    s->cot_theta = tan(M_PI / 2.0 - bc->theta_deg * M_PI / 180.0);
    d2q5_weights(p, s->w5);
    double S[9] = {p->s0, p->s_e, p->s_eps, p->s_j, p->s_q, p->s_j, p->s_q, s->sp, s->sp};
    memcpy(s->S, S, sizeof(S));
    double L[5] = {p->vs0, s->vs12, s->vs12, p->vs3, p->vs4};
    memcpy(s->Lam, L, sizeof(L));
    return ORC_OK;
}
