/*
 * FP64 CPU oracle of the three-dimensional form of the coupled step: a D3Q19
 * multiple-relaxation-time pseudopotential flow lattice with a D3Q7
 * temperature lattice carrying the same rho c_v-weighted streaming.  The
 * paper states the model extends to three dimensions (Section 1) and gives
 * the two-dimensional form; every 3-D choice below is a reading, marked
 * "reading:" where it is taken.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/ (and nothing in the product
 * path).  It shares no code with the CUDA library.
 *
 * Geometry: x and y periodic; z periodic, or walls at the bottom (z = -1/2)
 * and top (z = nz - 1/2) with halfway bounce-back, the wetting ghost layer and
 * Dirichlet (anti-bounce-back) or adiabatic thermal conditions.
 *
 * Per step, in the order of the two-dimensional oracle:
 *   1. rho = sum f, T = sum g
 *   2. psi from the Peng-Robinson EOS; wetting ghost layers of walls
 *   3. F_m = -G psi(x) sum_i varpi(|c_i|^2) psi(x + c_i) c_i, varpi = 1/6, 1/12
 *   4. F = F_m + (rho - rho_ave)(0, 0, -g); rho u = sum c f + F/2
 *   5. div u (isotropic central difference, D3Q19 weights)
 *   6. grad T from the local first moments of g
 *   7. (dp/dT)_rho, Q, P^n = Q/(rho c_v), S
 *   8. D3Q19 MRT collision with the forcing moments
 *   9. D3Q7 MRT collision
 *  10. pull streaming of f, halfway bounce-back at walls
 *  11. weighted streaming of g, anti-bounce-back / bounce-back at walls
 *  12. keep P^n
 *
 * Pins (tests/test_oracle_3d.py): velocity set and weights, the moment
 * matrices (orthogonality of M, inverses), M f^eq against the textbook
 * moments, the forcing moments against M of the discrete force term, mass
 * conservation, zero total momentum, the uniform fixed point, the cubic
 * symmetry of a centred droplet, the exact Fourier amplification of the
 * thermal lattice and its continuum limit, the reduction of the thermal
 * lattice to the textbook D3Q7 scheme when rho c_v = 1, steady conduction
 * between walls, flat-interface coexistence against Maxwell and the
 * two-dimensional oracle, and the Laplace law for spheres.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* D3Q19: rest, 6 axis, 12 edge directions; opposite pairs (2k-1, 2k) */
static const int CX[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CY[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZ[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
static const int OPP[19] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};
/* D3Q7: rest and the 6 axis directions */
static const int HX[7] = {0, 1, -1, 0, 0, 0, 0};
static const int HY[7] = {0, 0, 0, 1, -1, 0, 0};
static const int HZ[7] = {0, 0, 0, 0, 0, 1, -1};
static const int HOPP[7] = {0, 2, 1, 4, 3, 6, 5};

static double w19(int i) {
    int c2 = CX[i] * CX[i] + CY[i] * CY[i] + CZ[i] * CZ[i];
    return c2 == 0 ? 1.0 / 3.0 : (c2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
}

struct orc3_sim {
    int nx, ny, nz;
    orc_params p;
    orc_bc3 bc;
    double cot_theta, sp, vs1, cs2h;
    double M[361], Minv[361], Mh[49], Mhinv[49];
    double S[19], Lam[7], wh[7];
    double *f, *g, *Pprev;
    long step;
    double rho_ave_prev;
    int err;
    double *rho, *T, *psi, *Fmx, *Fmy, *Fmz, *Fx, *Fy, *Fz, *ux, *uy, *uz;
    double *divu, *dTx, *dTy, *dTz, *Q, *Pn, *Stot;
    double *fs, *gs, *fn, *gn;
    double *gpsi_b, *gpsi_t;   /* ghost-layer psi below z = 0 and above z = nz-1 */
};

/* ---------------------------------------------------------------------- */

static int gj_inv(const double* A, double* Ai, int n) {
    double* a = (double*)malloc(sizeof(double) * n * 2 * n);
    if (!a) return ORC_ENOMEM;
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < 2 * n; ++c)
            a[r * 2 * n + c] = c < n ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(a[r * 2 * n + c]) > fabs(a[piv * 2 * n + c])) piv = r;
        if (a[piv * 2 * n + c] == 0.0) {
            free(a);
            return ORC_EINVAL;
        }
        for (int k = 0; k < 2 * n; ++k) {
            double t = a[c * 2 * n + k];
            a[c * 2 * n + k] = a[piv * 2 * n + k];
            a[piv * 2 * n + k] = t;
        }
        double d = a[c * 2 * n + c];
        for (int k = 0; k < 2 * n; ++k) a[c * 2 * n + k] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double m = a[r * 2 * n + c];
            for (int k = 0; k < 2 * n; ++k) a[r * 2 * n + k] -= m * a[c * 2 * n + k];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) Ai[r * n + c] = a[r * 2 * n + n + c];
    free(a);
    return ORC_OK;
}

static void mv(const double* A, const double* x, double* y, int n) {
    for (int r = 0; r < n; ++r) {
        double s = 0.0;
        for (int c = 0; c < n; ++c) s += A[r * n + c] * x[c];
        y[r] = s;
    }
}

/* The D3Q19 moment basis of d'Humieres et al. (2002), written as polynomials
 * of the velocity c: rho, e, epsilon, j_x, q_x, j_y, q_y, j_z, q_z, 3p_xx,
 * 3pi_xx, p_ww, pi_ww, p_xy, p_yz, p_xz, m_x, m_y, m_z.
 * reading: the paper's matrix (Eq. 4) is the two-dimensional member of this
 * family (Lallemand & Luo), so the three-dimensional flow lattice takes it. */
static void moment_row(int k, int i, double* v) {
    const double x = CX[i], y = CY[i], z = CZ[i];
    const double c2 = x * x + y * y + z * z;
    switch (k) {
    case 0: *v = 1.0; break;
    case 1: *v = 19.0 * c2 - 30.0; break;
    case 2: *v = (21.0 * c2 * c2 - 53.0 * c2 + 24.0) / 2.0; break;
    case 3: *v = x; break;
    case 4: *v = (5.0 * c2 - 9.0) * x; break;
    case 5: *v = y; break;
    case 6: *v = (5.0 * c2 - 9.0) * y; break;
    case 7: *v = z; break;
    case 8: *v = (5.0 * c2 - 9.0) * z; break;
    case 9: *v = 3.0 * x * x - c2; break;
    case 10: *v = (3.0 * c2 - 5.0) * (3.0 * x * x - c2); break;
    case 11: *v = y * y - z * z; break;
    case 12: *v = (3.0 * c2 - 5.0) * (y * y - z * z); break;
    case 13: *v = x * y; break;
    case 14: *v = y * z; break;
    case 15: *v = x * z; break;
    case 16: *v = (y * y - z * z) * x; break;
    case 17: *v = (z * z - x * x) * y; break;
    default: *v = (x * x - y * y) * z; break;
    }
}

/* reading: the D3Q7 matrix is the three-dimensional form of Eq. 40 (the
 * paper's non-orthogonal D2Q5 matrix): rows 1, c_x, c_y, c_z, |c|^2,
 * c_x^2 - c_y^2, c_y^2 - c_z^2. */
static void moment_row7(int k, int i, double* v) {
    const double x = HX[i], y = HY[i], z = HZ[i];
    switch (k) {
    case 0: *v = 1.0; break;
    case 1: *v = x; break;
    case 2: *v = y; break;
    case 3: *v = z; break;
    case 4: *v = x * x + y * y + z * z; break;
    case 5: *v = x * x - y * y; break;
    default: *v = y * y - z * z; break;
    }
}

void orc3_matrices(double M[361], double Minv[361], double Mh[49], double Mhinv[49]) {
    for (int k = 0; k < 19; ++k)
        for (int i = 0; i < 19; ++i) moment_row(k, i, &M[k * 19 + i]);
    for (int k = 0; k < 7; ++k)
        for (int i = 0; i < 7; ++i) moment_row7(k, i, &Mh[k * 7 + i]);
    gj_inv(M, Minv, 19);
    gj_inv(Mh, Mhinv, 7);
}

void orc3_velocities(int cx[19], int cy[19], int cz[19], double w[19]) {
    for (int i = 0; i < 19; ++i) {
        cx[i] = CX[i];
        cy[i] = CY[i];
        cz[i] = CZ[i];
        w[i] = w19(i);
    }
}

/* second-order equilibrium, c_s^2 = 1/3 */
void orc3_feq(double rho, double ux, double uy, double uz, double f[19]) {
    const double uu = ux * ux + uy * uy + uz * uz;
    for (int i = 0; i < 19; ++i) {
        const double cu = CX[i] * ux + CY[i] * uy + CZ[i] * uz;
        f[i] = w19(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

/* the discrete force term whose moments are the forcing vector:
 * F_i = w_i [3 (c_i - u) + 9 (c_i . u) c_i] . F (Guo, Zheng & Shi 2002) */
void orc3_force_term(double ux, double uy, double uz, double Fx, double Fy, double Fz,
                     double out[19]) {
    for (int i = 0; i < 19; ++i) {
        const double cu = CX[i] * ux + CY[i] * uy + CZ[i] * uz;
        const double ax = 3.0 * (CX[i] - ux) + 9.0 * cu * CX[i];
        const double ay = 3.0 * (CY[i] - uy) + 9.0 * cu * CY[i];
        const double az = 3.0 * (CZ[i] - uz) + 9.0 * cu * CZ[i];
        out[i] = w19(i) * (ax * Fx + ay * Fy + az * Fz);
    }
}

/* ---------------------------------------------------------------------- */

static int valid_bc3(int nz, const orc_bc3* bc) {
    if (bc->flow_z != ORC_PERIODIC && bc->flow_z != ORC_WALL) return 0;
    for (int e = 0; e < 2; ++e) {
        if (bc->therm[e] < 0 || bc->therm[e] > 2) return 0;
        if ((bc->flow_z == ORC_PERIODIC) != (bc->therm[e] == ORC_T_PERIODIC)) return 0;
    }
    if (bc->flow_z == ORC_WALL && nz < 2) return 0;
    return 1;
}

static void derive(orc3_sim* s) {
    const orc_params* p = &s->p;
    s->sp = 1.0 / (3.0 * p->nu + 0.5);
    /* reading: c^_s^2 = w_dot / 3 for D3Q7 with rest weight 1 - w_dot and
     * moving weights w_dot / 6 (the D2Q5 choice of Section 3.2.1 in 3-D) */
    s->cs2h = p->w_dot / 3.0;
    s->vs1 = 1.0 / (p->lambda / s->cs2h + 0.5);
    s->cot_theta = tan(M_PI / 2.0 - s->bc.theta_deg * M_PI / 180.0);
    s->wh[0] = 1.0 - p->w_dot;
    for (int i = 1; i < 7; ++i) s->wh[i] = p->w_dot / 6.0;
    /* reading: s_rho = s_0, s_e, s_eps, s_j, s_q as in two dimensions; the
     * five stress moments (3p_xx, p_ww, p_xy, p_yz, p_xz) relax with s_p of
     * the viscosity; pi_xx, pi_ww and the third-order m_x,y,z with s_q. */
    const double sq = p->s_q;
    double S[19] = {p->s0, p->s_e, p->s_eps, p->s_j, sq, p->s_j, sq, p->s_j, sq,
                    s->sp, sq, s->sp, sq, s->sp, s->sp, s->sp, sq, sq, sq};
    memcpy(s->S, S, sizeof(S));
    double L[7] = {p->vs0, s->vs1, s->vs1, s->vs1, p->vs3, p->vs4, p->vs4};
    memcpy(s->Lam, L, sizeof(L));
}

orc3_sim* orc3_create(int nx, int ny, int nz, const orc_params* p, const orc_bc3* bc, int* err) {
    if (err) *err = ORC_OK;
    if (nx < 1 || ny < 1 || nz < 1 || !p || !bc || !valid_bc3(nz, bc) || p->cv <= 0 ||
        p->w_dot <= 0 || p->w_dot >= 1 || p->nu <= 0 || p->lambda <= 0) {
        if (err) *err = ORC_EINVAL;
        return NULL;
    }
    orc3_sim* s = (orc3_sim*)calloc(1, sizeof(orc3_sim));
    if (!s) {
        if (err) *err = ORC_ENOMEM;
        return NULL;
    }
    s->nx = nx;
    s->ny = ny;
    s->nz = nz;
    s->p = *p;
    s->bc = *bc;
    derive(s);
    orc3_matrices(s->M, s->Minv, s->Mh, s->Mhinv);
    const size_t N = (size_t)nx * ny * nz;
    double** one[] = {&s->rho, &s->T, &s->psi, &s->Fmx, &s->Fmy, &s->Fmz, &s->Fx, &s->Fy,
                      &s->Fz, &s->ux, &s->uy, &s->uz, &s->divu, &s->dTx, &s->dTy, &s->dTz,
                      &s->Q, &s->Pn, &s->Stot, &s->Pprev};
    for (size_t k = 0; k < sizeof(one) / sizeof(one[0]); ++k)
        if (!(*one[k] = (double*)calloc(N, sizeof(double)))) goto oom;
    if (!(s->f = (double*)calloc(19 * N, sizeof(double)))) goto oom;
    if (!(s->fs = (double*)calloc(19 * N, sizeof(double)))) goto oom;
    if (!(s->fn = (double*)calloc(19 * N, sizeof(double)))) goto oom;
    if (!(s->g = (double*)calloc(7 * N, sizeof(double)))) goto oom;
    if (!(s->gs = (double*)calloc(7 * N, sizeof(double)))) goto oom;
    if (!(s->gn = (double*)calloc(7 * N, sizeof(double)))) goto oom;
    if (!(s->gpsi_b = (double*)calloc((size_t)nx * ny, sizeof(double)))) goto oom;
    if (!(s->gpsi_t = (double*)calloc((size_t)nx * ny, sizeof(double)))) goto oom;
    return s;
oom:
    orc3_destroy(s);
    if (err) *err = ORC_ENOMEM;
    return NULL;
}

void orc3_destroy(orc3_sim* s) {
    if (!s) return;
    double* all[] = {s->rho, s->T, s->psi, s->Fmx, s->Fmy, s->Fmz, s->Fx, s->Fy, s->Fz,
                     s->ux, s->uy, s->uz, s->divu, s->dTx, s->dTy, s->dTz, s->Q, s->Pn,
                     s->Stot, s->Pprev, s->f, s->fs, s->fn, s->g, s->gs, s->gn, s->gpsi_b,
                     s->gpsi_t};
    for (size_t k = 0; k < sizeof(all) / sizeof(all[0]); ++k) free(all[k]);
    free(s);
}

static int wr(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

#define ID(x, y, z) (((size_t)(z) * s->ny + (y)) * s->nx + (x))

/* psi at a node one layer beyond the domain at most: x, y wrap; z wraps or
 * reads the wall's ghost layer */
static double psi_at(const orc3_sim* s, int x, int y, int z) {
    x = wr(x, s->nx);
    y = wr(y, s->ny);
    if (z >= 0 && z < s->nz) return s->psi[ID(x, y, z)];
    if (s->bc.flow_z == ORC_PERIODIC) return s->psi[ID(x, y, wr(z, s->nz))];
    return z < 0 ? s->gpsi_b[(size_t)y * s->nx + x] : s->gpsi_t[(size_t)y * s->nx + x];
}

/* velocity beyond the domain for div u: walls carry u = 0 */
static void u_at(const orc3_sim* s, int x, int y, int z, double* u) {
    x = wr(x, s->nx);
    y = wr(y, s->ny);
    if (z < 0 || z >= s->nz) {
        if (s->bc.flow_z == ORC_WALL) {
            u[0] = u[1] = u[2] = 0.0;
            return;
        }
        z = wr(z, s->nz);
    }
    const size_t n = ID(x, y, z);
    u[0] = s->ux[n];
    u[1] = s->uy[n];
    u[2] = s->uz[n];
}

static void macro3(orc3_sim* s) {
    const int nx = s->nx, ny = s->ny, nz = s->nz;
    const size_t N = (size_t)nx * ny * nz;
    const orc_params* p = &s->p;
    for (size_t n = 0; n < N; ++n) {
        double r = 0.0, t = 0.0;
        for (int i = 0; i < 19; ++i) r += s->f[i * N + n];
        for (int i = 0; i < 7; ++i) t += s->g[i * N + n];
        s->rho[n] = r;
        s->T[n] = t;
    }
    for (size_t n = 0; n < N; ++n) {
        const double q = orc_psi2(p, s->rho[n], s->T[n]);
        if (!(q >= 0.0)) s->err = ORC_EPSI;
        s->psi[n] = sqrt(q);
    }
    /* reading: the wetting ghost layer of Section 3.3 in 3-D,
     * rho_ghost = rho(layer 2) + tan(pi/2 - theta) |grad_t rho(layer 1)| with
     * the tangential differences taken over two spacings as in 2-D:
     * sqrt((rho(x+1) - rho(x-1))^2 + (rho(y+1) - rho(y-1))^2). */
    if (s->bc.flow_z == ORC_WALL) {
        for (int e = 0; e < 2; ++e) {
            const int z1 = e == 0 ? 0 : nz - 1, z2 = e == 0 ? 1 : nz - 2;
            double* gp = e == 0 ? s->gpsi_b : s->gpsi_t;
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    const double dx = s->rho[ID(wr(x + 1, nx), y, z1)] - s->rho[ID(wr(x - 1, nx), y, z1)];
                    const double dy = s->rho[ID(x, wr(y + 1, ny), z1)] - s->rho[ID(x, wr(y - 1, ny), z1)];
                    const double rg = s->rho[ID(x, y, z2)] + s->cot_theta * sqrt(dx * dx + dy * dy);
                    /* reading: psi of the ghost at the temperature of
                                     * the fluid node next to it (as in 2-D) */
                    const double tg = s->T[ID(x, y, z1)];
                    const double q = orc_psi2(p, rg, tg);
                    if (!(q >= 0.0)) s->err = ORC_EPSI;
                    gp[(size_t)y * nx + x] = sqrt(q);
                }
        }
    }
    /* F_m with the D3Q19 isotropy weights varpi(1) = 1/6, varpi(2) = 1/12 */
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double sx = 0.0, sy = 0.0, sz = 0.0;
                for (int i = 1; i < 19; ++i) {
                    const double wv = i < 7 ? 1.0 / 6.0 : 1.0 / 12.0;
                    const double pn = psi_at(s, x + CX[i], y + CY[i], z + CZ[i]);
                    sx += wv * pn * CX[i];
                    sy += wv * pn * CY[i];
                    sz += wv * pn * CZ[i];
                }
                const size_t n = ID(x, y, z);
                s->Fmx[n] = -p->G * s->psi[n] * sx;
                s->Fmy[n] = -p->G * s->psi[n] * sy;
                s->Fmz[n] = -p->G * s->psi[n] * sz;
            }
    for (size_t n = 0; n < N; ++n) {
        s->Fx[n] = s->Fmx[n];
        s->Fy[n] = s->Fmy[n];
        s->Fz[n] = s->Fmz[n] - (s->rho[n] - s->rho_ave_prev) * p->gravity;
        if (p->frozen_flow) {
            s->ux[n] = s->uy[n] = s->uz[n] = 0.0;
            continue;
        }
        double jx = 0.0, jy = 0.0, jz = 0.0;
        for (int i = 0; i < 19; ++i) {
            jx += CX[i] * s->f[i * N + n];
            jy += CY[i] * s->f[i * N + n];
            jz += CZ[i] * s->f[i * N + n];
        }
        s->ux[n] = (jx + 0.5 * s->Fx[n]) / s->rho[n];
        s->uy[n] = (jy + 0.5 * s->Fy[n]) / s->rho[n];
        s->uz[n] = (jz + 0.5 * s->Fz[n]) / s->rho[n];
    }
}

static int step3(orc3_sim* s) {
    const int nx = s->nx, ny = s->ny, nz = s->nz;
    const size_t N = (size_t)nx * ny * nz;
    const orc_params* p = &s->p;
    macro3(s);
    double rsum = 0.0;
    for (size_t n = 0; n < N; ++n) rsum += s->rho[n];
    /* div u: (1/c_s^2) sum_i w_i c_i . u(x + c_i) */
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double d = 0.0, u[3];
                for (int i = 1; i < 19; ++i) {
                    u_at(s, x + CX[i], y + CY[i], z + CZ[i], u);
                    d += 3.0 * w19(i) * (CX[i] * u[0] + CY[i] * u[1] + CZ[i] * u[2]);
                }
                s->divu[ID(x, y, z)] = d;
            }
    /* grad T: c^_s^2 d_a T = -varsigma_1 m^_a (first moments, m^eq = 0) */
    for (size_t n = 0; n < N; ++n) {
        double gl[7], m[7];
        for (int i = 0; i < 7; ++i) gl[i] = s->g[i * N + n];
        mv(s->Mh, gl, m, 7);
        s->dTx[n] = -s->Lam[1] * m[1] / s->cs2h;
        s->dTy[n] = -s->Lam[2] * m[2] / s->cs2h;
        s->dTz[n] = -s->Lam[3] * m[3] / s->cs2h;
    }
    /* Q, P^n, S as in two dimensions (Eqs. 20, 24) */
    for (size_t n = 0; n < N; ++n) {
        const double C = s->rho[n] * p->cv;
        const double q = -(C * (s->ux[n] * s->dTx[n] + s->uy[n] * s->dTy[n] + s->uz[n] * s->dTz[n]) +
                           s->T[n] * orc_dpdT(p, s->rho[n], s->T[n]) * s->divu[n]);
        const double Pn = q / C;
        const double Pp = s->step == 0 ? Pn : s->Pprev[n];
        s->Q[n] = q;
        s->Pn[n] = Pn;
        s->Stot[n] = C * 0.5 * (Pn - Pp);
    }
    /* D3Q19 MRT collision: m* = m - S (m - m^eq) + (I - S/2) Fbar, with
     * m^eq = M f^eq and Fbar = M F (the discrete force term).
     * reading: Li's sigma term acts on the energy moment e only, sized so the
     * diagonal of the momentum flux changes by the same amount as in 2-D:
     * e = sum (19 |c|^2 - 30) f gives sum |c|^2 f = (e + 30 rho)/19, so the
     * 2-D source 12 sigma |F_m|^2 / (psi^2 (tau_e - 1/2)) (per diagonal
     * entry / 6) becomes (19/2) sigma |F_m|^2 / (psi^2 (1/s_e - 1/2)). */
    if (!p->frozen_flow) {
        for (size_t n = 0; n < N; ++n) {
            double fl[19], m[19], fe[19], meq[19], ft[19], Fb[19], ms[19], fo[19];
            for (int i = 0; i < 19; ++i) fl[i] = s->f[i * N + n];
            mv(s->M, fl, m, 19);
            orc3_feq(s->rho[n], s->ux[n], s->uy[n], s->uz[n], fe);
            mv(s->M, fe, meq, 19);
            orc3_force_term(s->ux[n], s->uy[n], s->uz[n], s->Fx[n], s->Fy[n], s->Fz[n], ft);
            mv(s->M, ft, Fb, 19);
            const double Fm2 = s->Fmx[n] * s->Fmx[n] + s->Fmy[n] * s->Fmy[n] + s->Fmz[n] * s->Fmz[n];
            Fb[1] += 9.5 * p->sigma * Fm2 / (s->psi[n] * s->psi[n] * (1.0 / s->S[1] - 0.5));
            for (int k = 0; k < 19; ++k)
                ms[k] = m[k] - s->S[k] * (m[k] - meq[k]) + (1.0 - 0.5 * s->S[k]) * Fb[k];
            mv(s->Minv, ms, fo, 19);
            for (int i = 0; i < 19; ++i) s->fs[i * N + n] = fo[i];
        }
    }
    /* D3Q7 MRT collision: m^eq = [T, 0, 0, 0, w_dot T, 0, 0], source M^(w^ (Q + S)) */
    for (size_t n = 0; n < N; ++n) {
        double gl[7], m[7], src[7], msrc[7], ms[7], go[7];
        for (int i = 0; i < 7; ++i) gl[i] = s->g[i * N + n];
        mv(s->Mh, gl, m, 7);
        const double T = s->T[n];
        const double meq[7] = {T, 0.0, 0.0, 0.0, p->w_dot * T, 0.0, 0.0};
        for (int i = 0; i < 7; ++i) src[i] = s->wh[i] * (s->Q[n] + s->Stot[n]);
        mv(s->Mh, src, msrc, 7);
        for (int k = 0; k < 7; ++k) ms[k] = m[k] - s->Lam[k] * (m[k] - meq[k]) + msrc[k];
        mv(s->Mhinv, ms, go, 7);
        for (int i = 0; i < 7; ++i) s->gs[i * N + n] = go[i];
    }
    /* pull streaming of f; walls: halfway bounce-back */
    if (!p->frozen_flow) {
        for (int i = 0; i < 19; ++i)
            for (int z = 0; z < nz; ++z)
                for (int y = 0; y < ny; ++y)
                    for (int x = 0; x < nx; ++x) {
                        const int sz = z - CZ[i];
                        double v;
                        if ((sz < 0 || sz >= nz) && s->bc.flow_z == ORC_WALL)
                            v = s->fs[OPP[i] * N + ID(x, y, z)];
                        else
                            v = s->fs[i * N + ID(wr(x - CX[i], nx), wr(y - CY[i], ny), wr(sz, nz))];
                        s->fn[i * N + ID(x, y, z)] = v;
                    }
    }
    /* weighted streaming of g (Eq. 39 in 3-D); walls: anti-bounce-back
     * A = -g*_opp + 2 w^_i T_w (Dirichlet) or A = g*_opp (adiabatic) */
    for (int i = 0; i < 7; ++i)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    const size_t n = ID(x, y, z);
                    const int sz = z - HZ[i];
                    double A;
                    if ((sz < 0 || sz >= nz) && s->bc.flow_z == ORC_WALL) {
                        const int e = sz < 0 ? 0 : 1;
                        if (s->bc.therm[e] == ORC_T_DIRICHLET)
                            A = -s->gs[HOPP[i] * N + n] + 2.0 * s->wh[i] * s->bc.T_edge[e];
                        else
                            A = s->gs[HOPP[i] * N + n];
                    } else {
                        A = s->gs[i * N + ID(wr(x - HX[i], nx), wr(y - HY[i], ny), wr(sz, nz))];
                    }
                    const double C = s->rho[n] * p->cv;
                    const double go = s->g[i * N + n];
                    s->gn[i * N + n] = go + (A - go) / C;
                }
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
    s->rho_ave_prev = rsum / (double)N;
    s->step += 1;
    if (s->err) return s->err;
    for (size_t n = 0; n < N; ++n)
        if (!isfinite(s->rho[n]) || !isfinite(s->T[n])) return s->err = ORC_ENONFINITE;
    return ORC_OK;
}

int orc3_step(orc3_sim* s, int n) {
    if (!s || n < 0) return ORC_EINVAL;
    if (s->err) return s->err;
    for (int k = 0; k < n; ++k) {
        int rc = step3(s);
        if (rc) return rc;
    }
    return ORC_OK;
}

int orc3_init(orc3_sim* s, const double* rho, const double* ux, const double* uy,
              const double* uz, const double* T) {
    if (!s || !rho || !ux || !uy || !uz || !T) return ORC_EINVAL;
    const size_t N = (size_t)s->nx * s->ny * s->nz;
    double sum = 0.0;
    for (size_t n = 0; n < N; ++n) {
        double fe[19];
        orc3_feq(rho[n], ux[n], uy[n], uz[n], fe);
        for (int i = 0; i < 19; ++i) s->f[i * N + n] = fe[i];
        for (int i = 0; i < 7; ++i) s->g[i * N + n] = s->wh[i] * T[n];
        s->Pprev[n] = 0.0;
        sum += rho[n];
    }
    s->rho_ave_prev = sum / (double)N;
    s->step = 0;
    s->err = ORC_OK;
    return ORC_OK;
}

int orc3_fields(orc3_sim* s, double* rho, double* ux, double* uy, double* uz, double* T) {
    if (!s) return ORC_EINVAL;
    const int saved = s->err;
    macro3(s);
    const size_t N = (size_t)s->nx * s->ny * s->nz;
    if (rho) memcpy(rho, s->rho, N * sizeof(double));
    if (ux) memcpy(ux, s->ux, N * sizeof(double));
    if (uy) memcpy(uy, s->uy, N * sizeof(double));
    if (uz) memcpy(uz, s->uz, N * sizeof(double));
    if (T) memcpy(T, s->T, N * sizeof(double));
    const int rc = s->err;
    s->err = saved ? saved : rc;
    return rc;
}

int orc3_get_populations(const orc3_sim* s, double* f, double* g, double* P) {
    if (!s) return ORC_EINVAL;
    const size_t N = (size_t)s->nx * s->ny * s->nz;
    if (f) memcpy(f, s->f, 19 * N * sizeof(double));
    if (g) memcpy(g, s->g, 7 * N * sizeof(double));
    if (P) memcpy(P, s->Pprev, N * sizeof(double));
    return ORC_OK;
}

int orc3_set_populations(orc3_sim* s, const double* f, const double* g, const double* P,
                         long step, double rho_ave_prev) {
    if (!s || !f || !g || !P || step < 0) return ORC_EINVAL;
    const size_t N = (size_t)s->nx * s->ny * s->nz;
    memcpy(s->f, f, 19 * N * sizeof(double));
    memcpy(s->g, g, 7 * N * sizeof(double));
    memcpy(s->Pprev, P, N * sizeof(double));
    s->step = step;
    s->rho_ave_prev = rho_ave_prev;
    s->err = ORC_OK;
    return ORC_OK;
}

long orc3_step_count(const orc3_sim* s) { return s ? s->step : -1; }

/* mass, energy, liquid volume above rho_mid, smooth liquid volume, the
 * equivalent sphere (or hemisphere when sessile) diameters, max |u| */
int orc3_diagnostics(orc3_sim* s, double rho_l, double rho_g, int sessile, orc_diag* d) {
    if (!s || !d) return ORC_EINVAL;
    const int saved = s->err;
    macro3(s);
    s->err = saved;
    const size_t N = (size_t)s->nx * s->ny * s->nz;
    const double rmid = 0.5 * (rho_l + rho_g);
    memset(d, 0, sizeof(*d));
    for (size_t n = 0; n < N; ++n) {
        const double r = s->rho[n], T = s->T[n];
        const double ux = s->ux[n], uy = s->uy[n], uz = s->uz[n];
        if (!isfinite(r) || !isfinite(T) || !isfinite(ux) || !isfinite(uy) || !isfinite(uz))
            d->nonfinite += 1;
        d->mass += r;
        d->energy += r * s->p.cv * T;
        if (r > rmid) {
            d->liquid_mass += r;
            d->liquid_area += 1.0;
        }
        double ph = (r - rho_g) / (rho_l - rho_g);
        ph = ph < 0.0 ? 0.0 : (ph > 1.0 ? 1.0 : ph);
        d->liquid_area_smooth += ph;
        const double um = sqrt(ux * ux + uy * uy + uz * uz);
        if (um > d->max_u) d->max_u = um;
    }
    const double fac = sessile ? 12.0 / M_PI : 6.0 / M_PI;
    d->diameter = cbrt(fac * d->liquid_area);
    d->diameter_smooth = cbrt(fac * d->liquid_area_smooth);
    d->step = s->step;
    return ORC_OK;
}
