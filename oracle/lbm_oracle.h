/*
 * FP64 CPU oracle for the coupled time step of the thermal lattice Boltzmann
 * model for liquid-vapor phase change (Wang, Huang & He, arXiv 2205.00686).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference that the
 * CUDA path is checked against.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it; the product path never does.  It
 * shares no code, header, table or helper with the CUDA library.
 *
 * Every field array is row-major [ny][nx] (x fastest), node (0,0) at the
 * south-west corner.  Populations are [q][ny][nx].  Everything is double.
 *
 * Parity status per function (see the headers of lbm_oracle.c and
 * lbm_oracle_analysis.c for the pins): all functions declared here are pinned
 * by tests in tests/test_oracle_*.py.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* edge indices */
#define ORC_W 0
#define ORC_E 1
#define ORC_S 2
#define ORC_N 3

/* flow boundary kinds */
#define ORC_PERIODIC 0
#define ORC_WALL 1
#define ORC_OPEN 2

/* thermal boundary kinds */
#define ORC_T_PERIODIC 0
#define ORC_T_DIRICHLET 1
#define ORC_T_ADIABATIC 2

/* error codes */
#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_ENONFINITE (-3)
#define ORC_EPSI (-4)

typedef struct {
    /* Peng-Robinson EOS (Section 2): a, b, gas constant R, acentric factor */
    double a, b, R, omega;
    /* interaction strength G and the Li forcing parameter sigma (Section 2) */
    double G, sigma;
    /* kinematic viscosity -> s_p; the other D2Q9 rates */
    double nu, s0, s_e, s_eps, s_j, s_q;
    /* thermal conductivity lambda -> varsigma_1 = varsigma_2; c_v; w_dot */
    double lambda, cv, w_dot;
    /* the other D2Q5 rates varsigma_0, varsigma_3, varsigma_4 */
    double vs0, vs3, vs4;
    /* gravity magnitude g, body force (rho - rho_ave)(0, -g) (Section 4.3) */
    double gravity;
    /* test hook: u == 0 and rho fixed, only the thermal lattice advances */
    int frozen_flow;
    /* isothermal hook: g is left unchanged, only the flow lattice advances */
    int frozen_thermal;
} orc_params;

typedef struct {
    int flow[4];        /* ORC_PERIODIC / ORC_WALL / ORC_OPEN per edge W,E,S,N */
    int therm[4];       /* ORC_T_* per edge */
    double T_edge[4];   /* wall / Dirichlet temperature per edge */
    double theta_deg;   /* equilibrium contact angle of walls (Section 3.3) */
    int heater_x0, heater_x1;   /* heater segment [x0,x1) on the south edge */
    double T_heater;
} orc_bc;

typedef struct {
    double mass, energy, liquid_mass, liquid_area, liquid_area_smooth;
    double diameter, diameter_smooth, max_u;
    long step;
    int nonfinite;
} orc_diag;

/* contact angle of a sessile droplet on the south wall (Section 4.2) */
typedef struct {
    double theta_deg;        /* angle inside the liquid */
    double xc, yc, radius;   /* fitted circle, lattice units, node (0,0) at origin */
    double base_width;       /* chord of the circle on the wall line y = -1/2 */
    double height;           /* apex height above the wall line */
    int n_points;            /* interface points in the fit */
} orc_contact;

/* one 4-connected region of the vapour (or liquid) phase */
typedef struct {
    long long label;         /* smallest node index y * nx + x in the region */
    long long area;          /* nodes */
    long long sum_y;         /* sum of the nodes' row indices */
    int y_min, y_max;
    int touches_w, touches_e, touches_s, touches_n;
} orc_component;

typedef struct orc_sim orc_sim;

/* derived constants and closed forms ---------------------------------- */
double orc_Tc(const orc_params* p);
double orc_p_eos(const orc_params* p, double rho, double T);
double orc_dpdT(const orc_params* p, double rho, double T);
double orc_psi2(const orc_params* p, double rho, double T);
int orc_maxwell(const orc_params* p, double T, double* rho_g, double* rho_l);
void orc_feq(double rho, double ux, double uy, double f[9]);
void orc_geq(const orc_params* p, double T, double g[5]);
void orc_matrices(double M[81], double Minv[81], double Mh[25], double Mhinv[25]);
void orc_meq(double rho, double ux, double uy, double meq[9]);
void orc_set_defaults(orc_params* p);

/* simulation ----------------------------------------------------------- */
orc_sim* orc_create(int nx, int ny, const orc_params* p, const orc_bc* bc, int* err);
void orc_destroy(orc_sim* s);
int orc_init(orc_sim* s, const double* rho, const double* ux, const double* uy,
             const double* T);
int orc_step(orc_sim* s, int n);
int orc_fields(orc_sim* s, double* rho, double* ux, double* uy, double* T);
int orc_get_populations(const orc_sim* s, double* f, double* g, double* P);
int orc_set_populations(orc_sim* s, const double* f, const double* g, const double* P,
                        long step, double rho_ave_prev);
long orc_step_count(const orc_sim* s);
/* test hook: copies one per-node work array of the last step into out
 * ([ny][nx]; [9][ny][nx] for f*, [5][ny][nx] for g*, [nx] for a ghost row).
 * The values are those of the last orc_step (orc_fields and orc_diagnostics
 * refresh the phase 1-4 arrays from the current state). */
enum {
    ORC_W_RHO = 0, ORC_W_T, ORC_W_PSI,     /* phases 1-2 */
    ORC_W_FMX, ORC_W_FMY,                  /* phase 3, F_m (Eq. 9) */
    ORC_W_FX, ORC_W_FY, ORC_W_UX, ORC_W_UY, /* phase 4, F_n and u (Eq. 11) */
    ORC_W_DIVU,                            /* phase 5 */
    ORC_W_DTX, ORC_W_DTY,                  /* phase 6, Eqs. 49-50 */
    ORC_W_Q, ORC_W_PN, ORC_W_S,            /* phase 7: Q (Eq. 20), P^n, sum_i S_i (Eq. 24) */
    ORC_W_FSTAR, ORC_W_GSTAR,              /* phases 8-9, post-collision populations */
    ORC_W_GHOST_PSI_S, ORC_W_GHOST_PSI_N   /* Section 3.3 ghost rows of psi */
};
int orc_work(const orc_sim* s, int which, double* out);

int orc_diagnostics(orc_sim* s, double rho_l, double rho_g, int sessile, orc_diag* d);
int orc_last_error(const orc_sim* s);
/* replaces params and boundary values between steps; the flow boundary kinds
 * and w_dot must stay as created (ORC_EINVAL otherwise) */
int orc_reconfigure(orc_sim* s, const orc_params* p, const orc_bc* bc);

/* interface analyses on a density field [ny][nx] (lbm_oracle_analysis.c) -- */
/* interface points rho = rho_mid on lattice links at rows >= skip_rows; writes
 * at most max_points and returns the total count (or ORC_EINVAL) */
int orc_interface_points(const double* rho, int nx, int ny, double rho_mid, int skip_rows,
                         double* px, double* py, int max_points);
/* algebraic least-squares circle through n >= 3 points: out = (xc, yc, R) */
int orc_circle_fit(const double* px, const double* py, int n, double out[3]);
int orc_contact_angle(const double* rho, int nx, int ny, double rho_l, double rho_g,
                      int skip_rows, orc_contact* out);
/* labels [ny][nx]: the component label, -1 outside the phase; comps sorted by
 * label (at most max_comps written); *n_comps = number of components */
int orc_components(const double* rho, int nx, int ny, int periodic_x, int periodic_y,
                   double threshold, int below, int* labels, orc_component* comps,
                   int max_comps, int* n_comps);

/* three-dimensional form (lbm_oracle3d.c): D3Q19 MRT flow lattice, D3Q7
 * temperature lattice with the same weighted streaming.  x and y periodic;
 * z periodic or walls at both ends.  Arrays are [nz][ny][nx] (x fastest),
 * populations [q][nz][ny][nx]; gravity acts along -z. -------------------- */
typedef struct {
    int flow_z;          /* ORC_PERIODIC or ORC_WALL (bottom and top) */
    int therm[2];        /* bottom, top: ORC_T_* (periodic iff flow_z is) */
    double T_edge[2];    /* bottom, top wall temperatures */
    double theta_deg;    /* contact angle of both walls */
} orc_bc3;
typedef struct orc3_sim orc3_sim;
void orc3_velocities(int cx[19], int cy[19], int cz[19], double w[19]);
void orc3_matrices(double M[361], double Minv[361], double Mh[49], double Mhinv[49]);
void orc3_feq(double rho, double ux, double uy, double uz, double f[19]);
void orc3_force_term(double ux, double uy, double uz, double Fx, double Fy, double Fz,
                     double out[19]);
orc3_sim* orc3_create(int nx, int ny, int nz, const orc_params* p, const orc_bc3* bc, int* err);
void orc3_destroy(orc3_sim* s);
int orc3_init(orc3_sim* s, const double* rho, const double* ux, const double* uy,
              const double* uz, const double* T);
int orc3_step(orc3_sim* s, int n);
int orc3_fields(orc3_sim* s, double* rho, double* ux, double* uy, double* uz, double* T);
int orc3_get_populations(const orc3_sim* s, double* f, double* g, double* P);
int orc3_set_populations(orc3_sim* s, const double* f, const double* g, const double* P,
                         long step, double rho_ave_prev);
long orc3_step_count(const orc3_sim* s);
/* as orc_diagnostics; liquid_area is the liquid volume and the diameters are
 * those of the equivalent sphere (hemisphere when sessile) */
int orc3_diagnostics(orc3_sim* s, double rho_l, double rho_g, int sessile, orc_diag* d);

#ifdef __cplusplus
}
#endif
#endif
