// Internal definitions shared by the CUDA translation units of the library:
// device-resident descriptors, the per-launch physics constants and the
// closed-form pieces of the coupled step (Peng-Robinson EOS of Section 2,
// Eq. 10; the pseudopotential psi; (dp/dT)_rho used by Q of Eq. 20).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// flow / thermal boundary kinds (same values as the public header)
enum { PERIODIC = 0, WALL = 1, OPEN = 2 };
enum { T_PERIODIC = 0, T_DIRICHLET = 1, T_ADIABATIC = 2 };
enum { EW = 0, EE = 1, ES = 2, EN = 3 };

// sticky device error bits (ERR_TIMEOUT: a bounded wait for a staged row ran out)
enum { ERR_PSI = 1, ERR_NONFINITE = 2, ERR_TIMEOUT = 4 };

// Device-resident control block of one domain: the device-side step counter
// read by every launch, the three-slot ring of per-step density sums used by
// the buoyancy force (step n accumulates sum rho(n) into slot n % 3 and reads
// slot (n - 1) % 3), and the sticky error word.  The CTAs of a launch add
// their block sums as fixed-point integers (massq, see massq_scale), so the
// total does not depend on the order in which the CTAs finish; the launch's
// last CTA converts the finished slot to mass[] for the next step to read.
struct Ctl {
    long long step;
    double mass[3];
    long long massq[3];
    // the step count at which the domain stops (> 0), or 0 for none: a
    // launch skips the units of a domain that has reached it, so its state,
    // step counter and density ring stay as they are
    long long target;
    int err;
    int pad;
};

__device__ __forceinline__ bool ctl_stopped(const Ctl* c) {
    const long long tg = __ldcg(&c->target);
    return tg > 0 && __ldcg(&c->step) >= tg;
}

// fixed-point scale of Ctl::massq for a domain of N = 1 / inv_n nodes:
// 2^(58 - e) with N < 2^e.  Densities stay below 16 (the EOS ends at 1/b =
// 10.5), so a domain total stays below 2^62 and no sum overflows, while a
// block sum keeps at least 30 fraction bits (N < 2^28) and small domains keep
// the full double precision of their block sums
__host__ __device__ __forceinline__ double massq_scale(double inv_n) {
    int e = 0;
    frexp(1.0 / inv_n, &e);
    return ldexp(1.0, 58 - e);
}
__device__ __forceinline__ void massq_add(long long* slot, double block_sum, double scale) {
    atomicAdd(reinterpret_cast<unsigned long long*>(slot),
              (unsigned long long)__double2ll_rn(block_sum * scale));
}
__host__ __device__ __forceinline__ double massq_value(long long q, double scale) {
    return (double)q / scale;
}

// One domain as seen by the kernels.  Populations are stored as deviations
// f_i - w_i rho_ref and g_i - w^_i T_ref, SoA planes [q][ny][pitch].
struct Inst {
    void* f[2];
    void* g[2];
    void* P[2];
    Ctl* ctl;
    int nx, ny, pitch;
    int flow[4], therm[4];
    int heater_x0, heater_x1;
    double T_edge[4], T_heater, cot_theta;
    double rho_ref, T_ref, inv_n;
    // rows [own_y0, own_y1) enter the density sum behind rho_ave; inv_n is
    // 1 / (nodes the mean is taken over).  The whole domain unless it is one
    // slab of a larger domain (lbm_set_partition).
    int own_y0, own_y1;
};

// A work unit of the fused step: output columns [x0, x1), rows [y0, y1) of
// domain `inst`.
struct Unit {
    int inst, x0, x1, y0, y1;
};

// Physical constants shared by every domain of a launch, already combined
// into the factors the kernels use.
template <class R>
struct Phys {
    // EOS: p = rho Rg T/(1 - b rho) - a h^2 rho^2/(1 + 2 b rho - b^2 rho^2),
    // h = 1 + kpr (1 - sqrt(T/Tc))
    R a, b, Rg, kpr, inv_Tc, akTc;   // akTc = a kpr / Tc
    R two_over_G, negG;
    // D2Q9 MRT rates and Li forcing
    R s_e, s_eps, s_q, s_p;
    R hs_e, hs_eps, hs_q, hs_p;      // 1 - s/2
    R sig_e, sig_eps;                // sigma / (1/s - 1/2)
    // D2Q5
    R cv, inv_cv, w_dot, w5_0, w5_1, vs1_cs2h, vs3, vs4;   // vs1_cs2h = vs1 / cs2h
    R one_m_vs1, one_m_vs4;
    R gravity;
    int frozen_flow, frozen_thermal;
};

struct PhysD {
    double a, b, Rg, omega, G, sigma;
    double s_e, s_eps, s_q, s_p;
    double cv, w_dot, vs1, vs3, vs4;
    double gravity;
    int frozen_flow, frozen_thermal;
};

template <class R>
inline Phys<R> make_phys(const PhysD& d) {
    Phys<R> p;
    double kpr = 0.37464 + 1.54226 * d.omega - 0.26992 * d.omega * d.omega;
    double Tc = 0.0778 * d.a / (0.45724 * d.b * d.Rg);
    p.a = (R)d.a;
    p.b = (R)d.b;
    p.Rg = (R)d.Rg;
    p.kpr = (R)kpr;
    p.inv_Tc = (R)(1.0 / Tc);
    p.akTc = (R)(d.a * kpr / Tc);
    p.two_over_G = (R)(2.0 / d.G);
    p.negG = (R)(-d.G);
    p.s_e = (R)d.s_e;
    p.s_eps = (R)d.s_eps;
    p.s_q = (R)d.s_q;
    p.s_p = (R)d.s_p;
    p.hs_e = (R)(1.0 - 0.5 * d.s_e);
    p.hs_eps = (R)(1.0 - 0.5 * d.s_eps);
    p.hs_q = (R)(1.0 - 0.5 * d.s_q);
    p.hs_p = (R)(1.0 - 0.5 * d.s_p);
    p.sig_e = (R)(d.sigma / (1.0 / d.s_e - 0.5));
    p.sig_eps = (R)(d.sigma / (1.0 / d.s_eps - 0.5));
    p.cv = (R)d.cv;
    p.inv_cv = (R)(1.0 / d.cv);
    p.w_dot = (R)d.w_dot;
    p.w5_0 = (R)(1.0 - d.w_dot);
    p.w5_1 = (R)(0.25 * d.w_dot);
    p.vs1_cs2h = (R)(d.vs1 / (0.5 * d.w_dot));
    p.vs3 = (R)d.vs3;
    p.vs4 = (R)d.vs4;
    p.one_m_vs1 = (R)(1.0 - d.vs1);
    p.one_m_vs4 = (R)(1.0 - d.vs4);
    p.gravity = (R)d.gravity;
    p.frozen_flow = d.frozen_flow;
    p.frozen_thermal = d.frozen_thermal;
    return p;
}

// ---- storage conversions ------------------------------------------------
__device__ __forceinline__ float ld_st(const float* p) { return __ldg(p); }
__device__ __forceinline__ double ld_st(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ld_st(const __half* p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ void st_st(float* p, float v) { *p = v; }
__device__ __forceinline__ void st_st(double* p, double v) { *p = v; }
__device__ __forceinline__ void st_st(__half* p, float v) { *p = __float2half_rn(v); }
// a staged (shared-memory) storage value as arithmetic type
__device__ __forceinline__ float st_val(float v) { return v; }
__device__ __forceinline__ float st_val(__half v) { return __half2float(v); }

// ---- arithmetic helpers (precision-generic) -------------------------------
// FP64 keeps IEEE division and square root (parity with the FP64 oracle to
// ~1e-13); FP32 uses the hardware approximations (rcp.approx / sqrt.approx,
// relative error ~2^-23), well inside the FP32 tolerance.
__device__ __forceinline__ float rsq(float x) { return sqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return sqrt(x); }
__device__ __forceinline__ float rabs(float x) { return fabsf(x); }
__device__ __forceinline__ double rabs(double x) { return fabs(x); }
__device__ __forceinline__ float f_rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// FP64 reciprocal by the Newton-Raphson iteration for 1/x,
// r <- r + r (1 - x r), which squares the relative error at each step: from
// the hardware approximation rcp.approx.ftz.f64 two steps reach the FP64
// rounding level (within about one ulp of 1/x, not always the correctly
// rounded value).  The FP64 step divides six times per node and is bound by
// the GB300's FP64 pipe.  Operands are O(1) here (rho, 1 - b rho, rho c_v,
// sqrt(T/Tc)); a zero, infinite or NaN operand gives a non-finite result,
// which the step reports.
__device__ __forceinline__ double f_rcp(double x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}
__device__ __forceinline__ float f_sqrt(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double f_sqrt(double x) { return sqrt(x); }

// Two-lane arithmetic.  In float it maps to Blackwell's paired FP32
// instructions (one FADD2 / FMUL2 / FFMA2 does the work of two), each lane
// rounded as the scalar operation; in double it is componentwise.  Subtraction
// is a fused multiply-add with -1, which is exact in the product.
__device__ __forceinline__ float2 pr(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 pr(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double2 padd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ double2 pmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 pfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ double2 psub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// Peng-Robinson pressure (Eq. 10) and psi^2 = 2 (p_EOS - rho/3) / G.
template <class R>
__device__ __forceinline__ R eos_p(const Phys<R>& P, R rho, R T) {
    R st = rsq(T * P.inv_Tc);
    R h = R(1) + P.kpr * (R(1) - st);
    R br = P.b * rho;
    return rho * P.Rg * T / (R(1) - br) - P.a * h * h * rho * rho / (R(1) + R(2) * br - br * br);
}

// (dp_EOS/dT)_rho = rho Rg/(1 - b rho) + a k h rho^2 / (sqrt(T/Tc) Tc (1 + 2 b rho - b^2 rho^2))
template <class R>
__device__ __forceinline__ R eos_dpdT(const Phys<R>& P, R rho, R T) {
    R st = rsq(T * P.inv_Tc);
    R h = R(1) + P.kpr * (R(1) - st);
    R br = P.b * rho;
    return rho * P.Rg / (R(1) - br) + P.akTc * h * rho * rho / (st * (R(1) + R(2) * br - br * br));
}

template <class R>
__device__ __forceinline__ R psi2_of(const Phys<R>& P, R rho, R T) {
    return P.two_over_G * (eos_p(P, rho, T) - rho * R(1.0 / 3.0));
}

// psi^2 and T (dp/dT)_rho of one node from shared sub-expressions:
// st = sqrt(T/Tc), h = 1 + k (1 - st), ib = 1/(1 - b rho),
// r2id = rho^2 / (1 + 2 b rho - b^2 rho^2)
template <class R>
__device__ __forceinline__ void eos_node(const Phys<R>& P, R rho, R T, R* psi2, R* TdpdT) {
    const R st = f_sqrt(T * P.inv_Tc);
    const R h = R(1) + P.kpr * (R(1) - st);
    const R br = P.b * rho;
    const R ib = f_rcp(R(1) - br);
    const R r2id = rho * rho * f_rcp(R(1) + br * (R(2) - br));
    const R rRib = rho * P.Rg * ib;
    const R p = rRib * T - P.a * h * h * r2id;
    *psi2 = P.two_over_G * (p - rho * R(1.0 / 3.0));
    *TdpdT = T * (rRib + P.akTc * h * r2id * f_rcp(st));
}

__device__ __forceinline__ int wrapi(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

// wall / Dirichlet temperature along an edge, with the heater segment
__device__ __forceinline__ double wall_T(const Inst& I, int edge, int gx) {
    if (edge == ES && gx >= I.heater_x0 && gx < I.heater_x1) return I.T_heater;
    return I.T_edge[edge];
}

// Per-instance storage types by precision code
template <int PREC> struct Types;
template <> struct Types<0> { typedef double R; typedef double TF; typedef double TG; };
template <> struct Types<1> { typedef float R; typedef float TF; typedef float TG; };
template <> struct Types<2> { typedef float R; typedef float TF; typedef __half TG; };

inline size_t elem_f(int prec) { return prec == 0 ? 8 : 4; }
inline size_t elem_g(int prec) { return prec == 0 ? 8 : (prec == 1 ? 4 : 2); }
inline size_t elem_P(int prec) { return prec == 0 ? 8 : 4; }

// ---- launchers implemented in the .cu files ------------------------------
struct StepLaunch {
    Inst* insts;
    const Unit* units;
    int n_units;
    int n_inst;
    unsigned* sched;   // [0] next unit, [1] finished CTAs
    int grid;
    int walls;         // some domain has a wall: the launch carries the wall rings
    int staged;        // FP32 / FP16-g: rows arrive by bulk copies (stage_eligible)
    int wait_probe;    // test hook: staged CTAs also wait on an mbarrier nothing arms
    int targets;       // some domain has a target step (lbm_set_target)
    PhysD phys;
};

// The bulk-copy staged form (FP32 f and P; g in FP32 or FP16) needs every
// copied row piece to start on a 16-byte boundary: always true for open x
// edges (the copy of the last strip is rounded up into the row's pitch
// padding), and for periodic x when the wrapped pieces start on 16-byte
// column boundaries (nx a multiple of 4 for FP32 g, of 8 for FP16 g) and the
// window wraps at most a few times (nx >= 32).
inline bool stage_eligible(const Inst& I, int prec) {
    if (prec != 1 && prec != 2) return false;
    if (I.flow[EW] != PERIODIC) return true;
    return I.nx % (prec == 2 ? 8 : 4) == 0 && I.nx >= 32;
}

int step_launch(int prec, int threads, const StepLaunch& L, cudaStream_t st);
int step_occupancy(int prec, int threads, int walls, int staged, int* ctas_per_sm,
                   size_t* smem_bytes);

int init_launch(int prec, const Inst* I_dev, const Inst& I, const double* rho, const double* ux,
                const double* uy, const double* T, double w_dot, cudaStream_t st);
// rho, u (half-force velocity), T of the current state; psi is scratch of n doubles
int fields_launch(int prec, const Inst* I_dev, const Inst& I, const PhysD& phys, double* rho,
                  double* ux, double* uy, double* T, double* psi, cudaStream_t st);
int pop_get_launch(int prec, const Inst& I, int parity, double w_dot, double* f, double* g,
                   double* P, cudaStream_t st);
int pop_set_launch(int prec, const Inst& I, int parity, double w_dot, const double* f,
                   const double* g, const double* P, cudaStream_t st);
// reduction of device fields into 8 doubles + a nonfinite count; `scratch`
// holds diag_scratch_bytes(n) bytes
size_t diag_scratch_bytes(long long n);
int diag_launch(const double* rho, const double* ux, const double* uy, const double* T,
                long long n, double cv, double rho_l, double rho_g, double* out9,
                void* scratch, cudaStream_t st);
// out2 = (sum a, sum b) over n device doubles, fixed summation order; the
// same scratch as diag_launch
int sum2_launch(const double* a, const double* b, long long n, double* out2, void* scratch,
                cudaStream_t st);

// interface analyses (lbm_analysis.cu)
// contact-angle sums: out12[0..8] = n, sum u, sum v, sum uu, sum vv, sum uv,
// sum u z, sum v z, sum z about the mean point, out12[9..11] = n, sum x, sum y
size_t iface_scratch_bytes();
int iface_launch(const double* rho, int nx, int ny, double rho_mid, int skip, double* out12,
                 void* scratch, cudaStream_t st);
// one region of the phase: label = smallest node index, flags bit 0..3 = the
// region touches the W, E, S, N edge
struct RegionOut {
    long long label, area, sum_y;
    int y_min, y_max, flags, pad;
};
size_t regions_scratch_bytes(long long n);
// labels the phase; *parent_out -> n ints (root label or -1), *roots_out ->
// the first max_roots roots in no order, *count_out -> [roots found, error]
int regions_launch(const double* rho, int nx, int ny, int perx, int pery, double thr, int below,
                   void* scratch, int max_roots, int** parent_out, int** roots_out,
                   int** count_out, cudaStream_t st);
int regions_gather_launch(void* scratch, long long n, int m, RegionOut* out, cudaStream_t st);

}  // namespace lbm
