// Three-dimensional form of the coupled step: D3Q19 MRT pseudopotential flow
// lattice (d'Humieres moment basis, Li forcing with the sigma term on the
// energy moment) + D3Q7 temperature lattice with the rho c_v-weighted
// streaming of Eq. 39, x and y periodic, z periodic or walls.
//
// Two forms of the step give the same result.  k3_fused (below; the default
// in FP32) does the whole step in one kernel over z-marching tiles.  The other
// form (the default in FP64) is three kernels over the nodes plus a
// one-thread counter update, because every stage needs neighbours of the
// previous one:
//   k3_force    psi of the 18 neighbours (ghost layer at walls) -> F_m, F,
//               u = (j + F/2)/rho, |F_m|^2/psi^2                (Eqs. 9, 11)
//   k3_collide  div u (neighbour u), grad T (local moments), Q, P^n, S;
//               D3Q19 and D3Q7 collisions; f* pushed to its destination
//               (bounce-back at walls); g*_i blended into the destination's
//               g(t+1) = g + (g* - g)/(rho c_v) (anti-bounce-back at walls),
//               P^n stored                          (Eqs. 5, 20, 24, 39)
//   k3_macro    rho, j, T, psi, T dp/dT, 1/(rho c_v) of the new state from
//               f(t+1), g(t+1), and the density sum for buoyancy
// Per node and step (FP32) this moves about 1.9 times the 216 B of one read
// and one write of the state: f is read again after the push to build the
// next state's fields, and u, F and the per-node fields pass through memory.
//
// Reciprocals use f_rcp as in two dimensions (the hardware approximation in
// FP32; Newton-Raphson from it, within about one ulp, in FP64).
// Populations are stored as deviations f_i - w_i rho_ref and g_i - w^_i T_ref.
// Planes are [q][nz][ny][pitch], 64-bit offsets.
#include <math.h>
#include <string.h>

#include <new>
#include <string>
#include <type_traits>
#include <utility>

#include "lbm.h"
#include "lbm3d.h"
#include "lbm_internal.cuh"

namespace lbm {
namespace {

// ---- D3Q19 / D3Q7 tables as constexpr functions (folded after unrolling) --
__host__ __device__ constexpr int qx(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
           : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int qy(int i) {
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
           : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int qz(int i) {
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
           : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
__host__ __device__ constexpr int qopp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr int qc2(int i) { return qx(i) * qx(i) + qy(i) * qy(i) + qz(i) * qz(i); }
__host__ __device__ constexpr double qw(int i) {
    return qc2(i) == 0 ? 1.0 / 3.0 : (qc2(i) == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
}
// moment k of direction i (d'Humieres et al. 2002 basis), integer valued
__host__ __device__ constexpr int mrow(int k, int i) {
    return k == 0 ? 1
         : k == 1 ? 19 * qc2(i) - 30
         : k == 2 ? (21 * qc2(i) * qc2(i) - 53 * qc2(i) + 24) / 2
         : k == 3 ? qx(i)
         : k == 4 ? (5 * qc2(i) - 9) * qx(i)
         : k == 5 ? qy(i)
         : k == 6 ? (5 * qc2(i) - 9) * qy(i)
         : k == 7 ? qz(i)
         : k == 8 ? (5 * qc2(i) - 9) * qz(i)
         : k == 9 ? 3 * qx(i) * qx(i) - qc2(i)
         : k == 10 ? (3 * qc2(i) - 5) * (3 * qx(i) * qx(i) - qc2(i))
         : k == 11 ? qy(i) * qy(i) - qz(i) * qz(i)
         : k == 12 ? (3 * qc2(i) - 5) * (qy(i) * qy(i) - qz(i) * qz(i))
         : k == 13 ? qx(i) * qy(i)
         : k == 14 ? qy(i) * qz(i)
         : k == 15 ? qx(i) * qz(i)
         : k == 16 ? (qy(i) * qy(i) - qz(i) * qz(i)) * qx(i)
         : k == 17 ? (qz(i) * qz(i) - qx(i) * qx(i)) * qy(i)
                   : (qx(i) * qx(i) - qy(i) * qy(i)) * qz(i);
}
// squared norm of row k (the basis is orthogonal: M^-1 = M^T diag(1/norm))
__host__ __device__ constexpr int mnorm(int k) {
    int s = 0;
    for (int i = 0; i < 19; ++i) s += mrow(k, i) * mrow(k, i);
    return s;
}
// Parity of a moment row under c -> -c: the even rows take the same entry
// for a direction and its opposite, the odd rows opposite entries (and none
// for the rest direction).  Pairs are p = 1..9: directions 2p - 1 and 2p.
__host__ __device__ constexpr bool row_even(int k) {
    for (int p = 1; p <= 9; ++p)
        if (mrow(k, 2 * p - 1) != mrow(k, 2 * p)) return false;
    return true;
}
__host__ __device__ constexpr bool row_odd(int k) {
    if (mrow(k, 0) != 0) return false;
    for (int p = 1; p <= 9; ++p)
        if (mrow(k, 2 * p - 1) != -mrow(k, 2 * p)) return false;
    return true;
}
constexpr bool rows_split() {
    for (int k = 0; k < 19; ++k)
        if (row_even(k) == row_odd(k)) return false;
    for (int p = 1; p <= 9; ++p)
        if (qopp(2 * p - 1) != 2 * p) return false;
    return true;
}
static_assert(rows_split(), "every moment row is even or odd under c -> -c");

// f(integral_constant<int, 0>) ... f(integral_constant<int, N - 1>): the
// index is a constant in every call, whatever the unroller decides
template <class F, int... I>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// m = M f from the pair sums S_p = f_{2p-1} + f_{2p} (even rows) and
// differences D_p = f_{2p-1} - f_{2p} (odd rows): about half the operations
// of the plain product
template <class R>
__device__ __forceinline__ void moments19(const R (&f)[19], R (&m)[19]) {
    R S[10], Dp[10];
    static_for<9>([&](auto pc) {
        constexpr int p = decltype(pc)::value + 1;
        S[p] = f[2 * p - 1] + f[2 * p];
        Dp[p] = f[2 * p - 1] - f[2 * p];
    });
    static_for<19>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        R s = 0;
        if constexpr (mrow(k, 0) != 0) s = R(mrow(k, 0)) * f[0];
        static_for<9>([&](auto pc) {
            constexpr int p = decltype(pc)::value + 1;
            constexpr int c = mrow(k, 2 * p - 1);
            if constexpr (c != 0) s += R(c) * (row_odd(k) ? Dp[p] : S[p]);
        });
        m[k] = s;
    });
}

// f += M^T dm: for each pair the even rows give one term E_p for both
// directions, the odd rows a term O_p of opposite signs
template <class R>
__device__ __forceinline__ void add_inverse19(const R (&dm)[19], R (&f)[19]) {
    R E0 = 0;
    static_for<19>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        if constexpr (mrow(k, 0) != 0) E0 += R(mrow(k, 0)) * dm[k];
    });
    f[0] += E0;
    static_for<9>([&](auto pc) {
        constexpr int p = decltype(pc)::value + 1;
        R E = 0, O = 0;
        static_for<19>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            constexpr int c = mrow(k, 2 * p - 1);
            if constexpr (c != 0) {
                if constexpr (row_odd(k)) O += R(c) * dm[k];
                else E += R(c) * dm[k];
            }
        });
        f[2 * p - 1] += E + O;
        f[2 * p] += E - O;
    });
}

// D3Q7: rest, +-x, +-y, +-z
__host__ __device__ constexpr int hx(int i) { return i == 1 ? 1 : (i == 2 ? -1 : 0); }
__host__ __device__ constexpr int hy(int i) { return i == 3 ? 1 : (i == 4 ? -1 : 0); }
__host__ __device__ constexpr int hz(int i) { return i == 5 ? 1 : (i == 6 ? -1 : 0); }

enum { A_RHO = 0, A_T, A_PSI, A_TDPDT, A_JX, A_JY, A_JZ, A_IC, A_N };   // aux: 1/(rho c_v) last
enum { B_UX = 0, B_UY, B_UZ, B_FX, B_FY, B_FZ, B_FM2, B_N };            // aux2 planes

struct Dom3 {
    void* f[2];
    void* g[2];
    void* P[2];
    void* aux;
    void* aux2;
    void* ghost;      // wall ghost-layer psi [2][ny][pitch] (fused step)
    Ctl* ctl;
    int nx, ny, nz, pitch;
    size_t plane;
    int walls, therm[2];
    double T_edge[2], cot, rho_ref, T_ref, inv_n;
};

template <class R>
struct Lat3 {
    R s_e, s_eps, s_q, s_p;
    R sig_e3;            // (19/2) sigma / (1/s_e - 1/2), the sigma term of e
    R vs0, vs1, vs3, vs4, w7_0, w7_1, cs2h, cv, gravity;
    int frozen_flow, frozen_thermal;
};

template <class R>
Lat3<R> make_lat3(const lbm_params& p) {
    Lat3<R> L;
    L.s_e = (R)p.s_e;
    L.s_eps = (R)p.s_eps;
    L.s_q = (R)p.s_q;
    L.s_p = (R)(1.0 / (3.0 * p.nu + 0.5));
    L.sig_e3 = (R)(9.5 * p.sigma / (1.0 / p.s_e - 0.5));
    const double cs2h = p.w_dot / 3.0;
    L.cs2h = (R)cs2h;
    L.vs0 = (R)p.vs0;
    L.vs1 = (R)(1.0 / (p.lambda / cs2h + 0.5));
    L.vs3 = (R)p.vs3;
    L.vs4 = (R)p.vs4;
    L.w7_0 = (R)(1.0 - p.w_dot);
    L.w7_1 = (R)(p.w_dot / 6.0);
    L.cv = (R)p.cv;
    L.gravity = (R)p.gravity;
    L.frozen_flow = p.frozen_flow;
    L.frozen_thermal = p.frozen_thermal;
    return L;
}

// the EOS / interaction constants shared with the two-dimensional kernels
PhysD phys_of(const lbm_params& p) {
    PhysD d;
    memset(&d, 0, sizeof(d));
    d.a = p.a;
    d.b = p.b;
    d.Rg = p.R;
    d.omega = p.omega;
    d.G = p.G;
    d.sigma = p.sigma;
    d.s_e = p.s_e;
    d.s_eps = p.s_eps;
    d.s_q = p.s_q;
    d.s_p = 1.0 / (3.0 * p.nu + 0.5);
    d.cv = p.cv;
    d.w_dot = p.w_dot;
    d.vs1 = 1.0 / (p.lambda / (p.w_dot / 3.0) + 0.5);
    d.vs3 = p.vs3;
    d.vs4 = p.vs4;
    d.gravity = p.gravity;
    d.frozen_flow = p.frozen_flow;
    d.frozen_thermal = p.frozen_thermal;
    return d;
}

__device__ __forceinline__ int wrapn(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }
// any distance from the domain (tiles wider than a small domain wrap several times)
__device__ __forceinline__ int wrapm(int i, int n) { const int r = i % n; return r < 0 ? r + n : r; }

template <class R>
__device__ __forceinline__ size_t nid(const Dom3& D, int x, int y, int z) {
    return ((size_t)z * D.ny + y) * D.pitch + x;
}

// Element offsets from a node to its six axis neighbours, wrapped across the
// periodic seams; a lattice direction's offset is the sum of its components'.
// zlo / zhi: the node is next to the bottom / top wall.
struct Nbr {
    long long xp, xm, yp, ym, zp, zm;
    bool zlo, zhi;
};

__device__ __forceinline__ Nbr nbr_offsets(const Dom3& D, int x, int y, int z) {
    Nbr d;
    const long long P = D.pitch, S = (long long)D.ny * D.pitch;
    d.xp = x == D.nx - 1 ? -(long long)(D.nx - 1) : 1;
    d.xm = x == 0 ? (long long)(D.nx - 1) : -1;
    d.yp = y == D.ny - 1 ? -(long long)(D.ny - 1) * P : P;
    d.ym = y == 0 ? (long long)(D.ny - 1) * P : -P;
    d.zp = z == D.nz - 1 ? -(long long)(D.nz - 1) * S : S;
    d.zm = z == 0 ? (long long)(D.nz - 1) * S : -S;
    d.zlo = D.walls && z == 0;
    d.zhi = D.walls && z == D.nz - 1;
    return d;
}

// offset of the node at c = (cx, cy, cz) away (each component -1, 0 or 1)
__device__ __forceinline__ long long nbr_off(const Nbr& d, int cx, int cy, int cz) {
    long long o = 0;
    if (cx > 0) o += d.xp;
    if (cx < 0) o += d.xm;
    if (cy > 0) o += d.yp;
    if (cy < 0) o += d.ym;
    if (cz > 0) o += d.zp;
    if (cz < 0) o += d.zm;
    return o;
}

// the node c away lies beyond a wall
__device__ __forceinline__ bool nbr_solid(const Nbr& d, int cz) {
    return (cz < 0 && d.zlo) || (cz > 0 && d.zhi);
}

// ---------------------------------------------------------------------------
// psi of a node at most one layer beyond the domain: z wraps or, at walls,
// comes from the ghost layer built from rho / T of layers 1 and 2
template <class R>
__device__ R psi_nb(const Dom3& D, const Phys<R>& P, int x, int y, int z, int* err) {
    const R* A = (const R*)D.aux;
    x = wrapn(x, D.nx);
    y = wrapn(y, D.ny);
    if (z >= 0 && z < D.nz) return A[A_PSI * D.plane + nid<R>(D, x, y, z)];
    if (!D.walls) return A[A_PSI * D.plane + nid<R>(D, x, y, wrapn(z, D.nz))];
    const int e = z < 0 ? 0 : 1;
    const int z1 = e == 0 ? 0 : D.nz - 1, z2 = e == 0 ? 1 : D.nz - 2;
    const R* rho = A + A_RHO * D.plane;
    const R dx = rho[nid<R>(D, wrapn(x + 1, D.nx), y, z1)] - rho[nid<R>(D, wrapn(x - 1, D.nx), y, z1)];
    const R dy = rho[nid<R>(D, x, wrapn(y + 1, D.ny), z1)] - rho[nid<R>(D, x, wrapn(y - 1, D.ny), z1)];
    const R rg = rho[nid<R>(D, x, y, z2)] + (R)D.cot * rsq(dx * dx + dy * dy);
    const R tg = A[A_T * D.plane + nid<R>(D, x, y, z1)];   // the fluid node's temperature
    const R q2 = psi2_of(P, rg, tg);
    if (!(q2 >= R(0))) *err |= (q2 != q2) ? ERR_NONFINITE : ERR_PSI;
    return f_sqrt(q2);
}

// F_m from the psi of the 18 neighbours and F = F_m + F_b at node n
// (Eqs. 9, 11); |F_m|^2 / psi^2 for the sigma term
template <class R>
__device__ __forceinline__ void force_at(const Dom3& D, const Phys<R>& P, const Lat3<R>& L,
                                         int x, int y, int z, size_t n, const Nbr& nb,
                                         long long step, int* err, R* F, R* Fm2) {
    const R* A = (const R*)D.aux;
    const R* psi_p = A + A_PSI * D.plane;
    R sx = 0, sy = 0, sz = 0;
#pragma unroll 19
    for (int i = 1; i < 19; ++i) {
        const R wv = qc2(i) == 1 ? R(1.0 / 6.0) : R(1.0 / 12.0);
        // beyond a wall the neighbour is the ghost layer (Section 3.3)
        const R pn = nbr_solid(nb, qz(i))
                         ? psi_nb<R>(D, P, x + qx(i), y + qy(i), z + qz(i), err)
                         : psi_p[(size_t)((long long)n + nbr_off(nb, qx(i), qy(i), qz(i)))];
        if (qx(i)) sx += wv * pn * R(qx(i));
        if (qy(i)) sy += wv * pn * R(qy(i));
        if (qz(i)) sz += wv * pn * R(qz(i));
    }
    const R psi = psi_p[n];
    const R rho = A[A_RHO * D.plane + n];
    const R rho_ave = L.gravity != R(0) ? (R)(__ldcg(&D.ctl->mass[(step + 2) % 3]) * D.inv_n) : R(0);
    F[0] = P.negG * psi * sx;
    F[1] = P.negG * psi * sy;
    F[2] = P.negG * psi * sz - L.gravity * (rho - rho_ave);
    *Fm2 = P.negG * P.negG * (sx * sx + sy * sy + sz * sz);
}

template <class R>
__global__ void __launch_bounds__(128) k3_force(Dom3 D, Phys<R> P, Lat3<R> L) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= D.nx || y >= D.ny) return;
    const R* A = (const R*)D.aux;
    R* B = (R*)D.aux2;
    const size_t n = nid<R>(D, x, y, z);
    const Nbr nb = nbr_offsets(D, x, y, z);
    int err = 0;
    R F[3], Fm2;
    force_at<R>(D, P, L, x, y, z, n, nb, __ldcg(&D.ctl->step), &err, F, &Fm2);
    R ux = 0, uy = 0, uz = 0;
    if (!L.frozen_flow) {
        const R ir = f_rcp(A[A_RHO * D.plane + n]);
        ux = (A[A_JX * D.plane + n] + R(0.5) * F[0]) * ir;
        uy = (A[A_JY * D.plane + n] + R(0.5) * F[1]) * ir;
        uz = (A[A_JZ * D.plane + n] + R(0.5) * F[2]) * ir;
    }
    B[B_UX * D.plane + n] = ux;
    B[B_UY * D.plane + n] = uy;
    B[B_UZ * D.plane + n] = uz;
    B[B_FX * D.plane + n] = F[0];
    B[B_FY * D.plane + n] = F[1];
    B[B_FZ * D.plane + n] = F[2];
    B[B_FM2 * D.plane + n] = Fm2;
    if (err) atomicOr(&D.ctl->err, err);
}

// ---------------------------------------------------------------------------
template <class R>
__global__ void __launch_bounds__(128) k3_collide(Dom3 D, Phys<R> P, Lat3<R> L) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= D.nx || y >= D.ny) return;
    const long long step = __ldcg(&D.ctl->step);
    const int par = (int)(step & 1);
    const R* fc = (const R*)D.f[par];
    R* fn = (R*)D.f[par ^ 1];
    const R* gc = (const R*)D.g[par];
    const R* Pc = (const R*)D.P[par];
    R* Pn_out = (R*)D.P[par ^ 1];
    R* gn = (R*)D.g[par ^ 1];
    const R* A = (const R*)D.aux;
    const R* B = (const R*)D.aux2;
    const size_t n = nid<R>(D, x, y, z);
    const R rho = A[A_RHO * D.plane + n];
    const R TdpdT = A[A_TDPDT * D.plane + n];
    const R ux = B[B_UX * D.plane + n], uy = B[B_UY * D.plane + n], uz = B[B_UZ * D.plane + n];
    R g[7];
#pragma unroll 19
    for (int i = 0; i < 7; ++i) g[i] = gc[i * D.plane + n];

    const R Fx = B[B_FX * D.plane + n], Fy = B[B_FY * D.plane + n], Fz = B[B_FZ * D.plane + n];
    const R Fm2 = B[B_FM2 * D.plane + n];
    const Nbr nb = nbr_offsets(D, x, y, z);
    // div u: (1/c_s^2) sum_i w_i c_i . u(x + c_i); walls carry u = 0
    R divu = 0;
#pragma unroll 19
    for (int i = 1; i < 19; ++i) {
        if (nbr_solid(nb, qz(i))) continue;
        const size_t m = (size_t)((long long)n + nbr_off(nb, qx(i), qy(i), qz(i)));
        R cu = 0;
        if (qx(i)) cu += R(qx(i)) * B[B_UX * D.plane + m];
        if (qy(i)) cu += R(qy(i)) * B[B_UY * D.plane + m];
        if (qz(i)) cu += R(qz(i)) * B[B_UZ * D.plane + m];
        divu += R(3.0 * qw(i)) * cu;
    }
    // grad T from the local first moments: c^_s^2 d_a T = -vs1 m^_a
    const R m1 = g[1] - g[2], m2 = g[3] - g[4], m3 = g[5] - g[6];
    const R k = -L.vs1 / L.cs2h;
    const R dTx = k * m1, dTy = k * m2, dTz = k * m3;
    const R C = rho * L.cv;
    const R Q = -(C * (ux * dTx + uy * dTy + uz * dTz) + TdpdT * divu);
    const R Pn = Q * f_rcp(C);
    const R Qs = step == 0 ? Q : Q + R(0.5) * (Q - C * Pc[n]);

    // ---- D3Q19 MRT collision in moment space
    R f[19];
#pragma unroll 19
    for (int i = 0; i < 19; ++i) f[i] = fc[i * D.plane + n];
    if (L.frozen_flow) {
#pragma unroll 19
        for (int i = 0; i < 19; ++i) fn[i * D.plane + n] = f[i];
    } else {
        R m[19];
        moments19(f, m);
        // deviation storage: m(abs) = m(dev) + rho_ref M w, M w = (1, -11, 3, 0 ...)
        const R rr = (R)D.rho_ref;
        m[0] += rr;
        m[1] += R(-11) * rr;
        m[2] += R(3) * rr;
        const R uu = ux * ux + uy * uy + uz * uz;
        const R uF = ux * Fx + uy * Fy + uz * Fz;
        // equilibria (d'Humieres: w_eps = 3, w_epsj = -11/2, w_xx = -1/2)
        R meq[19], Fb[19], sk[19];
        meq[0] = rho;                            Fb[0] = 0;                  sk[0] = 0;
        meq[1] = rho * (R(-11) + R(19) * uu);    Fb[1] = R(38) * uF + L.sig_e3 * Fm2;  sk[1] = L.s_e;
        meq[2] = rho * (R(3) - R(5.5) * uu);     Fb[2] = R(-11) * uF;        sk[2] = L.s_eps;
        meq[3] = rho * ux;                       Fb[3] = Fx;                 sk[3] = 1;
        meq[4] = R(-2.0 / 3.0) * rho * ux;       Fb[4] = R(-2.0 / 3.0) * Fx; sk[4] = L.s_q;
        meq[5] = rho * uy;                       Fb[5] = Fy;                 sk[5] = 1;
        meq[6] = R(-2.0 / 3.0) * rho * uy;       Fb[6] = R(-2.0 / 3.0) * Fy; sk[6] = L.s_q;
        meq[7] = rho * uz;                       Fb[7] = Fz;                 sk[7] = 1;
        meq[8] = R(-2.0 / 3.0) * rho * uz;       Fb[8] = R(-2.0 / 3.0) * Fz; sk[8] = L.s_q;
        const R pxx = R(3) * ux * ux - uu, axx = R(2) * ux * Fx - uy * Fy - uz * Fz;
        const R pww = uy * uy - uz * uz, aww = uy * Fy - uz * Fz;
        meq[9] = rho * pxx;                      Fb[9] = R(2) * axx;         sk[9] = L.s_p;
        meq[10] = R(-0.5) * rho * pxx;           Fb[10] = -axx;              sk[10] = L.s_q;
        meq[11] = rho * pww;                     Fb[11] = R(2) * aww;        sk[11] = L.s_p;
        meq[12] = R(-0.5) * rho * pww;           Fb[12] = -aww;              sk[12] = L.s_q;
        meq[13] = rho * ux * uy;                 Fb[13] = ux * Fy + uy * Fx; sk[13] = L.s_p;
        meq[14] = rho * uy * uz;                 Fb[14] = uy * Fz + uz * Fy; sk[14] = L.s_p;
        meq[15] = rho * ux * uz;                 Fb[15] = ux * Fz + uz * Fx; sk[15] = L.s_p;
        meq[16] = 0;                             Fb[16] = 0;                 sk[16] = L.s_q;
        meq[17] = 0;                             Fb[17] = 0;                 sk[17] = L.s_q;
        meq[18] = 0;                             Fb[18] = 0;                 sk[18] = L.s_q;
        // dm = -S (m - m^eq) + (I - S/2) Fbar, scaled by 1/|row|^2
        R dm[19];
#pragma unroll 19
        for (int kk = 0; kk < 19; ++kk)
            dm[kk] = (-sk[kk] * (m[kk] - meq[kk]) + (R(1) - R(0.5) * sk[kk]) * Fb[kk]) *
                     R(1.0 / mnorm(kk));
        // f* = f + M^T dm, pushed to x + c_i (bounce-back through walls)
        add_inverse19(dm, f);
#pragma unroll 19
        for (int i = 0; i < 19; ++i) {
            const R v = f[i];
            if (nbr_solid(nb, qz(i)))
                fn[qopp(i) * D.plane + n] = v;
            else
                fn[i * D.plane + (size_t)((long long)n + nbr_off(nb, qx(i), qy(i), qz(i)))] = v;
        }
    }

    // ---- D3Q7 MRT collision (deviation form), closed-form inverse of the
    // moment matrix (rows 1, c_x, c_y, c_z, |c|^2, c_x^2 - c_y^2, c_y^2 - c_z^2)
    {
        const R Td = g[0] + g[1] + g[2] + g[3] + g[4] + g[5] + g[6];
        const R m4 = g[1] + g[2] + g[3] + g[4] + g[5] + g[6];
        const R m5 = (g[1] + g[2]) - (g[3] + g[4]);
        const R m6 = (g[3] + g[4]) - (g[5] + g[6]);
        const R wd = L.w7_1 * R(6);
        const R s0 = Td - L.vs0 * (Td - Td) + Qs;
        const R s1 = m1 - L.vs1 * m1, s2 = m2 - L.vs1 * m2, s3 = m3 - L.vs1 * m3;
        const R s4 = m4 - L.vs3 * (m4 - wd * Td) + wd * Qs;
        const R s5 = m5 - L.vs4 * m5, s6 = m6 - L.vs4 * m6;
        const R b = (s4 - s5 + s6) * R(1.0 / 3.0);
        const R a = b + s5, c = b - s6;
        R gs[7];
        gs[0] = s0 - s4;
        gs[1] = R(0.5) * (a + s1);
        gs[2] = R(0.5) * (a - s1);
        gs[3] = R(0.5) * (b + s2);
        gs[4] = R(0.5) * (b - s2);
        gs[5] = R(0.5) * (c + s3);
        gs[6] = R(0.5) * (c - s3);
        // weighted streaming (Eq. 39) from this node's side: g*_i lands on
        // x = y + c_i as g_i(x) + (g*_i - g_i(x)) / (rho(x) c_v), with g_i(x)
        // and rho(x) those of the current state; through a wall g*_i
        // returns to this node as the opposite direction, A = 2 w^ T_w - g*_i
        // (Dirichlet) or g*_i (adiabatic)
        if (L.frozen_thermal) {
#pragma unroll 7
            for (int i = 0; i < 7; ++i) gn[i * D.plane + n] = g[i];
        } else {
#pragma unroll 7
            for (int i = 0; i < 7; ++i) {
                if ((i == 5 && nb.zhi) || (i == 6 && nb.zlo)) {
                    const int e = i == 5 ? 1 : 0, o = i == 5 ? 6 : 5;
                    const R Ai = D.therm[e] == T_DIRICHLET
                                     ? R(2) * L.w7_1 * (R)(D.T_edge[e] - D.T_ref) - gs[i]
                                     : gs[i];
                    gn[o * D.plane + n] = g[o] + (Ai - g[o]) * A[A_IC * D.plane + n];
                } else {
                    const size_t m = (size_t)((long long)n + nbr_off(nb, hx(i), hy(i), hz(i)));
                    const R go = gc[i * D.plane + m];
                    gn[i * D.plane + m] = go + (gs[i] - go) * A[A_IC * D.plane + m];
                }
            }
        }
    }
    Pn_out[n] = Pn;
}

// ---------------------------------------------------------------------------
// macroscopic fields of a node from its (deviation) populations
template <class R>
__device__ __forceinline__ void macro_node(const Dom3& D, const Phys<R>& P, R cv, const R* f19,
                                           const R* g7, size_t n, int* err, R* rho_out) {
    R* A = (R*)D.aux;
    R rd = 0, jx = 0, jy = 0, jz = 0, Td = 0;
#pragma unroll 19
    for (int i = 0; i < 19; ++i) {
        rd += f19[i];
        if (qx(i)) jx += R(qx(i)) * f19[i];
        if (qy(i)) jy += R(qy(i)) * f19[i];
        if (qz(i)) jz += R(qz(i)) * f19[i];
    }
#pragma unroll 19
    for (int i = 0; i < 7; ++i) Td += g7[i];
    const R rho = rd + (R)D.rho_ref, T = Td + (R)D.T_ref;
    R q2, TdpdT;
    eos_node(P, rho, T, &q2, &TdpdT);
    if (!(q2 >= R(0))) *err |= (q2 != q2) ? ERR_NONFINITE : ERR_PSI;
    if (!(T == T) || !(rho == rho)) *err |= ERR_NONFINITE;
    A[A_RHO * D.plane + n] = rho;
    A[A_T * D.plane + n] = T;
    A[A_PSI * D.plane + n] = f_sqrt(q2);
    A[A_TDPDT * D.plane + n] = TdpdT;
    A[A_IC * D.plane + n] = f_rcp(rho * cv);
    A[A_JX * D.plane + n] = jx;
    A[A_JY * D.plane + n] = jy;
    A[A_JZ * D.plane + n] = jz;
    *rho_out = rho;
}

// block sum of rho into the density ring (FP64), for the buoyancy of the
// next step
__device__ __forceinline__ void add_mass(const Dom3& D, double v, int slot) {
    __shared__ double red[4];
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((t & 31) == 0) red[t >> 5] = v;
    __syncthreads();
    if (t == 0) massq_add(&D.ctl->massq[slot], red[0] + red[1] + red[2] + red[3], massq_scale(D.inv_n));
}

// macroscopic fields of the current state (next = 0) or of the state the
// step in progress has just written (next = 1), with its density sum into
// slot (step + next) % 3 for buoyancy
template <class R>
__global__ void __launch_bounds__(128) k3_macro(Dom3 D, Phys<R> P, R cv, int use_mass, int next) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    const bool in = x < D.nx && y < D.ny;
    double msum = 0.0;
    const long long step = __ldcg(&D.ctl->step);
    if (in) {
        const int par = (int)(step & 1) ^ next;
        const R* fc = (const R*)D.f[par];
        const R* gc = (const R*)D.g[par];
        const size_t n = nid<R>(D, x, y, z);
        R f[19], g[7];
#pragma unroll 19
        for (int i = 0; i < 19; ++i) f[i] = fc[i * D.plane + n];
#pragma unroll 19
        for (int i = 0; i < 7; ++i) g[i] = gc[i * D.plane + n];
        int err = 0;
        R rho;
        macro_node<R>(D, P, cv, f, g, n, &err, &rho);
        if (err) atomicOr(&D.ctl->err, err);
        msum = (double)rho;
    }
    if (use_mass) add_mass(D, in ? msum : 0.0, (int)((step + next) % 3));
}

// end of a step: publish the density sum the step's blend accumulated (the
// new state's, slot (s + 1) % 3), clear the slot the next step's blend
// accumulates into and advance the counter
__global__ void k3_advance(Ctl* ctl, double qscale) {
    const long long s = ctl->step;
    ctl->mass[(s + 1) % 3] = massq_value(ctl->massq[(s + 1) % 3], qscale);
    ctl->massq[(s + 2) % 3] = 0;
    ctl->step = s + 1;
}

// ---------------------------------------------------------------------------
// Fused step: one kernel for the whole step.  A CTA takes an xy tile of
// TX x TY nodes and a segment [z0, z1) of planes and marches k through the
// planes, the stages skewed so that each reads only planes its predecessors
// have finished (two barriers per plane):
//   A(k)     rho, j, T, psi, T dp/dT, 1/(rho c_v) on the tile + 2 halo nodes
//            from f(t), g(t) (beyond a wall: the ghost-layer psi, Section 3.3)
//   C(k-3)   on the tile: div u, grad T, Q, P^n, S and the D3Q7 collision
//            (Eqs. 20, 24, 49-50); g*_i blended into the destination's
//            g(t+1) = g + (g* - g)/(rho c_v) (Eq. 39; anti-bounce-back at
//            walls)
//   B(k-1)   F_m, F, u on the tile + 1 (Eqs. 9, 11); on the tile the D3Q19
//            collision (Eq. 5) with f*_i pushed to x + c_i (bounce-back at
//            walls) and the new state's density sum
// Shared-memory rings carry psi, rho, 1/(rho c_v), j, T dp/dT and u between
// the stages.  Each node is collided by the CTA that owns it, which writes
// its post-collision populations straight to their destinations in f(t+1)
// and g(t+1); only the fields the stencils need (two halo nodes of psi, one
// of u) are recomputed around the tile.  The step reads f, g, P once and
// writes them once (the halo and destination reads come from L2): no u, F
// or g* planes and no second read of f for the next state's fields.

// ring slot of plane k (k >= -8)
__device__ __forceinline__ int ring(int k, int s) { return (k + 24) % s; }

#ifndef K3_TILE_X
#define K3_TILE_X 16
#define K3_TILE_Y 16
#define K3_THREADS 256
#endif
template <class R>
struct Tile3 {
    static constexpr int TX = K3_TILE_X, TY = K3_TILE_Y, NT = K3_THREADS;
    static constexpr int W2 = TX + 4, N2 = W2 * (TY + 4);   // tile + 2: fields, psi
    static constexpr int W1 = TX + 2, N1 = W1 * (TY + 2);   // tile + 1: F, u
    static constexpr int NI = TX * TY;                       // the tile: collisions
    static constexpr int NB = N1 - NI;                       // tile + 1 outside the tile
    // psi 3, rho 4, 1/(rho c_v) 5, j 2 x 3, T dp/dT 4 planes of tile + 2; u 3 x 3 of tile + 1
    static constexpr int ELEMS = 22 * N2 + 9 * N1;
    static constexpr size_t BYTES = (size_t)ELEMS * sizeof(R);
    // FP32: three CTAs per SM (80 registers, no spills; 11.7 against 10.1
    // GLUPS with two at 120 registers, against 10.2 with four, which spill);
    // FP64 needs ~240 registers
    static constexpr int MIN_BLOCKS = (sizeof(R) == 4 && NT <= 256) ? 3 : 1;
    static_assert(NI <= NT, "the collisions take one tile node per thread");
    static_assert(N2 <= 2 * NT && N1 <= 2 * NT, "two passes per stage");
};

template <class R>
__global__ void __launch_bounds__(Tile3<R>::NT, Tile3<R>::MIN_BLOCKS)
k3_fused(Dom3 D, Phys<R> P, Lat3<R> L, int zseg, int use_mass) {
    using G = Tile3<R>;
    constexpr int TX = G::TX, TY = G::TY, NT = G::NT, W2 = G::W2, N2 = G::N2, W1 = G::W1,
                  N1 = G::N1, NI = G::NI, NB = G::NB;
    extern __shared__ __align__(16) unsigned char k3_smem[];
    R* const s_psi = reinterpret_cast<R*>(k3_smem);   // [3][N2]
    R* const s_rho = s_psi + 3 * N2;                   // [4][N2]
    R* const s_ic = s_rho + 4 * N2;                    // [5][N2] 1 / (rho c_v)
    R* const s_j = s_ic + 5 * N2;                      // [2][3][N2]
    R* const s_tdp = s_j + 6 * N2;                     // [4][N2]
    R* const s_u = s_tdp + 4 * N2;                     // [3][3][N1]

    const int tid = threadIdx.x;
    const int ntx = (D.nx + TX - 1) / TX;
    const int x0 = (int)(blockIdx.x % ntx) * TX, y0 = (int)(blockIdx.x / ntx) * TY;
    const int z0 = (int)blockIdx.y * zseg, z1 = min(D.nz, z0 + zseg);
    const long long step = __ldcg(&D.ctl->step);
    const int par = (int)(step & 1);
    const R* __restrict__ fc = (const R*)D.f[par];
    R* __restrict__ fnx = (R*)D.f[par ^ 1];
    const R* __restrict__ gc = (const R*)D.g[par];
    R* __restrict__ gnx = (R*)D.g[par ^ 1];
    const R* __restrict__ Pc = (const R*)D.P[par];
    R* __restrict__ Pnx = (R*)D.P[par ^ 1];
    const size_t PL = D.plane, ZS = (size_t)D.ny * D.pitch;
    const R rho_ref = (R)D.rho_ref, T_ref = (R)D.T_ref;
    const R rho_ave = L.gravity != R(0) ? (R)(__ldcg(&D.ctl->mass[(step + 2) % 3]) * D.inv_n) : R(0);

    // in-plane offsets of the nodes this thread takes in stage A (the tile's
    // local coordinates wrap periodically onto the domain)
    int oA[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int a = tid + r * NT;
        const int ax = a < N2 ? a % W2 - 2 : 0, ay = a < N2 ? a / W2 - 2 : 0;
        oA[r] = wrapm(y0 + ay, D.ny) * D.pitch + wrapm(x0 + ax, D.nx);
    }
    // this thread's node on the ring of tile + 1 around the tile (tid < NB),
    // where stage B computes F and u only
    int rx = 0, ry = 0;
    if (tid < NB) {
        if (tid < W1) { rx = tid - 1; ry = -1; }
        else if (tid < 2 * W1) { rx = tid - W1 - 1; ry = TY; }
        else if (tid < 2 * W1 + TY) { rx = -1; ry = tid - 2 * W1; }
        else { rx = TX; ry = tid - 2 * W1 - TY; }
    }
    // the tile node this thread takes in stages B (F, u and the collision)
    // and C; its wrapped neighbour offsets for the pushes
    const int cx = tid % TX, cy = tid / TX;
    const int gxo = x0 + cx, gyo = y0 + cy;
    const bool own_xy = tid < NI && gxo < D.nx && gyo < D.ny;
    const int oC = own_xy ? gyo * D.pitch + gxo : 0;
    const long long oxp = own_xy && gxo == D.nx - 1 ? -(long long)(D.nx - 1) : 1;
    const long long oxm = own_xy && gxo == 0 ? (long long)(D.nx - 1) : -1;
    const long long oyp = own_xy && gyo == D.ny - 1 ? -(long long)(D.ny - 1) * D.pitch : D.pitch;
    const long long oym = own_xy && gyo == 0 ? (long long)(D.ny - 1) * D.pitch : -(long long)D.pitch;
    auto inplane = [&](int qxv, int qyv) {
        return (qxv > 0 ? oxp : (qxv < 0 ? oxm : 0)) + (qyv > 0 ? oyp : (qyv < 0 ? oym : 0));
    };
    int err = 0;
    double msum = 0.0;
    int kzA = wrapm(z0 - 2, D.nz);   // the plane of A(k), wrapped; advanced with k

    for (int k = z0 - 2; k <= z1 + 2; ++k, kzA = kzA + 1 == D.nz ? 0 : kzA + 1) {
        // ================= phase 1: A(k), C(k - 3)
        if (k <= z1 + 1) {
            R* const psA = s_psi + ring(k, 3) * N2;
            if (D.walls && (k < 0 || k >= D.nz)) {
                if (k == -1 || k == D.nz) {
                    const R* gp = (const R*)D.ghost + (k < 0 ? (size_t)0 : ZS);
#pragma unroll
                    for (int r = 0; r < 2; ++r)
                        if (tid + r * NT < N2) psA[tid + r * NT] = gp[oA[r]];
                }
            } else {
                const size_t zo = (size_t)kzA * ZS;
                R* const rA = s_rho + ring(k, 4) * N2;
                R* const iA = s_ic + ring(k, 5) * N2;
                R* const jA = s_j + ring(k, 2) * 3 * N2;
                R* const tA = s_tdp + ring(k, 4) * N2;
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int a = tid + r * NT;
                    if (a < N2) {
                        const size_t n = zo + oA[r];
                        R f[19], g[7];
#pragma unroll
                        for (int i = 0; i < 19; ++i) f[i] = __ldg(fc + i * PL + n);
#pragma unroll
                        for (int i = 0; i < 7; ++i) g[i] = __ldg(gc + i * PL + n);
                        R rd = 0, jx = 0, jy = 0, jz = 0, Td = 0;
#pragma unroll
                        for (int i = 0; i < 19; ++i) {
                            rd += f[i];
                            if (qx(i)) jx += R(qx(i)) * f[i];
                            if (qy(i)) jy += R(qy(i)) * f[i];
                            if (qz(i)) jz += R(qz(i)) * f[i];
                        }
#pragma unroll
                        for (int i = 0; i < 7; ++i) Td += g[i];
                        const R rho = rd + rho_ref, T = Td + T_ref;
                        R q2, tdp;
                        eos_node(P, rho, T, &q2, &tdp);
                        if (!(q2 >= R(0))) err |= (q2 != q2) ? ERR_NONFINITE : ERR_PSI;
                        if (!(T == T) || !(rho == rho)) err |= ERR_NONFINITE;
                        psA[a] = f_sqrt(q2);
                        rA[a] = rho;
                        iA[a] = f_rcp(rho * L.cv);
                        jA[a] = jx;
                        jA[N2 + a] = jy;
                        jA[2 * N2 + a] = jz;
                        tA[a] = tdp;
                    }
                }
            }
        }
        {
            const int q = k - 3;
            if (q >= z0 && q < z1 && own_xy) {
                const size_t n = (size_t)q * ZS + oC;
                const bool lo_wall = D.walls && q == 0, hi_wall = D.walls && q == D.nz - 1;
                const R* const um = s_u + ring(q - 1, 3) * 3 * N1;
                const R* const u0 = s_u + ring(q, 3) * 3 * N1;
                const R* const up = s_u + ring(q + 1, 3) * 3 * N1;
                const int c1 = (cy + 1) * W1 + cx + 1, c2 = (cy + 2) * W2 + cx + 2;
                // div u: (1/c_s^2) sum_i w_i c_i . u(x + c_i); walls carry u = 0
                // (3 w_i = 1/6 on the axes, 1/12 on the diagonals, summed apart)
                R dva = 0, dvd = 0;
#pragma unroll
                for (int i = 1; i < 19; ++i) {
                    if ((qz(i) < 0 && lo_wall) || (qz(i) > 0 && hi_wall)) continue;
                    const R* us = (qz(i) < 0 ? um : (qz(i) > 0 ? up : u0)) + c1 + qy(i) * W1 + qx(i);
                    R& acc = qc2(i) == 1 ? dva : dvd;
                    if (qx(i)) acc += R(qx(i)) * us[0];
                    if (qy(i)) acc += R(qy(i)) * us[N1];
                    if (qz(i)) acc += R(qz(i)) * us[2 * N1];
                }
                const R divu = dva * R(1.0 / 6.0) + dvd * R(1.0 / 12.0);
                R g[7];
#pragma unroll
                for (int i = 0; i < 7; ++i) g[i] = gc[i * PL + n];
                const R ux = u0[c1], uy = u0[N1 + c1], uz = u0[2 * N1 + c1];
                const R rho = s_rho[ring(q, 4) * N2 + c2], TdpdT = s_tdp[ring(q, 4) * N2 + c2];
                // grad T from the local first moments: c^_s^2 d_a T = -vs1 m^_a
                const R m1 = g[1] - g[2], m2 = g[3] - g[4], m3 = g[5] - g[6];
                const R kT = -L.vs1 / L.cs2h;
                const R dTx = kT * m1, dTy = kT * m2, dTz = kT * m3;
                const R C = rho * L.cv;
                const R Q = -(C * (ux * dTx + uy * dTy + uz * dTz) + TdpdT * divu);
                const R Pn = Q * f_rcp(C);
                const R Qs = step == 0 ? Q : Q + R(0.5) * (Q - C * Pc[n]);
                Pnx[n] = Pn;
                // ---- D3Q7 MRT collision (deviation form), closed-form inverse
                const R Td = g[0] + g[1] + g[2] + g[3] + g[4] + g[5] + g[6];
                const R m4 = g[1] + g[2] + g[3] + g[4] + g[5] + g[6];
                const R m5 = (g[1] + g[2]) - (g[3] + g[4]);
                const R m6 = (g[3] + g[4]) - (g[5] + g[6]);
                const R wd = L.w7_1 * R(6);
                const R s0 = Td - L.vs0 * (Td - Td) + Qs;
                const R s1 = m1 - L.vs1 * m1, s2 = m2 - L.vs1 * m2, s3 = m3 - L.vs1 * m3;
                const R s4 = m4 - L.vs3 * (m4 - wd * Td) + wd * Qs;
                const R s5 = m5 - L.vs4 * m5, s6 = m6 - L.vs4 * m6;
                const R bq = (s4 - s5 + s6) * R(1.0 / 3.0);
                const R aq = bq + s5, cq = bq - s6;
                R gs[7];
                gs[0] = s0 - s4;
                gs[1] = R(0.5) * (aq + s1);
                gs[2] = R(0.5) * (aq - s1);
                gs[3] = R(0.5) * (bq + s2);
                gs[4] = R(0.5) * (bq - s2);
                gs[5] = R(0.5) * (cq + s3);
                gs[6] = R(0.5) * (cq - s3);
                // weighted streaming (Eq. 39) from this node's side: g*_i lands on
                // x = y + c_i as g_i(x) + (g*_i - g_i(x)) / (rho(x) c_v) of the
                // current state; through a wall it returns here as the opposite
                // direction, A = 2 w^ T_w - g*_i (Dirichlet) or g*_i (adiabatic)
                if (L.frozen_thermal) {
#pragma unroll
                    for (int i = 0; i < 7; ++i) gnx[i * PL + n] = g[i];
                } else {
                    const long long zp = q == D.nz - 1 ? -(long long)(D.nz - 1) * (long long)ZS : (long long)ZS;
                    const long long zm = q == 0 ? (long long)(D.nz - 1) * (long long)ZS : -(long long)ZS;
#pragma unroll
                    for (int i = 0; i < 7; ++i) {
                        if ((i == 5 && hi_wall) || (i == 6 && lo_wall)) {
                            const int e = i == 5 ? 1 : 0, o = i == 5 ? 6 : 5;
                            const R Ai = D.therm[e] == T_DIRICHLET
                                             ? R(2) * L.w7_1 * (R)(D.T_edge[e] - D.T_ref) - gs[i]
                                             : gs[i];
                            gnx[o * PL + n] = g[o] + (Ai - g[o]) * s_ic[ring(q, 5) * N2 + c2];
                        } else {
                            const long long off = inplane(hx(i), hy(i)) + (hz(i) > 0 ? zp : (hz(i) < 0 ? zm : 0));
                            const size_t m = (size_t)((long long)n + off);
                            const R go = gc[i * PL + m];
                            const R iCm = s_ic[ring(q + hz(i), 5) * N2 + c2 + hy(i) * W2 + hx(i)];
                            gnx[i * PL + m] = go + (gs[i] - go) * iCm;
                        }
                    }
                }
            }
        }
        __syncthreads();

        // ================= phase 2: B(k - 1)
        {
            const int p = k - 1;
            if (p >= z0 - 1 && p <= z1 && !(D.walls && (p < 0 || p >= D.nz))) {
                const bool own_z = p >= z0 && p < z1;
                const R* const psm = s_psi + ring(p - 1, 3) * N2;
                const R* const ps0 = s_psi + ring(p, 3) * N2;
                const R* const psp = s_psi + ring(p + 1, 3) * N2;
                const R* const rB = s_rho + ring(p, 4) * N2;
                const R* const jB = s_j + ring(p, 2) * 3 * N2;
                R* const uB = s_u + ring(p, 3) * 3 * N1;
                // pass 0: this thread's ring node of tile + 1; pass 1: its tile node
#pragma unroll 1
                for (int r = 0; r < 2; ++r) {
                    if (r == 0 ? tid >= NB : tid >= NI) continue;
                    const int lx = r ? cx : rx, ly = r ? cy : ry;
                    const int c2 = (ly + 2) * W2 + lx + 2;
                    // sum_i varpi(|c_i|^2) psi(x + c_i) c_i with the axis (1/6) and
                    // diagonal (1/12) neighbours summed apart and weighted once
                    R ax = 0, ay = 0, az = 0, dx = 0, dy = 0, dz = 0;
#pragma unroll
                    for (int i = 1; i < 19; ++i) {
                        const R* pp = qz(i) < 0 ? psm : (qz(i) > 0 ? psp : ps0);
                        const R pn = pp[c2 + qy(i) * W2 + qx(i)];
                        if (qc2(i) == 1) {
                            if (qx(i)) ax += R(qx(i)) * pn;
                            if (qy(i)) ay += R(qy(i)) * pn;
                            if (qz(i)) az += R(qz(i)) * pn;
                        } else {
                            if (qx(i)) dx += R(qx(i)) * pn;
                            if (qy(i)) dy += R(qy(i)) * pn;
                            if (qz(i)) dz += R(qz(i)) * pn;
                        }
                    }
                    const R sx = ax * R(1.0 / 6.0) + dx * R(1.0 / 12.0);
                    const R sy = ay * R(1.0 / 6.0) + dy * R(1.0 / 12.0);
                    const R sz = az * R(1.0 / 6.0) + dz * R(1.0 / 12.0);
                    const R psi = ps0[c2], rho = rB[c2];
                    const R Fx = P.negG * psi * sx, Fy = P.negG * psi * sy;
                    const R Fz = P.negG * psi * sz - L.gravity * (rho - rho_ave);
                    R ux = 0, uy = 0, uz = 0;
                    if (!L.frozen_flow) {
                        const R ir = f_rcp(rho);
                        ux = (jB[c2] + R(0.5) * Fx) * ir;
                        uy = (jB[N2 + c2] + R(0.5) * Fy) * ir;
                        uz = (jB[2 * N2 + c2] + R(0.5) * Fz) * ir;
                    }
                    const int c1 = (ly + 1) * W1 + lx + 1;
                    uB[c1] = ux;
                    uB[N1 + c1] = uy;
                    uB[2 * N1 + c1] = uz;
                    // the tile node: collide it if this CTA owns it
                    if (r == 0 || !own_z || !own_xy) continue;
                    const size_t n = (size_t)p * ZS + oC;
                    R f[19];
#pragma unroll
                    for (int i = 0; i < 19; ++i) f[i] = fc[i * PL + n];
                    if (L.frozen_flow) {
                        R rd = 0;
#pragma unroll
                        for (int i = 0; i < 19; ++i) {
                            fnx[i * PL + n] = f[i];
                            rd += f[i];
                        }
                        if (use_mass) msum += (double)(rd + rho_ref);
                        continue;
                    }
                    // ---- D3Q19 MRT collision in moment space
                    const R Fm2 = P.negG * P.negG * (sx * sx + sy * sy + sz * sz);
                    R m[19];
                    moments19(f, m);
                    m[0] += rho_ref;
                    m[1] += R(-11) * rho_ref;
                    m[2] += R(3) * rho_ref;
                    const R uu = ux * ux + uy * uy + uz * uz;
                    const R uF = ux * Fx + uy * Fy + uz * Fz;
                    R meq[19], Fb[19], sk[19];
                    meq[0] = rho;                            Fb[0] = 0;                  sk[0] = 0;
                    meq[1] = rho * (R(-11) + R(19) * uu);    Fb[1] = R(38) * uF + L.sig_e3 * Fm2;  sk[1] = L.s_e;
                    meq[2] = rho * (R(3) - R(5.5) * uu);     Fb[2] = R(-11) * uF;        sk[2] = L.s_eps;
                    meq[3] = rho * ux;                       Fb[3] = Fx;                 sk[3] = 1;
                    meq[4] = R(-2.0 / 3.0) * rho * ux;       Fb[4] = R(-2.0 / 3.0) * Fx; sk[4] = L.s_q;
                    meq[5] = rho * uy;                       Fb[5] = Fy;                 sk[5] = 1;
                    meq[6] = R(-2.0 / 3.0) * rho * uy;       Fb[6] = R(-2.0 / 3.0) * Fy; sk[6] = L.s_q;
                    meq[7] = rho * uz;                       Fb[7] = Fz;                 sk[7] = 1;
                    meq[8] = R(-2.0 / 3.0) * rho * uz;       Fb[8] = R(-2.0 / 3.0) * Fz; sk[8] = L.s_q;
                    const R pxx = R(3) * ux * ux - uu, axx = R(2) * ux * Fx - uy * Fy - uz * Fz;
                    const R pww = uy * uy - uz * uz, aww = uy * Fy - uz * Fz;
                    meq[9] = rho * pxx;                      Fb[9] = R(2) * axx;         sk[9] = L.s_p;
                    meq[10] = R(-0.5) * rho * pxx;           Fb[10] = -axx;              sk[10] = L.s_q;
                    meq[11] = rho * pww;                     Fb[11] = R(2) * aww;        sk[11] = L.s_p;
                    meq[12] = R(-0.5) * rho * pww;           Fb[12] = -aww;              sk[12] = L.s_q;
                    meq[13] = rho * ux * uy;                 Fb[13] = ux * Fy + uy * Fx; sk[13] = L.s_p;
                    meq[14] = rho * uy * uz;                 Fb[14] = uy * Fz + uz * Fy; sk[14] = L.s_p;
                    meq[15] = rho * ux * uz;                 Fb[15] = ux * Fz + uz * Fx; sk[15] = L.s_p;
                    meq[16] = 0;                             Fb[16] = 0;                 sk[16] = L.s_q;
                    meq[17] = 0;                             Fb[17] = 0;                 sk[17] = L.s_q;
                    meq[18] = 0;                             Fb[18] = 0;                 sk[18] = L.s_q;
                    R dm[19];
#pragma unroll
                    for (int kk = 0; kk < 19; ++kk)
                        dm[kk] = (-sk[kk] * (m[kk] - meq[kk]) + (R(1) - R(0.5) * sk[kk]) * Fb[kk]) *
                                 R(1.0 / mnorm(kk));
                    add_inverse19(dm, f);   // f* = f + M^T dm
                    // push to x + c_i; through a wall f*_i returns as f_opp(i)
                    const long long zp = p == D.nz - 1 ? -(long long)(D.nz - 1) * (long long)ZS : (long long)ZS;
                    const long long zm = p == 0 ? (long long)(D.nz - 1) * (long long)ZS : -(long long)ZS;
                    const bool lo_wall = D.walls && p == 0, hi_wall = D.walls && p == D.nz - 1;
                    R rd = 0;
                    static_for<19>([&](auto icn) {
                        constexpr int i = decltype(icn)::value;
                        rd += f[i];
                        if ((qz(i) < 0 && lo_wall) || (qz(i) > 0 && hi_wall)) {
                            fnx[qopp(i) * PL + n] = f[i];
                        } else {
                            const long long off = inplane(qx(i), qy(i)) + (qz(i) > 0 ? zp : (qz(i) < 0 ? zm : 0));
                            fnx[i * PL + (size_t)((long long)n + off)] = f[i];
                        }
                    });
                    // the new state's mass: streaming moves the f* without loss
                    if (use_mass) msum += (double)(rd + rho_ref);
                }
            }
        }
        __syncthreads();
    }

    // density sum of the new state for the buoyancy of the next step
    if (use_mass) {
        double* red = reinterpret_cast<double*>(k3_smem);
        for (int o = 16; o > 0; o >>= 1) msum += __shfl_down_sync(0xffffffffu, msum, o);
        if ((tid & 31) == 0) red[tid >> 5] = msum;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < NT / 32; ++w) s += red[w];
            massq_add(&D.ctl->massq[(step + 1) % 3], s, massq_scale(D.inv_n));
        }
    }
    if (err) atomicOr(&D.ctl->err, err);
}

// psi of the ghost layers beyond the two walls (Section 3.3) from the current
// state: rho_ghost = rho(layer 2) + tan(pi/2 - theta) |tangential difference of
// rho at layer 1|, at the temperature of layer 1
template <class R>
__global__ void k3_ghost(Dom3 D, Phys<R> P) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int e = blockIdx.z;
    if (x >= D.nx || y >= D.ny) return;
    const int par = (int)(__ldcg(&D.ctl->step) & 1);
    const R* fc = (const R*)D.f[par];
    const R* gc = (const R*)D.g[par];
    const int z1 = e == 0 ? 0 : D.nz - 1, z2 = e == 0 ? 1 : D.nz - 2;
    auto rho_at = [&](int xx, int yy, int zz) {
        const size_t n = nid<R>(D, xx, yy, zz);
        R rd = 0;
#pragma unroll
        for (int i = 0; i < 19; ++i) rd += fc[i * D.plane + n];
        return rd + (R)D.rho_ref;
    };
    const R dx = rho_at(wrapn(x + 1, D.nx), y, z1) - rho_at(wrapn(x - 1, D.nx), y, z1);
    const R dy = rho_at(x, wrapn(y + 1, D.ny), z1) - rho_at(x, wrapn(y - 1, D.ny), z1);
    const R rg = rho_at(x, y, z2) + (R)D.cot * rsq(dx * dx + dy * dy);
    const size_t n1 = nid<R>(D, x, y, z1);
    R Td = 0;
#pragma unroll
    for (int i = 0; i < 7; ++i) Td += gc[i * D.plane + n1];
    const R q2 = psi2_of(P, rg, Td + (R)D.T_ref);
    if (!(q2 >= R(0))) atomicOr(&D.ctl->err, (q2 != q2) ? ERR_NONFINITE : ERR_PSI);
    ((R*)D.ghost)[((size_t)e * D.ny + y) * D.pitch + x] = f_sqrt(q2);
}

// populations f = f^eq(rho, u), g = w^ T as deviations; P = 0
template <class R>
__global__ void k3_init(Dom3 D, Lat3<R> L, const double* rho, const double* ux,
                        const double* uy, const double* uz, const double* T) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= D.nx || y >= D.ny) return;
    const size_t h = ((size_t)z * D.ny + y) * D.nx + x, n = nid<R>(D, x, y, z);
    R* f = (R*)D.f[0];
    R* g = (R*)D.g[0];
    const double r = rho[h], a = ux[h], b = uy[h], c = uz[h], t = T[h];
    const double uu = a * a + b * b + c * c;
#pragma unroll 19
    for (int i = 0; i < 19; ++i) {
        const double cu = qx(i) * a + qy(i) * b + qz(i) * c;
        const double fe = qw(i) * r * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
        f[i * D.plane + n] = (R)(fe - qw(i) * D.rho_ref);
    }
    const double w0 = (double)L.w7_0, w1 = (double)L.w7_1;
#pragma unroll 19
    for (int i = 0; i < 7; ++i) g[i * D.plane + n] = (R)((i == 0 ? w0 : w1) * (t - D.T_ref));
    ((R*)D.P[0])[n] = R(0);
}

// state -> host-layout doubles: fields (rho, u, T) or absolute populations
template <class R>
__global__ void k3_export(Dom3 D, Lat3<R> L, int what, double* out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= D.nx || y >= D.ny) return;
    const size_t N = (size_t)D.nx * D.ny * D.nz;
    const size_t h = ((size_t)z * D.ny + y) * D.nx + x, n = nid<R>(D, x, y, z);
    const int par = (int)(__ldcg(&D.ctl->step) & 1);
    if (what == 0) {
        const R* A = (const R*)D.aux;
        const R* B = (const R*)D.aux2;
        out[0 * N + h] = (double)A[A_RHO * D.plane + n];
        out[1 * N + h] = (double)B[B_UX * D.plane + n];
        out[2 * N + h] = (double)B[B_UY * D.plane + n];
        out[3 * N + h] = (double)B[B_UZ * D.plane + n];
        out[4 * N + h] = (double)A[A_T * D.plane + n];
        const double ux = out[1 * N + h], uy = out[2 * N + h], uz = out[3 * N + h];
        out[5 * N + h] = sqrt(ux * ux + uy * uy + uz * uz);
    } else {
        const R* f = (const R*)D.f[par];
        const R* g = (const R*)D.g[par];
        for (int i = 0; i < 19; ++i) out[i * N + h] = (double)f[i * D.plane + n] + qw(i) * D.rho_ref;
        for (int i = 0; i < 7; ++i)
            out[(19 + i) * N + h] = (double)g[i * D.plane + n] +
                                    (double)(i == 0 ? L.w7_0 : L.w7_1) * D.T_ref;
        out[26 * N + h] = (double)((const R*)D.P[par])[n];
    }
}

}  // namespace
}  // namespace lbm

using namespace lbm;

struct lbm3d_ctx {
    int nx = 0, ny = 0, nz = 0, prec = 1;
    lbm_params params;
    lbm3d_bc bc;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void* mem = nullptr;
    Ctl* ctl = nullptr;
    Dom3 D;
    cudaGraphExec_t graph = nullptr;
    bool fused = true;       // one fused kernel per step (else three kernels)
    int zseg = 0;            // planes per CTA of the fused step
    bool aux_stale = false;  // the per-node planes lag the state (fused steps)
    long long step = 0;
    bool initialized = false;
    int sticky = LBM_OK;
    std::string err;
    double* host_buf = nullptr;   // device doubles: 27 N (export), reused
    void* diag_scratch = nullptr;
    double* diag_out = nullptr;
    double* zeros = nullptr;
};

namespace {

size_t pitch_for(int nx) { return ((size_t)nx + 31) / 32 * 32; }

size_t bytes_for(int nx, int ny, int nz, int prec) {
    const size_t es = prec == LBM_FP64 ? 8 : 4;
    const size_t plane = pitch_for(nx) * ny * nz;
    // f 2 x 19, g 2 x 7, P 2, aux 8, aux2 7, two ghost-layer planes
    return plane * es * (38 + 14 + 2 + A_N + B_N) + 2 * pitch_for(nx) * ny * es;
}

// planes per CTA of the fused step: enough (tile, segment) units for about
// three per resident CTA, segments of 16 to 48 planes
int auto_zseg(int nx, int ny, int nz, int prec) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        sms = 148;
    const int tx = Tile3<float>::TX, ty = Tile3<float>::TY;
    const long long tiles = (long long)((nx + tx - 1) / tx) * ((ny + ty - 1) / ty);
    const long long slots = (long long)sms * (prec == LBM_FP64 ? Tile3<double>::MIN_BLOCKS
                                                              : Tile3<float>::MIN_BLOCKS);
    const long long nseg = (3 * slots + tiles - 1) / tiles;
    int zs = (int)((nz + nseg - 1) / nseg);
    if (zs < 16) zs = 16;
    if (zs > 48) zs = 48;
    return zs > nz ? nz : zs;
}

int set_err3(lbm3d_ctx* c, int code, const char* msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_err3(lbm3d_ctx* c, cudaError_t e, const char* where) {
    if (e == cudaSuccess) return LBM_OK;
    if (c) c->err = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
}

// one thread per node
dim3 blk3() { return dim3(32, 4, 1); }
dim3 grd3(const lbm3d_ctx* c) { return dim3((c->nx + 31) / 32, (c->ny + 3) / 4, c->nz); }

template <class R>
int launch_fused(lbm3d_ctx* c) {
    using G = Tile3<R>;
    Phys<R> P = make_phys<R>(phys_of(c->params));
    Lat3<R> L = make_lat3<R>(c->params);
    if (c->D.walls)
        k3_ghost<R><<<dim3((c->nx + 31) / 32, (c->ny + 3) / 4, 2), blk3(), 0, c->stream>>>(c->D, P);
    const dim3 grid((unsigned)(((c->nx + G::TX - 1) / G::TX) * ((c->ny + G::TY - 1) / G::TY)),
                    (unsigned)((c->nz + c->zseg - 1) / c->zseg));
    k3_fused<R><<<grid, G::NT, G::BYTES, c->stream>>>(c->D, P, L, c->zseg, c->params.gravity != 0.0);
    k3_advance<<<1, 1, 0, c->stream>>>(c->ctl, massq_scale(c->D.inv_n));
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// the per-node planes (rho, T, psi, T dp/dT, j) of the current state
template <class R>
void launch_macro(lbm3d_ctx* c) {
    k3_macro<R><<<grd3(c), blk3(), 0, c->stream>>>(c->D, make_phys<R>(phys_of(c->params)),
                                                   (R)c->params.cv, 0, 0);
}

template <class R>
int launch_step(lbm3d_ctx* c) {
    if (c->fused) return launch_fused<R>(c);
    Phys<R> P = make_phys<R>(phys_of(c->params));
    Lat3<R> L = make_lat3<R>(c->params);
    const dim3 b = blk3(), g = grd3(c);
    k3_force<R><<<g, b, 0, c->stream>>>(c->D, P, L);
    k3_collide<R><<<g, b, 0, c->stream>>>(c->D, P, L);
    k3_macro<R><<<g, b, 0, c->stream>>>(c->D, make_phys<R>(phys_of(c->params)), (R)c->params.cv,
                                        c->params.gravity != 0.0, 1);
    k3_advance<<<1, 1, 0, c->stream>>>(c->ctl, massq_scale(c->D.inv_n));
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int step_once(lbm3d_ctx* c) { return c->prec == LBM_FP64 ? launch_step<double>(c) : launch_step<float>(c); }

int check3(lbm3d_ctx* c) {
    Ctl h;
    cudaError_t e = cudaMemcpyAsync(&h, c->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_err3(c, e, "reading the control block");
    if (h.err && c->sticky == LBM_OK) {
        c->sticky = (h.err & ERR_PSI) ? LBM_EPSI : LBM_ENONFINITE;
        c->err = c->sticky == LBM_EPSI ? "psi^2 < 0 at some node" : "non-finite density or temperature";
    }
    return c->sticky;
}

int ensure_buf(lbm3d_ctx* c) {
    if (c->host_buf) return LBM_OK;
    const size_t N = (size_t)c->nx * c->ny * c->nz;
    cudaError_t e = cudaMalloc(&c->host_buf, 27 * N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->diag_scratch, diag_scratch_bytes((long long)N));
    if (e == cudaSuccess) e = cudaMemset(c->diag_scratch, 0, diag_scratch_bytes((long long)N));
    if (e == cudaSuccess) e = cudaMalloc(&c->diag_out, 16 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->zeros, N * sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(c->zeros, 0, N * sizeof(double));
    return cuda_err3(c, e, "cudaMalloc(export buffers)");
}

// current fields (rho, u, T, |u|) into host_buf[0 .. 6N)
int export_fields(lbm3d_ctx* c) {
    int rc = ensure_buf(c);
    if (rc) return rc;
    const dim3 b = blk3(), g = grd3(c);
    if (c->prec == LBM_FP64) {
        launch_macro<double>(c);
        k3_force<double><<<g, b, 0, c->stream>>>(c->D, make_phys<double>(phys_of(c->params)),
                                                   make_lat3<double>(c->params));
        k3_export<double><<<g, b, 0, c->stream>>>(c->D, make_lat3<double>(c->params), 0, c->host_buf);
    } else {
        launch_macro<float>(c);
        k3_force<float><<<g, b, 0, c->stream>>>(c->D, make_phys<float>(phys_of(c->params)),
                                                  make_lat3<float>(c->params));
        k3_export<float><<<g, b, 0, c->stream>>>(c->D, make_lat3<float>(c->params), 0, c->host_buf);
    }
    return cuda_err3(c, cudaGetLastError(), "field export");
}

}  // namespace

extern "C" {

size_t lbm3d_state_bytes(int nx, int ny, int nz, int prec) {
    if (nx < 1 || ny < 1 || nz < 1 || (prec != LBM_FP64 && prec != LBM_FP32)) return 0;
    return bytes_for(nx, ny, nz, prec);
}

int lbm3d_create(int nx, int ny, int nz, const lbm_params* params, const lbm3d_bc* bc, int prec,
                 void* stream, lbm3d_ctx** out) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || !params || !bc || (prec != LBM_FP64 && prec != LBM_FP32))
        return LBM_EINVAL;
    if (nx > 65535 || ny > 65535 || nz > 65535) return LBM_EINVAL;
    if (bc->flow_z != LBM_PERIODIC && bc->flow_z != LBM_WALL) return LBM_EINVAL;
    for (int e = 0; e < 2; ++e) {
        if (bc->therm[e] < 0 || bc->therm[e] > 2) return LBM_EINVAL;
        if ((bc->flow_z == LBM_PERIODIC) != (bc->therm[e] == LBM_T_PERIODIC)) return LBM_EINVAL;
    }
    if (bc->flow_z == LBM_WALL && nz < 2) return LBM_EINVAL;
    if (!(params->cv > 0) || !(params->nu > 0) || !(params->lambda > 0) ||
        !(params->w_dot > 0 && params->w_dot < 1) || params->G == 0.0 || !(params->b > 0) ||
        !(params->s_e > 0 && params->s_e < 2))
        return LBM_EINVAL;
    lbm3d_ctx* c = new (std::nothrow) lbm3d_ctx();
    if (!c) return LBM_ENOMEM;
    c->nx = nx;
    c->ny = ny;
    c->nz = nz;
    c->prec = prec;
    c->params = *params;
    c->bc = *bc;
    cudaError_t e = cudaSuccess;
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        c->own_stream = e == cudaSuccess;
    }
    const size_t total = bytes_for(nx, ny, nz, prec);
    if (e == cudaSuccess) e = cudaMalloc(&c->mem, total);
    if (e == cudaSuccess) e = cudaMalloc(&c->ctl, sizeof(Ctl));
    if (e == cudaSuccess) e = cudaMemset(c->ctl, 0, sizeof(Ctl));
    if (e != cudaSuccess) {
        const int rc = e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
        lbm3d_destroy(c);
        return rc;
    }
    const size_t es = prec == LBM_FP64 ? 8 : 4;
    const size_t plane = pitch_for(nx) * ny * nz;
    char* m = (char*)c->mem;
    Dom3& D = c->D;
    memset(&D, 0, sizeof(D));
    size_t off = 0;
    for (int p = 0; p < 2; ++p) { D.f[p] = m + off; off += 19 * plane * es; }
    for (int p = 0; p < 2; ++p) { D.g[p] = m + off; off += 7 * plane * es; }
    for (int p = 0; p < 2; ++p) { D.P[p] = m + off; off += plane * es; }
    D.aux = m + off; off += A_N * plane * es;
    D.aux2 = m + off; off += B_N * plane * es;
    D.ghost = m + off;
    D.ctl = c->ctl;
    D.nx = nx;
    D.ny = ny;
    D.nz = nz;
    D.pitch = (int)pitch_for(nx);
    D.plane = plane;
    D.walls = bc->flow_z == LBM_WALL;
    D.therm[0] = bc->therm[0];
    D.therm[1] = bc->therm[1];
    D.T_edge[0] = bc->T_edge[0];
    D.T_edge[1] = bc->T_edge[1];
    D.cot = tan(M_PI / 2.0 - bc->theta_deg * M_PI / 180.0);
    D.rho_ref = 1.0;
    D.T_ref = 0.0;
    D.inv_n = 1.0 / ((double)nx * ny * nz);
    c->zseg = auto_zseg(nx, ny, nz, prec);
    // the fused step is the faster in FP32; in FP64 (bound by the FP64 pipe)
    // its recomputed halos cost more than the traffic it saves
    c->fused = prec == LBM_FP32;
    if (prec == LBM_FP64)
        e = cudaFuncSetAttribute(k3_fused<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Tile3<double>::BYTES);
    else
        e = cudaFuncSetAttribute(k3_fused<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Tile3<float>::BYTES);
    // the pitch padding is never read, but keep it defined
    if (e == cudaSuccess) e = cudaMemset(c->mem, 0, total);
    if (e != cudaSuccess) {
        lbm3d_destroy(c);
        return LBM_ECUDA;
    }
    *out = c;
    return LBM_OK;
}

int lbm3d_init_fields(lbm3d_ctx* c, const double* rho, const double* ux, const double* uy,
                      const double* uz, const double* T) {
    if (!c || !rho || !ux || !uy || !uz || !T) return LBM_EINVAL;
    const size_t N = (size_t)c->nx * c->ny * c->nz;
    int rc = ensure_buf(c);
    if (rc) return rc;
    const double* src[5] = {rho, ux, uy, uz, T};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 5 && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(c->host_buf + k * N, src[k], N * sizeof(double), cudaMemcpyHostToDevice,
                            c->stream);
    // storage references from device sums (fixed summation order)
    double sums[2];
    if (e == cudaSuccess && sum2_launch(c->host_buf, c->host_buf + 4 * N, (long long)N,
                                        c->diag_out + 8, c->diag_scratch, c->stream))
        e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sums, c->diag_out + 8, sizeof(sums), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_err3(c, e, "field sums");
    c->D.rho_ref = c->params.rho_ref > 0 ? c->params.rho_ref : sums[0] / (double)N;
    c->D.T_ref = c->params.T_ref > 0 ? c->params.T_ref : sums[1] / (double)N;
    Ctl h;
    memset(&h, 0, sizeof(h));
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->ctl, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_err3(c, e, "copying the initial fields");
    const dim3 b = blk3(), g = grd3(c);
    const int um = c->params.gravity != 0.0;
    if (c->prec == LBM_FP64) {
        k3_init<double><<<g, b, 0, c->stream>>>(c->D, make_lat3<double>(c->params), c->host_buf,
                                                c->host_buf + N, c->host_buf + 2 * N,
                                                c->host_buf + 3 * N, c->host_buf + 4 * N);
        k3_macro<double><<<g, b, 0, c->stream>>>(c->D, make_phys<double>(phys_of(c->params)),
                                                 c->params.cv, um, 0);
    } else {
        k3_init<float><<<g, b, 0, c->stream>>>(c->D, make_lat3<float>(c->params), c->host_buf,
                                               c->host_buf + N, c->host_buf + 2 * N,
                                               c->host_buf + 3 * N, c->host_buf + 4 * N);
        k3_macro<float><<<g, b, 0, c->stream>>>(c->D, make_phys<float>(phys_of(c->params)),
                                                (float)c->params.cv, um, 0);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err3(c, e, "init kernels");
    // the initial density sum (accumulated into massq[0]) is read by step 0
    // from slot 2 ((0 - 1) mod 3) and by step 1 from slot 0
    e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess && um) {
        long long q0 = 0;
        e = cudaMemcpy(&q0, &c->ctl->massq[0], sizeof(q0), cudaMemcpyDeviceToHost);
        const double m0 = massq_value(q0, massq_scale(c->D.inv_n));
        if (e == cudaSuccess) e = cudaMemcpy(&c->ctl->mass[0], &m0, sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(&c->ctl->mass[2], &m0, sizeof(double), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) return cuda_err3(c, e, "lbm3d_init_fields");
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;   // the launch arguments carry rho_ref / T_ref
    c->step = 0;
    c->aux_stale = false;
    c->sticky = LBM_OK;
    c->initialized = true;
    c->err.clear();
    return check3(c);
}

int lbm3d_step(lbm3d_ctx* c, int n) {
    if (!c || n < 0) return LBM_EINVAL;
    if (!c->initialized) return set_err3(c, LBM_ESTATE, "lbm3d_step before lbm3d_init_fields");
    if (c->sticky) return c->sticky;
    if (n == 0) return LBM_OK;
    if (!c->fused && c->aux_stale) {   // the three-kernel step starts from these planes
        if (c->prec == LBM_FP64) launch_macro<double>(c);
        else launch_macro<float>(c);
    }
    c->aux_stale = c->fused;
    const int kLen = 32;
    int left = n;
    if (left >= kLen) {
        if (!c->graph) {
            cudaGraph_t g;
            cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cuda_err3(c, e, "cudaStreamBeginCapture");
            for (int i = 0; i < kLen; ++i) step_once(c);
            e = cudaStreamEndCapture(c->stream, &g);
            if (e != cudaSuccess) return cuda_err3(c, e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&c->graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                c->graph = nullptr;
                return cuda_err3(c, e, "cudaGraphInstantiate");
            }
        }
        for (; left >= kLen; left -= kLen) {
            cudaError_t e = cudaGraphLaunch(c->graph, c->stream);
            if (e != cudaSuccess) return cuda_err3(c, e, "cudaGraphLaunch");
        }
    }
    for (; left > 0; --left)
        if (step_once(c)) return cuda_err3(c, cudaGetLastError(), "step launch");
    c->step += n;
    return LBM_OK;
}

int lbm3d_get_fields(lbm3d_ctx* c, double* rho, double* ux, double* uy, double* uz, double* T) {
    if (!c) return LBM_EINVAL;
    if (!c->initialized) return set_err3(c, LBM_ESTATE, "no state yet");
    int rc = export_fields(c);
    if (rc) return rc;
    const size_t N = (size_t)c->nx * c->ny * c->nz;
    double* dst[5] = {rho, ux, uy, uz, T};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 5 && e == cudaSuccess; ++k)
        if (dst[k])
            e = cudaMemcpyAsync(dst[k], c->host_buf + k * N, N * sizeof(double), cudaMemcpyDeviceToHost,
                                c->stream);
    if (e != cudaSuccess) return cuda_err3(c, e, "copying fields to the host");
    return check3(c);
}

int lbm3d_get_populations(lbm3d_ctx* c, double* f, double* g, double* P) {
    if (!c) return LBM_EINVAL;
    if (!c->initialized) return set_err3(c, LBM_ESTATE, "no state yet");
    int rc = ensure_buf(c);
    if (rc) return rc;
    const size_t N = (size_t)c->nx * c->ny * c->nz;
    const dim3 b = blk3(), gr = grd3(c);
    if (c->prec == LBM_FP64)
        k3_export<double><<<gr, b, 0, c->stream>>>(c->D, make_lat3<double>(c->params), 1, c->host_buf);
    else
        k3_export<float><<<gr, b, 0, c->stream>>>(c->D, make_lat3<float>(c->params), 1, c->host_buf);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && f)
        e = cudaMemcpyAsync(f, c->host_buf, 19 * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && g)
        e = cudaMemcpyAsync(g, c->host_buf + 19 * N, 7 * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && P)
        e = cudaMemcpyAsync(P, c->host_buf + 26 * N, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_err3(c, e, "copying populations to the host");
    return check3(c);
}

int lbm3d_diagnostics(lbm3d_ctx* c, double rho_l, double rho_g, int sessile, lbm_diag* out) {
    if (!c || !out || !(rho_l > rho_g)) return LBM_EINVAL;
    if (!c->initialized) return set_err3(c, LBM_ESTATE, "no state yet");
    int rc = export_fields(c);
    if (rc) return rc;
    const size_t N = (size_t)c->nx * c->ny * c->nz;
    // the reduction takes |u| in place of u_x and zeros for u_y
    if (diag_launch(c->host_buf, c->host_buf + 5 * N, c->zeros, c->host_buf + 4 * N, (long long)N,
                    c->params.cv, rho_l, rho_g, c->diag_out, c->diag_scratch, c->stream))
        return cuda_err3(c, cudaGetLastError(), "diagnostics kernel");
    double h[8];
    cudaError_t e = cudaMemcpyAsync(h, c->diag_out, 7 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_err3(c, e, "diagnostics");
    out->mass = h[0];
    out->energy = h[1];
    out->liquid_mass = h[2];
    out->liquid_area = h[3];
    out->liquid_area_smooth = h[4];
    out->max_u = h[5];
    out->nonfinite = (int)h[6];
    const double fac = sessile ? 12.0 / M_PI : 6.0 / M_PI;
    out->diameter = cbrt(fac * out->liquid_area);
    out->diameter_smooth = cbrt(fac * out->liquid_area_smooth);
    out->step = c->step;
    return check3(c);
}

long long lbm3d_step_count(const lbm3d_ctx* c) { return c ? c->step : -1; }

int lbm3d_set_path(lbm3d_ctx* c, int fused, int zseg) {
    if (!c || zseg < 0) return LBM_EINVAL;
    const bool f = fused != 0;
    const int zs = zseg == 0 ? auto_zseg(c->nx, c->ny, c->nz, c->prec) : (zseg > c->nz ? c->nz : zseg);
    if (f != c->fused || zs != c->zseg) {
        if (c->graph) cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    c->fused = f;
    c->zseg = zs;
    return LBM_OK;
}

int lbm3d_get_path(const lbm3d_ctx* c, int* fused, int* zseg) {
    if (!c) return LBM_EINVAL;
    if (fused) *fused = c->fused ? 1 : 0;
    if (zseg) *zseg = c->zseg;
    return LBM_OK;
}

int lbm3d_sync(lbm3d_ctx* c) {
    if (!c) return LBM_EINVAL;
    if (!c->initialized) return LBM_OK;
    return check3(c);
}

void lbm3d_destroy(lbm3d_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->host_buf) cudaFree(c->host_buf);
    if (c->diag_scratch) cudaFree(c->diag_scratch);
    if (c->diag_out) cudaFree(c->diag_out);
    if (c->zeros) cudaFree(c->zeros);
    if (c->mem) cudaFree(c->mem);
    if (c->ctl) cudaFree(c->ctl);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char* lbm3d_last_error(const lbm3d_ctx* c) { return c ? c->err.c_str() : "null context"; }

}  // extern "C"
