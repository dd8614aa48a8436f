// Auxiliary kernels around the fused step: initial equilibrium populations,
// macroscopic fields of the current state (rho, u with the half-force
// correction of Eq. 11, T), population import / export as absolute doubles,
// and the FP64 diagnostics reduction.  None of these is on the per-step path.
#include "lbm_internal.cuh"

namespace lbm {

__constant__ int dCX9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int dCY9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
__constant__ double dW9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                              1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

__device__ __forceinline__ double w5(int i, double w_dot) { return i == 0 ? 1.0 - w_dot : 0.25 * w_dot; }

// ---------------------------------------------------------------------------
// f = f^eq(rho, u) (Eq. 3), g = w^ T (Eq. 22), P = 0, stored as deviations
template <int PREC>
__global__ void k_init(Inst I, const double* rho, const double* ux, const double* uy,
                       const double* T, double w_dot) {
    typedef typename Types<PREC>::TF TF;
    typedef typename Types<PREC>::TG TG;
    typedef typename Types<PREC>::R R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= I.nx) return;
    const size_t n = (size_t)y * I.nx + x;
    const size_t plane = (size_t)I.ny * I.pitch;
    const size_t off = (size_t)y * I.pitch + x;
    const double r = rho[n], vx = ux[n], vy = uy[n], t = T[n];
    TF* f = (TF*)I.f[0];
    TG* g = (TG*)I.g[0];
    R* P = (R*)I.P[0];
    if (PREC == 0) {
        const double uu = vx * vx + vy * vy;
        for (int i = 0; i < 9; ++i) {
            const double cu = dCX9[i] * vx + dCY9[i] * vy;
            const double fe = dW9[i] * r * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
            st_st(f + i * plane + off, (TF)(fe - dW9[i] * I.rho_ref));
        }
        for (int i = 0; i < 5; ++i) st_st(g + i * plane + off, (R)(w5(i, w_dot) * (t - I.T_ref)));
    } else {
        // FP32 state: the deviation f^eq - w rho_ref = w [(rho - rho_ref) +
        // rho (3 c.u + 9/2 (c.u)^2 - 3/2 u^2)] in float (the reference
        // difference in double), which stays within the state's own rounding
        const float dr = (float)(r - I.rho_ref), rf = (float)r;
        const float fx = (float)vx, fy = (float)vy, uu = fx * fx + fy * fy;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const float cu = (float)dCX9[i] * fx + (float)dCY9[i] * fy;
            const float w = (float)dW9[i];
            st_st(f + i * plane + off, (TF)(w * (dr + rf * (3.0f * cu + 4.5f * cu * cu - 1.5f * uu))));
        }
        const float td = (float)(t - I.T_ref);
#pragma unroll
        for (int i = 0; i < 5; ++i) st_st(g + i * plane + off, (float)w5(i, w_dot) * td);
    }
    P[off] = R(0);
}

int init_launch(int prec, const Inst* I_dev, const Inst& I, const double* rho, const double* ux,
                const double* uy, const double* T, double w_dot, cudaStream_t st) {
    (void)I_dev;
    dim3 blk(128), grd((I.nx + 127) / 128, I.ny);
    if (prec == 0) k_init<0><<<grd, blk, 0, st>>>(I, rho, ux, uy, T, w_dot);
    else if (prec == 1) k_init<1><<<grd, blk, 0, st>>>(I, rho, ux, uy, T, w_dot);
    else k_init<2><<<grd, blk, 0, st>>>(I, rho, ux, uy, T, w_dot);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------------------
// fields of the current state, computed in double from the stored values
__device__ double psi_of(const PhysD& p, double rho, double T) {
    const double k = 0.37464 + 1.54226 * p.omega - 0.26992 * p.omega * p.omega;
    const double Tc = 0.0778 * p.a / (0.45724 * p.b * p.Rg);
    const double h = 1.0 + k * (1.0 - sqrt(T / Tc));
    const double pe = rho * p.Rg * T / (1.0 - p.b * rho) -
                      p.a * h * h * rho * rho / (1.0 + 2.0 * p.b * rho - p.b * p.b * rho * rho);
    return sqrt(2.0 * (pe - rho / 3.0) / p.G);
}

// pass 1: per node rho, T, j and psi of the current state (in double)
template <int PREC>
__global__ void k_fields_node(Inst I, PhysD p, const Ctl* ctl, double* orho, double* ojx,
                              double* ojy, double* oT, double* opsi) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= I.nx) return;
    const long long step = __ldcg(&ctl->step);
    const int par = (int)(step & 1);
    typedef typename Types<PREC>::TF TF;
    typedef typename Types<PREC>::TG TG;
    const TF* f = (const TF*)I.f[par];
    const TG* g = (const TG*)I.g[par];
    const size_t plane = (size_t)I.ny * I.pitch, off = (size_t)y * I.pitch + x;
    double r = 0.0, t = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i) {
        const double fi = (double)ld_st(f + i * plane + off) + dW9[i] * I.rho_ref;
        r += fi;
        jx += dCX9[i] * fi;
        jy += dCY9[i] * fi;
    }
    for (int i = 0; i < 5; ++i) t += (double)ld_st(g + i * plane + off) + w5(i, p.w_dot) * I.T_ref;
    const size_t n = (size_t)y * I.nx + x;
    orho[n] = r;
    oT[n] = t;
    ojx[n] = jx;
    ojy[n] = jy;
    opsi[n] = psi_of(p, r, t);
}

// FP32 state: the same fields from float sums of the stored deviations and
// the float EOS (the state's own precision; the GPU's FP64 rate would
// otherwise bound this pass)
template <int PREC>
__global__ void k_fields_node_f(Inst I, Phys<float> pf, const Ctl* ctl, double* orho,
                                double* ojx, double* ojy, double* oT, double* opsi) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= I.nx) return;
    const long long step = __ldcg(&ctl->step);
    const int par = (int)(step & 1);
    typedef typename Types<PREC>::TF TF;
    typedef typename Types<PREC>::TG TG;
    const TF* f = (const TF*)I.f[par];
    const TG* g = (const TG*)I.g[par];
    const size_t plane = (size_t)I.ny * I.pitch, off = (size_t)y * I.pitch + x;
    float rd = 0.f, jx = 0.f, jy = 0.f, td = 0.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float fi = (float)ld_st(f + i * plane + off);
        rd += fi;
        jx += (float)dCX9[i] * fi;
        jy += (float)dCY9[i] * fi;
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) td += (float)ld_st(g + i * plane + off);
    // sum_i w_i = sum_i w^_i = 1 and sum_i w_i c_i = 0: the references add
    // once to rho and T and not to j
    const float r = rd + (float)I.rho_ref, t = td + (float)I.T_ref;
    const size_t n = (size_t)y * I.nx + x;
    orho[n] = r;
    oT[n] = t;
    ojx[n] = jx;
    ojy[n] = jy;
    opsi[n] = f_sqrt(psi2_of(pf, r, t));
}

// pass 2: F_m from the psi field (Eq. 9, wetting ghost layer of Section 3.3),
// buoyancy, and u = (j + F/2) / rho (Eq. 11), in place over j
template <class C>
__global__ void k_fields_force(Inst I, PhysD p, Phys<float> pf, const Ctl* ctl, const double* rho,
                               double* ux, double* uy, const double* T, const double* psi) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= I.nx) return;
    const int nx = I.nx, ny = I.ny;
    const bool perx = I.flow[EW] == PERIODIC;
    auto extx = [&](int xx) { return perx ? wrapi(xx, nx) : min(max(xx, 0), nx - 1); };
    auto at = [&](const double* a, int xx, int yy) { return (C)a[(size_t)yy * nx + xx]; };
    const C cot = (C)I.cot_theta;
    auto psi_ext = [&](int xx, int yy) -> C {
        const int xe = extx(xx);
        if (yy >= 0 && yy < ny) return at(psi, xe, yy);
        const int edge = yy < 0 ? ES : EN;
        const int kind = I.flow[edge];
        if (kind == PERIODIC) return at(psi, xe, wrapi(yy, ny));
        if (kind == OPEN) return at(psi, xe, yy < 0 ? 0 : ny - 1);
        const int y1 = edge == ES ? 0 : ny - 1, y2 = edge == ES ? 1 : ny - 2;
        const C rg = at(rho, xe, y2) + cot * rabs(at(rho, extx(xe + 1), y1) - at(rho, extx(xe - 1), y1));
        const C tg = at(T, xe, y1);     // the fluid node's temperature
        if (sizeof(C) == 8) return (C)psi_of(p, (double)rg, (double)tg);
        return (C)f_sqrt(psi2_of(pf, (float)rg, (float)tg));
    };
    C sx = 0, sy = 0;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const C wv = i < 5 ? C(1.0 / 3.0) : C(1.0 / 12.0);
        const C pn = psi_ext(x + dCX9[i], y + dCY9[i]);
        sx += wv * pn * (C)dCX9[i];
        sy += wv * pn * (C)dCY9[i];
    }
    const size_t n = (size_t)y * nx + x;
    const C r = (C)rho[n], pc = (C)psi[n];
    const C G = (C)p.G;
    const C Fx = -G * pc * sx;
    const long long step = __ldcg(&ctl->step);
    const C rho_ave = (C)(__ldcg(&ctl->mass[(step + 2) % 3]) * I.inv_n);
    const C Fy = -G * pc * sy - (r - rho_ave) * (C)p.gravity;
    ux[n] = p.frozen_flow ? 0.0 : (double)(((C)ux[n] + C(0.5) * Fx) / r);
    uy[n] = p.frozen_flow ? 0.0 : (double)(((C)uy[n] + C(0.5) * Fy) / r);
}

int fields_launch(int prec, const Inst* I_dev, const Inst& I, const PhysD& phys, double* rho,
                  double* ux, double* uy, double* T, double* psi, cudaStream_t st) {
    (void)I_dev;
    dim3 blk(128), grd((I.nx + 127) / 128, I.ny);
    const Phys<float> pf = make_phys<float>(phys);
    if (prec == 0) {
        k_fields_node<0><<<grd, blk, 0, st>>>(I, phys, I.ctl, rho, ux, uy, T, psi);
        k_fields_force<double><<<grd, blk, 0, st>>>(I, phys, pf, I.ctl, rho, ux, uy, T, psi);
    } else {
        if (prec == 1) k_fields_node_f<1><<<grd, blk, 0, st>>>(I, pf, I.ctl, rho, ux, uy, T, psi);
        else k_fields_node_f<2><<<grd, blk, 0, st>>>(I, pf, I.ctl, rho, ux, uy, T, psi);
        k_fields_force<float><<<grd, blk, 0, st>>>(I, phys, pf, I.ctl, rho, ux, uy, T, psi);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------------------
// populations as absolute doubles, [q][ny][nx]
template <int PREC>
__global__ void k_pop(Inst I, int par, double w_dot, double* f, double* g, double* P, int set) {
    typedef typename Types<PREC>::TF TF;
    typedef typename Types<PREC>::TG TG;
    typedef typename Types<PREC>::R R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= I.nx) return;
    const size_t plane = (size_t)I.ny * I.pitch, off = (size_t)y * I.pitch + x;
    const size_t dplane = (size_t)I.ny * I.nx, doff = (size_t)y * I.nx + x;
    TF* fs = (TF*)I.f[par];
    TG* gs = (TG*)I.g[par];
    R* Ps = (R*)I.P[par];
    if (set) {
        for (int i = 0; i < 9; ++i)
            st_st(fs + i * plane + off, (TF)(f[i * dplane + doff] - dW9[i] * I.rho_ref));
        for (int i = 0; i < 5; ++i)
            st_st(gs + i * plane + off, (R)(g[i * dplane + doff] - w5(i, w_dot) * I.T_ref));
        Ps[off] = (R)P[doff];
    } else {
        if (f)
            for (int i = 0; i < 9; ++i)
                f[i * dplane + doff] = (double)fs[i * plane + off] + dW9[i] * I.rho_ref;
        if (g)
            for (int i = 0; i < 5; ++i)
                g[i * dplane + doff] = (double)ld_st(gs + i * plane + off) + w5(i, w_dot) * I.T_ref;
        if (P) P[doff] = (double)Ps[off];
    }
}

static int pop_launch(int prec, const Inst& I, int par, double w_dot, double* f, double* g,
                      double* P, int set, cudaStream_t st) {
    dim3 blk(128), grd((I.nx + 127) / 128, I.ny);
    if (prec == 0) k_pop<0><<<grd, blk, 0, st>>>(I, par, w_dot, f, g, P, set);
    else if (prec == 1) k_pop<1><<<grd, blk, 0, st>>>(I, par, w_dot, f, g, P, set);
    else k_pop<2><<<grd, blk, 0, st>>>(I, par, w_dot, f, g, P, set);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int pop_get_launch(int prec, const Inst& I, int par, double w_dot, double* f, double* g,
                   double* P, cudaStream_t st) {
    return pop_launch(prec, I, par, w_dot, f, g, P, 0, st);
}

int pop_set_launch(int prec, const Inst& I, int par, double w_dot, const double* f,
                   const double* g, const double* P, cudaStream_t st) {
    return pop_launch(prec, I, par, w_dot, (double*)f, (double*)g, (double*)P, 1, st);
}

// ---------------------------------------------------------------------------
// diagnostics: per-block partial sums in double, then the last block to finish
// folds the partials in block order (deterministic result)
enum { DIAG_BLOCKS = 304, DIAG_THREADS = 256, DIAG_VALS = 7 };

size_t diag_scratch_bytes(long long n) {
    (void)n;
    return (size_t)DIAG_BLOCKS * DIAG_VALS * sizeof(double) + 256;
}

__global__ void __launch_bounds__(DIAG_THREADS)
    k_diag(const double* rho, const double* ux, const double* uy, const double* T, long long n,
           double cv, double rho_l, double rho_g, double* out, double* partial,
           unsigned* ticket) {
    __shared__ double red[DIAG_VALS][DIAG_THREADS / 32];
    __shared__ bool last;
    const double rmid = 0.5 * (rho_l + rho_g);
    double v[DIAG_VALS] = {0, 0, 0, 0, 0, 0, 0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double r = rho[i], a = ux[i], b = uy[i], t = T[i];
        const bool fin = isfinite(r) && isfinite(a) && isfinite(b) && isfinite(t);
        v[0] += r;
        v[1] += r * cv * t;
        if (r > rmid) {
            v[2] += r;
            v[3] += 1.0;
        }
        double ph = (r - rho_g) / (rho_l - rho_g);
        ph = ph < 0.0 ? 0.0 : (ph > 1.0 ? 1.0 : ph);
        v[4] += ph;
        const double um = sqrt(a * a + b * b);
        v[5] = fmax(v[5], um);
        v[6] += fin ? 0.0 : 1.0;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < DIAG_VALS; ++k) {
        double x = v[k];
        for (int o = 16; o > 0; o >>= 1) {
            const double y = __shfl_down_sync(0xffffffffu, x, o);
            x = k == 5 ? fmax(x, y) : x + y;
        }
        if (lane == 0) red[k][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < DIAG_VALS) {
        const int k = threadIdx.x;
        double x = red[k][0];
        for (int w = 1; w < DIAG_THREADS / 32; ++w) x = k == 5 ? fmax(x, red[k][w]) : x + red[k][w];
        partial[blockIdx.x * DIAG_VALS + k] = x;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last && threadIdx.x < DIAG_VALS) {
        __threadfence();
        const int k = threadIdx.x;
        double x = __ldcg(&partial[k]);
        for (unsigned b = 1; b < gridDim.x; ++b) {
            const double y = __ldcg(&partial[b * DIAG_VALS + k]);
            x = k == 5 ? fmax(x, y) : x + y;
        }
        out[k] = x;
        if (k == 0) *ticket = 0u;
    }
}

// sum rho and sum T of device fields (the storage references and the first
// step's mean density), with the same fixed-order two-level reduction
__global__ void __launch_bounds__(DIAG_THREADS)
    k_sum2(const double* a, const double* b, long long n, double* out, double* partial,
           unsigned* ticket) {
    __shared__ double red[2][DIAG_THREADS / 32];
    __shared__ bool last;
    double v0 = 0.0, v1 = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        v0 += a[i];
        v1 += b[i];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_down_sync(0xffffffffu, v0, o);
        v1 += __shfl_down_sync(0xffffffffu, v1, o);
    }
    if (lane == 0) {
        red[0][wid] = v0;
        red[1][wid] = v1;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        const int k = threadIdx.x;
        double x = red[k][0];
        for (int w = 1; w < DIAG_THREADS / 32; ++w) x += red[k][w];
        partial[blockIdx.x * 2 + k] = x;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last && threadIdx.x < 2) {
        __threadfence();
        const int k = threadIdx.x;
        double x = __ldcg(&partial[k]);
        for (unsigned bk = 1; bk < gridDim.x; ++bk) x += __ldcg(&partial[bk * 2 + k]);
        out[k] = x;
        if (k == 0) *ticket = 0u;
    }
}

int sum2_launch(const double* a, const double* b, long long n, double* out2, void* scratch,
                cudaStream_t st) {
    double* partial = (double*)scratch;
    unsigned* ticket = (unsigned*)((char*)scratch + (size_t)DIAG_BLOCKS * DIAG_VALS * sizeof(double));
    k_sum2<<<DIAG_BLOCKS, DIAG_THREADS, 0, st>>>(a, b, n, out2, partial, ticket);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int diag_launch(const double* rho, const double* ux, const double* uy, const double* T,
                long long n, double cv, double rho_l, double rho_g, double* out9, void* scratch,
                cudaStream_t st) {
    double* partial = (double*)scratch;
    unsigned* ticket = (unsigned*)((char*)scratch + (size_t)DIAG_BLOCKS * DIAG_VALS * sizeof(double));
    k_diag<<<DIAG_BLOCKS, DIAG_THREADS, 0, st>>>(rho, ux, uy, T, n, cv, rho_l, rho_g, out9,
                                                 partial, ticket);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace lbm
