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
//   phase alpha of iteration k:  A(k)    load f, g, P of row k; rho, T, j,
//                                        psi and T (dp/dT)_rho (Eq. 10)
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
// Two load paths feed stage A.  In the register-prefetch form each thread
// loads its column of row k + 1 into registers during phase beta of
// iteration k.  In the staged form (FP32 f) the rows arrive in shared memory
// by bulk asynchronous copies (cp.async.bulk, one mbarrier per row in
// flight), issued two or three iterations ahead of their use (Ahead<NT>), and
// g and P^{n-1} stay in their staging slots until stages C and D5 have used
// them.  A bandwidth-bound sweep moves (bytes in flight per SM) / (loaded HBM
// latency); one row per thread in registers caps that at about 30 KB per SM,
// two staged rows per CTA of the 224-thread tile (two CTAs per SM) double it.
//
// The CTAs are persistent and pull (domain, strip, segment) units from an
// atomic counter, so one launch serves one domain or hundreds of domains of
// uneven size; the last CTA to finish advances every domain's device-side
// step counter, clears the next slot of its density-sum ring and resets the
// counter, which makes the launch replayable inside a CUDA graph.  No CTA
// ever waits on another.
#include <type_traits>

#include "lbm_internal.cuh"

namespace lbm {

template <class R>
struct Vec2;
template <>
struct Vec2<float> { typedef float2 T; };
template <>
struct Vec2<double> { typedef double2 T; };
template <class R>
struct Vec4;
template <>
struct Vec4<float> { typedef float4 T; };
template <>
struct Vec4<double> { typedef double4_32a T; };

template <class R, int NT>
struct StepSmem {
    R psi[3][NT];
    typename Vec2<R>::T u[3][NT];
    R fs[3][9][NT];     // post-collision f (deviation form)
    R gs[3][3][NT];     // post-collision g_1, g_2, g_3 (deviation form)
    // per column and row: g_dev[0..4], rho, then P^{n-1} and T (dp/dT)_rho,
    // which stage C replaces by the row's post-collision g*_0 and g*_4
    typename Vec4<R>::T own[5][2][NT];
    int unit;
};

// rho and T rings, read only by the wetting ghost layer of walls; they follow
// StepSmem in dynamic shared memory when a launch has a wall domain
template <class R, int NT>
struct WallRings {
    R rho[3][NT];
    R T[3][NT];
};

// Shared-memory layout of the bulk-copy staged form (FP32 state, g in FP32 or
// FP16 storage).  The rows of f,
// g and P^{n-1} arrive by cp.async.bulk (the copy engine of each SM, tracked
// by one mbarrier per in-flight row) instead of per-thread loads, two rows
// ahead of their use.  The step moves its bytes at the rate
// (bytes in flight per SM) / (loaded HBM latency); the register-prefetch form
// holds one row in flight, this form two, without spending registers.  f is
// needed only by stage A of its own row (three slots: the row being used, two
// rows in flight); g and P^{n-1} stay in their slots until stages C and D5 of
// the row, four iterations later (seven slots), which replaces the
// per-column ring of the register-prefetch form; only stage C reads them
// (stage D5 gets the row's g from C in registers), so no thread writes a
// slot that a copy fills.  g rows are kept in
// their storage type; FP16 rows are copied from the 8-column boundary at or
// below the window start (16 bytes), so they carry 8 columns of slack.
template <class TG>
struct GPad { static constexpr int value = sizeof(TG) == 2 ? 8 : 0; };
// rows in flight of the staged form: three on the narrower tiles (their
// shared memory leaves room: 128 threads -> 3 CTAs, 192 -> 2 CTAs per SM),
// two on 224 and 256 threads
template <int NT>
struct Ahead { static constexpr int value = NT <= 192 ? 3 : 2; };
template <class R, class TG, int NT>
struct StageSmem {
    static constexpr int D = Ahead<NT>::value;
    R fR[D + 1][9][NT];
    R pR[D + 5][NT];
    TG gR[D + 5][5][NT + GPad<TG>::value];
    R psi[3][NT];
    typename Vec2<R>::T u[3][NT];
    R fs[3][9][NT];
    R gs[3][3][NT];
    typename Vec2<R>::T own[5][NT];   // rho and T (dp/dT)_rho, from stage A to stage C
    unsigned long long mbar[D + 1];
    unsigned long long probe;   // never armed: the wait-timeout test hook waits on it
    int unit;
};

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* m, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* m, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)),
                 "r"(bytes)
                 : "memory");
}
// global -> shared bulk copy completing on mbarrier m; dst, src 16-byte
// aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* m) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(m))
        : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* m, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(m)), "r"(parity)
        : "memory");
    return ok != 0;
}
// a product rounded on its own, never fused into a later add (a value that
// one stage hands to another in a register then rounds as one passed through
// shared memory)
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
// bounded wait for an mbarrier phase: gives up after ~2^31 clocks (about a
// second at the GB300's clock), records ERR_TIMEOUT and sets *stalled; a
// thread that has stalled does not wait again on the same pipeline (its
// results are then invalid and the sticky error says so)
__device__ __forceinline__ void wait_row(unsigned long long* m, unsigned parity, int* err,
                                         bool* stalled) {
    if (*stalled) return;
    if (mbar_test(m, parity)) return;
    const long long t0 = clock64();
    while (!mbar_test(m, parity)) {
        if (clock64() - t0 > (1LL << 31)) {
            *err |= ERR_TIMEOUT;
            *stalled = true;
            return;
        }
    }
}

// ghost-layer psi of a wall (Section 3.3): rho_ghost = rho(layer 2) +
// tan(pi/2 - theta) |rho(x+1, layer 1) - rho(x-1, layer 1)|
template <class R>
__device__ __forceinline__ R ghost_psi(const Phys<R>& P, R rho_far, R rho_p, R rho_m, R cot, R Tg,
                                       int* err) {
    const R rg = rho_far + cot * rabs(rho_p - rho_m);
    const R q2 = psi2_of(P, rg, Tg);
    if (!(q2 >= R(0))) *err |= (q2 != q2) ? ERR_NONFINITE : ERR_PSI;
    return f_sqrt(q2);
}

// State of one CTA's sweep over one unit.  iter<STEADY>(k) runs both phases
// of iteration k.  The general form (STEADY = false) checks every row range
// and boundary rule; the steady form is used for iterations whose stages are
// all active on interior rows, so it carries no row conditions and no
// boundary branches and each phase compiles to one block of independent
// work (the stages only touch different rows and ring slots).
template <int PREC, int NT, bool UNIT, bool STG>
struct Sweep {
    typedef typename Types<PREC>::R R;
    typedef typename Types<PREC>::TF TF;
    typedef typename Types<PREC>::TG TG;
    typedef typename Vec2<R>::T R2;
    typedef typename Vec4<R>::T R4;
    typedef typename std::conditional<STG, StageSmem<R, TG, NT>, StepSmem<R, NT>>::type SM;
    static_assert(!STG || PREC != 0, "the staged form is FP32 / FP16-g only");
    static constexpr int NTG = NT + GPad<TG>::value;   // staged g row length
    static constexpr int DA = Ahead<NT>::value;        // staged rows in flight
    static constexpr int NF = DA + 1, NGS = DA + 5;    // f and g/P ring slots

    const Inst& I;
    const Phys<R>& P;
    SM& S;
    WallRings<R, NT>& WR;   // valid only for domains with walls
    int t, nx, ny, pitch, y0, y1, my0, my1;
    bool perx, pery, tperx, tpery, first, use_mass, wallS, wallN;
    unsigned plane;
    const TF* __restrict__ fsrc;
    const TG* __restrict__ gsrc;
    const R* __restrict__ Psrc;
    TF* __restrict__ fdst;
    TG* __restrict__ gdst;
    R* __restrict__ Pdst;
    R rho_ref, T_ref, rho_ave, cot;
    // columns
    bool colvalid, inB, inC, inD, left_edge, right_edge;
    bool dirW, dirE, dirS, dirN;
    int gx, gxl, xl1, xr1, cLL, cRR, cLR, cRL;
    R twW2, twE2, twS2, twN2;
    // carried from A(k-1) to B(k-1), and the next row's loads
    R fp[9], rhop, rhodp, jxp, jyp, psip, irp;
    // unit rates: of a row's populations stage B needs besides rho and j only
    // the stress moments m_7 and m_8, formed in stage A (fp is then unused)
    R m7p, m8p;
    R fa[9], ga[5], pa;
    R mass_acc;
    int errbits;
    int ra0, ra1, ra2, b0, kw;
    // staged form: window start column, this column's index in a staged row,
    // slot of row k in the g/P ring, slot and mbarrier of row k in the f ring
    // (both restart with each unit), and the phase parity each f mbarrier
    // completes next (bit m for mbarrier m; carried over from unit to unit)
    int X0w, sidx, gq, fq, kw2, scs, X0g, goff, gcs;
    unsigned mph, sbytes, gbytes, rbytes;
    // this thread's part in the row copies, fixed for the unit: the plane it
    // copies (-1: none; 0 f, 1 g, 2 P), the global address of that plane's
    // row 0 at the first copied column, the shared-memory byte offset of the
    // copy in slot 0, the bytes between slots, between rows and per copy
    int cp_kind;
    const char* cp_src;
    unsigned cp_dst, cp_slot, cp_row, cp_bytes;
    bool stalled;   // a staged-row wait ran out in this unit
    // staged form: what stage D5 of a row uses from its own column stays in
    // registers from stage C of that row (one iteration earlier) instead of
    // shared memory: the row's g, rho, g*_0, g*_2 and g*_4 (c: written by
    // C(k-3); d: read by D5(k-4)), and g*_2 of the row below (e)
    R cg[5], crho, cgs0, cgs2, cgs4;
    R dg[5], drho, dgs0, dgs2, dgs4, egs2;

    __device__ __forceinline__ Sweep(const Inst& I_, const Unit& U, const Phys<R>& P_, SM& S_,
                                     WallRings<R, NT>& WR_, unsigned mph0)
        : I(I_), P(P_), S(S_), WR(WR_) {
        t = threadIdx.x;
        nx = I.nx;
        ny = I.ny;
        pitch = I.pitch;
        y0 = U.y0;
        y1 = U.y1;
        // rows of this unit that enter the density sum (a slab's own rows)
        my0 = max(y0, I.own_y0);
        my1 = min(y1, I.own_y1);
        const int x0 = U.x0, x1 = U.x1;
        perx = I.flow[EW] == PERIODIC;
        pery = I.flow[ES] == PERIODIC;
        // the thermal lattice may have Dirichlet / adiabatic edges on an axis
        // along which the flow is periodic (Section 4.1)
        tperx = I.therm[EW] == T_PERIODIC;
        tpery = I.therm[ES] == T_PERIODIC;
        const long long step = __ldcg(&I.ctl->step);
        const int par = (int)(step & 1);
        first = step == 0;
        // plane stride in elements; lbm_create keeps 9 planes within 2^31 elements
        plane = (unsigned)ny * (unsigned)pitch;
        fsrc = (const TF*)I.f[par];
        gsrc = (const TG*)I.g[par];
        Psrc = (const R*)I.P[par];
        fdst = (TF*)I.f[par ^ 1];
        gdst = (TG*)I.g[par ^ 1];
        Pdst = (R*)I.P[par ^ 1];
        rho_ref = (R)I.rho_ref;
        T_ref = (R)I.T_ref;
        use_mass = P.gravity != R(0);
        rho_ave = use_mass ? (R)(__ldcg(&I.ctl->mass[(step + 2) % 3]) * I.inv_n) : R(0);
        cot = (R)I.cot_theta;
        wallS = I.flow[ES] == WALL;
        wallN = I.flow[EN] == WALL;

        // ---- column bookkeeping (fixed for the unit)
        const int X = x0 - 4 + t;
        colvalid = perx || (X >= 0 && X < nx);
        gx = perx ? wrapi(X, nx) : X;
        gxl = perx ? gx : min(max(X, 0), nx - 1);   // always a valid column to load
        // window index of a column one or two away, clamped at open x edges
        // and to the window (threads at the window ends compute unused values)
        const int xm1 = perx ? X - 1 : min(max(X - 1, 0), nx - 1);
        const int xp1 = perx ? X + 1 : min(max(X + 1, 0), nx - 1);
        auto win = [&](int c) { return min(max(c - x0 + 4, 0), NT - 1); };
        xl1 = win(xm1);
        xr1 = win(xp1);
        cLL = win(perx ? xm1 - 1 : min(max(xm1 - 1, 0), nx - 1));
        cRR = win(perx ? xp1 + 1 : min(max(xp1 + 1, 0), nx - 1));
        cLR = win(perx ? xm1 + 1 : min(max(xm1 + 1, 0), nx - 1));
        cRL = win(perx ? xp1 - 1 : min(max(xp1 - 1, 0), nx - 1));
        inB = colvalid && X >= x0 - 2 && X < x1 + 2;
        inC = colvalid && X >= x0 - 1 && X < x1 + 1;
        inD = X >= x0 && X < x1;
        left_edge = !tperx && X == 0;
        right_edge = !tperx && X == nx - 1;

        // thermal boundary values, as deviations from T_ref (halfway
        // anti-bounce-back A = -g*_opp + 2 w^ (T_w - T_ref) in deviation form)
        dirW = I.therm[EW] == T_DIRICHLET;
        dirE = I.therm[EE] == T_DIRICHLET;
        dirS = I.therm[ES] == T_DIRICHLET;
        dirN = I.therm[EN] == T_DIRICHLET;
        R twW = R(0), twE = R(0), twS = R(0), twN = R(0);
        if (!tperx) {
            twW = (R)(I.T_edge[EW] - I.T_ref);
            twE = (R)(I.T_edge[EE] - I.T_ref);
        }
        if (!tpery && inD) {
            twS = (R)(wall_T(I, ES, gx) - I.T_ref);
            twN = (R)(I.T_edge[EN] - I.T_ref);
        }
        twS2 = R(2) * P.w5_1 * twS;
        twN2 = R(2) * P.w5_1 * twN;
        twW2 = R(2) * P.w5_1 * twW;
        twE2 = R(2) * P.w5_1 * twE;

#pragma unroll
        for (int q = 0; q < 9; ++q) fp[q] = R(0);
        m7p = m8p = R(0);
        rhop = R(1);
        rhodp = jxp = jyp = psip = R(0);
        irp = R(1);
        mass_acc = R(0);
        errbits = 0;
#pragma unroll
        for (int q = 0; q < 5; ++q) cg[q] = dg[q] = R(0);
        crho = drho = R(1);
        cgs0 = cgs2 = cgs4 = dgs0 = dgs2 = dgs4 = egs2 = R(0);
        // rotating ring slots: a0 = slot of row k, a1 = row k-1, a2 = row k-2
        // (ring of 3, so row k-3 is a0 again); b0 = slot of row k in the ring of 5
        ra0 = 0;
        ra1 = 2;
        ra2 = 1;
        b0 = 0;
        // wrapped row of k for loads
        kw = pery ? wrapi(y0 - 3, ny) : y0 - 3;
        // the populations of the first row A works on
        X0w = x0 - 4;
        sidx = perx ? t : gxl - X0w;
        gq = 0;
        // the f ring restarts with each unit (every row of the previous unit
        // was waited for); the mbarriers' next phase parities carry over
        fq = 0;
        mph = mph0;
        stalled = false;
        if constexpr (STG) {
            // copy extent of one plane row: open x copies the columns inside
            // the domain, periodic x the whole window
            scs = perx ? X0w : max(X0w, 0);
            const int sce = perx ? X0w + NT : ((min(X0w + NT, nx) + 3) & ~3);
            sbytes = (unsigned)((sce - scs) * (int)sizeof(R));
            // g rows: FP32 as f; FP16 from the 8-column boundary X0g <= X0w
            constexpr int GA = 16 / (int)sizeof(TG);   // columns per 16 bytes
            X0g = X0w & ~(GA - 1);
            goff = X0w - X0g;
            gcs = perx ? X0g : max(X0g, 0);
            const int gce = perx ? X0g + NTG : ((min(X0g + NTG, nx) + GA - 1) & ~(GA - 1));
            gbytes = (unsigned)((gce - gcs) * (int)sizeof(TG));
            rbytes = 10u * sbytes + 5u * gbytes;
            // copy role: the 15 planes spread over the warps (plane = warp +
            // nwarps * lane: 0..8 f, 9..13 g, 14 P), so that no warp carries
            // the issue work alone
            {
                const int pl = (t >> 5) + (NT / 32) * (t & 31);
                cp_kind = pl < 9 ? 0 : (pl < 14 ? 1 : (pl < 15 ? 2 : -1));
                const bool isg = cp_kind == 1;
                const int es = isg ? (int)sizeof(TG) : (int)sizeof(R);
                const int w0 = isg ? X0g : X0w;
                const int cs = isg ? gcs : scs;
                const char* base = cp_kind == 0 ? (const char*)(fsrc + (size_t)pl * plane)
                                   : isg        ? (const char*)(gsrc + (size_t)(pl - 9) * plane)
                                                : (const char*)Psrc;
                // periodic x copies the window in wrapped pieces from column 0
                cp_src = base + (perx ? 0 : (size_t)cs * es);
                const char* s0 = (const char*)&S;
                const char* d0 = cp_kind == 0 ? (const char*)&S.fR[0][pl < 9 ? pl : 0][0]
                                 : isg        ? (const char*)&S.gR[0][isg ? pl - 9 : 0][0]
                                              : (const char*)&S.pR[0][0];
                cp_dst = (unsigned)(d0 - s0) + (perx ? 0u : (unsigned)((cs - w0) * es));
                cp_slot = cp_kind == 0 ? (unsigned)sizeof(S.fR[0])
                          : isg        ? (unsigned)sizeof(S.gR[0])
                                       : (unsigned)sizeof(S.pR[0]);
                cp_row = (unsigned)(pitch * es);
                cp_bytes = isg ? gbytes : sbytes;
            }
            // iteration k queues the copies of row k + DA and arms row
            // k + DA + 1
            // rows y0 - 3 .. y0 - 3 + DA armed, the first DA of them
            // issued; kw2 ends as the wrapped row y0 - 3 + DA
            {
                int fs = fq;
                for (int j = 0; j <= DA; ++j) {
                    arm_row(y0 - 3 + j, fs);
                    fs = fs == NF - 1 ? 0 : fs + 1;
                }
            }
            __syncthreads();
            {
                int fs = fq, kr = kw;
                for (int j = 0; j < DA; ++j) {
                    issue_row(y0 - 3 + j, kr, j, fs);
                    fs = fs == NF - 1 ? 0 : fs + 1;
                    kr = (pery && kr == ny - 1) ? 0 : kr + 1;
                }
                kw2 = kr;
            }
        } else {
            load_row(y0 - 3, kw);
        }
    }

    // staged form.  Thread 0 arms the mbarrier of row k (f slot fslot) with
    // the row's byte count one iteration before the row's copies go out, so
    // that a barrier orders the arming before every copy; a row outside a
    // non-periodic domain (or past the segment) arms with no bytes.
    __device__ __forceinline__ void arm_row(int k, int fslot) {
        if (t == 0) mbar_arrive_tx(&S.mbar[fslot], (k < y1 + 3 && rowvalid(k)) ? rbytes : 0u);
    }
    // This thread's bulk copy (its plane from the copy role) of row k (wrapped
    // row kwr) into f slot fslot or g/P slot gslot.  Open x: the columns
    // inside the domain (the last strip's copy rounded up to 4 columns, inside
    // the row pitch); clamped columns read their edge column's entry (sidx).
    // Periodic x: the window in pieces that wrap around the axis.
    __device__ __forceinline__ void issue_row(int k, int kwr, int gslot, int fslot) {
        if (cp_kind < 0 || !(k < y1 + 3 && rowvalid(k))) return;
        unsigned long long* mb = &S.mbar[fslot];
        char* dst = (char*)&S + cp_dst + (unsigned)(cp_kind == 0 ? fslot : gslot) * cp_slot;
        const char* src = cp_src + (size_t)kwr * cp_row;
        if (!perx) {
            bulk_g2s(dst, src, cp_bytes, mb);
        } else {
            const bool isg = cp_kind == 1;
            const int es = isg ? (int)sizeof(TG) : (int)sizeof(R);
            const int w0 = isg ? X0g : X0w;
            int c = w0;
            const int end = w0 + (isg ? NTG : NT);
            while (c < end) {
                const int wc = wrapi(c, nx);
                const int n = min(end - c, nx - wc);
                bulk_g2s(dst + (c - w0) * es, src + (size_t)wc * es, (unsigned)(n * es), mb);
                c += n;
            }
        }
    }

    __device__ __forceinline__ bool rowvalid(int r) const { return pery || (r >= 0 && r < ny); }

    // loads of row k (wrapped row kwr) into fa, ga, pa; rows outside a
    // non-periodic domain give zeros (A does not use them)
    __device__ __forceinline__ void load_row(int k, int kwr) {
#pragma unroll
        for (int q = 0; q < 9; ++q) fa[q] = R(0);
#pragma unroll
        for (int q = 0; q < 5; ++q) ga[q] = R(0);
        pa = R(0);
        if (k < y1 + 3 && rowvalid(k)) {
            const size_t off = (size_t)kwr * pitch + gxl;
            const TF* fr = fsrc + off;
            const TG* gr = gsrc + off;
#pragma unroll
            for (int q = 0; q < 9; ++q) fa[q] = (R)ld_st(fr + q * plane);
#pragma unroll
            for (int q = 0; q < 5; ++q) ga[q] = (R)ld_st(gr + q * plane);
            pa = ld_st(Psrc + off);
        }
    }

    // one iteration with the ring slots of rows k (a0), k - 1 (a1), k - 2 (a2);
    // the steady loop passes them as literals, so every shared-memory ring
    // address is a constant offset
    template <bool STEADY>
    __device__ __forceinline__ void iter(int k, const int a0, const int a1, const int a2) {
        const int bC = b0 >= 3 ? b0 - 3 : b0 + 2;   // slot5(k - 3)
        const int bD = b0 >= 4 ? b0 - 4 : b0 + 1;   // slot5(k - 4)
        const int kwn = (pery && kw == ny - 1) ? 0 : kw + 1;
        // staged form: g/P slot of row k - 3; the copies of row k + DA go out
        // now, DA iterations before stage A needs them (the f slot they fill
        // held row k - 1, the g/P slot row k - 5: both were last read before
        // the previous iteration's closing barrier)
        const int gC = gq >= 3 ? gq - 3 : gq + NGS - 3;
        if constexpr (STG) {
            if (k + DA <= y1 + 3)
                issue_row(k + DA, kw2, gq + DA >= NGS ? gq + DA - NGS : gq + DA,
                          NF == 3 ? a1 : (fq == 0 ? NF - 1 : fq - 1));
        }
        // ================= phase alpha =================
        const bool doA = STEADY || (k < y1 + 3 && rowvalid(k));

        // ---- C(k-3): div u, grad T, Q, S and the D2Q5 MRT collision (Eq. 39)
        {
            const int r = k - 3;
            if (STEADY || (r >= y0 - 1 && r < y1 + 1 && rowvalid(r) && inC)) {
                R g0, g1, g2, g3, g4, rho, Pp, TdpdT;
                if constexpr (STG) {
                    const TG* gr = &S.gR[gC][0][sidx + goff];
                    g0 = st_val(gr[0]);
                    g1 = st_val(gr[NTG]);
                    g2 = st_val(gr[2 * NTG]);
                    g3 = st_val(gr[3 * NTG]);
                    g4 = st_val(gr[4 * NTG]);
                    Pp = S.pR[gC][sidx];
                    const R2 ow = S.own[bC][t];
                    rho = ow.x;
                    TdpdT = ow.y;
                } else {
                    const R4 o0 = S.own[bC][0][t];
                    const R4 o1 = S.own[bC][1][t];
                    g0 = o0.x; g1 = o0.y; g2 = o0.z; g3 = o0.w; g4 = o1.x;
                    rho = o1.y; Pp = o1.z; TdpdT = o1.w;
                }
                // (m_1, m_2) = (g1 - g3, g2 - g4) and the pair sums (g1 + g3, g2 + g4)
                const R2 m12 = psub(pr(g1, g2), pr(g3, g4));
                const R2 p13 = padd(pr(g1, g2), pr(g3, g4));
                const R m1 = m12.x, m2 = m12.y;
                const R Td = (g0 + p13.x) + p13.y;
                const R m3d = p13.x + p13.y;
                const R m4 = p13.x - p13.y;
                // Eqs. 49-50: c_s^2 d_x T = -varsigma_1 m_1^(1), m_1^eq = 0
                const R2 dT = pmul(pr(-P.vs1_cs2h, -P.vs1_cs2h), m12);
                const R dTx = dT.x;
                const R dTy = dT.y;
                // neighbour rows: solid -> u = 0, open -> the boundary row
                const bool vd = STEADY || pery || r - 1 >= 0, vu = STEADY || pery || r + 1 < ny;
                const R2 uc = S.u[a0][t];
                const R2 uW = S.u[a0][xl1], uE = S.u[a0][xr1];
                R2 uS0, uS1, uS2, uN0, uN1, uN2;
                if (vd || !wallS) {
                    const int s = vd ? a1 : a0;
                    uS0 = S.u[s][xl1]; uS1 = S.u[s][t]; uS2 = S.u[s][xr1];
                } else {
                    uS0.x = uS0.y = uS1.x = uS1.y = uS2.x = uS2.y = R(0);
                }
                if (vu || !wallN) {
                    const int s = vu ? a2 : a0;
                    uN0 = S.u[s][xl1]; uN1 = S.u[s][t]; uN2 = S.u[s][xr1];
                } else {
                    uN0.x = uN0.y = uN1.x = uN1.y = uN2.x = uN2.y = R(0);
                }
                // isotropic central difference, (1/c_s^2) sum_i w_i c_i phi(x + c_i)
                const R divu = (uE.x - uW.x + uN1.y - uS1.y) * R(1.0 / 3.0) +
                               ((uN2.x + uS2.x - uN0.x - uS0.x) +
                                (uN2.y + uN0.y - uS2.y - uS0.y)) * R(1.0 / 12.0);
                const R C = rho * P.cv;
                // Q = -[rho c_v u.grad T + T (dp/dT)_rho div u]  (Eq. 20)
                const R Q = -(C * (uc.x * dTx + uc.y * dTy) + TdpdT * divu);
                // P^n = Q / (rho c_v); S = w^ rho c_v (dt/2) d_t^2 T with
                // d_t^2 T ~ P^n - P^{n-1} (Eq. 24), i.e. (Q - rho c_v P^{n-1}) / 2
                const R Pn = Q * f_rcp(rho) * P.inv_cv;
                const R Qs = first ? Q : Q + R(0.5) * (Q - C * Pp);
                // moment-space collision (Eqs. 39, 40, 47), deviation form
                const R hc = R(0.5) * P.one_m_vs1;
                const R2 h12 = pmul(pr(hc, hc), m12);
                const R h1 = h12.x, h2 = h12.y;
                R gs0, gs1, gs2, gs3, gs4;
                if (UNIT) {
                    // varsigma_3 = varsigma_4 = 1: m3* = w_dot (T + Qs), m4* = 0
                    const R TQ = Td + Qs;
                    const R a = R(0.25) * P.w_dot * TQ;
                    // unfused: stage D5 subtracts g_0 from g*_0, and the
                    // staged form hands g*_0 over in a register
                    gs0 = mul_rn(P.w5_0, TQ);
                    const R2 g12 = padd(pr(a, a), h12), g34 = psub(pr(a, a), h12);
                    gs1 = g12.x;
                    gs2 = g12.y;
                    gs3 = g34.x;
                    gs4 = g34.y;
                } else {
                    const R m0s = Td + Qs;
                    const R m3s = m3d - P.vs3 * (m3d - P.w_dot * Td) + P.w_dot * Qs;
                    const R m4s = P.one_m_vs4 * m4;
                    const R a = R(0.25) * (m3s + m4s), b = R(0.25) * (m3s - m4s);
                    gs0 = m0s - m3s;
                    gs1 = a + h1;
                    gs2 = b + h2;
                    gs3 = a - h1;
                    gs4 = b - h2;
                }
                // g*_1 and g*_3 are read by the neighbour columns; g*_0, g*_2
                // and g*_4 only by this column's stage D5 (rows r, r + 1 and
                // r - 1).  The register-prefetch form keeps g*_2 in the gs
                // ring and g*_0, g*_4 in the row's own slot in place of
                // P^{n-1} and T (dp/dT)_rho
                S.gs[a0][0][t] = gs1;
                S.gs[a0][2][t] = gs3;
                if constexpr (STG) {
                    // the rest is read only by this column's D5 (rows r and
                    // r + 1): registers
                    cg[0] = g0;
                    cg[1] = g1;
                    cg[2] = g2;
                    cg[3] = g3;
                    cg[4] = g4;
                    crho = rho;
                    cgs0 = gs0;
                    cgs2 = gs2;
                    cgs4 = gs4;
                } else {
                    S.gs[a0][1][t] = gs2;
                    R4 oo;
                    oo.x = g4;
                    oo.y = rho;
                    oo.z = gs0;
                    oo.w = gs4;
                    S.own[bC][1][t] = oo;
                }
                if (inD && (STEADY || (r >= y0 && r < y1))) Pdst[(size_t)r * pitch + gx] = Pn;
            }
        }

        // ---- D9(k-3): pull streaming of f* (Eq. 6) with wall / open rules
        {
            const int r = k - 3;
            if (STEADY || (r >= y0 && r < y1 && inD)) {
                const bool vd = STEADY || pery || r - 1 >= 0, vu = STEADY || pery || r + 1 < ny;
                const int rowS = vd ? a1 : a0;   // source row for c_y = +1 (open: own row)
                const int rowN = vu ? a2 : a0;   // source row for c_y = -1
                const bool bS = !vd && wallS, bN = !vu && wallN;
                R fo[9];
                if (P.frozen_flow) {
                    if constexpr (UNIT) {
                        const TF* fr = fsrc + (size_t)(pery ? wrapi(r, ny) : r) * pitch + gxl;
#pragma unroll
                        for (int q = 0; q < 9; ++q) fo[q] = (R)ld_st(fr + q * plane);
                    } else {
#pragma unroll
                        for (int q = 0; q < 9; ++q) fo[q] = S.fs[a0][q][t];
                    }
                } else {
                    fo[0] = S.fs[a0][0][t];
                    fo[1] = S.fs[a0][1][xl1];
                    fo[3] = S.fs[a0][3][xr1];
                    fo[2] = bS ? S.fs[a0][4][t] : S.fs[rowS][2][t];
                    fo[5] = bS ? S.fs[a0][7][t] : S.fs[rowS][5][xl1];
                    fo[6] = bS ? S.fs[a0][8][t] : S.fs[rowS][6][xr1];
                    fo[4] = bN ? S.fs[a0][2][t] : S.fs[rowN][4][t];
                    fo[7] = bN ? S.fs[a0][5][t] : S.fs[rowN][7][xr1];
                    fo[8] = bN ? S.fs[a0][6][t] : S.fs[rowN][8][xl1];
                }
                if (inD) {
                    TF* fw = fdst + (size_t)r * pitch + gx;
#pragma unroll
                    for (int q = 0; q < 9; ++q) st_st(fw + q * plane, (TF)fo[q]);
                }
            }
        }

        // ---- D5(k-4), staged form: rho c_v-weighted streaming of g* (Eq. 39).
        // It runs in phase alpha: the g*_1, g*_3 it reads from the neighbour
        // columns were written by C(k-4) before the last barrier, and the rest
        // is this column's own, in registers (g*_4 of row k-3 from C(k-3) just
        // above)
        if constexpr (STG) {
            const int r = k - 4;
            if (STEADY || (r >= y0 && r < y1 && inD)) {
                R go[5];
                if (P.frozen_thermal) {
#pragma unroll
                    for (int q = 0; q < 5; ++q) go[q] = dg[q];
                } else {
                    const bool vd = STEADY || tpery || r - 1 >= 0, vu = STEADY || tpery || r + 1 < ny;
                    // thermal walls: halfway anti-bounce-back (Dirichlet) or
                    // bounce-back (adiabatic) supplies the incoming g*
                    R A1, A3;
                    if (left_edge) A1 = dirW ? twW2 - S.gs[a1][2][t] : S.gs[a1][2][t];
                    else A1 = S.gs[a1][0][xl1];
                    if (right_edge) A3 = dirE ? twE2 - S.gs[a1][0][t] : S.gs[a1][0][t];
                    else A3 = S.gs[a1][2][xr1];
                    const R A2 = vd ? egs2 : (dirS ? twS2 - dgs4 : dgs4);
                    const R A4 = vu ? cgs4 : (dirN ? twN2 - dgs2 : dgs2);
                    const R iC = f_rcp(drho * P.cv);
                    go[0] = dg[0] + (dgs0 - dg[0]) * iC;
                    // g_i + (A_i - g_i) / (rho c_v) for (1, 3) and (2, 4) in pairs
                    const R2 iC2 = pr(iC, iC);
                    const R2 g13 = pr(dg[1], dg[3]), g24 = pr(dg[2], dg[4]);
                    const R2 o13 = pfma(psub(pr(A1, A3), g13), iC2, g13);
                    const R2 o24 = pfma(psub(pr(A2, A4), g24), iC2, g24);
                    go[1] = o13.x;
                    go[3] = o13.y;
                    go[2] = o24.x;
                    go[4] = o24.y;
                }
                if (inD) {
                    TG* gw = gdst + (size_t)r * pitch + gx;
#pragma unroll
                    for (int q = 0; q < 5; ++q) st_st(gw + q * plane, go[q]);
                }
            }
            // row k-3 is the next D5's own row, row k-4 the row below it
            egs2 = dgs2;
#pragma unroll
            for (int q = 0; q < 5; ++q) dg[q] = cg[q];
            drho = crho;
            dgs0 = cgs0;
            dgs2 = cgs2;
            dgs4 = cgs4;
        }

        // ---- A(k): moments, EOS, psi
        if constexpr (STG) {
            // with three f slots the f ring turns with the literal ring slots:
            // row k sits in slot a0
            const int fk = NF == 3 ? a0 : fq;
            wait_row(&S.mbar[fk], (mph >> fk) & 1u, &errbits, &stalled);
            mph ^= 1u << fk;
        }
        R rho_a = R(1), rhod_a = R(0), jx_a = R(0), jy_a = R(0), psi_a = R(0), ir_a = R(1);
        R m7_a = R(0), m8_a = R(0);
        if constexpr (STG) {
            if (doA && (STEADY || colvalid)) {
                const R* fr = &S.fR[NF == 3 ? a0 : fq][0][sidx];
#pragma unroll
                for (int q = 0; q < 9; ++q) fa[q] = fr[q * NT];
                const TG* gr = &S.gR[gq][0][sidx + goff];
#pragma unroll
                for (int q = 0; q < 5; ++q) ga[q] = st_val(gr[q * NTG]);
            } else {
#pragma unroll
                for (int q = 0; q < 9; ++q) fa[q] = R(0);
            }
        }
        if (doA && (STEADY || colvalid)) {
            // pair sums and differences of (f1, f2) & (f3, f4) and (f5, f6) & (f7, f8)
            const R2 sA = padd(pr(fa[1], fa[2]), pr(fa[3], fa[4]));   // (f1 + f3, f2 + f4)
            const R2 dA = psub(pr(fa[1], fa[2]), pr(fa[3], fa[4]));   // (f1 - f3, f2 - f4)
            const R2 sB = padd(pr(fa[5], fa[6]), pr(fa[7], fa[8]));   // (f5 + f7, f6 + f8)
            const R2 dB = psub(pr(fa[5], fa[6]), pr(fa[7], fa[8]));   // (f5 - f7, f6 - f8)
            rhod_a = (fa[0] + (sA.x + sA.y)) + (sB.x + sB.y);
            rho_a = rhod_a + rho_ref;
            ir_a = f_rcp(rho_a);
            const R Td = ((ga[0] + ga[1]) + (ga[2] + ga[3])) + ga[4];
            const R T_a = Td + T_ref;
            jx_a = dA.x + (dB.x - dB.y);    // (f1 - f3) + (f5 - f7) - (f6 - f8)
            jy_a = dA.y + (dB.x + dB.y);    // (f2 - f4) + (f5 - f7) + (f6 - f8)
            if constexpr (UNIT) {
                m7_a = sA.x - sA.y;
                m8_a = sB.x - sB.y;
            }
            R q2, TdpdT;
            eos_node(P, rho_a, T_a, &q2, &TdpdT);
            if (colvalid && !(q2 >= R(0))) errbits |= (q2 != q2) ? ERR_NONFINITE : ERR_PSI;
            psi_a = f_sqrt(q2);
            S.psi[a0][t] = psi_a;
            if (wallS || wallN) {
                // only the wetting ghost layer reads rho and T of neighbours
                WR.rho[a0][t] = rho_a;
                WR.T[a0][t] = T_a;
            }
            if constexpr (STG) {
                R2 ow;
                ow.x = rho_a;
                ow.y = TdpdT;
                S.own[b0][t] = ow;
            } else {
                R4 o0, o1;
                o0.x = ga[0]; o0.y = ga[1]; o0.z = ga[2]; o0.w = ga[3];
                o1.x = ga[4]; o1.y = rho_a; o1.z = pa; o1.w = TdpdT;
                S.own[b0][0][t] = o0;
                S.own[b0][1][t] = o1;
            }
            // this unit's output rows only (steady iterations also load the
            // three rows above the segment)
            mass_acc += (inD && k >= my0 && k < my1) ? rho_a : R(0);
        }
        __syncthreads();

        // ================= phase beta =================
        // keep row k's populations for B(k) and issue the loads of row k + 1
        R fpn[9];
        if constexpr (!UNIT) {
#pragma unroll
            for (int q = 0; q < 9; ++q) fpn[q] = fa[q];
        }
        if constexpr (!STG) load_row(k + 1, kwn);
        // staged form: every thread is past its wait for row k, so row k's
        // mbarrier (and f slot) can take row k + 3
        if constexpr (STG) {
            if (k + DA + 1 <= y1 + 3) arm_row(k + DA + 1, NF == 3 ? a0 : fq);
        }

        // ---- B(k-1): interaction force, velocity, D2Q9 MRT collision
        {
            const int r = k - 1;
            if (STEADY || (r >= y0 - 2 && r < y1 + 2 && rowvalid(r) && inB)) {
                const bool vd = STEADY || pery || r - 1 >= 0, vu = STEADY || pery || r + 1 < ny;
                R pSW, pS, pSE, pNW, pN, pNE;
                const R pW = S.psi[a1][xl1], pE = S.psi[a1][xr1];
                if (vd || !wallS) {
                    const int s = vd ? a2 : a1;
                    pSW = S.psi[s][xl1]; pS = S.psi[s][t]; pSE = S.psi[s][xr1];
                } else {
                    // south wall: layer 1 = row r (a1), layer 2 = row r + 1 (a0);
                    // the ghost's psi at the temperature of the fluid node above it
                    pSW = ghost_psi(P, WR.rho[a0][xl1], WR.rho[a1][cLR], WR.rho[a1][cLL], cot,
                                    WR.T[a1][xl1], &errbits);
                    pS = ghost_psi(P, WR.rho[a0][t], WR.rho[a1][xr1], WR.rho[a1][xl1], cot,
                                   WR.T[a1][t], &errbits);
                    pSE = ghost_psi(P, WR.rho[a0][xr1], WR.rho[a1][cRR], WR.rho[a1][cRL], cot,
                                    WR.T[a1][xr1], &errbits);
                }
                if (vu || !wallN) {
                    const int s = vu ? a0 : a1;
                    pNW = S.psi[s][xl1]; pN = S.psi[s][t]; pNE = S.psi[s][xr1];
                } else {
                    // north wall: layer 1 = row r (a1), layer 2 = row r - 1 (a2)
                    pNW = ghost_psi(P, WR.rho[a2][xl1], WR.rho[a1][cLR], WR.rho[a1][cLL], cot,
                                    WR.T[a1][xl1], &errbits);
                    pN = ghost_psi(P, WR.rho[a2][t], WR.rho[a1][xr1], WR.rho[a1][xl1], cot,
                                   WR.T[a1][t], &errbits);
                    pNE = ghost_psi(P, WR.rho[a2][xr1], WR.rho[a1][cRR], WR.rho[a1][cRL], cot,
                                    WR.T[a1][xr1], &errbits);
                }
                // Eq. 9 with varpi(1) = 1/3, varpi(2) = 1/12, both components
                // at once: s = (pE - pW, pN - pS) / 3 + (dA + dB, dA - dB) / 12
                const R dA = pNE - pSW, dB = pSE - pNW;
                const R2 sxy = pfma(psub(pr(pE, pN), pr(pW, pS)), pr(R(1.0 / 3.0), R(1.0 / 3.0)),
                                    pmul(pr(dA + dB, dA - dB), pr(R(1.0 / 12.0), R(1.0 / 12.0))));
                const R sx = sxy.x, sy = sxy.y;
                const R gp = P.negG * psip;
                const R2 Fm = pmul(pr(gp, gp), sxy);
                const R Fx = Fm.x;
                const R Fy = Fm.y - P.gravity * (rhop - rho_ave);
                R ux = R(0), uy = R(0);
                if (!P.frozen_flow) {
                    const R2 uu2 = pmul(pfma(pr(Fx, Fy), pr(R(0.5), R(0.5)), pr(jxp, jyp)), pr(irp, irp));
                    ux = uu2.x;
                    uy = uu2.y;
                }
                R2 uv;
                uv.x = ux;
                uv.y = uy;
                S.u[a1][t] = uv;
                if (STEADY || (r >= y0 - 1 && r < y1 + 1 && inC)) {
                    R* fsw = &S.fs[a1][0][t];
                    if (P.frozen_flow) {
                        // the populations stay as they are: stage D9 copies
                        // them from the source state (unit rates), or from here
                        if constexpr (!UNIT) {
#pragma unroll
                            for (int q = 0; q < 9; ++q) fsw[q * NT] = fp[q];
                        }
                    } else if (UNIT) {
                        // s_e = s_eps = s_q = 1: those moments leave the
                        // collision at m^eq + F/2, so f* = M^{-1} m* needs of f
                        // only rho, j and the stresses m_7, m_8 (Eqs. 5, 7, 8)
                        const R rr = rhop;
                        const R2 u2 = pr(ux, uy), F2 = pr(Fx, Fy);
                        const R2 ru = pmul(pr(rr, rr), u2);          // rho u
                        const R2 uu = pmul(ru, u2);                  // rho (ux^2, uy^2)
                        const R2 uFc = pmul(u2, F2);                 // (ux Fx, uy Fy)
                        const R2 s2 = pmul(sxy, sxy);
                        const R ruu = uu.x + uu.y;
                        const R uF = uFc.x + uFc.y;
                        const R Fm2 = P.negG * P.negG * (s2.x + s2.y);
                        const R m7 = m7p;
                        const R m8 = m8p;
                        const R F7 = R(2) * (uFc.x - uFc.y);
                        const R F8 = ux * Fy + uy * Fx;
                        // deviation-form m*_e, m*_eps (storage shifts them by
                        // -2 rho_ref and rho_ref)
                        const R t3 = R(3) * (ruu + uF);
                        const R m1s = R(-2) * rhodp + t3 + R(0.5) * P.sig_e * Fm2;
                        const R m2s = rhodp - t3 - R(0.5) * P.sig_eps * Fm2;
                        const R b0 = rhodp * R(1.0 / 9.0);
                        const R2 b12 = pmul(pr(m1s, m2s), pr(R(1.0 / 36.0), R(1.0 / 36.0)));
                        const R b1 = b12.x, b2 = b12.y;
                        const R b7 = (m7 - P.s_p * (m7 - (uu.x - uu.y)) + P.hs_p * F7) * R(0.25);
                        const R b8 = (m8 - P.s_p * (m8 - ru.x * uy) + P.hs_p * F8) * R(0.25);
                        // j* = j + F; q* = -(j + F) / 1 -> combined axis / diagonal terms
                        const R2 js = padd(pr(jxp, jyp), F2);
                        const R2 XY3 = pmul(js, pr(R(1.0 / 3.0), R(1.0 / 3.0)));
                        const R2 XY12 = pmul(js, pr(R(1.0 / 12.0), R(1.0 / 12.0)));
                        const R cax = b0 - b1 - R(2) * b2;
                        const R cdg = b0 + R(2) * b1 + b2;
                        // axis directions: (1, 2) = (cax + b7, cax - b7) + (X3, Y3),
                        // (3, 4) = the same minus (X3, Y3); diagonals: (5, 8) =
                        // (cdg + b8, cdg - b8) + (X12 + Y12, X12 - Y12), (7, 6) the
                        // same minus
                        const R2 cb = pr(cax + b7, cax - b7);
                        const R2 f12 = padd(cb, XY3), f34 = psub(cb, XY3);
                        const R2 db = pr(cdg + b8, cdg - b8);
                        const R2 sd = pr(XY12.x + XY12.y, XY12.x - XY12.y);
                        const R2 f58 = padd(db, sd), f76 = psub(db, sd);
                        fsw[0 * NT] = b0 + R(4) * (b2 - b1);
                        fsw[1 * NT] = f12.x;
                        fsw[2 * NT] = f12.y;
                        fsw[3 * NT] = f34.x;
                        fsw[4 * NT] = f34.y;
                        fsw[5 * NT] = f58.x;
                        fsw[6 * NT] = f76.y;
                        fsw[7 * NT] = f76.x;
                        fsw[8 * NT] = f58.y;
                    } else {
                        const R* f = fp;
                        const R rr = rhop;
                        const R rux = rr * ux, ruy = rr * uy;
                        const R ruu = rux * ux + ruy * uy;
                        const R s14 = (f[1] + f[3]) + (f[2] + f[4]);
                        const R s58 = (f[5] + f[7]) + (f[6] + f[8]);
                        // non-equilibrium parts m - m^eq of the moments of Eq. 7
                        // (deviation storage shifts m_e by -2 rho_ref, m_eps by rho_ref)
                        const R ne1 = R(2) * (s58 + rhodp - f[0]) - (R(2) * f[0] + s14) - R(3) * ruu;
                        const R ne2 = (R(4) * f[0] - R(2) * s14 + s58) - rhodp + R(3) * ruu;
                        const R d13 = f[1] - f[3], d24 = f[2] - f[4];
                        const R d58 = f[5] - f[7], d68 = f[6] - f[8];
                        const R ne4 = (d58 - d68 - R(2) * d13) + rux;
                        const R ne6 = (d58 + d68 - R(2) * d24) + ruy;
                        const R ne7 = (f[1] + f[3]) - (f[2] + f[4]) - (rux * ux - ruy * uy);
                        const R ne8 = (f[5] + f[7]) - (f[6] + f[8]) - rux * uy;
                        // Li forcing (Eq. 8); |F_m|^2 / psi^2 = G^2 |sum varpi psi c|^2
                        const R uF = ux * Fx + uy * Fy;
                        const R Fm2 = P.negG * P.negG * (sx * sx + sy * sy);
                        const R F1 = R(6) * uF + P.sig_e * Fm2;
                        const R F2 = R(-6) * uF - P.sig_eps * Fm2;
                        const R F7 = R(2) * (ux * Fx - uy * Fy);
                        const R F8 = ux * Fy + uy * Fx;
                        // m* - m = -S (m - m^eq) + (I - S/2) F; for j the
                        // change is exactly F because rho u = j + F/2
                        const R a1m = (P.hs_e * F1 - P.s_e * ne1) * R(1.0 / 36.0);
                        const R a2m = (P.hs_eps * F2 - P.s_eps * ne2) * R(1.0 / 36.0);
                        const R a3 = Fx * R(1.0 / 6.0), a5 = Fy * R(1.0 / 6.0);
                        const R a4 = -(P.s_q * ne4 + P.hs_q * Fx) * R(1.0 / 12.0);
                        const R a6 = -(P.s_q * ne6 + P.hs_q * Fy) * R(1.0 / 12.0);
                        const R a7 = (P.hs_p * F7 - P.s_p * ne7) * R(0.25);
                        const R a8 = (P.hs_p * F8 - P.s_p * ne8) * R(0.25);
                        // f* = f + M^{-1} (m* - m), M^{-1} = M^T diag(1/9, 1/36,
                        // 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4)
                        const R cax = -a1m - R(2) * a2m;   // common to the axis directions
                        const R cdg = R(2) * a1m + a2m;    // common to the diagonals
                        const R ex = a3 - R(2) * a4, ey = a5 - R(2) * a6;
                        const R dx = a3 + a4, dy = a5 + a6;
                        fsw[0 * NT] = f[0] + R(4) * (a2m - a1m);
                        fsw[1 * NT] = f[1] + cax + ex + a7;
                        fsw[2 * NT] = f[2] + cax + ey - a7;
                        fsw[3 * NT] = f[3] + cax - ex + a7;
                        fsw[4 * NT] = f[4] + cax - ey - a7;
                        fsw[5 * NT] = f[5] + cdg + dx + dy + a8;
                        fsw[6 * NT] = f[6] + cdg - dx + dy - a8;
                        fsw[7 * NT] = f[7] + cdg - dx - dy + a8;
                        fsw[8 * NT] = f[8] + cdg + dx - dy - a8;
                    }
                }
            }
        }

        // ---- D5(k-4), register-prefetch form: rho c_v-weighted streaming of
        // g* (Eq. 39)
        if constexpr (!STG) {
            const int r = k - 4;
            if (STEADY || (r >= y0 && r < y1 && inD)) {
                const R4 o0 = S.own[bD][0][t];
                const R4 o1 = S.own[bD][1][t];
                R go[5];
                if (P.frozen_thermal) {
                    go[0] = o0.x; go[1] = o0.y; go[2] = o0.z; go[3] = o0.w; go[4] = o1.x;
                } else {
                    const bool vd = STEADY || tpery || r - 1 >= 0, vu = STEADY || tpery || r + 1 < ny;
                    // gs planes hold g*_1, g*_2, g*_3; g*_0 and g*_4 of row r sit
                    // in the row's own slot, g*_4 of row r + 1 in that row's
                    const R* gsc = &S.gs[a1][0][t];
                    // thermal walls: halfway anti-bounce-back (Dirichlet) or
                    // bounce-back (adiabatic) supplies the incoming g*
                    R A1, A3;
                    if (left_edge) A1 = dirW ? twW2 - gsc[2 * NT] : gsc[2 * NT];
                    else A1 = S.gs[a1][0][xl1];
                    if (right_edge) A3 = dirE ? twE2 - gsc[0] : gsc[0];
                    else A3 = S.gs[a1][2][xr1];
                    R A2, A4;
                    if (vd) A2 = S.gs[a2][1][t];
                    else A2 = dirS ? twS2 - o1.w : o1.w;
                    if (vu) A4 = S.own[bC][1][t].w;
                    else A4 = dirN ? twN2 - gsc[1 * NT] : gsc[1 * NT];
                    const R A0 = o1.z;
                    const R iC = f_rcp(o1.y * P.cv);
                    go[0] = o0.x + (A0 - o0.x) * iC;
                    // as in the staged form: (1, 3) and (2, 4) in pairs
                    const R2 iC2 = pr(iC, iC);
                    const R2 g13 = pr(o0.y, o0.w), g24 = pr(o0.z, o1.x);
                    const R2 o13 = pfma(psub(pr(A1, A3), g13), iC2, g13);
                    const R2 o24 = pfma(psub(pr(A2, A4), g24), iC2, g24);
                    go[1] = o13.x;
                    go[3] = o13.y;
                    go[2] = o24.x;
                    go[4] = o24.y;
                }
                if (inD) {
                    TG* gw = gdst + (size_t)r * pitch + gx;
#pragma unroll
                    for (int q = 0; q < 5; ++q) st_st(gw + q * plane, go[q]);
                }
            }
        }
        __syncthreads();

        if constexpr (!UNIT) {
#pragma unroll
            for (int q = 0; q < 9; ++q) fp[q] = fpn[q];
        } else {
            m7p = m7_a;
            m8p = m8_a;
        }
        rhop = rho_a;
        rhodp = rhod_a;
        jxp = jx_a;
        jyp = jy_a;
        psip = psi_a;
        irp = ir_a;
        b0 = b0 == 4 ? 0 : b0 + 1;
        kw = kwn;
        gq = gq == NGS - 1 ? 0 : gq + 1;
        fq = fq == NF - 1 ? 0 : fq + 1;
        kw2 = (pery && kw2 == ny - 1) ? 0 : kw2 + 1;
    }

    // general iteration with the rotating slots
    __device__ __forceinline__ void iter_general(int k) {
        iter<false>(k, ra0, ra1, ra2);
        rotate();
    }
    __device__ __forceinline__ void rotate() {
        const int tmp = ra2;
        ra2 = ra1;
        ra1 = ra0;
        ra0 = tmp;
    }
};

template <int PREC, int NT, bool UNIT, bool STG>
__device__ __forceinline__ void process_unit(const Inst& I, const Unit& U,
                                             const Phys<typename Types<PREC>::R>& P,
                                             typename Sweep<PREC, NT, UNIT, STG>::SM& S,
                                             WallRings<typename Types<PREC>::R, NT>& WR,
                                             unsigned& mph, int probe) {
    Sweep<PREC, NT, UNIT, STG> w(I, U, P, S, WR, mph);
    const int y0 = U.y0, y1 = U.y1;
    if constexpr (STG) {
        // wait-timeout test hook: a bounded wait on an mbarrier that nothing
        // arms runs out and records ERR_TIMEOUT; the row pipeline keeps its
        // own waits, so the step itself is unaffected
        if (probe) {
            bool probe_stalled = false;
            wait_row(&S.probe, 0u, &w.errbits, &probe_stalled);
        }
    }
    // iterations whose five stages are all active on rows with interior
    // neighbours take the steady form
    int klo = y0 + 4, khi = y1 + 2;
    if (!w.pery || !w.tpery) {
        klo = max(klo, 5);
        khi = min(khi, I.ny - 2);
    }
    // the steady loop starts where the ring phase is back at its initial
    // (0, 2, 1) and runs in groups of three with literal slots
    klo += ((y0 - 3) - klo) % 3 + (((y0 - 3) - klo) % 3 < 0 ? 3 : 0);
    int k = y0 - 3;
    for (; k < klo && k <= y1 + 3; ++k) w.iter_general(k);
    for (; k + 2 <= khi; k += 3) {
        w.template iter<true>(k, 0, 2, 1);
        w.template iter<true>(k + 1, 1, 0, 2);
        w.template iter<true>(k + 2, 2, 1, 0);
    }
    for (; k <= y1 + 3; ++k) w.iter_general(k);
    mph = w.mph;
    if constexpr (STG) {
        // a row wait that ran out may leave copies in flight into this CTA's
        // shared memory: wait (again bounded) until each row mbarrier has
        // completed the last phase this unit used, before the CTA moves on
        if (w.stalled) {
            for (int m = 0; m < Sweep<PREC, NT, UNIT, STG>::NF; ++m) {
                bool st = false;
                wait_row(&S.mbar[m], ((mph >> m) & 1u) ^ 1u, &w.errbits, &st);
            }
        }
    }

    if (w.errbits) atomicOr(&I.ctl->err, w.errbits);
    {
        // warp sums of this unit's output densities -> ring slot step % 3, as
        // fixed-point integers (order-free, so no barrier is needed); kept
        // with gravity off too, so that lbm_reconfigure can switch buoyancy on
        // with the previous step's density sum in place
        double macc = (double)w.mass_acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) macc += __shfl_down_sync(0xffffffffu, macc, o);
        if ((w.t & 31) == 0) {
            const long long step = __ldcg(&I.ctl->step);
            massq_add(&I.ctl->massq[step % 3], macc, massq_scale(I.inv_n));
        }
    }
}

template <int PREC, int NT, bool UNIT, bool STG>
__global__ void __launch_bounds__(NT, (PREC == 0) ? 1 : (512 / NT))
    k_step(StepLaunch L, Phys<typename Types<PREC>::R> P) {
    typedef typename Types<PREC>::R R;
    typedef typename Sweep<PREC, NT, UNIT, STG>::SM SM;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SM& S = *reinterpret_cast<SM*>(smem_raw);
    WallRings<R, NT>& WR = *reinterpret_cast<WallRings<R, NT>*>(smem_raw + sizeof(SM));
    unsigned mph = 0;
    if constexpr (STG) {
        if (threadIdx.x == 0) {
            for (int m = 0; m <= Ahead<NT>::value; ++m) mbar_init(&S.mbar[m], 1);
            mbar_init(&S.probe, 1);
            mbar_init_fence();
        }
        __syncthreads();
    }
    for (;;) {
        if (threadIdx.x == 0) S.unit = (int)atomicAdd(&L.sched[0], 1u);
        __syncthreads();
        const int u = S.unit;
        __syncthreads();
        if (u >= L.n_units) break;
        const Unit U = L.units[u];
        // a domain at its target step sits this launch out (every thread
        // reads the same control block, so the branch is uniform); launches
        // without targets skip the check and its loads
        if (L.targets && ctl_stopped(L.insts[U.inst].ctl)) continue;
        process_unit<PREC, NT, UNIT, STG>(L.insts[U.inst], U, P, S, WR, mph, L.wait_probe);
    }
    // the last CTA to finish (its thread 0 finds the finished-CTA count at
    // gridDim.x - 1; S.unit is free once the unit loop has ended) publishes
    // each domain's density sum, clears the slot the next step accumulates
    // into, advances the step counters and resets the work counters for the
    // next launch; its threads share the domains, so a batch of hundreds of
    // domains costs a few dependent loads per thread, not per domain
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned done = atomicAdd(&L.sched[1], 1u);
        S.unit = done == gridDim.x - 1 ? 1 : 0;
    }
    __syncthreads();
    if (S.unit) {
        __threadfence();
        for (int i = threadIdx.x; i < L.n_inst; i += NT) {
            Ctl* c = L.insts[i].ctl;
            if (L.targets && ctl_stopped(c)) continue;
            const long long s = __ldcg(&c->step);
            c->mass[s % 3] = massq_value(__ldcg(&c->massq[s % 3]), massq_scale(L.insts[i].inv_n));
            c->massq[(s + 1) % 3] = 0;
            c->step = s + 1;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            L.sched[0] = 0u;
            L.sched[1] = 0u;
            __threadfence();
        }
    }
}

// The unit-rate form applies when every non-hydrodynamic rate is exactly 1
// (s_e = s_eps = s_q = 1 and varsigma_3 = varsigma_4 = 1, the paper's choice).
static bool unit_rates(const PhysD& d) {
    return d.s_e == 1.0 && d.s_eps == 1.0 && d.s_q == 1.0 && d.vs3 == 1.0 && d.vs4 == 1.0;
}

template <int PREC, int NT, bool STG>
static size_t smem_for(bool walls) {
    typedef typename Types<PREC>::R R;
    typedef typename Types<PREC>::TG TG;
    typedef typename std::conditional<STG, StageSmem<R, TG, NT>, StepSmem<R, NT>>::type SM;
    return sizeof(SM) + (walls ? sizeof(WallRings<R, NT>) : 0);
}

template <int PREC, int NT, bool UNIT, bool STG>
static int set_smem_attr() {
    static bool done = false;
    if (!done) {
        if (cudaFuncSetAttribute(k_step<PREC, NT, UNIT, STG>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_for<PREC, NT, STG>(true)) != cudaSuccess)
            return -1;
        done = true;
    }
    return 0;
}

template <int PREC, int NT, bool STG>
static int launch_form(const StepLaunch& L, cudaStream_t st) {
    typedef typename Types<PREC>::R R;
    const size_t smem = smem_for<PREC, NT, STG>(L.walls != 0);
    Phys<R> P = make_phys<R>(L.phys);
    if (unit_rates(L.phys)) {
        if (set_smem_attr<PREC, NT, true, STG>()) return -1;
        k_step<PREC, NT, true, STG><<<L.grid, NT, smem, st>>>(L, P);
    } else {
        if (set_smem_attr<PREC, NT, false, STG>()) return -1;
        k_step<PREC, NT, false, STG><<<L.grid, NT, smem, st>>>(L, P);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int PREC, int NT>
static int launch_one(const StepLaunch& L, cudaStream_t st) {
    if constexpr (PREC != 0) {
        if (L.staged) return launch_form<PREC, NT, true>(L, st);
    }
    return launch_form<PREC, NT, false>(L, st);
}

template <int PREC, int NT, bool STG>
static int occ_form(int walls, int* ctas, size_t* smem_bytes) {
    const size_t smem = smem_for<PREC, NT, STG>(walls != 0);
    if (set_smem_attr<PREC, NT, true, STG>() || set_smem_attr<PREC, NT, false, STG>()) return -1;
    int a = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_step<PREC, NT, true, STG>, NT, smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_step<PREC, NT, false, STG>, NT, smem) !=
            cudaSuccess)
        return -1;
    *ctas = a < b ? a : b;
    *smem_bytes = smem;
    return 0;
}

template <int PREC, int NT>
static int occ_one(int walls, int staged, int* ctas, size_t* smem_bytes) {
    if constexpr (PREC != 0) {
        if (staged) return occ_form<PREC, NT, true>(walls, ctas, smem_bytes);
    }
    return occ_form<PREC, NT, false>(walls, ctas, smem_bytes);
}

int step_launch(int prec, int threads, const StepLaunch& L, cudaStream_t st) {
    if (threads == 128) {
        if (prec == 0) return launch_one<0, 128>(L, st);
        if (prec == 1) return launch_one<1, 128>(L, st);
        return launch_one<2, 128>(L, st);
    }
    if (threads == 192) {
        if (prec == 0) return launch_one<0, 192>(L, st);
        if (prec == 1) return launch_one<1, 192>(L, st);
        return launch_one<2, 192>(L, st);
    }
    if (threads == 224) {
        if (prec == 0) return launch_one<0, 224>(L, st);
        if (prec == 1) return launch_one<1, 224>(L, st);
        return launch_one<2, 224>(L, st);
    }
    if (prec == 0) return launch_one<0, 256>(L, st);
    if (prec == 1) return launch_one<1, 256>(L, st);
    return launch_one<2, 256>(L, st);
}

int step_occupancy(int prec, int threads, int walls, int staged, int* ctas, size_t* smem) {
    if (threads == 128) {
        if (prec == 0) return occ_one<0, 128>(walls, staged, ctas, smem);
        if (prec == 1) return occ_one<1, 128>(walls, staged, ctas, smem);
        return occ_one<2, 128>(walls, staged, ctas, smem);
    }
    if (threads == 192) {
        if (prec == 0) return occ_one<0, 192>(walls, staged, ctas, smem);
        if (prec == 1) return occ_one<1, 192>(walls, staged, ctas, smem);
        return occ_one<2, 192>(walls, staged, ctas, smem);
    }
    if (threads == 224) {
        if (prec == 0) return occ_one<0, 224>(walls, staged, ctas, smem);
        if (prec == 1) return occ_one<1, 224>(walls, staged, ctas, smem);
        return occ_one<2, 224>(walls, staged, ctas, smem);
    }
    if (prec == 0) return occ_one<0, 256>(walls, staged, ctas, smem);
    if (prec == 1) return occ_one<1, 256>(walls, staged, ctas, smem);
    return occ_one<2, 256>(walls, staged, ctas, smem);
}

}  // namespace lbm
