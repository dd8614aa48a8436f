// C ABI of the library (declared in include/lbm.h): simulation contexts,
// device memory layout, work-unit lists, CUDA-graph replay of the fused step,
// batched stepping of many domains, the tile autotuner and checkpoints.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "lbm.h"
#include "lbm_internal.cuh"

using namespace lbm;

namespace {

const int kGraphLen = 32;      // launches per captured graph
const size_t kAlign = 256;

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Layout {
    int pitch;
    size_t planeF, planeG, planeP, total;
};

// Planes are [ny][pitch] with pitch a multiple of 64 elements, so every plane
// (and every row) starts on a 128-byte boundary; the kernels address plane q
// at q * ny * pitch elements, so planes are packed without extra padding.
Layout layout_for(int nx, int ny, int prec) {
    Layout L;
    L.pitch = (int)round_up((size_t)nx, 64);
    L.planeF = (size_t)L.pitch * ny * elem_f(prec);
    L.planeG = (size_t)L.pitch * ny * elem_g(prec);
    L.planeP = (size_t)L.pitch * ny * elem_P(prec);
    L.total = 2 * (9 * L.planeF + 5 * L.planeG + L.planeP);
    return L;
}

bool bc_valid(int nx, int ny, const lbm_bc* bc) {
    for (int e = 0; e < 4; ++e) {
        if (bc->flow[e] < 0 || bc->flow[e] > 2 || bc->therm[e] < 0 || bc->therm[e] > 2) return false;
        // a periodic thermal edge needs a periodic flow edge; a periodic flow
        // edge may carry a Dirichlet or adiabatic thermal edge (Section 4.1)
        if (bc->therm[e] == LBM_T_PERIODIC && bc->flow[e] != LBM_PERIODIC) return false;
    }
    if ((bc->flow[LBM_EDGE_W] == LBM_PERIODIC) != (bc->flow[LBM_EDGE_E] == LBM_PERIODIC)) return false;
    if ((bc->flow[LBM_EDGE_S] == LBM_PERIODIC) != (bc->flow[LBM_EDGE_N] == LBM_PERIODIC)) return false;
    if ((bc->therm[LBM_EDGE_W] == LBM_T_PERIODIC) != (bc->therm[LBM_EDGE_E] == LBM_T_PERIODIC))
        return false;
    if ((bc->therm[LBM_EDGE_S] == LBM_T_PERIODIC) != (bc->therm[LBM_EDGE_N] == LBM_T_PERIODIC))
        return false;
    if (bc->flow[LBM_EDGE_W] == LBM_WALL || bc->flow[LBM_EDGE_E] == LBM_WALL) return false;
    if (bc->flow[LBM_EDGE_W] != LBM_PERIODIC && nx < 2) return false;
    if (bc->flow[LBM_EDGE_S] != LBM_PERIODIC && ny < 2) return false;
    return true;
}

bool params_valid(const lbm_params* p) {
    return p->cv > 0 && p->nu > 0 && p->lambda > 0 && p->w_dot > 0 && p->w_dot < 1 &&
           p->G != 0.0 && p->b > 0 && p->s_e > 0 && p->s_e < 2 && p->s_eps > 0 && p->s_eps < 2;
}

PhysD phys_from(const lbm_params* p) {
    PhysD d;
    d.a = p->a;
    d.b = p->b;
    d.Rg = p->R;
    d.omega = p->omega;
    d.G = p->G;
    d.sigma = p->sigma;
    d.s_e = p->s_e;
    d.s_eps = p->s_eps;
    d.s_q = p->s_q;
    d.s_p = 1.0 / (3.0 * p->nu + 0.5);                       // nu = c_s^2 (1/s_p - 1/2)
    d.cv = p->cv;
    d.w_dot = p->w_dot;
    d.vs1 = 1.0 / (p->lambda / (0.5 * p->w_dot) + 0.5);      // lambda = (1/vs - 1/2) w_dot/2
    d.vs3 = p->vs3;
    d.vs4 = p->vs4;
    d.gravity = p->gravity;
    d.frozen_flow = p->frozen_flow;
    d.frozen_thermal = p->frozen_thermal;
    return d;
}

bool same_physics(const lbm_params& a, const lbm_params& b) {
    lbm_params x = a, y = b;
    x.rho_ref = y.rho_ref = 0.0;
    x.T_ref = y.T_ref = 0.0;
    return memcmp(&x, &y, sizeof(x)) == 0;
}

uint32_t crc32_update(uint32_t crc, const void* data, size_t n) {
    static uint32_t table[256];
    static bool init = false;
    if (!init) {
        for (uint32_t i = 0; i < 256; ++i) {
            uint32_t c = i;
            for (int k = 0; k < 8; ++k) c = (c & 1) ? 0xEDB88320u ^ (c >> 1) : c >> 1;
            table[i] = c;
        }
        init = true;
    }
    const unsigned char* p = (const unsigned char*)data;
    crc = ~crc;
    for (size_t i = 0; i < n; ++i) crc = table[(crc ^ p[i]) & 0xFF] ^ (crc >> 8);
    return ~crc;
}

// tile autotuner cache: (prec, nx, ny) -> (threads, rows, staged)
struct Tile {
    int threads, rows, staged;
};
std::map<std::tuple<int, int, int>, Tile>& tune_cache() {
    static std::map<std::tuple<int, int, int>, Tile> m;
    return m;
}

int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

void build_units(const Inst& I, int inst_index, int threads, int rows, std::vector<Unit>& out) {
    const int W = threads - 8;
    for (int y0 = 0; y0 < I.ny; y0 += rows)
        for (int x0 = 0; x0 < I.nx; x0 += W) {
            Unit u;
            u.inst = inst_index;
            u.x0 = x0;
            u.x1 = std::min(I.nx, x0 + W);
            u.y0 = y0;
            u.y1 = std::min(I.ny, y0 + rows);
            out.push_back(u);
        }
}

bool has_walls(const Inst& I) {
    return I.flow[2] == LBM_WALL || I.flow[3] == LBM_WALL;
}

// default load path and tile: bulk-copy staging on a 224-thread tile (two
// CTAs per SM, two rows in flight per CTA) where the domains can take it,
// have no walls (the wall rings would leave one CTA per SM) and are wide
// enough that 216-column strips need no more thread columns than 120-column
// ones (a 64-wide domain fills 29 % of a 224-thread strip, 50 % of a
// 128-thread one; on the 512-domain mix with sides 64..512, 9 % more thread
// columns already made the staged tile 12 % slower); otherwise the
// register-prefetch form on 128 threads (four CTAs per SM).  lbm_autotune /
// lbm_batch_autotune replace this guess by timed trials.
long long strip_columns(int nx, int threads) {
    return (long long)((nx + threads - 9) / (threads - 8)) * threads;
}
bool default_staged(const Inst* const* I, size_t n, int prec) {
    long long c224 = 0, c128 = 0;
    for (size_t i = 0; i < n; ++i) {
        if (!stage_eligible(*I[i], prec) || has_walls(*I[i])) return false;
        c224 += strip_columns(I[i]->nx, 224) * I[i]->ny;
        c128 += strip_columns(I[i]->nx, 128) * I[i]->ny;
    }
    return n > 0 && c224 <= c128;
}
int default_threads(int staged) { return staged ? 224 : 128; }

// default segment height: the work units of a launch should fill the
// persistent grid in whole waves (one unit per resident CTA; a second, partial
// wave doubles the time of the CTAs that take it), so take the most segments
// per strip that keep strips x segments within one wave, and the rows that
// gives; never below 8
int wave_rows(int ny, long long strips, long long slots, int waves) {
    const long long S = std::max<long long>(1, (long long)waves * slots / strips);
    return (int)std::max<long long>(1, std::min<long long>(ny, std::max<long long>(8, (ny + S - 1) / S)));
}

int default_rows(int prec, int threads, int walls, int staged, int nx, int ny) {
    int ctas = 1;
    size_t smem = 0;
    step_occupancy(prec, threads, walls, staged, &ctas, &smem);
    const long long slots = (long long)std::max(ctas, 1) * num_sms();
    const long long strips = (nx + threads - 9) / (threads - 8);
    return wave_rows(ny, strips, slots, 1);
}

}  // namespace

// ---------------------------------------------------------------------------
struct lbm_ctx {
    int nx = 0, ny = 0, prec = 0;
    lbm_params params;
    lbm_bc bc;
    PhysD phys;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void* mem = nullptr;
    bool own_mem = false;
    Layout lay;
    Inst inst;                 // host copy (pointers into mem)
    void* small = nullptr;     // Ctl | Inst | sched
    Ctl* ctl = nullptr;
    Inst* inst_dev = nullptr;
    unsigned* sched = nullptr;
    Unit* units = nullptr;
    int n_units = 0, grid = 1, threads = 128, rows = 64, staged = 0, wait_probe = 0;
    cudaGraphExec_t graph = nullptr;
    long long step = 0;
    long long target = 0;      // the step the domain stops at (0: none), as on the device
    bool initialized = false;
    int sticky = LBM_OK;
    std::string err;
    double* fields = nullptr;  // 5 N doubles (rho, ux, uy, T, psi scratch), lazily allocated
    void* diag_scratch = nullptr;
    double* diag_out = nullptr;
    void* iface_scratch = nullptr;   // contact-angle partial sums + 12 results
    void* region_scratch = nullptr;  // 32 bytes per node, lazily allocated
    lbm_batch* batch = nullptr;
};

struct lbm_batch {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<lbm_ctx*> members;
    Inst* insts = nullptr;
    Unit* units = nullptr;
    unsigned* sched = nullptr;
    int n_units = 0, grid = 1, threads = 128, rows = 64, prec = -1, walls = 0, staged = 0;
    // tile chosen by lbm_batch_autotune (kept across attach / detach)
    int tuned = 0, t_threads = 128, t_rows = 64, t_staged = 0;
    PhysD phys;
    lbm_params params;
    cudaGraphExec_t graph = nullptr;
    int* err_dev = nullptr;            // members' error words, gathered by lbm_batch_errors_async
    // pinned staging ring for the unit-list uploads of batch_rebuild: a slot
    // is reused only after its previous upload (event) has completed, so a
    // rebuild never waits for the work already queued on the batch stream
    static constexpr int kStage = 4;
    void* stage[kStage] = {};
    size_t stage_bytes[kStage] = {};
    cudaEvent_t stage_ev[kStage] = {};
    int stage_next = 0;
};

// a context attached to a batch is stepped on the batch's stream: wait for it
// before reading the state on the context's own stream
static void ctx_settle(lbm_ctx* c) {
    if (c->batch) cudaStreamSynchronize(c->batch->stream);
}

static int set_err(lbm_ctx* c, int code, const char* msg) {
    if (c) c->err = msg;
    return code;
}

static int cuda_err(lbm_ctx* c, cudaError_t e, const char* where) {
    if (e == cudaSuccess) return LBM_OK;
    if (c) c->err = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
}

static int map_device_err(int bits) {
    // a wait that ran out comes first: it can be the cause of the others
    if (bits & ERR_TIMEOUT) return LBM_ETIMEOUT;
    if (bits & ERR_PSI) return LBM_EPSI;
    if (bits & ERR_NONFINITE) return LBM_ENONFINITE;
    return LBM_OK;
}

static void drop_graph(cudaGraphExec_t* g) {
    if (*g) cudaGraphExecDestroy(*g);
    *g = nullptr;
}

// (re)builds the unit list and persistent grid of a context for its tile and
// load path (staged: bulk-copy staging of the FP32 rows where eligible)
static int ctx_apply_tile(lbm_ctx* c, int threads, int rows, int staged) {
    staged = staged && stage_eligible(c->inst, c->prec) ? 1 : 0;
    std::vector<Unit> us;
    build_units(c->inst, 0, threads, rows, us);
    int ctas = 1;
    size_t smem = 0;
    if (step_occupancy(c->prec, threads, has_walls(c->inst), staged, &ctas, &smem))
        return set_err(c, LBM_ECUDA, "occupancy query failed");
    if (ctas < 1) return set_err(c, LBM_EINVAL, "tile does not fit on an SM");
    cudaStreamSynchronize(c->stream);
    if (c->units) cudaFree(c->units);
    c->units = nullptr;
    cudaError_t e = cudaMalloc(&c->units, us.size() * sizeof(Unit));
    if (e != cudaSuccess) return cuda_err(c, e, "cudaMalloc(units)");
    e = cudaMemcpy(c->units, us.data(), us.size() * sizeof(Unit), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_err(c, e, "cudaMemcpy(units)");
    c->n_units = (int)us.size();
    c->grid = (int)std::min<long long>((long long)c->n_units, (long long)ctas * num_sms());
    c->threads = threads;
    c->rows = rows;
    c->staged = staged;
    drop_graph(&c->graph);
    return LBM_OK;
}

static StepLaunch ctx_launch(const lbm_ctx* c) {
    StepLaunch L;
    L.insts = c->inst_dev;
    L.units = c->units;
    L.n_units = c->n_units;
    L.n_inst = 1;
    L.sched = c->sched;
    L.grid = c->grid;
    L.walls = has_walls(c->inst) ? 1 : 0;
    L.staged = c->staged;
    L.wait_probe = c->wait_probe;
    L.targets = c->target > 0 ? 1 : 0;
    L.phys = c->phys;
    return L;
}

static int enqueue_steps(cudaStream_t st, cudaGraphExec_t* graph, const StepLaunch& L, int prec,
                         int threads, int n, lbm_ctx* errctx) {
    if (n >= kGraphLen) {
        if (!*graph) {
            cudaGraph_t g;
            cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cuda_err(errctx, e, "cudaStreamBeginCapture");
            for (int i = 0; i < kGraphLen; ++i) step_launch(prec, threads, L, st);
            e = cudaStreamEndCapture(st, &g);
            if (e != cudaSuccess) return cuda_err(errctx, e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                *graph = nullptr;
                return cuda_err(errctx, e, "cudaGraphInstantiate");
            }
        }
        for (int i = 0; i < n / kGraphLen; ++i) {
            cudaError_t e = cudaGraphLaunch(*graph, st);
            if (e != cudaSuccess) return cuda_err(errctx, e, "cudaGraphLaunch");
        }
        n %= kGraphLen;
    }
    for (int i = 0; i < n; ++i)
        if (step_launch(prec, threads, L, st)) return cuda_err(errctx, cudaGetLastError(), "step launch");
    return LBM_OK;
}

static int ctx_read_ctl(lbm_ctx* c, Ctl* out) {
    cudaError_t e = cudaMemcpyAsync(out, c->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_err(c, e, "reading the control block");
}

static int ctx_check(lbm_ctx* c) {
    Ctl h;
    int rc = ctx_read_ctl(c, &h);
    if (rc) return rc;
    if (h.err && c->sticky == LBM_OK) {
        c->sticky = map_device_err(h.err);
        c->err = c->sticky == LBM_ETIMEOUT ? "a bounded wait for a staged row ran out"
                 : c->sticky == LBM_EPSI ? "psi^2 < 0 at some node (density above the EOS range)"
                                         : "non-finite density or temperature";
    }
    return c->sticky;
}

static int ensure_fields(lbm_ctx* c) {
    if (c->fields) return LBM_OK;
    const size_t N = (size_t)c->nx * c->ny;
    cudaError_t e = cudaMalloc(&c->fields, 5 * N * sizeof(double));
    if (e != cudaSuccess) {
        c->fields = nullptr;
        return cuda_err(c, e, "cudaMalloc(fields)");
    }
    e = cudaMalloc(&c->diag_scratch, diag_scratch_bytes((long long)N));
    if (e == cudaSuccess) e = cudaMemset(c->diag_scratch, 0, diag_scratch_bytes((long long)N));
    if (e == cudaSuccess) e = cudaMalloc(&c->diag_out, 16 * sizeof(double));
    return cuda_err(c, e, "cudaMalloc(diagnostics)");
}

extern "C" {

int lbm_default_params(lbm_params* p) {
    if (!p) return LBM_EINVAL;
    memset(p, 0, sizeof(*p));
    p->a = 3.0 / 49.0;
    p->b = 2.0 / 21.0;
    p->R = 1.0;
    p->omega = 0.344;
    p->G = -1.0;
    p->sigma = 1.25;
    p->nu = 0.1;
    p->s0 = p->s_e = p->s_eps = p->s_j = p->s_q = 1.0;
    p->lambda = 1.0 / 3.0;
    p->cv = 5.0;
    p->w_dot = 2.0 / 3.0;
    p->vs0 = p->vs3 = p->vs4 = 1.0;
    return LBM_OK;
}

size_t lbm_state_bytes(int nx, int ny, int prec) {
    if (nx < 1 || ny < 1 || prec < 0 || prec > 2) return 0;
    return layout_for(nx, ny, prec).total;
}

int lbm_create(int nx, int ny, const lbm_params* params, const lbm_bc* bc, int prec,
               void* stream, void* device_mem, size_t device_bytes, lbm_ctx** out) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (nx < 1 || ny < 1 || !params || !bc || prec < 0 || prec > 2) return LBM_EINVAL;
    if (nx > (1 << 20) || ny > (1 << 20)) return LBM_EINVAL;
    // the kernels address the 9 planes of f with 32-bit element offsets
    if ((unsigned long long)layout_for(nx, ny, prec).pitch * ny * 9ull >= (1ull << 31)) return LBM_EINVAL;
    if (!bc_valid(nx, ny, bc) || !params_valid(params)) return LBM_EINVAL;
    if (device_mem && ((uintptr_t)device_mem % kAlign || device_bytes < lbm_state_bytes(nx, ny, prec)))
        return LBM_EINVAL;
    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return LBM_ENOMEM;
    c->nx = nx;
    c->ny = ny;
    c->prec = prec;
    c->params = *params;
    c->bc = *bc;
    c->phys = phys_from(params);
    c->lay = layout_for(nx, ny, prec);
    cudaError_t e = cudaSuccess;
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        c->own_stream = e == cudaSuccess;
    }
    if (e == cudaSuccess) {
        if (device_mem) {
            c->mem = device_mem;
        } else {
            e = cudaMalloc(&c->mem, c->lay.total);
            c->own_mem = e == cudaSuccess;
        }
    }
    if (e == cudaSuccess) e = cudaMalloc(&c->small, round_up(sizeof(Ctl), kAlign) + round_up(sizeof(Inst), kAlign) + kAlign);
    if (e != cudaSuccess) {
        int rc = e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
        lbm_destroy(c);
        return rc;
    }
    char* sp = (char*)c->small;
    c->ctl = (Ctl*)sp;
    c->inst_dev = (Inst*)(sp + round_up(sizeof(Ctl), kAlign));
    c->sched = (unsigned*)(sp + round_up(sizeof(Ctl), kAlign) + round_up(sizeof(Inst), kAlign));
    char* m = (char*)c->mem;
    Inst& I = c->inst;
    memset(&I, 0, sizeof(I));
    for (int p = 0; p < 2; ++p) {
        I.f[p] = m + p * 9 * c->lay.planeF;
        I.g[p] = m + 18 * c->lay.planeF + p * 5 * c->lay.planeG;
        I.P[p] = m + 18 * c->lay.planeF + 10 * c->lay.planeG + p * c->lay.planeP;
    }
    I.ctl = c->ctl;
    I.nx = nx;
    I.ny = ny;
    I.own_y0 = 0;
    I.own_y1 = ny;
    // the plane stride used by the kernels is ny * pitch elements: keep the
    // rounded plane sizes consistent with it
    I.pitch = c->lay.pitch;
    for (int k = 0; k < 4; ++k) {
        I.flow[k] = bc->flow[k];
        I.therm[k] = bc->therm[k];
        I.T_edge[k] = bc->T_edge[k];
    }
    I.heater_x0 = bc->heater_x0;
    I.heater_x1 = bc->heater_x1;
    I.T_heater = bc->T_heater;
    I.cot_theta = tan(M_PI / 2.0 - bc->theta_deg * M_PI / 180.0);
    I.rho_ref = params->rho_ref > 0 ? params->rho_ref : 1.0;
    I.T_ref = params->T_ref > 0 ? params->T_ref : 0.0;
    I.inv_n = 1.0 / ((double)nx * ny);
    e = cudaMemset(c->small, 0, round_up(sizeof(Ctl), kAlign) + round_up(sizeof(Inst), kAlign) + kAlign);
    if (e == cudaSuccess) e = cudaMemcpy(c->inst_dev, &I, sizeof(Inst), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        int rc = cuda_err(c, e, "lbm_create");
        lbm_destroy(c);
        return rc;
    }
    auto it = tune_cache().find(std::make_tuple(prec, nx, ny));
    const Inst* Ip = &I;
    int staged = default_staged(&Ip, 1, prec) ? 1 : 0, threads = default_threads(staged), rows = 0;
    if (it != tune_cache().end()) {
        threads = it->second.threads;
        rows = it->second.rows;
        staged = it->second.staged;
    } else {
        rows = default_rows(prec, threads, (bc->flow[2] == LBM_WALL || bc->flow[3] == LBM_WALL) ? 1 : 0,
                            staged, nx, ny);
    }
    int rc = ctx_apply_tile(c, threads, rows, staged);
    if (rc) {
        lbm_destroy(c);
        return rc;
    }
    *out = c;
    return LBM_OK;
}

static int ctx_upload_inst(lbm_ctx* c) {
    cudaError_t e = cudaMemcpyAsync(c->inst_dev, &c->inst, sizeof(Inst), cudaMemcpyHostToDevice, c->stream);
    return cuda_err(c, e, "uploading the domain descriptor");
}

int lbm_init_fields(lbm_ctx* c, const double* rho, const double* ux, const double* uy,
                    const double* T) {
    if (!c || !rho || !ux || !uy || !T) return LBM_EINVAL;
    if (c->batch) return set_err(c, LBM_ESTATE, "context is attached to a batch");
    const size_t N = (size_t)c->nx * c->ny;
    int rc = ensure_fields(c);
    if (rc) return rc;
    const double* src[4] = {rho, ux, uy, T};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(c->fields + k * N, src[k], N * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "copying the initial fields");
    // sum rho and sum T on the device (fixed summation order): the storage
    // references and the first step's mean density
    double sums[2];
    if (sum2_launch(c->fields, c->fields + 3 * N, (long long)N, c->diag_out + 8, c->diag_scratch,
                    c->stream))
        return cuda_err(c, cudaGetLastError(), "field sums");
    e = cudaMemcpyAsync(sums, c->diag_out + 8, sizeof(sums), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "field sums");
    const double sr = sums[0], sT = sums[1];
    c->inst.rho_ref = c->params.rho_ref > 0 ? c->params.rho_ref : sr / (double)N;
    c->inst.T_ref = c->params.T_ref > 0 ? c->params.T_ref : sT / (double)N;
    if ((rc = ctx_upload_inst(c))) return rc;
    if (init_launch(c->prec, c->inst_dev, c->inst, c->fields, c->fields + N, c->fields + 2 * N,
                    c->fields + 3 * N, c->params.w_dot, c->stream))
        return cuda_err(c, cudaGetLastError(), "init kernel");
    // state at t = 0: step 0 reads the initial mean density (slot 2)
    Ctl h;
    memset(&h, 0, sizeof(h));
    h.mass[2] = sr;
    e = cudaMemcpyAsync(c->ctl, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "lbm_init_fields");
    c->step = 0;
    c->target = 0;
    c->sticky = LBM_OK;
    c->initialized = true;
    c->err.clear();
    return LBM_OK;
}

// the step count after n more launches: a domain stops at its target
static long long step_after(const lbm_ctx* c, int n) {
    const long long s = c->step + n;
    return c->target > 0 ? std::min(s, std::max(c->step, c->target)) : s;
}

__global__ void k_set_target(Ctl* ctl, long long target) { ctl->target = target; }

int lbm_set_target(lbm_ctx* c, long long target) {
    if (!c || target < 0) return LBM_EINVAL;
    if (!c->initialized) return set_err(c, LBM_ESTATE, "lbm_set_target before lbm_init_fields");
    // in stream order with the steps that read it: the batch's stream while
    // the context is attached
    k_set_target<<<1, 1, 0, c->batch ? c->batch->stream : c->stream>>>(c->ctl, target);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(c, e, "lbm_set_target");
    // the launches carry whether any domain has a target: captured graphs
    // are rebuilt when that can change
    if ((c->target > 0) != (target > 0)) {
        drop_graph(&c->graph);
        if (c->batch) drop_graph(&c->batch->graph);
    }
    c->target = target;
    return LBM_OK;
}

int lbm_step(lbm_ctx* c, int n) {
    if (!c || n < 0) return LBM_EINVAL;
    if (!c->initialized) return set_err(c, LBM_ESTATE, "lbm_step before lbm_init_fields");
    if (c->batch) return set_err(c, LBM_ESTATE, "context is attached to a batch");
    if (c->sticky) return c->sticky;
    if (n == 0) return LBM_OK;
    int rc = enqueue_steps(c->stream, &c->graph, ctx_launch(c), c->prec, c->threads, n, c);
    if (rc == LBM_OK) c->step = step_after(c, n);
    return rc;
}

int lbm_sync(lbm_ctx* c) {
    if (!c) return LBM_EINVAL;
    if (!c->initialized) return LBM_OK;
    return ctx_check(c);
}

int lbm_get_rho_u_T(lbm_ctx* c, double* rho, double* ux, double* uy, double* T) {
    if (!c) return LBM_EINVAL;
    if (!c->initialized) return set_err(c, LBM_ESTATE, "no state yet");
    ctx_settle(c);
    int rc = ensure_fields(c);
    if (rc) return rc;
    const size_t N = (size_t)c->nx * c->ny;
    if (fields_launch(c->prec, c->inst_dev, c->inst, c->phys, c->fields, c->fields + N,
                      c->fields + 2 * N, c->fields + 3 * N, c->fields + 4 * N, c->stream))
        return cuda_err(c, cudaGetLastError(), "fields kernel");
    double* dst[4] = {rho, ux, uy, T};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
        if (dst[k])
            e = cudaMemcpyAsync(dst[k], c->fields + k * N, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "copying fields to the host");
    return ctx_check(c);
}

int lbm_diagnostics(lbm_ctx* c, double rho_l, double rho_g, int sessile, lbm_diag* out) {
    if (!c || !out || !(rho_l > rho_g)) return LBM_EINVAL;
    if (!c->initialized) return set_err(c, LBM_ESTATE, "no state yet");
    ctx_settle(c);
    int rc = ensure_fields(c);
    if (rc) return rc;
    const size_t N = (size_t)c->nx * c->ny;
    if (fields_launch(c->prec, c->inst_dev, c->inst, c->phys, c->fields, c->fields + N,
                      c->fields + 2 * N, c->fields + 3 * N, c->fields + 4 * N, c->stream))
        return cuda_err(c, cudaGetLastError(), "fields kernel");
    if (diag_launch(c->fields, c->fields + N, c->fields + 2 * N, c->fields + 3 * N, (long long)N,
                    c->params.cv, rho_l, rho_g, c->diag_out, c->diag_scratch, c->stream))
        return cuda_err(c, cudaGetLastError(), "diagnostics kernel");
    double h[8];
    cudaError_t e = cudaMemcpyAsync(h, c->diag_out, 7 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "diagnostics");
    out->mass = h[0];
    out->energy = h[1];
    out->liquid_mass = h[2];
    out->liquid_area = h[3];
    out->liquid_area_smooth = h[4];
    out->max_u = h[5];
    out->nonfinite = (int)h[6];
    const double fac = sessile ? 8.0 / M_PI : 4.0 / M_PI;
    out->diameter = sqrt(fac * out->liquid_area);
    out->diameter_smooth = sqrt(fac * out->liquid_area_smooth);
    out->step = c->step;
    return ctx_check(c);
}

int lbm_get_populations(lbm_ctx* c, double* f, double* g, double* P) {
    if (!c) return LBM_EINVAL;
    if (!c->initialized) return set_err(c, LBM_ESTATE, "no state yet");
    ctx_settle(c);
    const size_t N = (size_t)c->nx * c->ny;
    double* buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, 15 * N * sizeof(double));
    if (e != cudaSuccess) return cuda_err(c, e, "cudaMalloc(populations)");
    const int par = (int)(c->step & 1);
    int rc = LBM_OK;
    if (pop_get_launch(c->prec, c->inst, par, c->params.w_dot, buf, buf + 9 * N, buf + 14 * N, c->stream))
        rc = cuda_err(c, cudaGetLastError(), "population kernel");
    if (!rc && f) e = cudaMemcpyAsync(f, buf, 9 * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (!rc && g && e == cudaSuccess)
        e = cudaMemcpyAsync(g, buf + 9 * N, 5 * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (!rc && P && e == cudaSuccess)
        e = cudaMemcpyAsync(P, buf + 14 * N, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(buf);
    if (!rc) rc = cuda_err(c, e, "copying populations");
    return rc ? rc : ctx_check(c);
}

int lbm_set_populations(lbm_ctx* c, const double* f, const double* g, const double* P,
                        long long step, double rho_ave_prev) {
    if (!c || !f || !g || !P || step < 0) return LBM_EINVAL;
    if (c->batch) return set_err(c, LBM_ESTATE, "context is attached to a batch");
    const size_t N = (size_t)c->nx * c->ny;
    if (!c->initialized) {
        // storage references from the given state
        double sr = 0.0, sT = 0.0;
        for (size_t n = 0; n < N; ++n) {
            double r = 0.0, t = 0.0;
            for (int i = 0; i < 9; ++i) r += f[i * N + n];
            for (int i = 0; i < 5; ++i) t += g[i * N + n];
            sr += r;
            sT += t;
        }
        c->inst.rho_ref = c->params.rho_ref > 0 ? c->params.rho_ref : sr / (double)N;
        c->inst.T_ref = c->params.T_ref > 0 ? c->params.T_ref : sT / (double)N;
    }
    double* buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, 15 * N * sizeof(double));
    if (e != cudaSuccess) return cuda_err(c, e, "cudaMalloc(populations)");
    e = cudaMemcpyAsync(buf, f, 9 * N * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(buf + 9 * N, g, 5 * N * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(buf + 14 * N, P, N * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    int rc = cuda_err(c, e, "copying populations");
    if (!rc) rc = ctx_upload_inst(c);
    if (!rc && pop_set_launch(c->prec, c->inst, (int)(step & 1), c->params.w_dot, buf, buf + 9 * N,
                              buf + 14 * N, c->stream))
        rc = cuda_err(c, cudaGetLastError(), "population kernel");
    Ctl h;
    memset(&h, 0, sizeof(h));
    h.step = step;
    h.mass[(step + 2) % 3] = rho_ave_prev * (double)N;
    if (!rc) rc = cuda_err(c, cudaMemcpyAsync(c->ctl, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream), "ctl");
    if (!rc) rc = cuda_err(c, cudaStreamSynchronize(c->stream), "lbm_set_populations");
    cudaFree(buf);
    if (rc) return rc;
    c->step = step;
    c->target = 0;
    c->sticky = LBM_OK;
    c->initialized = true;
    c->err.clear();
    return LBM_OK;
}

long long lbm_step_count(const lbm_ctx* c) { return c ? c->step : -1; }

// ---- checkpoint ---------------------------------------------------------
namespace {
struct CkptHeader {
    char magic[8];
    int version, nx, ny, prec, pitch, pad;
    long long step;
    unsigned long long bytes;
    double mass[3], rho_ref, T_ref;
    lbm_params params;
    lbm_bc bc;
};
}  // namespace

static size_t ckpt_payload(const lbm_ctx* c) {
    return 9 * c->lay.planeF + 5 * c->lay.planeG + c->lay.planeP;
}

// ---------------------------------------------------------------------------
// one domain split into slabs of rows: halo rows between slabs and the
// combined density sum behind rho_ave

size_t lbm_rows_bytes(const lbm_ctx* c, int n) {
    if (!c || n < 0) return 0;
    return (size_t)n * c->nx * (9 * elem_f(c->prec) + 5 * elem_g(c->prec) + elem_P(c->prec));
}

// copies rows [y0, y0 + n) of every state plane (f 0..8, g 0..4, P) between
// the current state and a packed buffer [plane][row][nx], on the ctx stream
static int rows_copy(lbm_ctx* c, int y0, int n, void* buf, bool pack) {
    if (!c || !buf || n < 0 || y0 < 0 || y0 + n > c->ny) return LBM_EINVAL;
    if (!c->initialized) return set_err(c, LBM_ESTATE, "no state yet");
    if (c->batch) return set_err(c, LBM_ESTATE, "context is attached to a batch");
    if (n == 0) return LBM_OK;
    const int par = (int)(c->step & 1);
    const size_t ef = elem_f(c->prec), eg = elem_g(c->prec), ep = elem_P(c->prec);
    char* b = (char*)buf;
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < 15 && e == cudaSuccess; ++q) {
        const size_t es = q < 9 ? ef : (q < 14 ? eg : ep);
        char* plane = q < 9 ? (char*)c->inst.f[par] + q * c->lay.planeF
                            : (q < 14 ? (char*)c->inst.g[par] + (q - 9) * c->lay.planeG
                                      : (char*)c->inst.P[par]);
        char* rows = plane + (size_t)y0 * c->lay.pitch * es;
        const size_t spitch = (size_t)c->lay.pitch * es, w = (size_t)c->nx * es;
        if (pack)
            e = cudaMemcpy2DAsync(b, w, rows, spitch, w, n, cudaMemcpyDeviceToDevice, c->stream);
        else
            e = cudaMemcpy2DAsync(rows, spitch, b, w, w, n, cudaMemcpyDeviceToDevice, c->stream);
        b += w * n;
    }
    return cuda_err(c, e, pack ? "lbm_pack_rows" : "lbm_unpack_rows");
}

int lbm_pack_rows(lbm_ctx* c, int y0, int n, void* dev_buf) { return rows_copy(c, y0, n, dev_buf, true); }

int lbm_unpack_rows(lbm_ctx* c, int y0, int n, const void* dev_buf) {
    return rows_copy(c, y0, n, const_cast<void*>(dev_buf), false);
}

int lbm_set_partition(lbm_ctx* c, int own_y0, int own_y1, long long global_nodes) {
    if (!c || own_y0 < 0 || own_y1 > c->ny || own_y0 >= own_y1 ||
        global_nodes < (long long)c->nx * (own_y1 - own_y0))
        return LBM_EINVAL;
    if (c->batch) return set_err(c, LBM_ESTATE, "context is attached to a batch");
    c->inst.own_y0 = own_y0;
    c->inst.own_y1 = own_y1;
    c->inst.inv_n = 1.0 / (double)global_nodes;
    drop_graph(&c->graph);
    return ctx_upload_inst(c);
}

int lbm_mass_ring(lbm_ctx* c, double** dev_ring) {
    if (!c || !dev_ring) return LBM_EINVAL;
    *dev_ring = c->ctl->mass;
    return LBM_OK;
}

int lbm_save(lbm_ctx* c, const char* path) {
    if (!c || !path) return LBM_EINVAL;
    if (!c->initialized) return set_err(c, LBM_ESTATE, "no state yet");
    ctx_settle(c);
    int rc = ctx_check(c);
    if (rc) return rc;
    Ctl h;
    if ((rc = ctx_read_ctl(c, &h))) return rc;
    const int par = (int)(c->step & 1);
    const size_t bytes = ckpt_payload(c);
    std::vector<char> buf(bytes);
    cudaError_t e = cudaMemcpy(buf.data(), c->inst.f[par], 9 * c->lay.planeF, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(buf.data() + 9 * c->lay.planeF, c->inst.g[par], 5 * c->lay.planeG, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(buf.data() + 9 * c->lay.planeF + 5 * c->lay.planeG, c->inst.P[par], c->lay.planeP,
                       cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(c, e, "lbm_save");
    CkptHeader hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.magic, "LBMGB300", 8);
    hd.version = 1;
    hd.nx = c->nx;
    hd.ny = c->ny;
    hd.prec = c->prec;
    hd.pitch = c->lay.pitch;
    hd.step = c->step;
    hd.bytes = bytes;
    for (int k = 0; k < 3; ++k) hd.mass[k] = h.mass[k];
    hd.rho_ref = c->inst.rho_ref;
    hd.T_ref = c->inst.T_ref;
    hd.params = c->params;
    hd.bc = c->bc;
    uint32_t crc = crc32_update(0, &hd, sizeof(hd));
    crc = crc32_update(crc, buf.data(), bytes);
    FILE* fp = fopen(path, "wb");
    if (!fp) return set_err(c, LBM_EIO, "cannot open checkpoint for writing");
    bool ok = fwrite(&hd, sizeof(hd), 1, fp) == 1 && fwrite(buf.data(), 1, bytes, fp) == bytes &&
              fwrite(&crc, sizeof(crc), 1, fp) == 1;
    ok = (fclose(fp) == 0) && ok;
    return ok ? LBM_OK : set_err(c, LBM_EIO, "short write to checkpoint");
}

int lbm_load(lbm_ctx* c, const char* path) {
    if (!c || !path) return LBM_EINVAL;
    if (c->batch) return set_err(c, LBM_ESTATE, "context is attached to a batch");
    FILE* fp = fopen(path, "rb");
    if (!fp) return set_err(c, LBM_EIO, "cannot open checkpoint");
    CkptHeader hd;
    const size_t bytes = ckpt_payload(c);
    std::vector<char> buf(bytes);
    uint32_t crc_file = 0;
    bool ok = fread(&hd, sizeof(hd), 1, fp) == 1;
    ok = ok && memcmp(hd.magic, "LBMGB300", 8) == 0 && hd.version == 1 && hd.nx == c->nx &&
         hd.ny == c->ny && hd.prec == c->prec && hd.pitch == c->lay.pitch && hd.bytes == bytes;
    ok = ok && fread(buf.data(), 1, bytes, fp) == bytes && fread(&crc_file, sizeof(crc_file), 1, fp) == 1;
    fclose(fp);
    if (!ok) return set_err(c, LBM_EIO, "checkpoint header or size mismatch");
    uint32_t crc = crc32_update(0, &hd, sizeof(hd));
    crc = crc32_update(crc, buf.data(), bytes);
    if (crc != crc_file) return set_err(c, LBM_EIO, "checkpoint CRC mismatch");
    const int par = (int)(hd.step & 1);
    cudaStreamSynchronize(c->stream);
    cudaError_t e = cudaMemcpy(c->inst.f[par], buf.data(), 9 * c->lay.planeF, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->inst.g[par], buf.data() + 9 * c->lay.planeF, 5 * c->lay.planeG, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->inst.P[par], buf.data() + 9 * c->lay.planeF + 5 * c->lay.planeG, c->lay.planeP,
                       cudaMemcpyHostToDevice);
    c->inst.rho_ref = hd.rho_ref;
    c->inst.T_ref = hd.T_ref;
    Ctl h;
    memset(&h, 0, sizeof(h));
    h.step = hd.step;
    for (int k = 0; k < 3; ++k) h.mass[k] = hd.mass[k];
    if (e == cudaSuccess) e = cudaMemcpy(c->ctl, &h, sizeof(h), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->inst_dev, &c->inst, sizeof(Inst), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_err(c, e, "lbm_load");
    c->step = hd.step;
    c->target = 0;
    c->sticky = LBM_OK;
    c->initialized = true;
    c->err.clear();
    return LBM_OK;
}

void lbm_destroy(lbm_ctx* c) {
    if (!c) return;
    if (c->batch) lbm_batch_detach(c->batch, c);
    if (c->stream) cudaStreamSynchronize(c->stream);
    drop_graph(&c->graph);
    if (c->units) cudaFree(c->units);
    if (c->fields) cudaFree(c->fields);
    if (c->diag_scratch) cudaFree(c->diag_scratch);
    if (c->diag_out) cudaFree(c->diag_out);
    if (c->iface_scratch) cudaFree(c->iface_scratch);
    if (c->region_scratch) cudaFree(c->region_scratch);
    if (c->small) cudaFree(c->small);
    if (c->own_mem && c->mem) cudaFree(c->mem);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char* lbm_last_error(const lbm_ctx* c) {
    if (!c) return "null context";
    return c->err.c_str();
}

// ---- reconfiguration and interface analyses -----------------------------
int lbm_reconfigure(lbm_ctx* c, const lbm_params* params, const lbm_bc* bc) {
    if (!c || !params || !bc) return LBM_EINVAL;
    if (c->batch) return set_err(c, LBM_ESTATE, "context is attached to a batch");
    if (!params_valid(params) || !bc_valid(c->nx, c->ny, bc))
        return set_err(c, LBM_EINVAL, "invalid parameters or boundaries");
    if (params->w_dot != c->params.w_dot) return set_err(c, LBM_EINVAL, "w_dot cannot change");
    for (int e = 0; e < 4; ++e)
        if (bc->flow[e] != c->bc.flow[e]) return set_err(c, LBM_EINVAL, "flow boundary kinds cannot change");
    lbm_params np = *params;
    np.rho_ref = c->params.rho_ref;
    np.T_ref = c->params.T_ref;
    c->params = np;
    c->bc = *bc;
    c->phys = phys_from(&np);
    Inst& I = c->inst;
    for (int k = 0; k < 4; ++k) {
        I.therm[k] = bc->therm[k];
        I.T_edge[k] = bc->T_edge[k];
    }
    I.heater_x0 = bc->heater_x0;
    I.heater_x1 = bc->heater_x1;
    I.T_heater = bc->T_heater;
    I.cot_theta = tan(M_PI / 2.0 - bc->theta_deg * M_PI / 180.0);
    // the captured graph holds the old constants as launch arguments
    drop_graph(&c->graph);
    return ctx_upload_inst(c);
}

int lbm_contact_angle(lbm_ctx* c, double rho_l, double rho_g, int skip_rows, lbm_contact* out) {
    if (!c || !out || !(rho_l > rho_g) || skip_rows < 0) return LBM_EINVAL;
    memset(out, 0, sizeof(*out));
    if (c->bc.flow[LBM_EDGE_S] != LBM_WALL) return set_err(c, LBM_EINVAL, "no south wall");
    if (!c->initialized) return set_err(c, LBM_ESTATE, "no state yet");
    ctx_settle(c);
    int rc = ensure_fields(c);
    if (rc) return rc;
    cudaError_t e = cudaSuccess;
    if (!c->iface_scratch) {
        e = cudaMalloc(&c->iface_scratch, iface_scratch_bytes() + 16 * sizeof(double));
        if (e == cudaSuccess) e = cudaMemset(c->iface_scratch, 0, iface_scratch_bytes() + 16 * sizeof(double));
        if (e != cudaSuccess) {
            if (c->iface_scratch) cudaFree(c->iface_scratch);
            c->iface_scratch = nullptr;
            return cuda_err(c, e, "cudaMalloc(contact-angle scratch)");
        }
    }
    const size_t N = (size_t)c->nx * c->ny;
    double* res = (double*)((char*)c->iface_scratch + iface_scratch_bytes());
    if (fields_launch(c->prec, c->inst_dev, c->inst, c->phys, c->fields, c->fields + N,
                      c->fields + 2 * N, c->fields + 3 * N, c->fields + 4 * N, c->stream) ||
        iface_launch(c->fields, c->nx, c->ny, 0.5 * (rho_l + rho_g), skip_rows, res,
                     c->iface_scratch, c->stream))
        return cuda_err(c, cudaGetLastError(), "contact-angle kernels");
    double h[12];
    e = cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "contact angle");
    rc = ctx_check(c);
    if (rc) return rc;
    const double n = h[0];
    out->n_points = (int)n;
    if (n < 3) return set_err(c, LBM_EINVAL, "fewer than 3 interface points");
    // normal equations of min sum (z + D u + E v + F)^2 about the mean point,
    // solved by Cramer's rule
    const double Su = h[1], Sv = h[2], Suu = h[3], Svv = h[4], Suv = h[5];
    const double Suz = h[6], Svz = h[7], Sz = h[8];
    const double A[3][3] = {{Suu, Suv, Su}, {Suv, Svv, Sv}, {Su, Sv, n}};
    const double b[3] = {-Suz, -Svz, -Sz};
    auto det3 = [](const double M[3][3]) {
        return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
               M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
               M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    };
    const double d = det3(A);
    if (!(fabs(d) > 0.0)) return set_err(c, LBM_EINVAL, "degenerate interface points");
    double sol[3];
    for (int k = 0; k < 3; ++k) {
        double M[3][3];
        for (int r = 0; r < 3; ++r)
            for (int q = 0; q < 3; ++q) M[r][q] = q == k ? b[r] : A[r][q];
        sol[k] = det3(M) / d;
    }
    const double uc = -0.5 * sol[0], vc = -0.5 * sol[1];
    const double R2 = uc * uc + vc * vc - sol[2];
    if (!(R2 > 0.0)) return set_err(c, LBM_EINVAL, "no circle through the interface points");
    const double xm = h[10] / h[9], ym = h[11] / h[9];
    out->xc = xm + uc;
    out->yc = ym + vc;
    out->radius = sqrt(R2);
    const double yw = -0.5;   // halfway bounce-back wall line
    double cs = (yw - out->yc) / out->radius;
    cs = cs < -1.0 ? -1.0 : (cs > 1.0 ? 1.0 : cs);
    out->theta_deg = acos(cs) * (180.0 / M_PI);
    const double hh = R2 - (yw - out->yc) * (yw - out->yc);
    out->base_width = hh > 0.0 ? 2.0 * sqrt(hh) : 0.0;
    out->height = out->yc + out->radius - yw;
    return LBM_OK;
}

int lbm_regions(lbm_ctx* c, double threshold, int below, int* labels, lbm_region* regions,
                int max_regions, int* n_regions) {
    if (!c || !n_regions || max_regions < 0 || (max_regions > 0 && !regions)) return LBM_EINVAL;
    *n_regions = 0;
    if (!c->initialized) return set_err(c, LBM_ESTATE, "no state yet");
    ctx_settle(c);
    int rc = ensure_fields(c);
    if (rc) return rc;
    const long long N = (long long)c->nx * c->ny;
    cudaError_t e = cudaSuccess;
    if (!c->region_scratch) {
        e = cudaMalloc(&c->region_scratch, regions_scratch_bytes(N));
        if (e != cudaSuccess) {
            c->region_scratch = nullptr;
            return cuda_err(c, e, "cudaMalloc(region scratch)");
        }
    }
    int *parent = nullptr, *roots = nullptr, *count = nullptr;
    if (fields_launch(c->prec, c->inst_dev, c->inst, c->phys, c->fields, c->fields + N,
                      c->fields + 2 * N, c->fields + 3 * N, c->fields + 4 * N, c->stream) ||
        regions_launch(c->fields, c->nx, c->ny, c->bc.flow[LBM_EDGE_W] == LBM_PERIODIC,
                       c->bc.flow[LBM_EDGE_S] == LBM_PERIODIC, threshold, below,
                       c->region_scratch, (int)N, &parent, &roots, &count, c->stream))
        return cuda_err(c, cudaGetLastError(), "region kernels");
    int hc[2];
    e = cudaMemcpyAsync(hc, count, sizeof(hc), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && labels)
        e = cudaMemcpyAsync(labels, parent, N * sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "region labels");
    if (hc[1]) return set_err(c, LBM_ECUDA, "region labelling did not converge");
    const int m = hc[0];
    *n_regions = m;
    if (max_regions > 0 && m > 0) {
        RegionOut* dev = nullptr;
        e = cudaMalloc(&dev, (size_t)m * sizeof(RegionOut));
        if (e != cudaSuccess) return cuda_err(c, e, "cudaMalloc(regions)");
        std::vector<RegionOut> h(m);
        if (regions_gather_launch(c->region_scratch, N, m, dev, c->stream)) e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h.data(), dev, (size_t)m * sizeof(RegionOut), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        cudaFree(dev);
        if (e != cudaSuccess) return cuda_err(c, e, "region statistics");
        std::sort(h.begin(), h.end(), [](const RegionOut& a, const RegionOut& b) { return a.label < b.label; });
        for (int k = 0; k < m && k < max_regions; ++k) {
            lbm_region& r = regions[k];
            r.label = h[k].label;
            r.area = h[k].area;
            r.sum_y = h[k].sum_y;
            r.y_min = h[k].y_min;
            r.y_max = h[k].y_max;
            r.touches_w = (h[k].flags >> 0) & 1;
            r.touches_e = (h[k].flags >> 1) & 1;
            r.touches_s = (h[k].flags >> 2) & 1;
            r.touches_n = (h[k].flags >> 3) & 1;
        }
    }
    return ctx_check(c);
}

// ---- tile / autotune ------------------------------------------------------
int lbm_set_tile(lbm_ctx* c, int threads, int rows) {
    if (!c || (threads != 128 && threads != 192 && threads != 224 && threads != 256) || rows < 1)
        return LBM_EINVAL;
    if (c->batch) return set_err(c, LBM_ESTATE, "context is attached to a batch");
    return ctx_apply_tile(c, threads, std::min(rows, c->ny), c->staged);
}

int lbm_set_staging(lbm_ctx* c, int on) {
    if (!c) return LBM_EINVAL;
    if (c->batch) return set_err(c, LBM_ESTATE, "context is attached to a batch");
    if (on && !stage_eligible(c->inst, c->prec))
        return set_err(c, LBM_EINVAL,
                       "bulk-copy staging needs FP32 storage of f and open x, or periodic x "
                       "with nx >= 32 a multiple of 4 (FP32 g) or 8 (FP16 g)");
    return ctx_apply_tile(c, c->threads, c->rows, on ? 1 : 0);
}

int lbm_get_staging(const lbm_ctx* c) { return c ? c->staged : LBM_EINVAL; }

int lbm_set_wait_probe(lbm_ctx* c, int on) {
    if (!c) return LBM_EINVAL;
    if (c->batch) return set_err(c, LBM_ESTATE, "context is attached to a batch");
    c->wait_probe = on ? 1 : 0;
    drop_graph(&c->graph);
    return LBM_OK;
}

int lbm_get_tile(const lbm_ctx* c, int* threads, int* rows) {
    if (!c) return LBM_EINVAL;
    if (threads) *threads = c->threads;
    if (rows) *rows = c->rows;
    return LBM_OK;
}

int lbm_autotune(lbm_ctx* c, int steps) {
    if (!c || steps < 1) return LBM_EINVAL;
    if (c->batch) return set_err(c, LBM_ESTATE, "context is attached to a batch");
    // a scratch domain of the same size, precision and boundaries in a
    // uniform vapour state, so the caller's state is untouched
    lbm_ctx* s = nullptr;
    int rc = lbm_create(c->nx, c->ny, &c->params, &c->bc, c->prec, nullptr, nullptr, 0, &s);
    if (rc) return set_err(c, rc, "autotune: cannot create the scratch domain");
    const size_t N = (size_t)c->nx * c->ny;
    std::vector<double> rho(N, c->inst.rho_ref > 0 ? c->inst.rho_ref : 1.0), z(N, 0.0),
        T(N, c->inst.T_ref > 0 ? c->inst.T_ref : 0.09);
    rc = lbm_init_fields(s, rho.data(), z.data(), z.data(), T.data());
    if (rc) {
        lbm_destroy(s);
        return set_err(c, rc, "autotune: init failed");
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int bt = c->threads, br = c->rows, bs = c->staged;
    const int thr_c[4] = {128, 192, 224, 256};
    const int n_paths = stage_eligible(c->inst, c->prec) ? 2 : 1;
    for (int si = 0; si < n_paths; ++si)
        for (int ti = 0; ti < 4; ++ti) {
            const int staged = n_paths == 2 ? 1 - si : 0;
            // powers of two, and the heights that fill the grid in 1, 2, 3
            // whole waves
            std::vector<int> rows_c = {16, 32, 64, 128, 256, 512};
            {
                int ctas = 0;
                size_t smem = 0;
                if (step_occupancy(c->prec, thr_c[ti], has_walls(c->inst), staged, &ctas, &smem) ||
                    ctas < 1)
                    continue;
                const long long strips = (c->nx + thr_c[ti] - 9) / (thr_c[ti] - 8);
                for (int w = 1; w <= 3; ++w)
                    rows_c.push_back(wave_rows(c->ny, strips, (long long)ctas * num_sms(), w));
            }
            std::sort(rows_c.begin(), rows_c.end());
            for (int& r : rows_c) r = std::min(r, c->ny);
            rows_c.erase(std::unique(rows_c.begin(), rows_c.end()), rows_c.end());
            for (int rows : rows_c) {
                if (ctx_apply_tile(s, thr_c[ti], rows, staged)) continue;
                lbm_step(s, 2);
                cudaEventRecord(e0, s->stream);
                lbm_step(s, steps);
                cudaEventRecord(e1, s->stream);
                if (cudaEventSynchronize(e1) != cudaSuccess) continue;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) {
                    best = ms;
                    bt = thr_c[ti];
                    br = rows;
                    bs = staged;
                }
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    lbm_destroy(s);
    tune_cache()[std::make_tuple(c->prec, c->nx, c->ny)] = Tile{bt, br, bs};
    return ctx_apply_tile(c, bt, br, bs);
}

// ---- batch ---------------------------------------------------------------
// Rebuilds the batch's instance table and work-unit list after a member
// joined or left.  Stream-ordered: the old device arrays are freed, and the
// new ones allocated and filled, on the batch stream (cudaFreeAsync,
// cudaMallocAsync, copies from a pinned staging slot), so launches already
// queued keep their own arrays and the host does not wait for them.
static int batch_rebuild(lbm_batch* b) {
    drop_graph(&b->graph);
    if (b->insts) cudaFreeAsync(b->insts, b->stream);
    if (b->units) cudaFreeAsync(b->units, b->stream);
    if (b->err_dev) cudaFreeAsync(b->err_dev, b->stream);
    b->insts = nullptr;
    b->units = nullptr;
    b->err_dev = nullptr;
    b->n_units = 0;
    if (b->members.empty()) return LBM_OK;
    std::vector<Inst> hi;
    std::vector<Unit> us;
    b->walls = 0;
    std::vector<const Inst*> ip;
    for (size_t i = 0; i < b->members.size(); ++i) {
        hi.push_back(b->members[i]->inst);
        ip.push_back(&b->members[i]->inst);
        if (has_walls(b->members[i]->inst)) b->walls = 1;
    }
    if (b->tuned) {
        // the autotuned tile; staging only while every member can take it
        bool all = true;
        for (const Inst* I : ip) all = all && stage_eligible(*I, b->prec);
        b->threads = b->t_threads;
        b->rows = b->t_rows;
        b->staged = b->t_staged && all ? 1 : 0;
    } else {
        // bulk-copy staging (224-thread tile) when the members as a whole take it
        b->staged = default_staged(ip.data(), ip.size(), b->prec) ? 1 : 0;
        b->threads = default_threads(b->staged);
    }
    for (size_t i = 0; i < b->members.size(); ++i) {
        build_units(b->members[i]->inst, (int)i, b->threads, std::min(b->rows, b->members[i]->ny), us);
    }
    // longest first: a unit's sweep takes (rows + 6) iterations whatever its
    // width, and the persistent CTAs take units in list order, so the tall
    // units go first and the short ones fill the tail; units of equal height
    // keep domain order, so neighbouring units share halos in L2
    std::stable_sort(us.begin(), us.end(),
                     [](const Unit& a, const Unit& b) { return a.y1 - a.y0 > b.y1 - b.y0; });
    const size_t bi = hi.size() * sizeof(Inst), bu = us.size() * sizeof(Unit);
    const size_t off_u = round_up(bi, kAlign), need = off_u + bu;
    const int slot = b->stage_next;
    b->stage_next = (slot + 1) % lbm_batch::kStage;
    cudaError_t e = cudaSuccess;
    if (b->stage_ev[slot]) e = cudaEventSynchronize(b->stage_ev[slot]);
    else e = cudaEventCreateWithFlags(&b->stage_ev[slot], cudaEventDisableTiming);
    if (e == cudaSuccess && b->stage_bytes[slot] < need) {
        if (b->stage[slot]) cudaFreeHost(b->stage[slot]);
        b->stage[slot] = nullptr;
        b->stage_bytes[slot] = 0;
        e = cudaMallocHost(&b->stage[slot], need);
        if (e == cudaSuccess) b->stage_bytes[slot] = need;
    }
    if (e == cudaSuccess) {
        char* st = (char*)b->stage[slot];
        memcpy(st, hi.data(), bi);
        memcpy(st + off_u, us.data(), bu);
        e = cudaMallocAsync((void**)&b->insts, bi, b->stream);
    }
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&b->units, bu, b->stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&b->err_dev, hi.size() * sizeof(int), b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->insts, b->stage[slot], bi, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->units, (char*)b->stage[slot] + off_u, bu, cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->stage_ev[slot], b->stream);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
    b->n_units = (int)us.size();
    int ctas = 1;
    size_t smem = 0;
    step_occupancy(b->prec, b->threads, b->walls, b->staged, &ctas, &smem);
    b->grid = (int)std::min<long long>((long long)b->n_units, (long long)std::max(ctas, 1) * num_sms());
    return LBM_OK;
}

// makes `waiter` wait for the work queued so far on `first` (no host wait)
static cudaError_t stream_after(cudaStream_t waiter, cudaStream_t first) {
    if (waiter == first) return cudaSuccess;
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(ev, first);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(waiter, ev, 0);
    cudaEventDestroy(ev);
    return e;
}

// error words of a batch's members (attach order) -> out
__global__ void k_gather_err(const Inst* insts, int n, int* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = insts[i].ctl->err;
}

int lbm_batch_create(void* stream, lbm_batch** out) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ENOMEM;
    cudaError_t e = cudaSuccess;
    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        b->own_stream = e == cudaSuccess;
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->sched, 2 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(b->sched, 0, 2 * sizeof(unsigned));
    if (e != cudaSuccess) {
        lbm_batch_destroy(b);
        return LBM_ECUDA;
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_attach(lbm_batch* b, lbm_ctx* c) {
    if (!b || !c) return LBM_EINVAL;
    if (c->batch) return set_err(c, LBM_ESTATE, "context already in a batch");
    if (!c->initialized) return set_err(c, LBM_ESTATE, "attach after lbm_init_fields");
    if (b->members.empty()) {
        b->prec = c->prec;
        b->params = c->params;
        b->phys = c->phys;
        b->threads = 128;
        b->rows = 64;
    } else if (b->prec != c->prec || !same_physics(b->params, c->params)) {
        return set_err(c, LBM_EINVAL, "batch members must share precision and physics");
    }
    // the batch stream waits for the context's queued work (its
    // initialisation); the host waits for neither stream
    cudaError_t e = stream_after(b->stream, c->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "lbm_batch_attach");
    b->members.push_back(c);
    c->batch = b;
    int rc = batch_rebuild(b);
    if (rc) {
        b->members.pop_back();
        c->batch = nullptr;
        batch_rebuild(b);
    }
    return rc;
}

int lbm_batch_detach(lbm_batch* b, lbm_ctx* c) {
    if (!b || !c || c->batch != b) return LBM_EINVAL;
    // the context's own stream waits for the batch's steps queued so far, so
    // whatever it does next sees the state they leave; the host does not wait
    cudaError_t e = stream_after(c->stream, b->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "lbm_batch_detach");
    b->members.erase(std::remove(b->members.begin(), b->members.end(), c), b->members.end());
    c->batch = nullptr;
    return batch_rebuild(b);
}

int lbm_batch_errors_async(lbm_batch* b, int* host_out) {
    if (!b || !host_out) return LBM_EINVAL;
    const int n = (int)b->members.size();
    if (n == 0) return LBM_OK;
    k_gather_err<<<(n + 127) / 128, 128, 0, b->stream>>>(b->insts, n, b->err_dev);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host_out, b->err_dev, n * sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

int lbm_batch_size(const lbm_batch* b) { return b ? (int)b->members.size() : 0; }

int lbm_batch_step(lbm_batch* b, int n) {
    if (!b || n < 0) return LBM_EINVAL;
    if (b->members.empty() || n == 0) return LBM_OK;
    for (lbm_ctx* c : b->members)
        if (c->sticky) return c->sticky;
    StepLaunch L;
    L.insts = b->insts;
    L.units = b->units;
    L.n_units = b->n_units;
    L.n_inst = (int)b->members.size();
    L.sched = b->sched;
    L.grid = b->grid;
    L.walls = b->walls;
    L.staged = b->staged;
    L.wait_probe = 0;
    L.targets = 0;
    for (lbm_ctx* c : b->members) L.targets |= c->target > 0 ? 1 : 0;
    L.phys = b->phys;
    int rc = enqueue_steps(b->stream, &b->graph, L, b->prec, b->threads, n, b->members[0]);
    if (rc == LBM_OK)
        for (lbm_ctx* c : b->members) c->step = step_after(c, n);
    return rc;
}

int lbm_batch_sync(lbm_batch* b) {
    if (!b) return LBM_EINVAL;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return LBM_ECUDA;
    int first = LBM_OK;
    for (lbm_ctx* c : b->members) {
        Ctl h;
        if (cudaMemcpy(&h, c->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost) != cudaSuccess) return LBM_ECUDA;
        if (h.err && c->sticky == LBM_OK) {
            c->sticky = map_device_err(h.err);
            c->err = "device error in batched step";
        }
        if (c->sticky && first == LBM_OK) first = c->sticky;
    }
    return first;
}

int lbm_batch_get_tile(const lbm_batch* b, int* threads, int* rows, int* staged) {
    if (!b) return LBM_EINVAL;
    if (threads) *threads = b->threads;
    if (rows) *rows = b->rows;
    if (staged) *staged = b->staged;
    return LBM_OK;
}

int lbm_batch_autotune(lbm_batch* b, int steps) {
    if (!b || steps < 1) return LBM_EINVAL;
    if (b->members.empty()) return LBM_OK;
    cudaStreamSynchronize(b->stream);
    // a shadow batch of scratch domains with the members' sizes, precision,
    // boundaries and parameters in a uniform state: the members' states are
    // untouched
    std::vector<lbm_ctx*> sh;
    lbm_batch* s = nullptr;
    int rc = lbm_batch_create(nullptr, &s);
    for (size_t i = 0; rc == LBM_OK && i < b->members.size(); ++i) {
        const lbm_ctx* m = b->members[i];
        lbm_ctx* c = nullptr;
        rc = lbm_create(m->nx, m->ny, &m->params, &m->bc, m->prec, nullptr, nullptr, 0, &c);
        if (rc) break;
        sh.push_back(c);
        const size_t N = (size_t)m->nx * m->ny;
        std::vector<double> rho(N, m->inst.rho_ref > 0 ? m->inst.rho_ref : 1.0), z(N, 0.0),
            T(N, m->inst.T_ref > 0 ? m->inst.T_ref : 0.09);
        rc = lbm_init_fields(c, rho.data(), z.data(), z.data(), T.data());
        if (rc == LBM_OK) rc = lbm_batch_attach(s, c);
    }
    int bt = b->threads, br = b->rows, bs = b->staged;
    if (rc == LBM_OK) {
        bool elig = true;
        for (lbm_ctx* c : sh) elig = elig && stage_eligible(c->inst, c->prec);
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = 1e30f;
        const int thr_c[4] = {128, 192, 224, 256};
        const int rows_c[5] = {16, 32, 64, 128, 256};
        for (int si = 0; si < (elig ? 2 : 1); ++si)
            for (int ti = 0; ti < 4; ++ti)
                for (int ri = 0; ri < 5; ++ri) {
                    const int staged = elig ? 1 - si : 0;
                    s->tuned = 1;
                    s->t_threads = thr_c[ti];
                    s->t_rows = rows_c[ri];
                    s->t_staged = staged;
                    int ctas = 0;
                    size_t smem = 0;
                    if (step_occupancy(s->prec, thr_c[ti], s->walls, staged, &ctas, &smem) ||
                        ctas < 1)
                        continue;
                    if (batch_rebuild(s) != LBM_OK) continue;
                    if (lbm_batch_step(s, 2) != LBM_OK) continue;
                    cudaEventRecord(e0, s->stream);
                    lbm_batch_step(s, steps);
                    cudaEventRecord(e1, s->stream);
                    if (cudaEventSynchronize(e1) != cudaSuccess) continue;
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (ms < best) {
                        best = ms;
                        bt = thr_c[ti];
                        br = rows_c[ri];
                        bs = staged;
                    }
                }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    if (s) lbm_batch_destroy(s);
    for (lbm_ctx* c : sh) lbm_destroy(c);
    if (rc) return rc;
    b->tuned = 1;
    b->t_threads = bt;
    b->t_rows = br;
    b->t_staged = bs;
    return batch_rebuild(b);
}

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (lbm_ctx* c : b->members) c->batch = nullptr;
    b->members.clear();
    drop_graph(&b->graph);
    if (b->stream) {
        if (b->insts) cudaFreeAsync(b->insts, b->stream);
        if (b->units) cudaFreeAsync(b->units, b->stream);
        if (b->err_dev) cudaFreeAsync(b->err_dev, b->stream);
        cudaStreamSynchronize(b->stream);
    }
    for (int k = 0; k < lbm_batch::kStage; ++k) {
        if (b->stage[k]) cudaFreeHost(b->stage[k]);
        if (b->stage_ev[k]) cudaEventDestroy(b->stage_ev[k]);
    }
    if (b->sched) cudaFree(b->sched);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"
