// lbm_diag_reduce_noalloc: the diagnostics reduction for callers that cannot
// allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is off limits -- a host
// process whose device memory is owned entirely by another framework's pool
// (a serving stack that pre-reserves the GPU), a real-time loop that cannot
// afford the implicit device synchronisation of cudaMalloc / cudaFree, or a
// plugin that is handed device pointers and a stream and nothing else.  The
// regular lbm_diagnostics path keeps its scratch in memory the context
// allocated; this entry point instead keeps its per-block partial sums in one
// file-scope device array of fixed size that lives as long as the library is
// loaded, so a call allocates nothing.
//
// The array is shared by every call on a device and keeps whatever the last
// call left in it; the ticket that elects the final block is cleared before
// each launch.  Two calls whose kernels overlap on the GPU (different streams
// without ordering) race on the array: order them on one stream.
#include <mutex>

#include "lbm.h"
#include "lbm_internal.cuh"

namespace {

const int NA_THREADS = 256;
const int NA_PER_THREAD = 32;
const long long NA_CHUNK = (long long)NA_THREADS * NA_PER_THREAD;   // nodes per block
const int NA_MAX_BLOCKS = (int)(LBM_NOALLOC_MAX_NODES / NA_CHUNK);  // 4096
const int NA_VALS = 7;
const int NA_STRIDE = 8;                                             // doubles per block

static_assert(LBM_NOALLOC_MAX_NODES % (256 * 32) == 0, "chunk must divide the maximum");

// per-block partial sums (NA_MAX_BLOCKS x 8 doubles) followed by the ticket
static __device__ __align__(256) double g_noalloc_scratch[NA_MAX_BLOCKS * NA_STRIDE + 32];

const int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

__global__ void __launch_bounds__(NA_THREADS)
    k_diag_noalloc(const double* __restrict__ rho, const double* __restrict__ ux,
                   const double* __restrict__ uy, const double* __restrict__ T, long long n,
                   double cv, double rho_l, double rho_g, double* __restrict__ out,
                   double* partial, unsigned* ticket) {
    __shared__ double red[NA_VALS][NA_THREADS / 32];
    __shared__ bool last;
    const double rmid = 0.5 * (rho_l + rho_g);
    double v[NA_VALS] = {0, 0, 0, 0, 0, 0, 0};
    const long long base = (long long)blockIdx.x * NA_CHUNK;
    for (int j = 0; j < NA_PER_THREAD; ++j) {
        const long long i = base + (long long)j * NA_THREADS + threadIdx.x;
        if (i >= n) break;
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
        v[5] = fmax(v[5], sqrt(a * a + b * b));
        v[6] += fin ? 0.0 : 1.0;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < NA_VALS; ++k) {
        double x = v[k];
        for (int o = 16; o > 0; o >>= 1) {
            const double y = __shfl_down_sync(0xffffffffu, x, o);
            x = k == 5 ? fmax(x, y) : x + y;
        }
        if (lane == 0) red[k][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < NA_VALS) {
        const int k = threadIdx.x;
        double x = red[k][0];
        for (int w = 1; w < NA_THREADS / 32; ++w) x = k == 5 ? fmax(x, red[k][w]) : x + red[k][w];
        partial[(size_t)blockIdx.x * NA_STRIDE + k] = x;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last && threadIdx.x < NA_VALS) {
        __threadfence();
        const int k = threadIdx.x;
        double x = __ldcg(&partial[k]);
        for (unsigned b = 1; b < gridDim.x; ++b) {
            const double y = __ldcg(&partial[(size_t)b * NA_STRIDE + k]);
            x = k == 5 ? fmax(x, y) : x + y;
        }
        out[k] = x;
    }
}

// Device address of the scratch array for the current device, looked up once
// per device (the array's host-side name is only a stand-in and must never be
// handed to a kernel).
int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_ECUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return LBM_ECUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return LBM_OK;
}

}  // namespace

extern "C" int lbm_diag_reduce_noalloc(const double* rho, const double* ux, const double* uy,
                                       const double* T, long long n, double cv, double rho_l,
                                       double rho_g, double* out7, void* stream) {
    if (!rho || !ux || !uy || !T || !out7 || n < 0 || !(rho_l > rho_g)) return LBM_EINVAL;
    if (n > LBM_NOALLOC_MAX_NODES) return LBM_ETOOBIG;
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0) {
        // nothing to reduce: every sum, the maximum and the count are zero
        return cudaMemsetAsync(out7, 0, NA_VALS * sizeof(double), st) == cudaSuccess ? LBM_OK
                                                                                     : LBM_ECUDA;
    }
    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    double* partial = (double*)base;
    unsigned* ticket = (unsigned*)(partial + (size_t)NA_MAX_BLOCKS * NA_STRIDE);
    // the array keeps the previous call's contents: the ticket must start at 0
    if (cudaMemsetAsync(ticket, 0, sizeof(unsigned), st) != cudaSuccess) return LBM_ECUDA;
    const int blocks = (int)((n + NA_CHUNK - 1) / NA_CHUNK);
    k_diag_noalloc<<<blocks, NA_THREADS, 0, st>>>(rho, ux, uy, T, n, cv, rho_l, rho_g, out7,
                                                  partial, ticket);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}
