// Interface analyses of the density field, on the device:
//  * the contact angle of a sessile droplet (Section 4.2 relaxes the droplet
//    without evaporation until it shows the prescribed angle, then heats);
//  * the 4-connected regions of the vapour (or liquid) phase, from which the
//    departure of a bubble from the heated wall and its size follow
//    (Section 4.3, the Fritz relation D_d ~ g^-1/2).
//
// Contact angle.  Every lattice link between horizontally or vertically
// adjacent nodes whose densities lie on opposite sides of rho_mid contributes
// one interface point, placed on the link by linear interpolation; links
// with a node below row skip_rows are left out.  Two passes over the field
// accumulate, in double, first the count and mean of the points and then the
// centred moment sums of the algebraic circle fit
//   min sum (u^2 + v^2 + D u + E v + F)^2,  (u, v) = point - mean,
// which the host solves for the circle.  Each pass keeps per-block partials
// and the last block to finish folds them in block order, so the result does
// not depend on scheduling.
//
// Regions.  A union-find over node indices: every node in the phase starts
// as its own root; for each pair of 4-neighbours in the phase (across the
// seams of periodic axes) the two roots are merged by an atomicMin that
// makes the larger root point to the smaller one, so a parent index is never
// above its node's index and every region ends with its smallest node index
// as root.  Loops that chase parents or retry a merge strictly decrease an
// index, so they end within n iterations; they are still capped and report
// an error word instead of running on.  A flattening pass then writes each
// node's root, and a statistics pass accumulates per-root area, row sums,
// row range and edge contacts with atomics (integers only: the result is
// exact and independent of order).
#include "lbm_internal.cuh"

namespace lbm {

namespace {

enum { ANA_BLOCKS = 304, ANA_THREADS = 256, ANA_VALS = 9 };

struct IfaceScratch {
    double partial[ANA_BLOCKS * ANA_VALS];
    double mean[ANA_VALS];
    unsigned ticket;
};

__device__ __forceinline__ void add_point(double* v, int pass, const double* mean, double px,
                                          double py) {
    if (pass == 0) {
        v[0] += 1.0;
        v[1] += px;
        v[2] += py;
    } else {
        const double u = px - mean[1] / mean[0], w = py - mean[2] / mean[0];
        const double z = u * u + w * w;
        v[0] += 1.0;
        v[1] += u;
        v[2] += w;
        v[3] += u * u;
        v[4] += w * w;
        v[5] += u * w;
        v[6] += u * z;
        v[7] += w * z;
        v[8] += z;
    }
}

__global__ void __launch_bounds__(ANA_THREADS)
    k_iface(const double* __restrict__ rho, int nx, int ny, double rho_mid, int skip, int pass,
            double* out, IfaceScratch* sc) {
    __shared__ double red[ANA_VALS][ANA_THREADS / 32];
    __shared__ bool last;
    double v[ANA_VALS] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const double* mean = sc->mean;
    const long long n = (long long)nx * (ny - skip);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = skip + (int)(i / nx);
        const long long c = (long long)y * nx + x;
        const double a = rho[c] - rho_mid;
        if (x + 1 < nx) {
            const double b = rho[c + 1] - rho_mid;
            if ((a >= 0.0) != (b >= 0.0)) add_point(v, pass, mean, x + a / (a - b), (double)y);
        }
        if (y + 1 < ny) {
            const double b = rho[c + nx] - rho_mid;
            if ((a >= 0.0) != (b >= 0.0)) add_point(v, pass, mean, (double)x, y + a / (a - b));
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < ANA_VALS; ++k) {
        double x = v[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[k][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < ANA_VALS) {
        const int k = threadIdx.x;
        double x = red[k][0];
        for (int w = 1; w < ANA_THREADS / 32; ++w) x += red[k][w];
        sc->partial[blockIdx.x * ANA_VALS + k] = x;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&sc->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last && threadIdx.x < ANA_VALS) {
        __threadfence();
        const int k = threadIdx.x;
        double x = __ldcg(&sc->partial[k]);
        for (unsigned b = 1; b < gridDim.x; ++b) x += __ldcg(&sc->partial[b * ANA_VALS + k]);
        if (pass == 0) sc->mean[k] = x;
        else out[k] = x;
        if (pass == 1 && k < 3) out[ANA_VALS + k] = sc->mean[k];
        if (k == 0) sc->ticket = 0u;
    }
}

// ---- regions -----------------------------------------------------------
enum { CC_THREADS = 256 };

struct CCArrays {
    unsigned long long* sum_y;
    int* parent;
    unsigned* area;
    int* y_min;
    int* y_max;
    int* flags;     // bit 0 W, 1 E, 2 S, 3 N
    int* roots;
    int* count;     // [0] roots found, [1] error word
};

__device__ __forceinline__ int find_root(const int* parent, int x, long long cap, int* err) {
    long long it = 0;
    int p = __ldcg(&parent[x]);
    while (p != x) {
        x = p;
        p = __ldcg(&parent[x]);
        if (++it > cap) {
            atomicOr(err, 1);
            break;
        }
    }
    return x;
}

__global__ void k_cc_init(const double* __restrict__ rho, long long n, double thr, int below,
                          CCArrays A) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double r = rho[i];
        const bool in = below ? (r < thr) : (r > thr);
        A.parent[i] = in ? (int)i : -1;
        A.area[i] = 0u;
        A.sum_y[i] = 0ull;
        A.y_min[i] = 0x7fffffff;
        A.y_max[i] = -1;
        A.flags[i] = 0;
    }
}

__device__ void unite(int* parent, int a, int b, long long cap, int* err) {
    for (long long it = 0; it <= cap; ++it) {
        a = find_root(parent, a, cap, err);
        b = find_root(parent, b, cap, err);
        if (a == b) return;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        // link the larger root b under a; if b stopped being a root meanwhile,
        // continue from its new parent
        const int old = atomicMin(&parent[b], a);
        if (old == b) return;
        b = old;
    }
    atomicOr(err, 2);
}

__global__ void k_cc_union(int nx, int ny, int perx, int pery, CCArrays A) {
    const long long n = (long long)nx * ny;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (A.parent[i] < 0) continue;
        const int x = (int)(i % nx), y = (int)(i / nx);
        // east and north neighbours cover every pair once (the seams through
        // x = nx-1 -> 0 and y = ny-1 -> 0 when periodic)
        int xe = x + 1, yn = y + 1;
        if (xe == nx) xe = perx ? 0 : -1;
        if (yn == ny) yn = pery ? 0 : -1;
        if (xe >= 0) {
            const long long j = (long long)y * nx + xe;
            if (j != i && __ldcg(&A.parent[j]) >= 0) unite(A.parent, (int)i, (int)j, n, &A.count[1]);
        }
        if (yn >= 0) {
            const long long j = (long long)yn * nx + x;
            if (j != i && __ldcg(&A.parent[j]) >= 0) unite(A.parent, (int)i, (int)j, n, &A.count[1]);
        }
    }
}

__global__ void k_cc_flatten(long long n, CCArrays A) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        if (A.parent[i] >= 0) A.parent[i] = find_root(A.parent, (int)i, n, &A.count[1]);
}

__global__ void k_cc_stats(int nx, int ny, int max_roots, CCArrays A) {
    const long long n = (long long)nx * ny;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = A.parent[i];
        if (r < 0) continue;
        const int x = (int)(i % nx), y = (int)(i / nx);
        atomicAdd(&A.area[r], 1u);
        atomicAdd(&A.sum_y[r], (unsigned long long)y);
        atomicMin(&A.y_min[r], y);
        atomicMax(&A.y_max[r], y);
        const int f = (x == 0 ? 1 : 0) | (x == nx - 1 ? 2 : 0) | (y == 0 ? 4 : 0) | (y == ny - 1 ? 8 : 0);
        if (f) atomicOr(&A.flags[r], f);
        if (r == (int)i) {
            const int slot = atomicAdd(&A.count[0], 1);
            if (slot < max_roots) A.roots[slot] = r;
        }
    }
}

__global__ void k_cc_gather(const int* roots, int m, CCArrays A, RegionOut* out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    const int r = roots[k];
    RegionOut o;
    o.label = r;
    o.area = A.area[r];
    o.sum_y = (long long)A.sum_y[r];
    o.y_min = A.y_min[r];
    o.y_max = A.y_max[r];
    o.flags = A.flags[r];
    out[k] = o;
}

// sum_y (8n bytes) | parent, area, y_min, y_max, flags, roots (4n each) | count
CCArrays cc_arrays(void* scratch, long long n) {
    char* p = (char*)scratch;
    CCArrays A;
    A.sum_y = (unsigned long long*)p;
    A.parent = (int*)(p + 8 * n);
    A.area = (unsigned*)(p + 12 * n);
    A.y_min = (int*)(p + 16 * n);
    A.y_max = (int*)(p + 20 * n);
    A.flags = (int*)(p + 24 * n);
    A.roots = (int*)(p + 28 * n);
    A.count = (int*)(p + 32 * n);
    return A;
}

int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b > 4096) b = 4096;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

size_t iface_scratch_bytes() { return sizeof(IfaceScratch); }

int iface_launch(const double* rho, int nx, int ny, double rho_mid, int skip, double* out12,
                 void* scratch, cudaStream_t st) {
    if (skip >= ny) skip = ny;
    IfaceScratch* sc = (IfaceScratch*)scratch;
    for (int pass = 0; pass < 2; ++pass)
        k_iface<<<ANA_BLOCKS, ANA_THREADS, 0, st>>>(rho, nx, ny, rho_mid, skip, pass, out12, sc);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

size_t regions_scratch_bytes(long long n) { return (size_t)n * 32 + 64; }

int regions_launch(const double* rho, int nx, int ny, int perx, int pery, double thr, int below,
                   void* scratch, int max_roots, int** parent_out, int** roots_out,
                   int** count_out, cudaStream_t st) {
    const long long n = (long long)nx * ny;
    const CCArrays A = cc_arrays(scratch, n);
    if (cudaMemsetAsync(A.count, 0, 2 * sizeof(int), st) != cudaSuccess) return -1;
    const int g = grid_for(n, CC_THREADS);
    k_cc_init<<<g, CC_THREADS, 0, st>>>(rho, n, thr, below, A);
    k_cc_union<<<g, CC_THREADS, 0, st>>>(nx, ny, perx, pery, A);
    k_cc_flatten<<<g, CC_THREADS, 0, st>>>(n, A);
    k_cc_stats<<<g, CC_THREADS, 0, st>>>(nx, ny, max_roots < n ? max_roots : (int)n, A);
    *parent_out = A.parent;
    *roots_out = A.roots;
    *count_out = A.count;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int regions_gather_launch(void* scratch, long long n, int m, RegionOut* out, cudaStream_t st) {
    const CCArrays A = cc_arrays(scratch, n);
    if (m <= 0) return 0;
    k_cc_gather<<<(m + 127) / 128, 128, 0, st>>>(A.roots, m, A, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace lbm
