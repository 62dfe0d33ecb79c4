// Dynamics around the polarizable FMM: the short-range repulsive wall and the
// kicks, drifts and kinetic energy of velocity Verlet and of the reversible
// multiple-time-step integrator (Sec. IV.B runs the long-range forces on a
// longer step than the short-range ones).  None of this is part of the FMM:
// the paper's force field has its own short-range terms, which are out of
// scope, and the wall only keeps undamped point dipoles and light opposite
// charges from collapsing onto each other during a run.
//
// The wall: U = sum over pairs closer than r_c = 2^(1/6) sigma of
// 4 eps [(sigma/r)^12 - (sigma/r)^6] + eps (the repulsive part of a
// Lennard-Jones pair, shifted to zero at its minimum), FP64 throughout.
// Neighbours come from a spatial hash of cells of side r_c: every pair closer
// than r_c sits in the same or in adjacent cells.  Each site sums its own
// pairs (no atomics on the forces) over the 27 cells in a fixed order and,
// within a cell, over its members in ascending site index, so that the output
// is bitwise reproducible.
#include <cmath>
#include <new>

#include "internal.cuh"

struct polfmm_wall {
    int64_t cap = 0;      // sites the scratch holds
    int nbucket = 0;      // hash table size, a power of two >= 2 cap
    cudaStream_t stream = nullptr;
    int* count = nullptr;  // [nbucket] members per bucket
    int* start = nullptr;  // [nbucket + 1] exclusive prefix sum of count
    int* scan_part = nullptr;  // per-level block sums of the prefix sum
    int* member = nullptr;     // [cap] site indices, grouped by bucket
    int4* cell = nullptr;      // [cap] cell coordinates and bucket of each site
    double* e_site = nullptr;  // [cap] half the wall energy of each site's pairs
    double* part = nullptr;    // [kWallRedBlocks] partial sums of the energy
};

namespace polfmm {

constexpr int kScanBlock = 1024;
constexpr int kWallRedThreads = 256;
constexpr int kWallRedBlocks = 512;  // fixed, so that the summation order depends on n only

__device__ inline uint32_t wall_bucket(int cx, int cy, int cz, uint32_t mask) {
    // three large odd multipliers and xor: a common spatial hash for integer cells
    return ((uint32_t)cx * 73856093u ^ (uint32_t)cy * 19349663u ^ (uint32_t)cz * 83492791u) & mask;
}

__device__ inline int wall_cell_coord(double x, double inv_rc) {
    double c = floor(x * inv_rc);
    // far beyond any physical coordinate; keeps the integer conversion defined
    c = fmin(fmax(c, -1.0e9), 1.0e9);
    return (int)c;
}

__global__ void wall_count_kernel(const double* __restrict__ x, int64_t n, double inv_rc, uint32_t mask,
                                  int4* __restrict__ cell, int* __restrict__ count) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int cx = wall_cell_coord(x[3 * i], inv_rc), cy = wall_cell_coord(x[3 * i + 1], inv_rc),
        cz = wall_cell_coord(x[3 * i + 2], inv_rc);
    uint32_t b = wall_bucket(cx, cy, cz, mask);
    cell[i] = make_int4(cx, cy, cz, (int)b);
    atomicAdd(&count[b], 1);
}

// exclusive prefix sum of kScanBlock entries per block; the block total goes to part
__global__ void __launch_bounds__(kScanBlock) wall_scan_block_kernel(const int* __restrict__ in, int* __restrict__ out,
                                                                     int* __restrict__ part, int n) {
    __shared__ int warp_tot[kScanBlock / 32];
    int i = blockIdx.x * kScanBlock + threadIdx.x;
    int v = i < n ? in[i] : 0;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int s = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += t;
    }
    if (lane == 31) warp_tot[w] = s;
    __syncthreads();
    if (w == 0) {
        int t = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        warp_tot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    int before = w > 0 ? warp_tot[w - 1] : 0;
    if (i < n) out[i] = before + s - v;
    if (threadIdx.x == kScanBlock - 1) part[blockIdx.x] = before + s;
}

__global__ void wall_scan_add_kernel(int* __restrict__ out, const int* __restrict__ part_scanned, int n) {
    int i = blockIdx.x * kScanBlock + threadIdx.x;
    if (i < n) out[i] += part_scanned[blockIdx.x];
}

__global__ void wall_fill_kernel(int64_t n, const int4* __restrict__ cell, int* __restrict__ start, int nbucket,
                                 int* __restrict__ count, int* __restrict__ member) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i == 0) start[nbucket] = (int)n;  // the end of the last bucket; no thread here reads it
    if (i >= n) return;
    int b = cell[i].w;
    int k = atomicSub(&count[b], 1) - 1;  // count[b] was the bucket's size: k in [0, size)
    member[start[b] + k] = (int)i;
}

// ascending site index within each bucket (buckets hold a handful of sites)
__global__ void wall_order_kernel(int nbucket, const int* __restrict__ start, int* __restrict__ member) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbucket) return;
    int s = start[b], e = start[b + 1];
    for (int k = s + 1; k < e; k++) {
        int v = member[k], m = k - 1;
        while (m >= s && member[m] > v) {
            member[m + 1] = member[m];
            m--;
        }
        member[m + 1] = v;
    }
}

__global__ void wall_pairs_kernel(const double* __restrict__ x, int64_t n, const int4* __restrict__ cell,
                                  const int* __restrict__ start, const int* __restrict__ member, uint32_t mask,
                                  double rc2, double sigma6, double eps4, double eps, double* __restrict__ F,
                                  double* __restrict__ e_site) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int4 ci = cell[i];
    const double xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2];
    double fx = 0.0, fy = 0.0, fz = 0.0, e = 0.0;
    for (int dz = -1; dz <= 1; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                const int cx = ci.x + dx, cy = ci.y + dy, cz = ci.z + dz;
                const uint32_t b = wall_bucket(cx, cy, cz, mask);
                const int s = start[b], t = start[b + 1];
                for (int k = s; k < t; k++) {
                    const int j = member[k];
                    if (j == (int)i) continue;
                    const int4 cj = cell[j];
                    if (cj.x != cx || cj.y != cy || cj.z != cz) continue;  // another cell in the same bucket
                    const double rx = xi - x[3 * j], ry = yi - x[3 * j + 1], rz = zi - x[3 * j + 2];
                    const double r2 = rx * rx + ry * ry + rz * rz;
                    if (!(r2 < rc2)) continue;
                    const double inv_r2 = 1.0 / r2;
                    const double t6 = sigma6 * inv_r2 * inv_r2 * inv_r2;  // (sigma / r)^6
                    e += 0.5 * (eps4 * (t6 * t6 - t6) + eps);
                    const double g = eps4 * (12.0 * t6 * t6 - 6.0 * t6) * inv_r2;  // -dU/dr / r
                    fx += g * rx;
                    fy += g * ry;
                    fz += g * rz;
                }
            }
    F[3 * i] = fx;
    F[3 * i + 1] = fy;
    F[3 * i + 2] = fz;
    e_site[i] = e;
}

// fixed-shape sum: kWallRedBlocks blocks stride over the array, then one block adds
// the partials; the order depends on n only
__device__ inline double block_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = kWallRedThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    return sh[0];
}

__global__ void __launch_bounds__(kWallRedThreads) sum_partial_kernel(const double* __restrict__ a, int64_t n,
                                                                  double* __restrict__ part) {
    __shared__ double sh[kWallRedThreads];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kWallRedThreads + threadIdx.x; i < n; i += (int64_t)kWallRedBlocks * kWallRedThreads)
        s += a[i];
    double t = block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kWallRedThreads) sum_final_kernel(const double* __restrict__ part, double scale,
                                                                double* __restrict__ out) {
    __shared__ double sh[kWallRedThreads];
    double s = 0.0;
    for (int k = threadIdx.x; k < kWallRedBlocks; k += kWallRedThreads) s += part[k];
    double t = block_sum(s, sh);
    if (threadIdx.x == 0) *out = scale * t;
}

// kinetic energy of each site, 1/2 m |v|^2
__global__ void kinetic_site_kernel(const double* __restrict__ v, const double* __restrict__ m, int64_t n,
                                    double* __restrict__ e) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a = v[3 * i], b = v[3 * i + 1], c = v[3 * i + 2];
    e[i] = 0.5 * m[i] * (a * a + b * b + c * c);
}

__global__ void kick_kernel(double* __restrict__ v, const double* __restrict__ F, const double* __restrict__ m,
                            double coef, int64_t n3) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n3) return;
    v[k] += coef * F[k] / m[k / 3];
}

__global__ void drift_kernel(double* __restrict__ x, const double* __restrict__ v, double dt, int64_t n3) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n3) return;
    x[k] += dt * v[k];
}

// exclusive prefix sum of n ints into out (n <= kScanBlock^3), with the block
// sums of each level in part (at least scan_part_need(n) ints)
static size_t scan_part_need(int n) {
    size_t need = 0;
    while (n > 1) {
        n = (n + kScanBlock - 1) / kScanBlock;
        need += (size_t)2 * n;
    }
    return need + 2;
}

static cudaError_t scan_levels(cudaStream_t st, const int* in, int* out, int* part, int n) {
    int nb = (n + kScanBlock - 1) / kScanBlock;
    wall_scan_block_kernel<<<nb, kScanBlock, 0, st>>>(in, out, part, n);
    if (nb > 1) {
        int* part_scanned = part + nb;
        cudaError_t e = scan_levels(st, part, part_scanned, part + 2 * nb, nb);
        if (e != cudaSuccess) return e;
        wall_scan_add_kernel<<<nb, kScanBlock, 0, st>>>(out, part_scanned, n);
    }
    return cudaGetLastError();
}

static void wall_free(polfmm_wall* w) {
    cudaFree(w->count);
    cudaFree(w->start);
    cudaFree(w->scan_part);
    cudaFree(w->member);
    cudaFree(w->cell);
    cudaFree(w->e_site);
    cudaFree(w->part);
}

static int sum_to(cudaStream_t st, const double* a, int64_t n, double scale, double* part, double* out) {
    sum_partial_kernel<<<kWallRedBlocks, kWallRedThreads, 0, st>>>(a, n, part);
    sum_final_kernel<<<1, kWallRedThreads, 0, st>>>(part, scale, out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? POLFMM_OK : cuda_fail(e, "reduction kernel launch");
}

}  // namespace polfmm

using namespace polfmm;

extern "C" POLFMM_API int fmm_wall_create(polfmm_wall** out, int64_t max_sites, void* cuda_stream) {
    if (!out) return POLFMM_ERR_INVALID_ARG;
    *out = nullptr;
    if (max_sites < 1 || max_sites > (int64_t)1 << 28) return POLFMM_ERR_INVALID_ARG;
    polfmm_wall* w = new (std::nothrow) polfmm_wall();
    if (!w) return POLFMM_ERR_OUT_OF_MEMORY;
    w->cap = max_sites;
    w->stream = (cudaStream_t)cuda_stream;
    int nb = kScanBlock;
    while ((int64_t)nb < 2 * max_sites) nb <<= 1;
    w->nbucket = nb;
    bool ok = dev_alloc(reinterpret_cast<void**>(&w->count), sizeof(int) * nb) == cudaSuccess &&
              dev_alloc(reinterpret_cast<void**>(&w->start), sizeof(int) * (nb + 1)) == cudaSuccess &&
              dev_alloc(reinterpret_cast<void**>(&w->scan_part), sizeof(int) * scan_part_need(nb)) == cudaSuccess &&
              dev_alloc(reinterpret_cast<void**>(&w->member), sizeof(int) * max_sites) == cudaSuccess &&
              dev_alloc(reinterpret_cast<void**>(&w->cell), sizeof(int4) * max_sites) == cudaSuccess &&
              dev_alloc(reinterpret_cast<void**>(&w->e_site), sizeof(double) * max_sites) == cudaSuccess &&
              dev_alloc(reinterpret_cast<void**>(&w->part), sizeof(double) * kWallRedBlocks) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        wall_free(w);
        delete w;
        return POLFMM_ERR_OUT_OF_MEMORY;
    }
    *out = w;
    return POLFMM_OK;
}

extern "C" POLFMM_API void fmm_wall_destroy(polfmm_wall* w) {
    if (!w) return;
    cudaStreamSynchronize(w->stream);
    wall_free(w);
    cudaGetLastError();
    delete w;
}

extern "C" POLFMM_API int fmm_wall_forces(polfmm_wall* w, const double* positions, int64_t n, double eps, double sigma,
                                          double* energy, double* forces) {
    if (!w || n < 0 || n > w->cap || !(eps >= 0.0) || !(sigma > 0.0) || !energy || (n > 0 && (!positions || !forces)))
        return POLFMM_ERR_INVALID_ARG;
    cudaStream_t st = w->stream;
    cudaError_t e;
    if (n == 0) {
        e = cudaMemsetAsync(energy, 0, sizeof(double), st);
        return e == cudaSuccess ? POLFMM_OK : cuda_fail(e, "wall memset");
    }
    const double rc = std::pow(2.0, 1.0 / 6.0) * sigma;
    const double sigma6 = sigma * sigma * sigma * sigma * sigma * sigma;
    const uint32_t mask = (uint32_t)w->nbucket - 1u;
    const int nb = w->nbucket;
    if ((e = cudaMemsetAsync(w->count, 0, sizeof(int) * nb, st)) != cudaSuccess) return cuda_fail(e, "wall memset");
    wall_count_kernel<<<grid_for(n, 256), 256, 0, st>>>(positions, n, 1.0 / rc, mask, w->cell, w->count);
    if ((e = scan_levels(st, w->count, w->start, w->scan_part, nb)) != cudaSuccess) return cuda_fail(e, "wall scan");
    wall_fill_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, w->cell, w->start, nb, w->count, w->member);
    wall_order_kernel<<<grid_for(nb, 256), 256, 0, st>>>(nb, w->start, w->member);
    wall_pairs_kernel<<<grid_for(n, 128), 128, 0, st>>>(positions, n, w->cell, w->start, w->member, mask, rc * rc,
                                                        sigma6, 4.0 * eps, eps, forces, w->e_site);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "wall kernel launch");
    return sum_to(st, w->e_site, n, 1.0, w->part, energy);
}

extern "C" POLFMM_API int fmm_md_kick(double* velocities, const double* forces, const double* masses, double coef,
                                      int64_t n, void* cuda_stream) {
    if (n < 0 || (n > 0 && (!velocities || !forces || !masses))) return POLFMM_ERR_INVALID_ARG;
    if (n == 0) return POLFMM_OK;
    kick_kernel<<<grid_for(3 * n, 256), 256, 0, (cudaStream_t)cuda_stream>>>(velocities, forces, masses, coef, 3 * n);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? POLFMM_OK : cuda_fail(e, "kick kernel launch");
}

extern "C" POLFMM_API int fmm_md_drift(double* positions, const double* velocities, double dt, int64_t n,
                                       void* cuda_stream) {
    if (n < 0 || (n > 0 && (!positions || !velocities))) return POLFMM_ERR_INVALID_ARG;
    if (n == 0) return POLFMM_OK;
    drift_kernel<<<grid_for(3 * n, 256), 256, 0, (cudaStream_t)cuda_stream>>>(positions, velocities, dt, 3 * n);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? POLFMM_OK : cuda_fail(e, "drift kernel launch");
}

// site i's momentum component k, m_i v_ik
__global__ void momentum_site_kernel(const double* __restrict__ v, const double* __restrict__ m, int64_t n, int k,
                                     double* __restrict__ e) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    e[i] = m[i] * v[3 * i + k];
}

extern "C" POLFMM_API int fmm_md_momentum(polfmm_wall* w, const double* velocities, const double* masses, int64_t n,
                                          double* momentum) {
    if (!w || n < 0 || n > w->cap || !momentum || (n > 0 && (!velocities || !masses))) return POLFMM_ERR_INVALID_ARG;
    cudaStream_t st = w->stream;
    if (n == 0) {
        cudaError_t e = cudaMemsetAsync(momentum, 0, 3 * sizeof(double), st);
        return e == cudaSuccess ? POLFMM_OK : cuda_fail(e, "momentum memset");
    }
    for (int k = 0; k < 3; k++) {
        momentum_site_kernel<<<grid_for(n, 256), 256, 0, st>>>(velocities, masses, n, k, w->e_site);
        int rc = sum_to(st, w->e_site, n, 1.0, w->part, momentum + k);
        if (rc != POLFMM_OK) return rc;
    }
    return POLFMM_OK;
}

extern "C" POLFMM_API int fmm_md_kinetic(polfmm_wall* w, const double* velocities, const double* masses, int64_t n,
                                         double scale, double* energy) {
    if (!w || n < 0 || n > w->cap || !energy || (n > 0 && (!velocities || !masses))) return POLFMM_ERR_INVALID_ARG;
    cudaStream_t st = w->stream;
    if (n == 0) {
        cudaError_t e = cudaMemsetAsync(energy, 0, sizeof(double), st);
        return e == cudaSuccess ? POLFMM_OK : cuda_fail(e, "kinetic memset");
    }
    kinetic_site_kernel<<<grid_for(n, 256), 256, 0, st>>>(velocities, masses, n, w->e_site);
    return sum_to(st, w->e_site, n, scale, w->part, energy);
}
