// The adaptive kd-tree FMM of Sec. III on the GPU, in FP64: the paper's own
// tree (split the longest dimension of a cell's particles at their geometric
// centre, stop at n_bucket particles), the opening criterion
// theta |z_A - z_B| > r_enc,A + r_enc,B (Eq. mac) and the mutual dual-tree
// walk, with the single-box operators of Sec. II.B evaluated per pair.
//
// Every stage is level-synchronous and deterministic:
// - the tree grows one level per round: a block per cell reduces its
//   particles (centre, box, r_enc), decides the split, and partitions its
//   index range stably; the children of a level get consecutive ids;
// - the multipoles go up one level per launch (P2M at the leaves, M2M of the
//   two children in order), the locals down one level per launch;
// - the walk expands a frontier of cell pairs one round at a time; every pair
//   counts what it emits (a direct pair, a multipole pair, child pairs), a
//   scan places the outputs, so that the lists come out in a fixed order;
// - the multipole-to-local terms and the direct terms are gathered per target
//   (a cell, or the particles of a leaf and its ancestors) from lists sorted
//   by source, so that every sum runs in a fixed order.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace polfmm {

constexpr int kKdThreads = 128;

struct KdCells {
    int* start = nullptr;   // [cap] first particle (index into perm)
    int* end = nullptr;     // [cap]
    int* left = nullptr;    // [cap] first child, -1 for a leaf
    int* parent = nullptr;  // [cap]
    double* z = nullptr;    // [cap][3] geometric centre of the particles
    double* renc = nullptr; // [cap] distance from z to the farthest corner of the (padded) box
    int* split = nullptr;   // [cap] 1 if the cell splits
    int* sdim = nullptr;    // [cap] split dimension
    double* M = nullptr;    // [cap][nc] multipoles about z
    double* F = nullptr;    // [cap][nc] locals about z
};

// ---------------------------------------------------------------------------
// deterministic block reductions and a two-level exclusive scan
// ---------------------------------------------------------------------------
__device__ inline double kd_block_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = kKdThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__device__ inline double kd_block_max(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = kKdThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__device__ inline int kd_block_scan_excl(int v, int* sh, int* total) {
    // inclusive scan through shared memory (Hillis-Steele), then exclusive
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < kKdThreads; o <<= 1) {
        const int t = (int)threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    const int incl = sh[threadIdx.x];
    *total = sh[kKdThreads - 1];
    __syncthreads();
    return incl - v;
}

constexpr int kKdScanBlock = 1024;

__global__ void kd_scan_block_kernel(const int* __restrict__ in, int* __restrict__ out, int* __restrict__ part, int n) {
    __shared__ int wt[kKdScanBlock / 32];
    const int i = blockIdx.x * kKdScanBlock + threadIdx.x;
    const int v = i < n ? in[i] : 0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int s = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += t;
    }
    if (lane == 31) wt[w] = s;
    __syncthreads();
    if (w == 0) {
        int t = wt[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        wt[lane] = t;
    }
    __syncthreads();
    const int before = w > 0 ? wt[w - 1] : 0;
    if (i < n) out[i] = before + s - v;
    if (threadIdx.x == kKdScanBlock - 1) part[blockIdx.x] = before + s;
}

__global__ void kd_scan_add_kernel(int* __restrict__ out, const int* __restrict__ add, int n) {
    const int i = blockIdx.x * kKdScanBlock + threadIdx.x;
    if (i < n) out[i] += add[blockIdx.x];
}

// exclusive scan of n ints; scratch holds at least kd_scan_need(n) ints; the
// total is returned through the host (one synchronisation)
static size_t kd_scan_need(int n) {
    size_t need = 2;
    while (n > 1) {
        n = (n + kKdScanBlock - 1) / kKdScanBlock;
        need += 2 * (size_t)n;
    }
    return need;
}

static void kd_scan(cudaStream_t st, const int* in, int* out, int* scratch, int n) {
    if (n <= 0) return;
    const int nb = (n + kKdScanBlock - 1) / kKdScanBlock;
    kd_scan_block_kernel<<<nb, kKdScanBlock, 0, st>>>(in, out, scratch, n);
    if (nb > 1) {
        kd_scan(st, scratch, scratch + nb, scratch + 2 * nb, nb);
        kd_scan_add_kernel<<<nb, kKdScanBlock, 0, st>>>(out, scratch + nb, n);
    }
}

// ---------------------------------------------------------------------------
// tree
// ---------------------------------------------------------------------------
// one block per cell of the level: centre, padded box, r_enc, and the split
// (the longest dimension of the unpadded box, at the centre along it; no split
// when the cell holds at most n_bucket particles, when they coincide along that
// dimension, or when the centre would leave one side empty)
__global__ void __launch_bounds__(kKdThreads) kd_stats_kernel(int begin, KdCells C, const int* __restrict__ perm,
                                                              const double* __restrict__ x, int n_bucket, double pad) {
    __shared__ double sh[kKdThreads];
    __shared__ int shi[kKdThreads];
    const int c = begin + blockIdx.x;
    const int s = C.start[c], e = C.end[c], cnt = e - s;
    double sum[3] = {0, 0, 0}, mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int k = s + threadIdx.x; k < e; k += kKdThreads) {
        const int i = perm[k];
        for (int d = 0; d < 3; d++) {
            const double v = x[3 * (int64_t)i + d];
            sum[d] += v;
            mn[d] = fmin(mn[d], v);
            mx[d] = fmax(mx[d], v);
        }
    }
    double z[3], lo[3], hi[3];
    for (int d = 0; d < 3; d++) {
        z[d] = kd_block_sum(sum[d], sh) / (double)cnt;
        lo[d] = -kd_block_max(-mn[d], sh);
        hi[d] = kd_block_max(mx[d], sh);
    }
    int dim = 0;
    double ext = hi[0] - lo[0];
    for (int d = 1; d < 3; d++)
        if (hi[d] - lo[d] > ext) {
            ext = hi[d] - lo[d];
            dim = d;
        }
    int go = cnt > n_bucket && ext > 0.0;
    if (go) {
        // the particles left of the centre: the split must leave both sides non-empty
        int nl = 0;
        for (int k = s + threadIdx.x; k < e; k += kKdThreads) nl += x[3 * (int64_t)perm[k] + dim] < z[dim];
        int tot;
        kd_block_scan_excl(nl, shi, &tot);
        go = tot > 0 && tot < cnt;
    }
    if (threadIdx.x == 0) {
        // the box, padded on every side when the cell holds fewer than three particles
        double bl[3], bh[3];
        for (int d = 0; d < 3; d++) {
            bl[d] = cnt < 3 ? lo[d] - pad : lo[d];
            bh[d] = cnt < 3 ? hi[d] + pad : hi[d];
        }
        double r2 = 0.0;
        for (int corner = 0; corner < 8; corner++) {
            double q = 0.0;
            for (int d = 0; d < 3; d++) {
                const double v = ((corner >> d) & 1) ? bh[d] : bl[d];
                q += (v - z[d]) * (v - z[d]);
            }
            r2 = fmax(r2, q);
        }
        for (int d = 0; d < 3; d++) C.z[3 * c + d] = z[d];
        C.renc[c] = sqrt(r2);
        C.split[c] = go;
        C.sdim[c] = dim;
        C.left[c] = -1;
    }
}

// one block per cell of the level that splits: stable partition of its index
// range about the centre, children at next + 2 rank(c)
__global__ void __launch_bounds__(kKdThreads) kd_split_kernel(int begin, KdCells C, const int* __restrict__ rank,
                                                              int next, int* __restrict__ perm, int* __restrict__ tmp,
                                                              const double* __restrict__ x) {
    __shared__ int sh[kKdThreads];
    const int c = begin + blockIdx.x;
    if (!C.split[c]) return;
    const int s = C.start[c], e = C.end[c];
    const int dim = C.sdim[c];
    const double zc = C.z[3 * c + dim];
    // left particles first, then right, each in their current order
    int nl_total = 0;
    {
        int carry = 0;
        for (int base = s; base < e; base += kKdThreads) {
            const int k = base + threadIdx.x;
            const int f = k < e && x[3 * (int64_t)perm[k] + dim] < zc;
            int tot;
            const int off = kd_block_scan_excl(f, sh, &tot);
            if (f) tmp[s + carry + off] = perm[k];
            carry += tot;
        }
        nl_total = carry;
    }
    {
        int carry = 0;
        for (int base = s; base < e; base += kKdThreads) {
            const int k = base + threadIdx.x;
            const int f = k < e && !(x[3 * (int64_t)perm[k] + dim] < zc);
            int tot;
            const int off = kd_block_scan_excl(f, sh, &tot);
            if (f) tmp[s + nl_total + carry + off] = perm[k];
            carry += tot;
        }
    }
    __syncthreads();
    for (int k = s + threadIdx.x; k < e; k += kKdThreads) perm[k] = tmp[k];
    if (threadIdx.x == 0) {
        const int l = next + 2 * rank[blockIdx.x], r = l + 1;
        C.left[c] = l;
        C.start[l] = s;
        C.end[l] = s + nl_total;
        C.start[r] = s + nl_total;
        C.end[r] = e;
        C.parent[l] = C.parent[r] = c;
    }
}

// ---------------------------------------------------------------------------
// expansions (Sec. II.B, un-normalised, about each cell's centre z):
//   P2M  M_n = sum_a q_a (-1)^|n| (x_a - z)^n / n!
//            + (-1)^|n| sum_d mu_a,d (x_a - z)^(n - e_d) / (n - e_d)!   (point dipole)
//   M2M  M_n(z + s) = sum_{k <= n} s^k / k! M_(n-k)(z)
//   M2L  F_n(z_B) = sum_{|m| <= p - |n|} M_m(z_A) d^(n+m) (1/r)(z_B - z_A)
//   L2L  F_n(z + s) = sum_{|k| <= p - |n|} s^k / k! F_(n+k)(z)
//   L2P  d^k Phi(x) = sum_{|n| <= p - |k|} (x - z)^n / n! F_(n+k)
// ---------------------------------------------------------------------------
struct KdOrder {
    int p, nc;
    const int* mi;          // [nc] packed x | y << 8 | z << 16 | |n| << 24
    const double* ifact;    // [p + 1] 1 / k!
};

__device__ inline void kd_unpack(int pk, int& x, int& y, int& z) {
    x = pk & 0xff;
    y = (pk >> 8) & 0xff;
    z = (pk >> 16) & 0xff;
}

__device__ inline double kd_pow(double v, int k) {
    double r = 1.0;
    for (int i = 0; i < k; i++) r *= v;
    return r;
}

// one block per cell of a level: P2M at a leaf, else M2M of its two children
__global__ void __launch_bounds__(kKdThreads) kd_upward_kernel(int begin, KdCells C, KdOrder O,
                                                               const int* __restrict__ perm, const double* __restrict__ x,
                                                               const double* __restrict__ q, const double* __restrict__ mu,
                                                               double dl) {
    const int c = begin + blockIdx.x;
    const double zc[3] = {C.z[3 * c], C.z[3 * c + 1], C.z[3 * c + 2]};
    double* M = C.M + (int64_t)c * O.nc;
    const int l = C.left[c];
    for (int cc = threadIdx.x; cc < O.nc; cc += kKdThreads) {
        int nx, ny, nz;
        kd_unpack(O.mi[cc], nx, ny, nz);
        const int n[3] = {nx, ny, nz};
        const double sgn = ((nx + ny + nz) & 1) ? -1.0 : 1.0;
        double acc = 0.0;
        if (l < 0) {
            for (int k = C.start[c]; k < C.end[c]; k++) {
                const int i = perm[k];
                const double r[3] = {x[3 * (int64_t)i] - zc[0], x[3 * (int64_t)i + 1] - zc[1], x[3 * (int64_t)i + 2] - zc[2]};
                const double qi = q ? q[i] : 0.0;
                const double m[3] = {mu ? mu[3 * (int64_t)i] : 0.0, mu ? mu[3 * (int64_t)i + 1] : 0.0,
                                     mu ? mu[3 * (int64_t)i + 2] : 0.0};
                const double mn = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
                if (dl > 0.0) {
                    // the dipole as +-q^mu at x +- dl mu/|mu| (Sec. II.C)
                    double v = qi;
                    double t = v * kd_pow(r[0], nx) * kd_pow(r[1], ny) * kd_pow(r[2], nz);
                    if (mn > 0.0)
                        for (int sg = -1; sg <= 1; sg += 2) {
                            const double qq = sg * mn / (2.0 * dl);
                            const double y[3] = {r[0] + sg * dl * m[0] / mn, r[1] + sg * dl * m[1] / mn,
                                                 r[2] + sg * dl * m[2] / mn};
                            t += qq * kd_pow(y[0], nx) * kd_pow(y[1], ny) * kd_pow(y[2], nz);
                        }
                    acc += t;
                } else {
                    double t = qi * kd_pow(r[0], nx) * kd_pow(r[1], ny) * kd_pow(r[2], nz);
                    // d/dx_d of (x - z)^n: n_d (x - z)^(n - e_d); with 1/n! this is (x - z)^(n - e_d) / (n - e_d)!
                    for (int d = 0; d < 3; d++) {
                        if (n[d] == 0 || m[d] == 0.0) continue;
                        int e[3] = {nx, ny, nz};
                        e[d] -= 1;
                        t += m[d] * n[d] * kd_pow(r[0], e[0]) * kd_pow(r[1], e[1]) * kd_pow(r[2], e[2]);
                    }
                    acc += t;
                }
            }
            acc *= sgn * O.ifact[nx] * O.ifact[ny] * O.ifact[nz];
        } else {
            for (int h = 0; h < 2; h++) {
                const int ch = l + h;
                const double s[3] = {zc[0] - C.z[3 * ch], zc[1] - C.z[3 * ch + 1], zc[2] - C.z[3 * ch + 2]};
                const double* Mc = C.M + (int64_t)ch * O.nc;
                double part = 0.0;
                for (int kx = 0; kx <= nx; kx++)
                    for (int ky = 0; ky <= ny; ky++)
                        for (int kz = 0; kz <= nz; kz++)
                            part += kd_pow(s[0], kx) * kd_pow(s[1], ky) * kd_pow(s[2], kz) * O.ifact[kx] * O.ifact[ky] *
                                    O.ifact[kz] * Mc[mi_index(nx - kx, ny - ky, nz - kz)];
                acc += part;
            }
        }
        M[cc] = acc;
    }
}

// ---------------------------------------------------------------------------
// walk (Sec. III): one round of the frontier.  A pair (A, B) emits
//   a self pair that is a leaf or holds fewer than n_direct particles: direct;
//   a self pair otherwise: (L, L), (R, R), (L, R);
//   A != B with n_A + n_B < n_direct, or two leaves: direct;
//   theta |z_A - z_B| > r_A + r_B: a multipole pair (both directions);
//   else the larger r_enc is split (the other one if it is a leaf): (small, c1), (small, c2)
// ---------------------------------------------------------------------------
__device__ inline int kd_walk_decide(int2 pr, const KdCells& C, double theta, int n_direct, int* kids) {
    const int a = pr.x, b = pr.y;
    const int na = C.end[a] - C.start[a], nb = C.end[b] - C.start[b];
    const int la = C.left[a], lb = C.left[b];
    if (a == b) {
        if (la < 0 || na < n_direct) return 0;  // direct
        kids[0] = la; kids[1] = la; kids[2] = la + 1; kids[3] = la + 1; kids[4] = la; kids[5] = la + 1;
        return 3;
    }
    if (na + nb < n_direct || (la < 0 && lb < 0)) return 0;
    const double d0 = C.z[3 * a] - C.z[3 * b], d1 = C.z[3 * a + 1] - C.z[3 * b + 1], d2 = C.z[3 * a + 2] - C.z[3 * b + 2];
    if (theta * sqrt(d0 * d0 + d1 * d1 + d2 * d2) > C.renc[a] + C.renc[b]) return 1;  // multipole
    int big = a, small = b;
    if (!(C.renc[a] >= C.renc[b])) { big = b; small = a; }
    if (C.left[big] < 0) { const int t = big; big = small; small = t; }
    const int c1 = C.left[big];
    kids[0] = small; kids[1] = c1; kids[2] = small; kids[3] = c1 + 1;
    return 2;
}

__global__ void kd_walk_count_kernel(int m, const int2* __restrict__ fr, KdCells C, double theta, int n_direct,
                                     int* __restrict__ cnt_direct, int* __restrict__ cnt_multi, int* __restrict__ cnt_kids) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    int kids[6];
    const int r = kd_walk_decide(fr[t], C, theta, n_direct, kids);
    cnt_direct[t] = r == 0;
    cnt_multi[t] = r == 1;
    cnt_kids[t] = r >= 2 ? r : 0;
}

__global__ void kd_walk_write_kernel(int m, const int2* __restrict__ fr, KdCells C, double theta, int n_direct,
                                     const int* __restrict__ off_direct, const int* __restrict__ off_multi,
                                     const int* __restrict__ off_kids, int base_direct, int base_multi,
                                     int2* __restrict__ direct, int2* __restrict__ multi, int2* __restrict__ next) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    int kids[6];
    const int2 pr = fr[t];
    const int r = kd_walk_decide(pr, C, theta, n_direct, kids);
    if (r == 0) direct[base_direct + off_direct[t]] = pr;
    else if (r == 1) multi[base_multi + off_multi[t]] = pr;
    else
        for (int k = 0; k < r; k++) next[off_kids[t] + k] = make_int2(kids[2 * k], kids[2 * k + 1]);
}

// ---------------------------------------------------------------------------
// per-target lists: entries (target, source), grouped by target, ascending
// source within a target
// ---------------------------------------------------------------------------
__global__ void kd_entry_count_kernel(int m, const int2* __restrict__ pairs, int* __restrict__ cnt) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    const int2 p = pairs[t];
    atomicAdd(&cnt[p.x], 1);
    if (p.y != p.x) atomicAdd(&cnt[p.y], 1);
}

__global__ void kd_entry_fill_kernel(int m, const int2* __restrict__ pairs, const int* __restrict__ ptr,
                                     int* __restrict__ fill, int* __restrict__ src) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    const int2 p = pairs[t];
    src[ptr[p.x] + atomicAdd(&fill[p.x], 1)] = p.y;
    if (p.y != p.x) src[ptr[p.y] + atomicAdd(&fill[p.y], 1)] = p.x;
}

__global__ void kd_entry_sort_kernel(int ncell, const int* __restrict__ ptr, int* __restrict__ src) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int s = ptr[c], e = ptr[c + 1];
    for (int k = s + 1; k < e; k++) {
        const int v = src[k];
        int j = k - 1;
        while (j >= s && src[j] > v) {
            src[j + 1] = src[j];
            j--;
        }
        src[j + 1] = v;
    }
}

// ---------------------------------------------------------------------------
// M2L per target cell: F_t += sum over its sources s (ascending) of the
// contraction with the derivatives of 1/r at z_t - z_s, by the recurrence
//   |n| r^2 D_n = -(2|n| - 1) sum_d n_d R_d D_(n - e_d) - (|n| - 1) sum_d n_d (n_d - 1) D_(n - 2 e_d)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kKdThreads) kd_m2l_kernel(KdCells C, KdOrder O, const int* __restrict__ ptr,
                                                            const int* __restrict__ src) {
    extern __shared__ double kd_sm[];  // [nc] derivatives
    const int t = blockIdx.x;
    const int s0 = ptr[t], s1 = ptr[t + 1];
    if (s0 == s1) return;
    double* D = kd_sm;
    double acc[4] = {0, 0, 0, 0};  // up to 4 coefficients per thread (nc <= 512)
    for (int k = s0; k < s1; k++) {
        const int s = src[k];
        const double R[3] = {C.z[3 * t] - C.z[3 * s], C.z[3 * t + 1] - C.z[3 * s + 1], C.z[3 * t + 2] - C.z[3 * s + 2]};
        const double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
        __syncthreads();
        if (threadIdx.x == 0) D[0] = 1.0 / sqrt(r2);
        __syncthreads();
        for (int o = 1; o <= O.p; o++) {
            const int b0 = o * (o + 1) * (o + 2) / 6, b1 = (o + 1) * (o + 2) * (o + 3) / 6;
            for (int cc = b0 + threadIdx.x; cc < b1; cc += kKdThreads) {
                int nx, ny, nz;
                kd_unpack(O.mi[cc], nx, ny, nz);
                const int n[3] = {nx, ny, nz};
                double v = 0.0;
                for (int d = 0; d < 3; d++) {
                    if (n[d] >= 1) {
                        int e[3] = {nx, ny, nz};
                        e[d] -= 1;
                        v -= (2.0 * o - 1.0) * n[d] * R[d] * D[mi_index(e[0], e[1], e[2])];
                    }
                    if (n[d] >= 2) {
                        int e[3] = {nx, ny, nz};
                        e[d] -= 2;
                        v -= (o - 1.0) * n[d] * (n[d] - 1.0) * D[mi_index(e[0], e[1], e[2])];
                    }
                }
                D[cc] = v / (o * r2);
            }
            __syncthreads();
        }
        const double* Ms = C.M + (int64_t)s * O.nc;
        for (int j = 0; j < 4; j++) {
            const int cc = threadIdx.x + j * kKdThreads;
            if (cc >= O.nc) break;
            int nx, ny, nz;
            kd_unpack(O.mi[cc], nx, ny, nz);
            const int rest = O.p - (nx + ny + nz);
            double a = 0.0;
            for (int mm = 0; mm < O.nc; mm++) {
                int mx, my, mz;
                kd_unpack(O.mi[mm], mx, my, mz);
                if (mx + my + mz > rest) break;  // the coefficients come in ascending degree
                a += Ms[mm] * D[mi_index(nx + mx, ny + my, nz + mz)];
            }
            acc[j] += a;
        }
    }
    double* F = C.F + (int64_t)t * O.nc;
    for (int j = 0; j < 4; j++) {
        const int cc = threadIdx.x + j * kKdThreads;
        if (cc < O.nc) F[cc] += acc[j];
    }
}

// one block per cell of a level (>= 1): F += L2L of the parent's locals
__global__ void __launch_bounds__(kKdThreads) kd_downward_kernel(int begin, KdCells C, KdOrder O) {
    const int c = begin + blockIdx.x;
    const int pa = C.parent[c];
    const double s[3] = {C.z[3 * c] - C.z[3 * pa], C.z[3 * c + 1] - C.z[3 * pa + 1], C.z[3 * c + 2] - C.z[3 * pa + 2]};
    const double* Fp = C.F + (int64_t)pa * O.nc;
    double* F = C.F + (int64_t)c * O.nc;
    for (int cc = threadIdx.x; cc < O.nc; cc += kKdThreads) {
        int nx, ny, nz;
        kd_unpack(O.mi[cc], nx, ny, nz);
        const int rest = O.p - (nx + ny + nz);
        double a = 0.0;
        for (int kx = 0; kx <= rest; kx++)
            for (int ky = 0; ky <= rest - kx; ky++)
                for (int kz = 0; kz <= rest - kx - ky; kz++)
                    a += kd_pow(s[0], kx) * kd_pow(s[1], ky) * kd_pow(s[2], kz) * O.ifact[kx] * O.ifact[ky] * O.ifact[kz] *
                         Fp[mi_index(nx + kx, ny + ky, nz + kz)];
        F[cc] += a;
    }
}

// one block per leaf, one thread per particle: L2P of the leaf's locals, then
// the direct terms of every source cell listed for the leaf or its ancestors
// (ancestors from the leaf up, sources ascending), excluding the particle itself
__global__ void __launch_bounds__(kKdThreads) kd_leaf_kernel(const int* __restrict__ leaves, KdCells C, KdOrder O,
                                                             const int* __restrict__ perm, const double* __restrict__ x,
                                                             const double* __restrict__ q, const double* __restrict__ mu,
                                                             const int* __restrict__ dptr, const int* __restrict__ dsrc,
                                                             double* __restrict__ phi, double* __restrict__ E,
                                                             double* __restrict__ G) {
    const int c = leaves[blockIdx.x];
    const int s = C.start[c], e = C.end[c];
    const double* F = C.F + (int64_t)c * O.nc;
    for (int k = s + threadIdx.x; k < e; k += kKdThreads) {
        const int i = perm[k];
        const double xi[3] = {x[3 * (int64_t)i], x[3 * (int64_t)i + 1], x[3 * (int64_t)i + 2]};
        const double r[3] = {xi[0] - C.z[3 * c], xi[1] - C.z[3 * c + 1], xi[2] - C.z[3 * c + 2]};
        double ph = 0.0, dp[3] = {0, 0, 0}, ddp[6] = {0, 0, 0, 0, 0, 0};
        const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
        for (int cc = 0; cc < O.nc; cc++) {
            int nx, ny, nz;
            kd_unpack(O.mi[cc], nx, ny, nz);
            const int deg = nx + ny + nz;
            const double w = kd_pow(r[0], nx) * kd_pow(r[1], ny) * kd_pow(r[2], nz) * O.ifact[nx] * O.ifact[ny] * O.ifact[nz];
            ph += w * F[cc];
            if (deg <= O.p - 1) {
                dp[0] += w * F[mi_index(nx + 1, ny, nz)];
                dp[1] += w * F[mi_index(nx, ny + 1, nz)];
                dp[2] += w * F[mi_index(nx, ny, nz + 1)];
            }
            if (deg <= O.p - 2)
                for (int g = 0; g < 6; g++) {
                    int m[3] = {nx, ny, nz};
                    m[ia[g]] += 1;
                    m[ib[g]] += 1;
                    ddp[g] += w * F[mi_index(m[0], m[1], m[2])];
                }
        }
        double ef[3] = {-dp[0], -dp[1], -dp[2]}, gf[6];
        for (int g = 0; g < 6; g++) gf[g] = -ddp[g];
        // direct terms: phi = q/r + mu.r/r^3, E = q r/r^3 + 3 (mu.r) r/r^5 - mu/r^3,
        // G_ab = q (delta_ab/r^3 - 3 r_a r_b/r^5) + 3 (mu_a r_b + mu_b r_a + (mu.r) delta_ab)/r^5 - 15 (mu.r) r_a r_b/r^7
        for (int a = c; a >= 0; a = C.parent[a]) {
            for (int kk = dptr[a]; kk < dptr[a + 1]; kk++) {
                const int b = dsrc[kk];
                for (int m = C.start[b]; m < C.end[b]; m++) {
                    const int j = perm[m];
                    if (j == i) continue;
                    const double rr[3] = {xi[0] - x[3 * (int64_t)j], xi[1] - x[3 * (int64_t)j + 1], xi[2] - x[3 * (int64_t)j + 2]};
                    const double r2 = rr[0] * rr[0] + rr[1] * rr[1] + rr[2] * rr[2];
                    const double ri = 1.0 / sqrt(r2), ri2 = ri * ri, ri3 = ri * ri2, ri5 = ri3 * ri2, ri7 = ri5 * ri2;
                    const double qj = q ? q[j] : 0.0;
                    const double mj[3] = {mu ? mu[3 * (int64_t)j] : 0.0, mu ? mu[3 * (int64_t)j + 1] : 0.0,
                                          mu ? mu[3 * (int64_t)j + 2] : 0.0};
                    const double mr = mj[0] * rr[0] + mj[1] * rr[1] + mj[2] * rr[2];
                    ph += qj * ri + mr * ri3;
                    for (int d = 0; d < 3; d++) ef[d] += qj * ri3 * rr[d] + 3.0 * mr * rr[d] * ri5 - mj[d] * ri3;
                    for (int g = 0; g < 6; g++) {
                        const int aa = ia[g], bb = ib[g];
                        const double dl = aa == bb ? 1.0 : 0.0;
                        gf[g] += qj * (dl * ri3 - 3.0 * rr[aa] * rr[bb] * ri5) +
                                 3.0 * (mj[aa] * rr[bb] + mj[bb] * rr[aa] + mr * dl) * ri5 - 15.0 * mr * rr[aa] * rr[bb] * ri7;
                    }
                }
            }
        }
        if (phi) phi[i] = ph;
        if (E)
            for (int d = 0; d < 3; d++) E[3 * (int64_t)i + d] = ef[d];
        if (G)
            for (int g = 0; g < 6; g++) G[6 * (int64_t)i + g] = gf[g];
    }
}

__global__ void kd_iota_kernel(int n, int* __restrict__ v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = i;
}

__global__ void kd_leaves_kernel(int ncell, const int* __restrict__ left, const int* __restrict__ rank,
                                 int* __restrict__ leaves) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncell && left[c] < 0) leaves[rank[c]] = c;
}

__global__ void kd_isleaf_kernel(int ncell, const int* __restrict__ left, int* __restrict__ f) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncell) f[c] = left[c] < 0;
}

}  // namespace polfmm

using namespace polfmm;

namespace {

// device allocations of one call, freed together
struct KdMem {
    std::vector<void*> ptrs;
    bool ok = true;
    template <typename T>
    T* get(size_t count) {
        void* p = nullptr;
        if (!ok) return nullptr;
        if (dev_alloc(&p, sizeof(T) * std::max<size_t>(count, 1)) != cudaSuccess) {
            ok = false;
            cudaGetLastError();
            return nullptr;
        }
        ptrs.push_back(p);
        return static_cast<T*>(p);
    }
    ~KdMem() {
        for (void* p : ptrs) cudaFree(p);
    }
};

int read_int(cudaStream_t st, const int* dev, int* out) {
    cudaError_t e = cudaMemcpyAsync(out, dev, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? POLFMM_OK : cuda_fail(e, "kd-tree counts");
}

// exclusive scan with the total read back (the host sizes the next stage)
int scan_total(cudaStream_t st, const int* in, int* out, int* scratch, int n, int* total) {
    *total = 0;
    if (n <= 0) return POLFMM_OK;
    kd_scan(st, in, out, scratch, n);
    int last_in = 0, last_out = 0;
    cudaError_t e = cudaMemcpyAsync(&last_in, in + n - 1, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&last_out, out + n - 1, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "kd-tree scan");
    *total = last_in + last_out;
    return POLFMM_OK;
}

// per-target lists of the pairs (both directions, a self pair once), sorted by source
int target_lists(cudaStream_t st, const int2* pairs, int m, int ncell, KdMem& mem, int* scratch, int** ptr_out,
                 int** src_out) {
    int* cnt = mem.get<int>(ncell + 1);
    int* ptr = mem.get<int>(ncell + 1);
    int* fill = mem.get<int>(ncell + 1);
    if (!mem.ok) return POLFMM_ERR_OUT_OF_MEMORY;
    cudaMemsetAsync(cnt, 0, sizeof(int) * (ncell + 1), st);
    cudaMemsetAsync(fill, 0, sizeof(int) * (ncell + 1), st);
    if (m > 0) kd_entry_count_kernel<<<grid_for(m, 256), 256, 0, st>>>(m, pairs, cnt);
    int total = 0;
    int rc = scan_total(st, cnt, ptr, scratch, ncell + 1, &total);
    if (rc != POLFMM_OK) return rc;
    int* src = mem.get<int>(total);
    if (!mem.ok) return POLFMM_ERR_OUT_OF_MEMORY;
    if (m > 0) kd_entry_fill_kernel<<<grid_for(m, 256), 256, 0, st>>>(m, pairs, ptr, fill, src);
    kd_entry_sort_kernel<<<grid_for(ncell, 128), 128, 0, st>>>(ncell, ptr, src);
    *ptr_out = ptr;
    *src_out = src;
    return POLFMM_OK;
}

int kdtree_impl(int64_t n64, const double* x, const double* q, const double* mu, int p, double theta, int n_bucket,
                int n_direct, double pad, double dl, double* phi, double* E, double* G, int64_t* stats,
                cudaStream_t st) {
    const int n = (int)n64;
    const int nc = ncoef_of(p);
    const int cap = 2 * n + 1;
    KdMem mem;
    KdCells C;
    C.start = mem.get<int>(cap);
    C.end = mem.get<int>(cap);
    C.left = mem.get<int>(cap);
    C.parent = mem.get<int>(cap);
    C.z = mem.get<double>(3 * (size_t)cap);
    C.renc = mem.get<double>(cap);
    C.split = mem.get<int>(cap);
    C.sdim = mem.get<int>(cap);
    C.M = mem.get<double>((size_t)cap * nc);
    C.F = mem.get<double>((size_t)cap * nc);
    int* perm = mem.get<int>(n);
    int* tmp = mem.get<int>(n);
    int* rank = mem.get<int>(cap + 1);
    int* scratch = mem.get<int>(kd_scan_need(cap + 1) + 64);
    // multi-indices in ascending degree, and 1/k!
    std::vector<int> mi_h(nc);
    for (int o = 0; o <= p; o++)
        for (int x_ = o; x_ >= 0; x_--)
            for (int y_ = o - x_; y_ >= 0; y_--) {
                const int z_ = o - x_ - y_;
                mi_h[mi_index(x_, y_, z_)] = x_ | (y_ << 8) | (z_ << 16) | (o << 24);
            }
    std::vector<double> if_h(p + 1, 1.0);
    for (int k = 1; k <= p; k++) if_h[k] = if_h[k - 1] / k;
    int* mi = mem.get<int>(nc);
    double* ifact = mem.get<double>(p + 1);
    if (!mem.ok) return POLFMM_ERR_OUT_OF_MEMORY;
    cudaMemcpyAsync(mi, mi_h.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(ifact, if_h.data(), sizeof(double) * (p + 1), cudaMemcpyHostToDevice, st);
    const KdOrder O{p, nc, mi, ifact};
    cudaMemsetAsync(C.F, 0, sizeof(double) * (size_t)cap * nc, st);

    // tree, one level per round
    kd_iota_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, perm);
    const int zero = 0, minus1 = -1;
    cudaMemcpyAsync(C.start, &zero, sizeof(int), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(C.end, &n, sizeof(int), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(C.parent, &minus1, sizeof(int), cudaMemcpyHostToDevice, st);
    std::vector<int> lbeg{0}, lend{1};
    int rc;
    for (int level = 0;; level++) {
        const int b = lbeg.back(), m = lend.back() - lbeg.back();
        if (m == 0) break;
        kd_stats_kernel<<<m, kKdThreads, 0, st>>>(b, C, perm, x, n_bucket, pad);
        int nsplit = 0;
        if ((rc = scan_total(st, C.split + b, rank, scratch, m, &nsplit)) != POLFMM_OK) return rc;
        const int next = lend.back();
        if (nsplit > 0) kd_split_kernel<<<m, kKdThreads, 0, st>>>(b, C, rank, next, perm, tmp, x);
        lbeg.push_back(next);
        lend.push_back(next + 2 * nsplit);
        if (level > 200) return POLFMM_ERR_INVALID_ARG;  // cannot happen with both sides non-empty
    }
    const int ncell = lend.back();
    const int nlev = (int)lbeg.size() - 1;
    // multipoles, deepest level first
    for (int L = nlev - 1; L >= 0; L--)
        kd_upward_kernel<<<lend[L] - lbeg[L], kKdThreads, 0, st>>>(lbeg[L], C, O, perm, x, q, mu, dl);

    // walk
    int2* fr = mem.get<int2>(4);
    if (!mem.ok) return POLFMM_ERR_OUT_OF_MEMORY;
    const int2 root = make_int2(0, 0);
    cudaMemcpyAsync(fr, &root, sizeof(int2), cudaMemcpyHostToDevice, st);
    int nfr = 1;
    size_t cap_d = 1024, cap_m = 1024;
    int2* direct = mem.get<int2>(cap_d);
    int2* multi = mem.get<int2>(cap_m);
    int nd = 0, nm = 0;
    while (nfr > 0) {
        int* cd = mem.get<int>(nfr);
        int* cm = mem.get<int>(nfr);
        int* ck = mem.get<int>(nfr);
        int* od = mem.get<int>(nfr);
        int* om = mem.get<int>(nfr);
        int* ok = mem.get<int>(nfr);
        int* wscr = nfr > cap + 1 ? mem.get<int>(kd_scan_need(nfr) + 64) : scratch;
        if (!mem.ok) return POLFMM_ERR_OUT_OF_MEMORY;
        kd_walk_count_kernel<<<grid_for(nfr, 256), 256, 0, st>>>(nfr, fr, C, theta, n_direct, cd, cm, ck);
        int td, tm, tk;
        if ((rc = scan_total(st, cd, od, wscr, nfr, &td)) != POLFMM_OK ||
            (rc = scan_total(st, cm, om, wscr, nfr, &tm)) != POLFMM_OK ||
            (rc = scan_total(st, ck, ok, wscr, nfr, &tk)) != POLFMM_OK)
            return rc;
        if ((size_t)(nd + td) > cap_d || (size_t)(nm + tm) > cap_m) {
            const size_t nd_cap = std::max(cap_d, (size_t)(nd + td)) * 2, nm_cap = std::max(cap_m, (size_t)(nm + tm)) * 2;
            int2* d2 = mem.get<int2>(nd_cap);
            int2* m2 = mem.get<int2>(nm_cap);
            if (!mem.ok) return POLFMM_ERR_OUT_OF_MEMORY;
            if (nd) cudaMemcpyAsync(d2, direct, sizeof(int2) * nd, cudaMemcpyDeviceToDevice, st);
            if (nm) cudaMemcpyAsync(m2, multi, sizeof(int2) * nm, cudaMemcpyDeviceToDevice, st);
            direct = d2;
            multi = m2;
            cap_d = nd_cap;
            cap_m = nm_cap;
        }
        int2* nx = mem.get<int2>(tk);
        if (!mem.ok) return POLFMM_ERR_OUT_OF_MEMORY;
        kd_walk_write_kernel<<<grid_for(nfr, 256), 256, 0, st>>>(nfr, fr, C, theta, n_direct, od, om, ok, nd, nm,
                                                                  direct, multi, nx);
        nd += td;
        nm += tm;
        fr = nx;
        nfr = tk;
    }

    // multipole-to-local per target cell, then down the tree
    int *mptr = nullptr, *msrc = nullptr, *dptr = nullptr, *dsrc = nullptr;
    if ((rc = target_lists(st, multi, nm, ncell, mem, scratch, &mptr, &msrc)) != POLFMM_OK) return rc;
    if ((rc = target_lists(st, direct, nd, ncell, mem, scratch, &dptr, &dsrc)) != POLFMM_OK) return rc;
    kd_m2l_kernel<<<ncell, kKdThreads, sizeof(double) * nc, st>>>(C, O, mptr, msrc);
    for (int L = 1; L < nlev; L++) kd_downward_kernel<<<lend[L] - lbeg[L], kKdThreads, 0, st>>>(lbeg[L], C, O);
    // leaves
    int* isleaf = mem.get<int>(ncell);
    int* lrank = mem.get<int>(ncell);
    if (!mem.ok) return POLFMM_ERR_OUT_OF_MEMORY;
    kd_isleaf_kernel<<<grid_for(ncell, 256), 256, 0, st>>>(ncell, C.left, isleaf);
    int nleaf = 0;
    if ((rc = scan_total(st, isleaf, lrank, scratch, ncell, &nleaf)) != POLFMM_OK) return rc;
    int* leaves = mem.get<int>(nleaf);
    if (!mem.ok) return POLFMM_ERR_OUT_OF_MEMORY;
    kd_leaves_kernel<<<grid_for(ncell, 256), 256, 0, st>>>(ncell, C.left, lrank, leaves);
    kd_leaf_kernel<<<nleaf, kKdThreads, 0, st>>>(leaves, C, O, perm, x, q, mu, dptr, dsrc, phi, E, G);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kd-tree FMM");
    if (stats) {
        stats[0] = ncell;
        stats[1] = nleaf;
        stats[2] = nlev;
        stats[3] = nm;
        stats[4] = nd;
    }
    return POLFMM_OK;
}

}  // namespace

extern "C" POLFMM_API int fmm_kdtree_fields(int64_t n, const double* positions, const double* charges,
                                            const double* dipoles, int order_p, double theta, int n_bucket,
                                            int n_direct, double pad, double dipole_dl, double* phi, double* E,
                                            double* G, int64_t* stats, void* cuda_stream, int on_device) {
    if (n < 1 || n > (int64_t)1 << 26 || !positions || order_p < 1 || order_p > 7 || !(theta >= 0.0) || !(theta < 1.0) ||
        n_bucket < 1 || n_direct < 0 || !(pad >= 0.0) || !isfinite(pad) || !(dipole_dl >= 0.0) || !isfinite(dipole_dl))
        return POLFMM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // inputs and outputs on the device
    KdMem io;
    const double *xd = positions, *qd = charges, *md = dipoles;
    double *pd = phi, *ed = E, *gd = G;
    if (!on_device) {
        double* t = io.get<double>(3 * (size_t)n);
        double* tq = charges ? io.get<double>(n) : nullptr;
        double* tm = dipoles ? io.get<double>(3 * (size_t)n) : nullptr;
        pd = phi ? io.get<double>(n) : nullptr;
        ed = E ? io.get<double>(3 * (size_t)n) : nullptr;
        gd = G ? io.get<double>(6 * (size_t)n) : nullptr;
        if (!io.ok) return POLFMM_ERR_OUT_OF_MEMORY;
        cudaMemcpyAsync(t, positions, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st);
        if (tq) cudaMemcpyAsync(tq, charges, sizeof(double) * n, cudaMemcpyHostToDevice, st);
        if (tm) cudaMemcpyAsync(tm, dipoles, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st);
        xd = t;
        qd = tq;
        md = tm;
    }
    int rc = kdtree_impl(n, xd, qd, md, order_p, theta, n_bucket, n_direct, pad, dipole_dl, pd, ed, gd, stats, st);
    if (rc != POLFMM_OK) return rc;
    if (!on_device) {
        cudaError_t e = cudaSuccess;
        if (phi && e == cudaSuccess) e = cudaMemcpyAsync(phi, pd, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
        if (E && e == cudaSuccess) e = cudaMemcpyAsync(E, ed, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st);
        if (G && e == cudaSuccess) e = cudaMemcpyAsync(G, gd, sizeof(double) * 6 * n, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "kd-tree FMM outputs");
    }
    return POLFMM_OK;
}
