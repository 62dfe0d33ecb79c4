// Octree construction on the GPU: bounding cube, Morton keys of the leaf
// cells, a stable LSD radix sort of the sites by key, and the per-level box
// tables (occupied boxes in Morton order, parents, child ranges, dense
// key -> slot maps, octant-class grouping).
//
// The paper builds an adaptive kd-tree (Sec. III); this library uses a
// uniform octree of fixed depth instead, whose boxes at one level all share a
// side length, so that multipole-to-local translations depend only on the
// integer offset between boxes.
#include <math.h>

#include <mutex>

#include "internal.cuh"

namespace polfmm {

// ---------------------------------------------------------------------------
// bounding box (deterministic: min / max are exact in any order)
// ---------------------------------------------------------------------------
constexpr int kBBoxBlocks = 128;

__global__ void bbox_partial_kernel(const double* __restrict__ x, int64_t n, double* __restrict__ part) {
    double mn[3] = {INFINITY, INFINITY, INFINITY};
    double mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        for (int d = 0; d < 3; d++) {
            double v = x[3 * i + d];
            mn[d] = fmin(mn[d], v);
            mx[d] = fmax(mx[d], v);
        }
    }
    __shared__ double s[6][256];
    for (int d = 0; d < 3; d++) {
        s[d][threadIdx.x] = mn[d];
        s[3 + d][threadIdx.x] = mx[d];
    }
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int d = 0; d < 3; d++) {
                s[d][threadIdx.x] = fmin(s[d][threadIdx.x], s[d][threadIdx.x + w]);
                s[3 + d][threadIdx.x] = fmax(s[3 + d][threadIdx.x], s[3 + d][threadIdx.x + w]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) part[threadIdx.x * gridDim.x + blockIdx.x] = s[threadIdx.x][0];
}

// one warp per component (min x, y, z, max x, y, z): lanes stride over the
// block partials, then a shuffle reduction (min / max are exact in any order)
__global__ void bbox_final_kernel(const double* __restrict__ part, int nblk, double* __restrict__ out) {
    const int a = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (a >= 6) return;
    const bool is_min = a < 3;
    double v = is_min ? INFINITY : -INFINITY;
    for (int b = lane; b < nblk; b += 32) v = is_min ? fmin(v, part[a * nblk + b]) : fmax(v, part[a * nblk + b]);
    for (int o = 16; o > 0; o >>= 1) {
        const double w = __shfl_down_sync(0xffffffffu, v, o);
        v = is_min ? fmin(v, w) : fmax(v, w);
    }
    if (lane == 0) out[a] = v;
}

// ---------------------------------------------------------------------------
// Morton keys of the leaf cells
// ---------------------------------------------------------------------------
__global__ void keys_kernel(const double* __restrict__ x, int64_t n, double lo0, double lo1, double lo2, double h,
                            int nside, uint32_t* __restrict__ key, int* __restrict__ idx, int* __restrict__ err) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double lo[3] = {lo0, lo1, lo2};
    uint32_t c[3];
    for (int d = 0; d < 3; d++) {
        double v = x[3 * i + d];
        if (!isfinite(v)) atomicOr(err, 1);
        // floor((x - lo) / h): no contraction into an FMA, IEEE division
        double u = __ddiv_rn(__dsub_rn(v, lo[d]), h);
        double f = floor(u);
        int ci = f < 0.0 ? 0 : (f > (double)(nside - 1) ? nside - 1 : (int)f);
        if (!(f == f)) ci = 0;
        c[d] = (uint32_t)ci;
    }
    key[i] = morton3(c[0], c[1], c[2]);
    idx[i] = (int)i;
}

// ---------------------------------------------------------------------------
// exclusive scan of int32 (three-phase, recursive over block sums)
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ inline int block_exclusive_scan(int v, int* total) {
    __shared__ int warp_tot[kScanThreads / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        int t = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
        int ti = t;
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += u;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = ti - t;  // exclusive warp offsets
        if (lane == kScanThreads / 32 - 1) *total = ti;
    }
    __syncthreads();
    int r = warp_tot[w] + incl - v;
    __syncthreads();
    return r;
}

__global__ void scan_block_kernel(const int* __restrict__ in, int* __restrict__ out, const int* __restrict__ n_dev,
                                  int n_host, int* __restrict__ block_sums) {
    int n = n_dev ? *n_dev : n_host;
    __shared__ int tot;
    int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int pre = block_exclusive_scan(s, &tot);
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        if (base + k < n) out[base + k] = pre;
        pre += v[k];
    }
    if (threadIdx.x == 0 && block_sums) block_sums[blockIdx.x] = tot;
}

__global__ void scan_add_kernel(int* __restrict__ out, const int* __restrict__ n_dev, int n_host,
                                const int* __restrict__ offs) {
    int n = n_dev ? *n_dev : n_host;
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    int o = offs[blockIdx.x];
    for (int k = threadIdx.x; k < kScanTile; k += blockDim.x)
        if (base + k < n) out[base + k] += o;
}

__global__ void copy_int_kernel(const int* src, int* dst) { *dst = *src; }

// Exclusive scan of in[0..n) into out; if total_dev, *total_dev = sum.  n may
// be given on the device (n_dev) with n_cap an upper bound for the grid.
static void scan_rec(polfmm_ctx* c, const int* in, int* out, const int* n_dev, int n_cap, int* total_dev,
                     int* scratch) {
    int nb = grid_for(n_cap, kScanTile);
    int* sums = scratch;
    int* offs = scratch + nb;
    {
        LaunchScope ls(c, F_TREE);
        scan_block_kernel<<<nb, kScanThreads, 0, c->stream>>>(in, out, n_dev, n_cap, sums);
    }
    if (nb == 1) {
        if (total_dev) {
            LaunchScope ls(c, F_TREE);
            copy_int_kernel<<<1, 1, 0, c->stream>>>(sums, total_dev);
        }
        return;
    }
    // scan the (up to nb) block sums; entries past the live blocks are zero
    // because those blocks saw no elements
    scan_rec(c, sums, offs, nullptr, nb, total_dev, scratch + 2 * nb);
    LaunchScope ls(c, F_TREE);
    scan_add_kernel<<<nb, kScanThreads, 0, c->stream>>>(out, n_dev, n_cap, offs);
}

static size_t scan_scratch_need(int n_cap) {
    size_t need = 0;
    int m = n_cap;
    do {
        int nb = grid_for(m, kScanTile);
        need += 2 * (size_t)nb;
        m = nb;
        if (nb == 1) break;
    } while (true);
    return need + 8;
}

int scan_exclusive(polfmm_ctx* c, const int* in, int* out, int n, int* total_dev) {
    scan_rec(c, in, out, nullptr, n, total_dev, c->scan_tmp);
    return POLFMM_OK;
}

static void scan_exclusive_dev(polfmm_ctx* c, const int* in, int* out, const int* n_dev, int n_cap, int* total_dev) {
    scan_rec(c, in, out, n_dev, n_cap, total_dev, c->scan_tmp);
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of (uint32 key, int32 value) pairs
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;

template <int BITS>
__global__ void radix_hist_kernel(const uint32_t* __restrict__ key, const int* __restrict__ n_dev, int n_host,
                                  int shift, int ntiles, int* __restrict__ counts) {
    constexpr int RADIX = 1 << BITS;
    int n = n_dev ? *n_dev : n_host;
    __shared__ int h[RADIX];
    for (int d = threadIdx.x; d < RADIX; d += blockDim.x) h[d] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int k = threadIdx.x; k < kSortTile; k += blockDim.x) {
        int64_t i = base + k;
        if (i < n) atomicAdd(&h[(key[i] >> shift) & (RADIX - 1)], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RADIX; d += blockDim.x) counts[d * ntiles + blockIdx.x] = h[d];
}

template <int BITS>
__global__ void radix_scatter_kernel(const uint32_t* __restrict__ kin, const int* __restrict__ vin,
                                     uint32_t* __restrict__ kout, int* __restrict__ vout,
                                     const int* __restrict__ n_dev, int n_host, int shift, int ntiles,
                                     const int* __restrict__ offsets) {
    constexpr int RADIX = 1 << BITS;
    constexpr int NW = kSortThreads / 32;
    int n = n_dev ? *n_dev : n_host;
    __shared__ int s_base[RADIX];
    __shared__ int s_warp[NW][RADIX];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < RADIX; d += blockDim.x) s_base[d] = offsets[d * ntiles + blockIdx.x];
    const unsigned lt_mask = (1u << lane) - 1u;
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int round = 0; round < kSortItems; round++) {
        for (int d = threadIdx.x; d < NW * RADIX; d += blockDim.x) (&s_warp[0][0])[d] = 0;
        __syncthreads();
        int64_t i = base + (int64_t)round * kSortThreads + threadIdx.x;
        bool valid = i < n;
        uint32_t k = valid ? kin[i] : 0u;
        int v = valid ? vin[i] : 0;
        int digit = valid ? (int)((k >> shift) & (RADIX - 1)) : RADIX;
        unsigned peers = __match_any_sync(0xffffffffu, digit);
        int rank = __popc(peers & lt_mask);
        bool leader = (__ffs(peers) - 1) == lane;
        if (valid && leader) s_warp[w][digit] = __popc(peers);
        __syncthreads();
        if (valid) {
            int pre = 0;
            for (int u = 0; u < w; u++) pre += s_warp[u][digit];
            int pos = s_base[digit] + pre + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
        for (int d = threadIdx.x; d < RADIX; d += blockDim.x) {
            int t = 0;
            for (int u = 0; u < NW; u++) t += s_warp[u][d];
            s_base[d] += t;
        }
        __syncthreads();
    }
}

// Sort pairs stably by the bits [0, nbits) of the keys.  Results end in
// (key_a, val_a); (key_b, val_b) is scratch of the same size.
template <int BITS>
static void radix_pass(polfmm_ctx* c, const uint32_t* kin, const int* vin, uint32_t* kout, int* vout,
                       const int* n_dev, int n_cap, int shift) {
    constexpr int RADIX = 1 << BITS;
    int ntiles = grid_for(n_cap, kSortTile);
    {
        LaunchScope ls(c, F_TREE);
        radix_hist_kernel<BITS><<<ntiles, kSortThreads, 0, c->stream>>>(kin, n_dev, n_cap, shift, ntiles, c->counts);
    }
    scan_exclusive_dev(c, c->counts, c->counts + (size_t)RADIX * ntiles, nullptr, RADIX * ntiles, nullptr);
    LaunchScope ls(c, F_TREE);
    radix_scatter_kernel<BITS><<<ntiles, kSortThreads, 0, c->stream>>>(
        kin, vin, kout, vout, n_dev, n_cap, shift, ntiles, c->counts + (size_t)RADIX * ntiles);
}

// ---------------------------------------------------------------------------
// sorted site arrays
// ---------------------------------------------------------------------------
template <typename R>
__global__ void gather_sorted_kernel(int64_t n, const int* __restrict__ perm, const uint32_t* __restrict__ key,
                                     const double* __restrict__ x, const double* __restrict__ q,
                                     const double* __restrict__ a, double* __restrict__ xs, double* __restrict__ qs,
                                     double* __restrict__ as, double* __restrict__ ias, R* __restrict__ ploc,
                                     double lo0, double lo1, double lo2, double h, int* __restrict__ err) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int j = perm[i];
    uint32_t k = key[i];
    uint32_t cc[3] = {compact3(k), compact3(k >> 1), compact3(k >> 2)};
    double lo[3] = {lo0, lo1, lo2};
    for (int d = 0; d < 3; d++) {
        double v = x[3 * (int64_t)j + d];
        xs[3 * i + d] = v;
        double zc = lo[d] + ((double)cc[d] + 0.5) * h;
        ploc[3 * i + d] = (R)(v - zc);
    }
    double qq = q[j], aa = a[j];
    if (!isfinite(qq) || !isfinite(aa) || aa < 0.0) atomicOr(err, 1);
    qs[i] = qq;
    as[i] = aa;
    ias[i] = aa > 0.0 ? 1.0 / aa : 0.0;  // the solver multiplies by 1/alpha (FP64 division is slow here)
}

// ---------------------------------------------------------------------------
// box tables
// ---------------------------------------------------------------------------
// leaf level: run starts of the sorted keys
__global__ void leaf_flags_kernel(const uint32_t* __restrict__ key, int64_t n, int* __restrict__ flags) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    flags[i] = (i == 0 || key[i] != key[i - 1]) ? 1 : 0;
}

__global__ void leaf_scatter_kernel(const uint32_t* __restrict__ key, int64_t n, const int* __restrict__ flags,
                                    const int* __restrict__ pos, int* __restrict__ lkey, int* __restrict__ lstart) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (flags[i]) {
        lkey[pos[i]] = (int)key[i];
        lstart[pos[i]] = (int)i;
    }
}

__global__ void leaf_count_kernel(const int* __restrict__ nleaf_dev, int64_t n, const int* __restrict__ lstart,
                                  int* __restrict__ lcount) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    int nl = *nleaf_dev;
    if (b >= nl) return;
    int e = (b + 1 < nl) ? lstart[b + 1] : (int)n;
    lcount[b] = e - lstart[b];
}

// parent level from a sorted child key list
__global__ void parent_flags_kernel(const int* __restrict__ ckey, const int* __restrict__ nc_dev, int* __restrict__ flags) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int nc = *nc_dev;
    if (i >= nc) return;
    flags[i] = (i == 0 || (ckey[i] >> 3) != (ckey[i - 1] >> 3)) ? 1 : 0;
}

__global__ void parent_scatter_kernel(const int* __restrict__ ckey, const int* __restrict__ nc_dev,
                                      const int* __restrict__ flags, const int* __restrict__ pos,
                                      int* __restrict__ pkey, int* __restrict__ child0, int* __restrict__ cparent) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int nc = *nc_dev;
    if (i >= nc) return;
    int pslot = pos[i] + flags[i] - 1;
    cparent[i] = pslot;
    if (flags[i]) {
        pkey[pos[i]] = ckey[i] >> 3;
        child0[pos[i]] = i;
    }
}

__global__ void nchild_kernel(const int* __restrict__ np_dev, const int* __restrict__ nc_dev,
                              const int* __restrict__ child0, int* __restrict__ nchild) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    int np = *np_dev;
    if (b >= np) return;
    int e = (b + 1 < np) ? child0[b + 1] : *nc_dev;
    nchild[b] = e - child0[b];
}

__global__ void map_scatter_kernel(const int* __restrict__ key, const int* __restrict__ nb_dev, int* __restrict__ map) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= *nb_dev) return;
    map[key[b]] = b;
}

__global__ void iota_kernel(int* __restrict__ v, const int* __restrict__ n_dev) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < *n_dev) v[b] = b;
}

__global__ void class_count_kernel(const int* __restrict__ key, const int* __restrict__ nb_dev, int* __restrict__ cnt8) {
    __shared__ int h[8];
    if (threadIdx.x < 8) h[threadIdx.x] = 0;
    __syncthreads();
    int nb = *nb_dev;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) atomicAdd(&h[key[b] & 7], 1);
    __syncthreads();
    if (threadIdx.x < 8) atomicAdd(&cnt8[threadIdx.x], h[threadIdx.x]);
}

// near-field work of each leaf (targets x sources in the 27 adjacent leaves),
// as an ascending sort key for descending work
__global__ void leaf_work_kernel(int nleaf, int depth, const int* __restrict__ lkey, const int* __restrict__ lcount,
                                 const int* __restrict__ lmap, uint32_t* __restrict__ key, int* __restrict__ idx) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    const uint32_t k = (uint32_t)lkey[b];
    const int bx = (int)compact3(k), by = (int)compact3(k >> 1), bz = (int)compact3(k >> 2);
    const int nside = 1 << depth;
    long src = 0;
    for (int dz = -1; dz <= 1; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                int ax = bx + dx, ay = by + dy, az = bz + dz;
                if (ax < 0 || ay < 0 || az < 0 || ax >= nside || ay >= nside || az >= nside) continue;
                int s = lmap[morton3(ax, ay, az)];
                if (s >= 0) src += lcount[s];
            }
    long w = (long)lcount[b] * src;
    long q = w >> 4;
    key[b] = 0xFFFFu - (uint32_t)(q > 0xFFFF ? 0xFFFF : q);
    idx[b] = b;
}

// near-field blocks: leaf r of the work order covers ceil(count / targets)
// blocks of at most targets targets each
__global__ void leaf_split_count_kernel(int nleaf, const int* __restrict__ order, const int* __restrict__ lcount,
                                        int targets, int* __restrict__ nsplit) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nleaf) return;
    nsplit[r] = (lcount[order[r]] + targets - 1) / targets;
}

__global__ void leaf_items_kernel(int nleaf, const int* __restrict__ order, const int* __restrict__ lcount,
                                  const int* __restrict__ first, int targets, int2* __restrict__ items, int cap) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nleaf) return;
    const int b = order[r], cnt = lcount[b];
    int o = first[r];
    for (int t = 0; t < cnt && o < cap; t += targets) items[o++] = make_int2(b, t);
}

int tree_build(polfmm_ctx* c, const double* x_in) {
    const int64_t n = c->n;
    const int d = c->depth;
    const int nside = 1 << d;
    cudaStream_t st = c->stream;
    double h = c->side / (double)nside;

    // keys and stable sort
    {
        LaunchScope ls(c, F_TREE);
        keys_kernel<<<grid_for(n, 256), 256, 0, st>>>(x_in, n, c->lo[0],
                                                      c->lo[1], c->lo[2], h, nside, c->key_tmp, c->val_tmp, c->err);
    }
    // pairs start in (key_tmp, val_tmp); passes alternate between the two buffers
    uint32_t* ka = c->key_tmp;
    int* va = c->val_tmp;
    uint32_t* kb = c->key_s;
    int* vb = c->perm;
    int nbits = 3 * d;
    int npass = (nbits + 7) / 8;
    for (int ps = 0; ps < npass; ps++) {
        radix_pass<8>(c, ka, va, kb, vb, nullptr, (int)n, 8 * ps);
        uint32_t* tk = ka; ka = kb; kb = tk;
        int* tv = va; va = vb; vb = tv;
    }
    if (ka != c->key_s) {
        cudaMemcpyAsync(c->key_s, ka, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(c->perm, va, sizeof(int) * n, cudaMemcpyDeviceToDevice, st);
    }
    return POLFMM_OK;
}

int tree_tables(polfmm_ctx* c, const double* x_in, const double* q_in, const double* a_in) {
    const int64_t n = c->n;
    const int d = c->depth;
    cudaStream_t st = c->stream;
    double h = c->side / (double)(1 << d);
    {
        LaunchScope ls(c, F_TREE);
        if (c->mixed)
            gather_sorted_kernel<float><<<grid_for(n, 256), 256, 0, st>>>(
                n, c->perm, c->key_s, x_in, q_in, a_in, c->pos_s, c->q_s, c->alpha_s, c->inv_alpha_s, (float*)c->ploc, c->lo[0],
                c->lo[1], c->lo[2], h, c->err);
        else
            gather_sorted_kernel<double><<<grid_for(n, 256), 256, 0, st>>>(
                n, c->perm, c->key_s, x_in, q_in, a_in, c->pos_s, c->q_s, c->alpha_s, c->inv_alpha_s, (double*)c->ploc, c->lo[0],
                c->lo[1], c->lo[2], h, c->err);
    }
    // device counters: [kMaxDepth + 1] box counts, then [kMaxDepth + 1][8] class counts
    int* nbox_dev = c->tree_cnt;
    int* cls_dev = nbox_dev + (kMaxDepth + 1);
    cudaMemsetAsync(nbox_dev, 0, sizeof(int) * (kMaxDepth + 1) * 9, st);

    // leaf level
    Level& L = c->lv[d];
    {
        LaunchScope ls(c, F_TREE);
        leaf_flags_kernel<<<grid_for(n, 256), 256, 0, st>>>(c->key_s, n, c->flags);
    }
    scan_exclusive_dev(c, c->flags, c->val_a, nullptr, (int)n, nbox_dev + d);
    {
        LaunchScope ls(c, F_TREE);
        leaf_scatter_kernel<<<grid_for(n, 256), 256, 0, st>>>(c->key_s, n, c->flags, c->val_a, L.key, c->lstart);
    }
    {
        LaunchScope ls(c, F_TREE);
        leaf_count_kernel<<<grid_for(L.cap, 256), 256, 0, st>>>(nbox_dev + d, n, c->lstart, c->lcount);
    }
    // coarser levels
    for (int l = d - 1; l >= 0; l--) {
        Level& C = c->lv[l + 1];
        Level& P = c->lv[l];
        {
            LaunchScope ls(c, F_TREE);
            parent_flags_kernel<<<grid_for(C.cap, 256), 256, 0, st>>>(C.key, nbox_dev + l + 1, c->flags);
        }
        scan_exclusive_dev(c, c->flags, c->val_a, nbox_dev + l + 1, C.cap, nbox_dev + l);
        {
            LaunchScope ls(c, F_TREE);
            parent_scatter_kernel<<<grid_for(C.cap, 256), 256, 0, st>>>(C.key, nbox_dev + l + 1, c->flags, c->val_a,
                                                                        P.key, P.child0, C.parent);
        }
        {
            LaunchScope ls(c, F_TREE);
            nchild_kernel<<<grid_for(P.cap, 256), 256, 0, st>>>(nbox_dev + l, nbox_dev + l + 1, P.child0, P.nchild);
        }
    }
    // maps and octant-class grouping
    for (int l = 0; l <= d; l++) {
        Level& B = c->lv[l];
        size_t mapn = (size_t)1 << (3 * l);
        cudaMemsetAsync(B.map, 0xff, sizeof(int) * mapn, st);
        {
            LaunchScope ls(c, F_TREE);
            map_scatter_kernel<<<grid_for(B.cap, 256), 256, 0, st>>>(B.key, nbox_dev + l, B.map);
        }
        if (l >= 2) {
            {
                LaunchScope ls(c, F_TREE);
                iota_kernel<<<grid_for(B.cap, 256), 256, 0, st>>>(c->val_tmp, nbox_dev + l);
            }
            {
                LaunchScope ls(c, F_TREE);
                class_count_kernel<<<std::min(grid_for(B.cap, 256), 64), 256, 0, st>>>(B.key, nbox_dev + l,
                                                                                       cls_dev + 8 * l);
            }
            radix_pass<3>(c, (const uint32_t*)B.key, c->val_tmp, c->key_tmp, B.by_class, nbox_dev + l, B.cap, 0);
        }
    }
    cudaMemcpyAsync(c->h_counts, nbox_dev, sizeof(int) * (kMaxDepth + 1) * 9, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return POLFMM_ERR_CUDA;
    // leaves in descending order of near-field work, so that the heaviest
    // leaf blocks start first and the lighter ones fill in behind them
    {
        const int nl = c->h_counts[d];
        {
            LaunchScope ls(c, F_TREE);
            leaf_work_kernel<<<grid_for(nl, 256), 256, 0, st>>>(nl, d, L.key, c->lcount, L.map, c->key_tmp,
                                                                c->val_tmp);
        }
        uint32_t* kb = reinterpret_cast<uint32_t*>(c->flags);
        radix_pass<8>(c, c->key_tmp, c->val_tmp, kb, c->val_a, nullptr, nl, 0);
        radix_pass<8>(c, kb, c->val_a, c->key_tmp, c->leaf_order, nullptr, nl, 8);
        // heavy leaves split by targets, in the same order
        {
            LaunchScope ls(c, F_TREE);
            leaf_split_count_kernel<<<grid_for(nl, 256), 256, 0, st>>>(nl, c->leaf_order, c->lcount,
                                                                       leaf_targets(c->mixed), c->flags);
        }
        scan_exclusive_dev(c, c->flags, c->val_a, nullptr, nl, c->leaf_nitems);
        {
            LaunchScope ls(c, F_TREE);
            leaf_items_kernel<<<grid_for(nl, 256), 256, 0, st>>>(nl, c->leaf_order, c->lcount, c->val_a,
                                                                 leaf_targets(c->mixed), c->leaf_items,
                                                                 c->leaf_items_cap);
        }
    }
    c->leaf_items_grid =
        (int)std::min<int64_t>(c->leaf_items_cap, (int64_t)c->h_counts[d] + n / leaf_targets(c->mixed) + 1);
    for (int l = 0; l <= d; l++) {
        Level& B = c->lv[l];
        B.nbox = c->h_counts[l];
        int s = 0;
        for (int k = 0; k < 8; k++) {
            B.class_count[k] = l >= 2 ? c->h_counts[kMaxDepth + 1 + 8 * l + k] : 0;
            B.class_start[k] = s;
            s += B.class_count[k];
        }
    }
    return POLFMM_OK;
}

size_t tree_scan_scratch(int64_t n) { return scan_scratch_need((int)std::max<int64_t>(n, 1 << 12)) + 64; }

size_t tree_count_scratch(int64_t n) {
    int ntiles = grid_for(std::max<int64_t>(n, 1), kSortTile);
    return 2 * 256 * (size_t)ntiles + 64;
}

// bounding cube: device reduction, then the same FP64 arithmetic as the
// documented rule (centre of the box, side = largest extent * (1 + 1e-6))
int tree_root_box(polfmm_ctx* c, const double* x_dev, double* part_dev, double* h_pinned) {
    {
        LaunchScope ls(c, F_TREE);
        bbox_partial_kernel<<<kBBoxBlocks, 256, 0, c->stream>>>(x_dev, c->n, part_dev);
    }
    {
        LaunchScope ls(c, F_TREE);
        bbox_final_kernel<<<1, 6 * 32, 0, c->stream>>>(part_dev, kBBoxBlocks, part_dev + 6 * kBBoxBlocks);
    }
    cudaMemcpyAsync(h_pinned, part_dev + 6 * kBBoxBlocks, 6 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return POLFMM_ERR_CUDA;
    double ext = 0.0;
    for (int d = 0; d < 3; d++) {
        double e = h_pinned[3 + d] - h_pinned[d];
        if (!(e == e)) return POLFMM_ERR_INVALID_ARG;
        if (e > ext) ext = e;
    }
    if (!isfinite(ext)) return POLFMM_ERR_INVALID_ARG;
    double s = ext > 0.0 ? ext * (1.0 + 1e-6) : 1.0;
    for (int d = 0; d < 3; d++) {
        volatile double cen = 0.5 * (h_pinned[d] + h_pinned[3 + d]);
        volatile double half = 0.5 * s;
        c->lo[d] = cen - half;
    }
    c->side = s;
    return POLFMM_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the tree set-up (fmm_sort_sites_noalloc).
//
// Some callers cannot call cudaMalloc: code whose host framework owns every
// byte of device memory through its own pool, or a time-critical loop that
// cannot afford the device-wide synchronisation of cudaMalloc / cudaFree.
// For them this variant runs the bounding-cube reduction, the Morton keys and
// the stable radix sort with all temporaries in one file-scope device array of
// fixed size instead of context-owned buffers.  The paper has no counterpart.
// ---------------------------------------------------------------------------
constexpr int64_t kNoAllocMaxSites = POLFMM_NOALLOC_MAX_SITES;
constexpr int kNoAllocTiles = (int)((kNoAllocMaxSites + kSortTile - 1) / kSortTile);
constexpr size_t kNAKeys = 0;                                                // uint32 [max sites]
constexpr size_t kNAVals = kNAKeys + 4 * (size_t)kNoAllocMaxSites;          // int32 [max sites]
constexpr size_t kNACounts = kNAVals + 4 * (size_t)kNoAllocMaxSites;        // int32 [2 * 256 * tiles]
constexpr size_t kNAScan = kNACounts + 4 * 2 * 256 * (size_t)kNoAllocTiles;  // int32 [4096]
constexpr size_t kNABBox = kNAScan + 4 * 4096;                               // double [1024]
constexpr size_t kNAErr = kNABBox + 8 * 1024;                                // int32 [64]
constexpr size_t kNoAllocBytes = kNAErr + 256;

// Held by every device that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static std::mutex g_noalloc_mutex;
static void* g_noalloc_ptr[64];

// Device address of the scratch array on the current device.  The host-side
// name g_noalloc_scratch is not a device address; it is resolved once per
// device with cudaGetSymbolAddress, with that device current.
static int noalloc_scratch(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return POLFMM_ERR_CUDA;
    }
    std::lock_guard<std::mutex> guard(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return POLFMM_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = reinterpret_cast<unsigned char*>(g_noalloc_ptr[dev]);
    return POLFMM_OK;
}

__global__ void cells_from_keys_kernel(const uint32_t* __restrict__ key, int64_t n, int32_t* __restrict__ cells) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t k = key[i];
    cells[3 * i] = (int32_t)compact3(k);
    cells[3 * i + 1] = (int32_t)compact3(k >> 1);
    cells[3 * i + 2] = (int32_t)compact3(k >> 2);
}

static void noalloc_scan(cudaStream_t st, const int* in, int* out, int n, int* scratch) {
    int nb = grid_for(n, kScanTile);
    int* sums = scratch;
    int* offs = scratch + nb;
    scan_block_kernel<<<nb, kScanThreads, 0, st>>>(in, out, nullptr, n, sums);
    if (nb == 1) return;
    noalloc_scan(st, sums, offs, nb, scratch + 2 * nb);
    scan_add_kernel<<<nb, kScanThreads, 0, st>>>(out, nullptr, n, offs);
}

static void noalloc_radix_pass(cudaStream_t st, const uint32_t* kin, const int* vin, uint32_t* kout, int* vout,
                               int n, int shift, int* counts, int* scan_scratch) {
    int ntiles = grid_for(n, kSortTile);
    radix_hist_kernel<8><<<ntiles, kSortThreads, 0, st>>>(kin, nullptr, n, shift, ntiles, counts);
    noalloc_scan(st, counts, counts + 256 * ntiles, 256 * ntiles, scan_scratch);
    radix_scatter_kernel<8><<<ntiles, kSortThreads, 0, st>>>(kin, vin, kout, vout, nullptr, n, shift, ntiles,
                                                            counts + 256 * ntiles);
}

}  // namespace polfmm

extern "C" POLFMM_API int fmm_sort_sites_noalloc(int64_t n, const double* positions, int tree_depth, double* root_lo,
                                      double* root_side, int32_t* cells, uint32_t* keys, int32_t* perm,
                                      void* cuda_stream) {
    using namespace polfmm;
    if (n < 1 || !positions || !root_lo || !root_side || !cells || !keys || !perm) return POLFMM_ERR_INVALID_ARG;
    if (n > kNoAllocMaxSites) return POLFMM_ERR_INVALID_ARG;
    if (tree_depth < 1 || tree_depth > kMaxDepth) return POLFMM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned char* S = nullptr;
    int rc = noalloc_scratch(&S);
    if (rc != POLFMM_OK) return rc;
    uint32_t* key_tmp = reinterpret_cast<uint32_t*>(S + kNAKeys);
    int* val_tmp = reinterpret_cast<int*>(S + kNAVals);
    int* counts = reinterpret_cast<int*>(S + kNACounts);
    int* scan_scratch = reinterpret_cast<int*>(S + kNAScan);
    double* bbox = reinterpret_cast<double*>(S + kNABBox);
    int* err = reinterpret_cast<int*>(S + kNAErr);
    // the array keeps the previous call's contents: clear the error word
    if (cudaMemsetAsync(err, 0, sizeof(int) * 4, st) != cudaSuccess) return POLFMM_ERR_CUDA;
    // root cube: same reduction and the same FP64 rule as fmm_build
    bbox_partial_kernel<<<kBBoxBlocks, 256, 0, st>>>(positions, n, bbox);
    bbox_final_kernel<<<1, 6 * 32, 0, st>>>(bbox, kBBoxBlocks, bbox + 6 * kBBoxBlocks);
    double hb[6];
    if (cudaMemcpyAsync(hb, bbox + 6 * kBBoxBlocks, sizeof(hb), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return POLFMM_ERR_CUDA;
    double ext = 0.0;
    for (int d = 0; d < 3; d++) {
        double e = hb[3 + d] - hb[d];
        if (!(e == e)) return POLFMM_ERR_INVALID_ARG;
        if (e > ext) ext = e;
    }
    if (!isfinite(ext)) return POLFMM_ERR_INVALID_ARG;
    double side = ext > 0.0 ? ext * (1.0 + 1e-6) : 1.0;
    for (int d = 0; d < 3; d++) {
        volatile double cen = 0.5 * (hb[d] + hb[3 + d]);
        volatile double half = 0.5 * side;
        root_lo[d] = cen - half;
    }
    *root_side = side;
    const int nside = 1 << tree_depth;
    const double h = side / (double)nside;
    // keys start in the buffer that makes the last pass land in keys / perm
    const int npass = (3 * tree_depth + 7) / 8;
    uint32_t* ka = (npass & 1) ? key_tmp : keys;
    int* va = (npass & 1) ? val_tmp : perm;
    uint32_t* kb = (npass & 1) ? keys : key_tmp;
    int* vb = (npass & 1) ? perm : val_tmp;
    keys_kernel<<<grid_for(n, 256), 256, 0, st>>>(positions, n, root_lo[0], root_lo[1], root_lo[2], h, nside, ka,
                                                  va, err);
    cells_from_keys_kernel<<<grid_for(n, 256), 256, 0, st>>>(ka, n, cells);
    for (int ps = 0; ps < npass; ps++) {
        noalloc_radix_pass(st, ka, va, kb, vb, (int)n, 8 * ps, counts, scan_scratch);
        uint32_t* tk = ka; ka = kb; kb = tk;
        int* tv = va; va = vb; vb = tv;
    }
    int herr[4] = {0, 0, 0, 0};
    if (cudaMemcpyAsync(herr, err, sizeof(herr), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return POLFMM_ERR_CUDA;
    return herr[0] ? POLFMM_ERR_INVALID_ARG : POLFMM_OK;
}
