// Exclusion lists and field charges (the Polaris specifics of Sec. II.A and
// Sec. III): the starred sums of the Coulomb energy, the static field and the
// dipole field skip a list of excluded pairs, and only the field charges q^E
// (which may differ from the Coulomb charges q) generate the field that
// polarizes the sites.
//
// The FMM passes sum over all pairs; the kernel here then subtracts, at every
// site that has excluded partners, the direct terms of those partners (the
// near field evaluated them directly, the far field through the expansions):
// FMM(all pairs) - direct(excluded pairs).  One thread per such site adds its
// partners in a fixed (ascending) order, so the result is deterministic.
//
// Thole damping of the dipole-dipole tensor (Sec. II.A cites Thole's model;
// the form is Thole's exponential model as used by AMOEBA, Ren and Ponder
// 2003): lambda3 = 1 - exp(-a u^3), lambda5 = 1 - (1 + a u^3) exp(-a u^3),
// u = r / (alpha_i alpha_j)^(1/6).  Per tree, a spatial hash lists the pairs
// with a u^3 < 40; the solve adds (T^damp - T) mu over them after the near
// field, and the force pass forms the damped-minus-undamped dipole field,
// dipole-dipole force and dU/dalpha part in FP64.
#include <cmath>

#include "internal.cuh"

namespace polfmm {

// MODE 0: charges w -> Phi, E;  1: dipoles mu -> E;  2: charges w and dipoles mu -> Phi, E, grad E
// (xx xy xz yy yz zz), with r = x_target - x_source:
//   charge: Phi = w/r, E = w r/r^3, G_ab = w (delta_ab/r^3 - 3 r_a r_b/r^5)
//   dipole: Phi = mu.r/r^3, E = 3 (mu.r) r/r^5 - mu/r^3,
//           G_ab = 3 (mu_a r_b + mu_b r_a + (mu.r) delta_ab)/r^5 - 15 (mu.r) r_a r_b/r^7
template <int MODE>
__global__ void exclusion_kernel(int ntarget, const int* __restrict__ targets, const int* __restrict__ ptr,
                                 const int* __restrict__ partner, const int* __restrict__ inv_perm,
                                 const double* __restrict__ pos, const double* __restrict__ w,
                                 const double* __restrict__ mu, double* __restrict__ phi, double* __restrict__ E,
                                 double* __restrict__ G) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntarget) return;
    const int si = inv_perm[targets[t]];
    const double xi = pos[3 * (int64_t)si], yi = pos[3 * (int64_t)si + 1], zi = pos[3 * (int64_t)si + 2];
    double p = 0.0, e[3] = {0.0, 0.0, 0.0}, g[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    // component c of grad E is (a, b): xx xy xz yy yz zz
    auto ga = [](int c) { return c < 3 ? 0 : (c < 5 ? 1 : 2); };
    auto gb = [](int c) { return c < 3 ? c : (c < 5 ? c - 2 : 2); };
    for (int k = ptr[t]; k < ptr[t + 1]; k++) {
        const int sj = inv_perm[partner[k]];
        const double r[3] = {xi - pos[3 * (int64_t)sj], yi - pos[3 * (int64_t)sj + 1], zi - pos[3 * (int64_t)sj + 2]};
        const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        if (!(r2 > 0.0)) continue;  // coincident sites are reported by the near-field pass
        const double ri = 1.0 / sqrt(r2), ri2 = ri * ri, ri3 = ri * ri2, ri5 = ri3 * ri2;
        if (MODE != 1) {
            const double q = w[sj];
            p += q * ri;
            for (int d = 0; d < 3; d++) e[d] += q * ri3 * r[d];
            if (MODE == 2)
                for (int c = 0; c < 6; c++) g[c] += q * ((ga(c) == gb(c) ? ri3 : 0.0) - 3.0 * r[ga(c)] * r[gb(c)] * ri5);
        }
        if (MODE != 0) {
            const double m[3] = {mu[3 * (int64_t)sj], mu[3 * (int64_t)sj + 1], mu[3 * (int64_t)sj + 2]};
            const double mr = m[0] * r[0] + m[1] * r[1] + m[2] * r[2];
            if (MODE == 2) p += mr * ri3;
            for (int d = 0; d < 3; d++) e[d] += 3.0 * mr * r[d] * ri5 - m[d] * ri3;
            if (MODE == 2) {
                const double ri7 = ri5 * ri2;
                for (int c = 0; c < 6; c++) {
                    const int a = ga(c), b = gb(c);
                    g[c] += 3.0 * (m[a] * r[b] + m[b] * r[a] + (a == b ? mr : 0.0)) * ri5 - 15.0 * mr * r[a] * r[b] * ri7;
                }
            }
        }
    }
    if (MODE != 1 && phi) phi[si] -= p;
    for (int d = 0; d < 3; d++) E[3 * (int64_t)si + d] -= e[d];
    if (MODE == 2 && G)
        for (int c = 0; c < 6; c++) G[6 * (int64_t)si + c] -= g[c];
}

__global__ void inv_perm_kernel(int64_t n, const int* __restrict__ perm, int* __restrict__ inv) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < n) inv[perm[k]] = (int)k;
}

void exclusion_correct(polfmm_ctx* c, int leaf_mode, const double* w_sorted, const double* mu_sorted, double* phi,
                       double* E, double* G, cudaStream_t st) {
    if (c->n_excl == 0 || c->n_excl_targets == 0) return;
    LaunchScope ls(c, F_LEAF_STATIC);
    const int nt = c->n_excl_targets, grid = grid_for(nt, 128);
    if (leaf_mode == LEAF_DIPOLE_E)
        exclusion_kernel<1><<<grid, 128, 0, st>>>(nt, c->excl_targets, c->excl_ptr, c->excl_idx, c->inv_perm, c->pos_s,
                                                   nullptr, mu_sorted, nullptr, E, nullptr);
    else if (leaf_mode == LEAF_CHARGE_PHI_E || !mu_sorted)
        exclusion_kernel<0><<<grid, 128, 0, st>>>(nt, c->excl_targets, c->excl_ptr, c->excl_idx, c->inv_perm, c->pos_s,
                                                   w_sorted, nullptr, phi, E, nullptr);
    else
        exclusion_kernel<2><<<grid, 128, 0, st>>>(nt, c->excl_targets, c->excl_ptr, c->excl_idx, c->inv_perm, c->pos_s,
                                                   w_sorted, mu_sorted, phi, E, G);
}

// ---------------------------------------------------------------------------
// Thole damping
// ---------------------------------------------------------------------------
constexpr double kTholeAu3Max = 40.0;  // exp(-40) = 4e-18: beyond, the damping is 1 in FP64

__device__ inline uint32_t th_bucket_of(int cx, int cy, int cz, uint32_t mask) {
    return ((uint32_t)cx * 73856093u ^ (uint32_t)cy * 19349663u ^ (uint32_t)cz * 83492791u) & mask;
}

__device__ inline int th_coord(double x, double inv_l) {
    double c = floor(x * inv_l);
    c = fmin(fmax(c, -1.0e9), 1.0e9);
    return (int)c;
}

// alpha^(1/6) per sorted site and their maximum (non-negative doubles order as
// their bit patterns)
__global__ void th_a16_kernel(int64_t n, const double* __restrict__ alpha, const double* __restrict__ pos,
                              double* __restrict__ a16, float4* __restrict__ xa, unsigned long long* __restrict__ amax) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = alpha[i] > 0.0 ? cbrt(sqrt(alpha[i])) : 0.0;
    a16[i] = v;
    xa[i] = make_float4(float(pos[3 * i]), float(pos[3 * i + 1]), float(pos[3 * i + 2]), float(v));
    atomicMax(amax, (unsigned long long)__double_as_longlong(v));
}

__global__ void th_cell_kernel(int64_t n, const double* __restrict__ pos, double inv_l, uint32_t mask,
                               int4* __restrict__ cell, int* __restrict__ count) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int cx = th_coord(pos[3 * i], inv_l), cy = th_coord(pos[3 * i + 1], inv_l), cz = th_coord(pos[3 * i + 2], inv_l);
    const uint32_t b = th_bucket_of(cx, cy, cz, mask);
    cell[i] = make_int4(cx, cy, cz, (int)b);
    atomicAdd(&count[b], 1);
}

__global__ void th_fill_kernel(int64_t n, const int4* __restrict__ cell, int* __restrict__ start, int nb,
                               int* __restrict__ count, int* __restrict__ member) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i == 0) start[nb] = (int)n;
    if (i >= n) return;
    const int b = cell[i].w;
    const int k = atomicSub(&count[b], 1) - 1;
    member[start[b] + k] = (int)i;
}

// ascending site index within each bucket, so that the pair lists come out in
// a fixed order: one warp per bucket, each member placed at its rank (the
// number of smaller indices in the bucket; indices are distinct)
__global__ void th_order_kernel(int nb, const int* __restrict__ start, const int* __restrict__ member_in,
                                int* __restrict__ member_out) {
    const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (w >= nb) return;
    const int s = start[w], e = start[w + 1];
    for (int a = s + lane; a < e; a += 32) {
        const int v = member_in[a];
        int rank = 0;
        for (int b = s; b < e; b++) rank += member_in[b] < v;
        member_out[s + rank] = v;
    }
}

// damped partners of every sorted site i, G lanes per site: lane g takes the
// neighbour cells g, g + G, ... of the 27.  COUNT: per-site totals; else each
// lane writes its partners at ptr[i] + (partners of the lanes before it), so
// the list order is fixed
constexpr int kThLanes = 8;
template <bool COUNT>
__global__ void th_pairs_kernel(int64_t n, const float4* __restrict__ xa,
                                const int4* __restrict__ cell, const int* __restrict__ start,
                                const int* __restrict__ member, uint32_t mask, float umax,
                                const int* __restrict__ perm, const int* __restrict__ excl_row,
                                const int* __restrict__ excl_ptr, const int* __restrict__ excl_idx,
                                int* __restrict__ cnt, const int* __restrict__ ptr, int* __restrict__ idx) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t i = t / kThLanes;
    const int g = (int)(t % kThLanes);
    const bool live = i < n;
    const float4 me = live ? xa[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float si = me.w;
    int4 ci = make_int4(0, 0, 0, 0);
    int row = -1;
    if (live && si > 0.f) {
        ci = cell[i];
        row = excl_row ? excl_row[perm[i]] : -1;
    }
    // pass 0 counts this lane's partners; the write pass repeats it to find the
    // lane's offset, then writes
    int out = 0;
    for (int pass = 0; pass < (COUNT ? 1 : 2); pass++) {
        int k = 0;
        if (live && si > 0.f) {
            for (int cc = g; cc < 27; cc += kThLanes) {
                const int cx = ci.x + cc % 3 - 1, cy = ci.y + (cc / 3) % 3 - 1, cz = ci.z + cc / 9 - 1;
                const uint32_t b = th_bucket_of(cx, cy, cz, mask);
                for (int m = start[b]; m < start[b + 1]; m++) {
                    const int j = member[m];
                    if (j == (int)i) continue;
                    const int4 cj = cell[j];
                    if (cj.x != cx || cj.y != cy || cj.z != cz) continue;
                    // in FP32 (a pair at the cut-off contributes exp(-40) either way, and FP64
                    // is a narrow unit here); every pass takes the same decisions
                    const float4 o = xa[j];
                    if (!(o.w > 0.f)) continue;
                    const float rx = me.x - o.x, ry = me.y - o.y, rz = me.z - o.z;
                    const float rc = umax * si * o.w;
                    if (!(rx * rx + ry * ry + rz * rz < rc * rc)) continue;
                    if (row >= 0) {
                        // excluded pairs stay excluded: binary search in the ascending partners
                        const int pj = perm[j];
                        int lo = excl_ptr[row], hi = excl_ptr[row + 1];
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if (excl_idx[mid] < pj) lo = mid + 1; else hi = mid;
                        }
                        if (lo < excl_ptr[row + 1] && excl_idx[lo] == pj) continue;
                    }
                    if (!COUNT && pass == 1) idx[out++] = j;
                    k++;
                }
            }
        }
        // inclusive scan of the lane counts within the group of G lanes
        int incl = k;
        for (int o = 1; o < kThLanes; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o, kThLanes);
            if (g >= o) incl += v;
        }
        if (COUNT) {
            if (live && g == kThLanes - 1) cnt[i] = incl;
        } else if (pass == 0) {
            out = live ? ptr[i] + incl - k : 0;
        }
    }
}

// MIXED: the geometry of every pair once per tree (the solve's passes then only
// load it): r_ij = x_i - x_j from the FP64 positions, 3 (lambda5 - 1) / r^5 and
// (lambda3 - 1) / r^3, in FP32
__global__ void th_coef_kernel(int64_t n, const int* __restrict__ ptr, const int* __restrict__ idx,
                               const double* __restrict__ pos, const double* __restrict__ a16, double a_in,
                               float4* __restrict__ rr, float* __restrict__ t3) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t i = t / kThLanes;
    const int g = (int)(t % kThLanes);
    if (i >= n) return;
    const double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
    const float si = float(a16[i]), a = float(a_in);
    for (int k = ptr[i] + g; k < ptr[i + 1]; k += kThLanes) {
        const int j = idx[k];
        const float rx = float(xi - pos[3 * (int64_t)j]), ry = float(yi - pos[3 * (int64_t)j + 1]),
                    rz = float(zi - pos[3 * (int64_t)j + 2]);
        const float r2 = rx * rx + ry * ry + rz * rz;
        const float ri = 1.f / sqrtf(r2), ri2 = ri * ri, ri3 = ri * ri2, ri5 = ri3 * ri2;
        const float u = (r2 * ri) / (si * float(a16[j]));
        const float au3 = a * u * u * u;
        const float ex = expf(-au3);
        rr[k] = make_float4(rx, ry, rz, 3.f * (-(1.f + au3) * ex) * ri5);
        t3[k] = -ex * ri3;
    }
}

int thole_pairs(polfmm_ctx* c) {
    c->th_npairs = 0;
    if (!(c->thole_a > 0.0)) return POLFMM_OK;
    const int64_t n = c->n;
    cudaStream_t st = c->stream;
    if (!c->a16) return POLFMM_ERR_STATE;  // fmm_set_thole allocates the scratch
    const int nb = c->th_nb;
    const uint32_t mask = (uint32_t)nb - 1u;
    const double umax = std::cbrt(kTholeAu3Max / c->thole_a);
    {
        LaunchScope ls(c, F_TREE);
        cudaMemsetAsync(c->th_max, 0, sizeof(double), st);
        th_a16_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, c->alpha_s, c->pos_s, c->a16, c->th_xa,
                                                          reinterpret_cast<unsigned long long*>(c->th_max));
    }
    double amax = 0.0;
    cudaError_t e = cudaMemcpyAsync(c->h_scal + S_COUNT, c->th_max, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "Thole pair list (largest polarizability)");
    amax = c->h_scal[S_COUNT];
    if (!(amax > 0.0)) return POLFMM_OK;  // no polarizable site: nothing to damp
    const double cellside = umax * amax * amax;  // the largest cut-off of any pair
    cudaMemsetAsync(c->th_count, 0, sizeof(int) * nb, st);
    {
        LaunchScope ls(c, F_TREE);
        th_cell_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, c->pos_s, 1.0 / cellside, mask, c->th_cell, c->th_count);
    }
    scan_exclusive(c, c->th_count, c->th_bucket, nb, nullptr);
    {
        LaunchScope ls(c, F_TREE);
        th_fill_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, c->th_cell, c->th_bucket, nb, c->th_count, c->th_cnt);
        th_order_kernel<<<grid_for((int64_t)nb * 32, 256), 256, 0, st>>>(nb, c->th_bucket, c->th_cnt, c->th_member);
        th_pairs_kernel<true><<<grid_for(n * kThLanes, 128), 128, 0, st>>>(
            n, c->th_xa, c->th_cell, c->th_bucket, c->th_member, mask, float(umax), c->perm,
            c->n_excl ? c->excl_row : nullptr, c->excl_ptr, c->excl_idx, c->th_cnt, nullptr, nullptr);
    }
    scan_exclusive(c, c->th_cnt, c->th_ptr, (int)n, c->th_ptr + n);
    int total = 0;
    e = cudaMemcpyAsync(&total, c->th_ptr + n, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "Thole pair count");
    if (total > c->th_cap) {
        if (c->th_idx) cudaFree(c->th_idx);
        if (c->th_r) cudaFree(c->th_r);
        if (c->th_t3) cudaFree(c->th_t3);
        c->th_idx = nullptr;
        c->th_r = nullptr;
        c->th_t3 = nullptr;
        c->th_cap = 0;
        const size_t m = (size_t)std::max(total, 1);
        if (dev_alloc(reinterpret_cast<void**>(&c->th_idx), sizeof(int) * m) != cudaSuccess ||
            (c->mixed && (dev_alloc(reinterpret_cast<void**>(&c->th_r), sizeof(float4) * m) != cudaSuccess ||
                          dev_alloc(reinterpret_cast<void**>(&c->th_t3), sizeof(float) * m) != cudaSuccess))) {
            cudaGetLastError();
            return POLFMM_ERR_OUT_OF_MEMORY;
        }
        c->th_cap = total;
    }
    {
        LaunchScope ls(c, F_TREE);
        th_pairs_kernel<false><<<grid_for(n * kThLanes, 128), 128, 0, st>>>(
            n, c->th_xa, c->th_cell, c->th_bucket, c->th_member, mask, float(umax), c->perm,
            c->n_excl ? c->excl_row : nullptr, c->excl_ptr, c->excl_idx, nullptr, c->th_ptr, c->th_idx);
    }
    if (c->mixed && total > 0) {
        LaunchScope ls(c, F_TREE);
        th_coef_kernel<<<grid_for(n * kThLanes, 128), 128, 0, st>>>(n, c->th_ptr, c->th_idx, c->pos_s, c->a16,
                                                                    c->thole_a, c->th_r, c->th_t3);
    }
    c->th_npairs = total;
    e = cudaGetLastError();
    return e == cudaSuccess ? POLFMM_OK : cuda_fail(e, "Thole pair list");
}

// E_i += sum_j (T^damp - T) mu_j = sum_j 3 (lambda5 - 1) (mu_j.r) r / r^5 - (lambda3 - 1) mu_j / r^3,
// in R (the mode's precision); one thread per site, partners in list order
template <typename R>
__global__ void th_field_kernel(int64_t n, const int* __restrict__ ptr, const int* __restrict__ idx,
                                const double* __restrict__ pos, const double* __restrict__ a16,
                                const double* __restrict__ mu, double a, double* __restrict__ E) {
    // kThLanes lanes per site take every kThLanes-th partner; the lane sums are
    // added in a fixed shuffle order
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t i = t / kThLanes;
    const int g = (int)(t % kThLanes);
    const bool live = i < n;
    const int k0 = live ? ptr[i] : 0, k1 = live ? ptr[i + 1] : 0;
    double xi = 0.0, yi = 0.0, zi = 0.0;
    R si = R(1);
    if (live && k1 > k0) {
        xi = pos[3 * i];
        yi = pos[3 * i + 1];
        zi = pos[3 * i + 2];
        si = R(a16[i]);
    }
    const R ra = R(a);
    R e0 = R(0), e1 = R(0), e2 = R(0);
    for (int k = k0 + g; k < k1; k += kThLanes) {
        const int j = idx[k];
        const R rx = R(xi - pos[3 * (int64_t)j]), ry = R(yi - pos[3 * (int64_t)j + 1]), rz = R(zi - pos[3 * (int64_t)j + 2]);
        const R r2 = rx * rx + ry * ry + rz * rz;
        const R ri = R(1) / sqrt(r2);
        const R ri2 = ri * ri, ri3 = ri * ri2, ri5 = ri3 * ri2;
        const R u = (r2 * ri) / (si * R(a16[j]));
        const R au3 = ra * u * u * u;
        const R ex = exp(-au3);
        const R d3 = -ex;                   // lambda3 - 1
        const R d5 = -(R(1) + au3) * ex;    // lambda5 - 1
        const R m0 = R(mu[3 * (int64_t)j]), m1 = R(mu[3 * (int64_t)j + 1]), m2 = R(mu[3 * (int64_t)j + 2]);
        const R mr = m0 * rx + m1 * ry + m2 * rz;
        const R tt = R(3) * d5 * mr * ri5;
        const R s3 = d3 * ri3;
        e0 += tt * rx - s3 * m0;
        e1 += tt * ry - s3 * m1;
        e2 += tt * rz - s3 * m2;
    }
    for (int o = kThLanes / 2; o > 0; o >>= 1) {
        e0 += __shfl_down_sync(0xffffffffu, e0, o, kThLanes);
        e1 += __shfl_down_sync(0xffffffffu, e1, o, kThLanes);
        e2 += __shfl_down_sync(0xffffffffu, e2, o, kThLanes);
    }
    if (live && g == 0 && k1 > k0) {
        E[3 * i] += double(e0);
        E[3 * i + 1] += double(e1);
        E[3 * i + 2] += double(e2);
    }
}

// MIXED: E_i += sum_j t5_ij (mu_j.r) r - t3_ij mu_j from the stored pair geometry
// and the dipoles of the near field's pair records (packed for this pass)
__global__ void th_field_coef_kernel(int64_t n, const int* __restrict__ ptr, const int* __restrict__ idx,
                                     const float4* __restrict__ rr, const float* __restrict__ t3,
                                     const float* __restrict__ P, const int* __restrict__ slot,
                                     double* __restrict__ E) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t i = t / kThLanes;
    const int g = (int)(t % kThLanes);
    const bool live = i < n;
    const int k0 = live ? ptr[i] : 0, k1 = live ? ptr[i + 1] : 0;
    float e0 = 0.f, e1 = 0.f, e2 = 0.f;
    for (int k = k0 + g; k < k1; k += kThLanes) {
        const int j = idx[k];
        const float4 r = rr[k];
        const float s3 = t3[k];
        // the dipole from the near field's pair records (FP32, stored negated)
        const int sl = slot[j];
        const float* q = P + 12 * (int64_t)(sl >> 1) + (sl & 1);
        const float m0 = -q[6], m1 = -q[8], m2 = -q[10];
        const float tt = r.w * (m0 * r.x + m1 * r.y + m2 * r.z);
        e0 += tt * r.x - s3 * m0;
        e1 += tt * r.y - s3 * m1;
        e2 += tt * r.z - s3 * m2;
    }
    for (int o = kThLanes / 2; o > 0; o >>= 1) {
        e0 += __shfl_down_sync(0xffffffffu, e0, o, kThLanes);
        e1 += __shfl_down_sync(0xffffffffu, e1, o, kThLanes);
        e2 += __shfl_down_sync(0xffffffffu, e2, o, kThLanes);
    }
    if (live && g == 0 && k1 > k0) {
        E[3 * i] += double(e0);
        E[3 * i + 1] += double(e1);
        E[3 * i + 2] += double(e2);
    }
}

void thole_field(polfmm_ctx* c, const double* mu_sorted, double* E, cudaStream_t st) {
    if (c->th_npairs == 0 || !mu_sorted) return;
    LaunchScope ls(c, F_LEAF_DIPOLE);
    if (c->mixed)
        th_field_coef_kernel<<<grid_for(c->n * kThLanes, 128), 128, 0, st>>>(
            c->n, c->th_ptr, c->th_idx, c->th_r, c->th_t3, c->near_pairs, c->near_slot, E);
    else
        th_field_kernel<double><<<grid_for(c->n * kThLanes, 128), 128, 0, st>>>(c->n, c->th_ptr, c->th_idx, c->pos_s,
                                                                                 c->a16, mu_sorted, c->thole_a, E);
}

// force pass, in R (the mode's precision): for the converged dipoles, per sorted site i,
//   thE_i  = sum_j (T^damp - T)(r_ij) mu_j                         (energy: -1/2 mu.E^mu)
//   thF_i  = sum_j grad_i [mu_i . (T^damp - T)(r_ij) mu_j]          (dipole-dipole force)
//   thdA_i = -sum_j mu_i . (d T^damp / d alpha_i) mu_j               (dU/dalpha)
// with f = 3 lambda5 (mu_i.r)(mu_j.r) / r^5 - lambda3 (mu_i.mu_j) / r^3,
//   grad_i f = 3 lambda5 (mu_i (mu_j.r) + mu_j (mu_i.r)) / r^5
//            + [3 (mu_i.r)(mu_j.r) (lambda5' / r^6 - 5 lambda5 / r^7) - (mu_i.mu_j)(lambda3' / r^4 - 3 lambda3 / r^5)] r,
//   lambda3' = 3 a u^2 e / s, lambda5' = 3 a^2 u^5 e / s (d/dr), s = (alpha_i alpha_j)^(1/6), e = exp(-a u^3),
//   d lambda / d alpha_i = (d lambda / du) (-u / (6 alpha_i)); the undamped parts (lambda = 1) are the FMM's
template <typename R>
__global__ void th_force_kernel(int64_t n, const int* __restrict__ ptr, const int* __restrict__ idx,
                                const double* __restrict__ pos, const float4* __restrict__ rr,
                                const double* __restrict__ a16,
                                const double* __restrict__ alpha, const double* __restrict__ mu, double a_in,
                                double* __restrict__ thE, double* __restrict__ thF, double* __restrict__ thdA) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t i = t / kThLanes;
    const int g = (int)(t % kThLanes);
    const bool live = i < n;
    const int k0 = live ? ptr[i] : 0, k1 = live ? ptr[i + 1] : 0;
    double xi = 0.0, yi = 0.0, zi = 0.0;
    R mi[3] = {R(0), R(0), R(0)}, si = R(1), ai = R(0);
    if (live) {
        xi = pos[3 * i];
        yi = pos[3 * i + 1];
        zi = pos[3 * i + 2];
        for (int d = 0; d < 3; d++) mi[d] = R(mu[3 * i + d]);
        si = R(a16[i]);
        ai = R(alpha[i]);
    }
    const R a = R(a_in);
    // e[0..2] field, e[3..5] force, e[6] dU/dalpha part
    R e[7] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
    for (int k = k0 + g; k < k1; k += kThLanes) {
        const int j = idx[k];
        R r[3];
        if (rr) {  // MIXED: the stored pair geometry
            const float4 g4 = rr[k];
            r[0] = R(g4.x);
            r[1] = R(g4.y);
            r[2] = R(g4.z);
        } else {
            r[0] = R(xi - pos[3 * (int64_t)j]);
            r[1] = R(yi - pos[3 * (int64_t)j + 1]);
            r[2] = R(zi - pos[3 * (int64_t)j + 2]);
        }
        const R r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        const R rn = sqrt(r2), ri = R(1) / rn;
        const R ri2 = ri * ri, ri3 = ri * ri2, ri5 = ri3 * ri2, ri7 = ri5 * ri2;
        const R s = si * R(a16[j]);
        const R u = rn / s, au3 = a * u * u * u, ex = exp(-au3);
        const R d3 = -ex, d5 = -(R(1) + au3) * ex;                           // lambda - 1
        const R d3u = R(3) * a * u * u * ex, d5u = R(3) * a * a * u * u * u * u * u * ex;  // d lambda / du
        const R d3r = d3u / s, d5r = d5u / s;
        const R mj[3] = {R(mu[3 * (int64_t)j]), R(mu[3 * (int64_t)j + 1]), R(mu[3 * (int64_t)j + 2])};
        const R Bi = mi[0] * r[0] + mi[1] * r[1] + mi[2] * r[2];
        const R Bj = mj[0] * r[0] + mj[1] * r[1] + mj[2] * r[2];
        const R Aij = mi[0] * mj[0] + mi[1] * mj[1] + mi[2] * mj[2];
        const R cr = R(3) * Bi * Bj * (d5r * ri * ri5 - R(5) * d5 * ri7) - Aij * (d3r * ri * ri3 - R(3) * d3 * ri5);
        const R cm = R(3) * d5 * ri5;
        for (int d = 0; d < 3; d++) {
            e[d] += R(3) * d5 * Bj * r[d] * ri5 - d3 * mj[d] * ri3;
            e[3 + d] += cr * r[d] + cm * (mi[d] * Bj + mj[d] * Bi);
        }
        if (ai > R(0)) {
            const R du = -u / (R(6) * ai);
            e[6] -= (R(3) * Bi * Bj * ri5 * d5u - Aij * ri3 * d3u) * du;
        }
    }
    for (int o = kThLanes / 2; o > 0; o >>= 1)
        for (int c = 0; c < 7; c++) e[c] += __shfl_down_sync(0xffffffffu, e[c], o, kThLanes);
    if (live && g == 0) {
        for (int d = 0; d < 3; d++) {
            thE[3 * i + d] = double(e[d]);
            thF[3 * i + d] = double(e[3 + d]);
        }
        thdA[i] = double(e[6]);
    }
}

void thole_forces(polfmm_ctx* c) {
    if (c->th_npairs == 0) return;
    LaunchScope ls(c, F_ASSEMBLE);
    if (c->mixed)
        th_force_kernel<float><<<grid_for(c->n * kThLanes, 128), 128, 0, c->stream>>>(
            c->n, c->th_ptr, c->th_idx, c->pos_s, c->th_r, c->a16, c->alpha_s, c->mu, c->thole_a, c->thE, c->thF,
            c->thdA);
    else
        th_force_kernel<double><<<grid_for(c->n * kThLanes, 128), 128, 0, c->stream>>>(
            c->n, c->th_ptr, c->th_idx, c->pos_s, nullptr, c->a16, c->alpha_s, c->mu, c->thole_a, c->thE, c->thF,
            c->thdA);
}

void exclusion_inv_perm(polfmm_ctx* c) {
    if (c->n_excl == 0) return;
    LaunchScope ls(c, F_TREE);
    inv_perm_kernel<<<grid_for(c->n, 256), 256, 0, c->stream>>>(c->n, c->perm, c->inv_perm);
}

}  // namespace polfmm
