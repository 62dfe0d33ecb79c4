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
__global__ void th_a16_kernel(int64_t n, const double* __restrict__ alpha, double* __restrict__ a16,
                              unsigned long long* __restrict__ amax) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = alpha[i] > 0.0 ? cbrt(sqrt(alpha[i])) : 0.0;
    a16[i] = v;
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

// ascending site index within each bucket: the pair lists come out in a fixed order
__global__ void th_order_kernel(int nb, const int* __restrict__ start, int* __restrict__ member) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int s = start[b], e = start[b + 1];
    for (int k = s + 1; k < e; k++) {
        const int v = member[k];
        int m = k - 1;
        while (m >= s && member[m] > v) {
            member[m + 1] = member[m];
            m--;
        }
        member[m + 1] = v;
    }
}

// COUNT: damped partners of every sorted site i; else write them from ptr[i]
template <bool COUNT>
__global__ void th_pairs_kernel(int64_t n, const double* __restrict__ pos, const double* __restrict__ a16,
                                const int4* __restrict__ cell, const int* __restrict__ start,
                                const int* __restrict__ member, uint32_t mask, double umax,
                                const int* __restrict__ perm, const int* __restrict__ excl_row,
                                const int* __restrict__ excl_ptr, const int* __restrict__ excl_idx,
                                int* __restrict__ cnt, const int* __restrict__ ptr, int* __restrict__ idx) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double si = a16[i];
    int k = 0;
    if (si > 0.0) {
        const int4 ci = cell[i];
        const double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
        const int row = excl_row ? excl_row[perm[i]] : -1;
        int out = COUNT ? 0 : ptr[i];
        for (int dz = -1; dz <= 1; dz++)
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    const int cx = ci.x + dx, cy = ci.y + dy, cz = ci.z + dz;
                    const uint32_t b = th_bucket_of(cx, cy, cz, mask);
                    for (int m = start[b]; m < start[b + 1]; m++) {
                        const int j = member[m];
                        if (j == (int)i) continue;
                        const int4 cj = cell[j];
                        if (cj.x != cx || cj.y != cy || cj.z != cz) continue;
                        const double sj = a16[j];
                        if (!(sj > 0.0)) continue;
                        const double rx = xi - pos[3 * (int64_t)j], ry = yi - pos[3 * (int64_t)j + 1],
                                     rz = zi - pos[3 * (int64_t)j + 2];
                        const double rc = umax * si * sj;
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
                        if (!COUNT) idx[out++] = j;
                        k++;
                    }
                }
    }
    if (COUNT) cnt[i] = k;
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
        th_a16_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, c->alpha_s, c->a16,
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
        th_fill_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, c->th_cell, c->th_bucket, nb, c->th_count, c->th_member);
        th_order_kernel<<<grid_for(nb, 256), 256, 0, st>>>(nb, c->th_bucket, c->th_member);
        th_pairs_kernel<true><<<grid_for(n, 128), 128, 0, st>>>(
            n, c->pos_s, c->a16, c->th_cell, c->th_bucket, c->th_member, mask, umax, c->perm,
            c->n_excl ? c->excl_row : nullptr, c->excl_ptr, c->excl_idx, c->th_cnt, nullptr, nullptr);
    }
    scan_exclusive(c, c->th_cnt, c->th_ptr, (int)n, c->th_ptr + n);
    int total = 0;
    e = cudaMemcpyAsync(&total, c->th_ptr + n, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "Thole pair count");
    if (total > c->th_cap) {
        if (c->th_idx) cudaFree(c->th_idx);
        c->th_idx = nullptr;
        c->th_cap = 0;
        if (dev_alloc(reinterpret_cast<void**>(&c->th_idx), sizeof(int) * std::max(total, 1)) != cudaSuccess) {
            cudaGetLastError();
            return POLFMM_ERR_OUT_OF_MEMORY;
        }
        c->th_cap = total;
    }
    {
        LaunchScope ls(c, F_TREE);
        th_pairs_kernel<false><<<grid_for(n, 128), 128, 0, st>>>(
            n, c->pos_s, c->a16, c->th_cell, c->th_bucket, c->th_member, mask, umax, c->perm,
            c->n_excl ? c->excl_row : nullptr, c->excl_ptr, c->excl_idx, nullptr, c->th_ptr, c->th_idx);
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
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k0 = ptr[i], k1 = ptr[i + 1];
    if (k0 == k1) return;
    const double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
    const R si = R(a16[i]), ra = R(a);
    R e0 = R(0), e1 = R(0), e2 = R(0);
    for (int k = k0; k < k1; k++) {
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
        const R t = R(3) * d5 * mr * ri5;
        const R s3 = d3 * ri3;
        e0 += t * rx - s3 * m0;
        e1 += t * ry - s3 * m1;
        e2 += t * rz - s3 * m2;
    }
    E[3 * i] += double(e0);
    E[3 * i + 1] += double(e1);
    E[3 * i + 2] += double(e2);
}

void thole_field(polfmm_ctx* c, const double* mu_sorted, double* E, cudaStream_t st) {
    if (c->th_npairs == 0 || !mu_sorted) return;
    LaunchScope ls(c, F_LEAF_DIPOLE);
    if (c->mixed)
        th_field_kernel<float><<<grid_for(c->n, 128), 128, 0, st>>>(c->n, c->th_ptr, c->th_idx, c->pos_s, c->a16,
                                                                     mu_sorted, c->thole_a, E);
    else
        th_field_kernel<double><<<grid_for(c->n, 128), 128, 0, st>>>(c->n, c->th_ptr, c->th_idx, c->pos_s, c->a16,
                                                                      mu_sorted, c->thole_a, E);
}

// force pass, FP64: for the converged dipoles, per sorted site i,
//   thE_i  = sum_j (T^damp - T)(r_ij) mu_j                         (energy: -1/2 mu.E^mu)
//   thF_i  = sum_j grad_i [mu_i . (T^damp - T)(r_ij) mu_j]          (dipole-dipole force)
//   thdA_i = -sum_j mu_i . (d T^damp / d alpha_i) mu_j               (dU/dalpha)
// with f = 3 lambda5 (mu_i.r)(mu_j.r) / r^5 - lambda3 (mu_i.mu_j) / r^3,
//   grad_i f = 3 lambda5 (mu_i (mu_j.r) + mu_j (mu_i.r)) / r^5
//            + [3 (mu_i.r)(mu_j.r) (lambda5' / r^6 - 5 lambda5 / r^7) - (mu_i.mu_j)(lambda3' / r^4 - 3 lambda3 / r^5)] r,
//   lambda3' = 3 a u^2 e / s, lambda5' = 3 a^2 u^5 e / s (d/dr), s = (alpha_i alpha_j)^(1/6), e = exp(-a u^3),
//   d lambda / d alpha_i = (d lambda / du) (-u / (6 alpha_i)); the undamped parts (lambda = 1) are the FMM's
__global__ void th_force_kernel(int64_t n, const int* __restrict__ ptr, const int* __restrict__ idx,
                                const double* __restrict__ pos, const double* __restrict__ a16,
                                const double* __restrict__ alpha, const double* __restrict__ mu, double a,
                                double* __restrict__ thE, double* __restrict__ thF, double* __restrict__ thdA) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
    const double mi0 = mu[3 * i], mi1 = mu[3 * i + 1], mi2 = mu[3 * i + 2];
    const double si = a16[i], ai = alpha[i];
    double e[3] = {0, 0, 0}, f[3] = {0, 0, 0}, da = 0.0;
    for (int k = ptr[i]; k < ptr[i + 1]; k++) {
        const int j = idx[k];
        const double r[3] = {xi - pos[3 * (int64_t)j], yi - pos[3 * (int64_t)j + 1], zi - pos[3 * (int64_t)j + 2]};
        const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        const double rr = sqrt(r2), ri = 1.0 / rr;
        const double ri2 = ri * ri, ri3 = ri * ri2, ri5 = ri3 * ri2, ri7 = ri5 * ri2;
        const double s = si * a16[j];
        const double u = rr / s, au3 = a * u * u * u, ex = exp(-au3);
        const double d3 = -ex, d5 = -(1.0 + au3) * ex;          // lambda - 1
        const double d3u = 3.0 * a * u * u * ex, d5u = 3.0 * a * a * u * u * u * u * u * ex;  // d lambda / du
        const double d3r = d3u / s, d5r = d5u / s;
        const double mj[3] = {mu[3 * (int64_t)j], mu[3 * (int64_t)j + 1], mu[3 * (int64_t)j + 2]};
        const double Bi = mi0 * r[0] + mi1 * r[1] + mi2 * r[2];
        const double Bj = mj[0] * r[0] + mj[1] * r[1] + mj[2] * r[2];
        const double Aij = mi0 * mj[0] + mi1 * mj[1] + mi2 * mj[2];
        const double cr = 3.0 * Bi * Bj * (d5r * ri * ri5 - 5.0 * d5 * ri7) - Aij * (d3r * ri * ri3 - 3.0 * d3 * ri5);
        const double cm = 3.0 * d5 * ri5;
        const double mi[3] = {mi0, mi1, mi2};
        for (int d = 0; d < 3; d++) {
            e[d] += 3.0 * d5 * Bj * r[d] * ri5 - d3 * mj[d] * ri3;
            f[d] += cr * r[d] + cm * (mi[d] * Bj + mj[d] * Bi);
        }
        if (ai > 0.0) {
            const double du = -u / (6.0 * ai);
            da -= (3.0 * Bi * Bj * ri5 * d5u - Aij * ri3 * d3u) * du;
        }
    }
    for (int d = 0; d < 3; d++) {
        thE[3 * i + d] = e[d];
        thF[3 * i + d] = f[d];
    }
    thdA[i] = da;
}

void thole_forces(polfmm_ctx* c) {
    if (c->th_npairs == 0) return;
    LaunchScope ls(c, F_ASSEMBLE);
    th_force_kernel<<<grid_for(c->n, 128), 128, 0, c->stream>>>(c->n, c->th_ptr, c->th_idx, c->pos_s, c->a16,
                                                                 c->alpha_s, c->mu, c->thole_a, c->thE, c->thF,
                                                                 c->thdA);
}

void exclusion_inv_perm(polfmm_ctx* c) {
    if (c->n_excl == 0) return;
    LaunchScope ls(c, F_TREE);
    inv_perm_kernel<<<grid_for(c->n, 256), 256, 0, c->stream>>>(c->n, c->perm, c->inv_perm);
}

}  // namespace polfmm
