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

void exclusion_inv_perm(polfmm_ctx* c) {
    if (c->n_excl == 0) return;
    LaunchScope ls(c, F_TREE);
    inv_perm_kernel<<<grid_for(c->n, 256), 256, 0, c->stream>>>(c->n, c->perm, c->inv_perm);
}

}  // namespace polfmm
