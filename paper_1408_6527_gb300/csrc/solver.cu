// Induced-dipole solver and energy / gradient assembly, all in FP64.
//
// The dipoles solve mu_i = alpha_i (E^q_i + E^mu_i) (Sec. II.A, Eq. dipole
// moment), i.e. (diag(1/alpha) - T) mu = E^q with T the (symmetric) FMM
// dipole-field operator.  Default: preconditioned conjugate gradients with
// the Jacobi preconditioner diag(alpha), started from mu = alpha E^q; the
// fixed point mu <- alpha (E^q + T mu) is available as well.  The paper only
// refers to an earlier publication for its iteration (Sec. III).
//
// Reductions are deterministic: a fixed grid of kRedBlocks blocks writes
// per-block partial sums in a fixed order, and one block adds them up.
#include <math.h>

#include "internal.cuh"

namespace polfmm {

constexpr int kRedThreads = 256;

// block-wide sum in a fixed order (warp shuffles, then the warp sums in warp
// order); every thread gets the result.  sh holds kRedThreads doubles.
__device__ inline double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5;
    __syncthreads();  // sh may still be read by a previous call
    if ((threadIdx.x & 31) == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    for (int k = 0; k < kRedThreads / 32; k++) r += sh[k];
    return r;
}

// true in exactly one block: the last to finish.  Its caller then adds the
// per-block partials in fixed order (deterministic) and re-arms the ticket.
__device__ inline bool last_block(int* ticket) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (last) __threadfence();
    return last;
}

__device__ inline double sum_partials(const double* __restrict__ partial, int row, double* sh) {
    double v = 0.0;
    for (int b = threadIdx.x; b < kRedBlocks; b += kRedThreads) v += __ldcg(partial + row * kRedBlocks + b);
    return block_sum(v, sh);
}

// packed (mu_x, mu_y, mu_z, 0) record of site i for the near-field kernels
// the near-field source copy of a dipole-like vector: FP64 (x, y, z, 0)
// records per site; FP32 into the site's slot of the pair records
template <typename R>
__device__ inline void store_packed(void* base, const int* __restrict__ slot, int64_t i, double x, double y,
                                    double z) {
    if constexpr (sizeof(R) == 4) {
        const int sl = slot[i];
        float* q = reinterpret_cast<float*>(base) + 12 * (int64_t)(sl >> 1) + (sl & 1);
        q[6] = -(float)x;  // the pair records hold the negated dipole
        q[8] = -(float)y;
        q[10] = -(float)z;
    } else {
        R* p = reinterpret_cast<R*>(base) + 4 * i;
        p[0] = R(x);
        p[1] = R(y);
        p[2] = R(z);
        p[3] = R(0);
    }
}

// single-block final reduction of nslot partial rows
// post: 0 = store sums into scal[dst[k]]; 1 = PCG direction update
// (scal[S_BETA] = sum0 / scal[S_RZ], scal[S_RZ] = sum0, scal[S_RR] = sum1);
// 2 = store, and restart the residual-growth count of a new solve
__global__ void reduce_final_kernel(const double* __restrict__ partial, int nslot, int s0, int s1, int s2, int s3,
                                    double* __restrict__ scal, int post) {
    __shared__ double sh[kRedThreads];
    int dst[4] = {s0, s1, s2, s3};
    double res[4] = {0, 0, 0, 0};
    for (int k = 0; k < nslot; k++) {
        double v = 0.0;
        for (int b = threadIdx.x; b < kRedBlocks; b += kRedThreads) v += partial[k * kRedBlocks + b];
        res[k] = block_sum(v, sh);
    }
    if (threadIdx.x == 0) {
        if (post == 1) {
            double rz_old = scal[S_RZ];
            scal[S_BETA] = res[0] / rz_old;  // beta
            scal[S_RZ] = res[0];
            scal[S_RR] = res[1];
        } else {
            for (int k = 0; k < nslot; k++) scal[dst[k]] = res[k];
            if (post == 2) scal[S_GROW] = 0.0;
        }
    }
}

// 32-bit indices: fmm_build limits n to 2^28, so 3 n < 2^31 (i / 3 is then a
// multiply and shift)
#define RED_LOOP(i, n) for (int i = blockIdx.x * kRedThreads + threadIdx.x; i < (int)(n); i += kRedBlocks * kRedThreads)

__device__ inline bool active_site(const double* alpha, int64_t site) { return alpha[site] > 0.0; }

// mu = alpha E^q (masked)
__global__ void mu_init_kernel(int64_t n, const double* __restrict__ alpha, const double* __restrict__ Eq,
                               double* __restrict__ mu) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    double a = alpha[i / 3];
    mu[i] = a > 0.0 ? a * Eq[i] : 0.0;
}

__global__ void mask_kernel(int64_t n, const double* __restrict__ alpha, double* __restrict__ v) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    if (!(alpha[i / 3] > 0.0)) v[i] = 0.0;
}

// r = E^q - (mu/alpha - T mu); z = alpha r; d = z; partials r.z, r.r, Eq.Eq
__global__ void pcg_init_kernel(int64_t n, const double* __restrict__ alpha, const double* __restrict__ Eq,
                                const double* __restrict__ mu, const double* __restrict__ Tmu, double* __restrict__ r,
                                double* __restrict__ z, double* __restrict__ d, double* __restrict__ partial) {
    __shared__ double sh[kRedThreads];
    double rz = 0, rr = 0, bb = 0;
    RED_LOOP(i, 3 * n) {
        double a = alpha[i / 3];
        double ri = 0, zi = 0;
        if (a > 0.0) {
            ri = Eq[i] - (mu[i] / a - Tmu[i]);
            zi = a * ri;
            bb += Eq[i] * Eq[i];
        }
        r[i] = ri;
        z[i] = zi;
        d[i] = zi;
        rz += ri * zi;
        rr += ri * ri;
    }
    rz = block_sum(rz, sh);
    rr = block_sum(rr, sh);
    bb = block_sum(bb, sh);
    if (threadIdx.x == 0) {
        partial[0 * kRedBlocks + blockIdx.x] = rz;
        partial[1 * kRedBlocks + blockIdx.x] = rr;
        partial[2 * kRedBlocks + blockIdx.x] = bb;
    }
}

// Ad = d/alpha - T d; d.Ad (partials, then the last block stores the sum).
// Inside the solve graph (cond != 0) it also clears the loop condition, which
// only the last kernel of the iteration sets again.
__global__ void pcg_ad_kernel(int64_t n, const double* __restrict__ inv_alpha, const double* __restrict__ d,
                              const double* __restrict__ Td, double* __restrict__ Ad, double* __restrict__ partial,
                              double* __restrict__ scal, int* __restrict__ ticket, cudaGraphConditionalHandle cond) {
    __shared__ double sh[kRedThreads];
    if (cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
    double s = 0;
    RED_LOOP(i, 3 * n) {
        const double ia = inv_alpha[i / 3];
        const double v = ia > 0.0 ? d[i] * ia - Td[i] : 0.0;
        Ad[i] = v;
        s += d[i] * v;
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
    if (last_block(ticket)) {
        double t = sum_partials(partial, 0, sh);
        if (threadIdx.x == 0) {
            scal[S_DAD] = t;
            *ticket = 0;
        }
    }
}

// step = rz / dAd; mu += step d; r -= step Ad; z = alpha r; r.z and r.r; the
// last block stores beta = (r.z)_new / (r.z)_old, (r.z)_new and r.r, and counts
// the iterations in a row whose residual grew.  A direction with d.Ad <= 0 (the
// operator is not positive definite: polarization catastrophe) or a non-finite
// d.Ad is not applied, so mu, r and z keep the last good iterate.  Inside the
// solve graph (cond != 0) it counts the iteration and keeps the loop going while
// d.Ad > 0, the relative residual is finite and above tol, the residual has not
// grown kStagnationIters times in a row, and fewer than max_iter iterations are done.
__global__ void pcg_update_kernel(int64_t n, const double* __restrict__ alpha, double* __restrict__ scal,
                                  const double* __restrict__ d, const double* __restrict__ Ad, double* __restrict__ mu,
                                  double* __restrict__ r, double* __restrict__ z, double* __restrict__ partial,
                                  int* __restrict__ ticket, cudaGraphConditionalHandle cond) {
    __shared__ double sh[kRedThreads];
    __shared__ double step_sh;
    pdl_wait();  // d.Ad and Ad come from the kernel before
    const double dad = scal[S_DAD];
    const bool ok = dad > 0.0 && isfinite(dad);
    // one FP64 division per block, not per thread (FP64 is a narrow unit here)
    if (threadIdx.x == 0) step_sh = ok ? scal[S_RZ] / dad : 0.0;
    __syncthreads();
    const double step = step_sh;
    double rz = 0, rr = 0;
    RED_LOOP(i, 3 * n) {
        double a = alpha[i / 3];
        if (a > 0.0) {
            double ri = r[i];
            if (ok) {
                mu[i] += step * d[i];
                ri -= step * Ad[i];
                r[i] = ri;
            }
            double zi = a * ri;
            z[i] = zi;
            rz += ri * zi;
            rr += ri * ri;
        }
    }
    rz = block_sum(rz, sh);
    rr = block_sum(rr, sh);
    if (threadIdx.x == 0) {
        partial[0 * kRedBlocks + blockIdx.x] = rz;
        partial[1 * kRedBlocks + blockIdx.x] = rr;
    }
    if (last_block(ticket)) {
        double rz_new = sum_partials(partial, 0, sh);
        double rr_all = sum_partials(partial, 1, sh);
        if (threadIdx.x == 0) {
            const double grow = rr_all > scal[S_RR] ? scal[S_GROW] + 1.0 : 0.0;
            scal[S_GROW] = grow;
            scal[S_BETA] = rz_new / scal[S_RZ];
            scal[S_RZ] = rz_new;
            scal[S_RR] = rr_all;
            *ticket = 0;
            if (cond) {
                const double it = scal[S_ITER] + 1.0;
                scal[S_ITER] = it;
                const double res = sqrt(rr_all / scal[S_BB]);
                const bool go = ok && isfinite(res) && res > scal[S_TOL] && it < scal[S_MAXIT] &&
                                grow < (double)kStagnationIters;
                cudaGraphSetConditional(cond, go ? 1u : 0u);
            }
        }
    }
    pdl_launch_dependents();
}

// solve-graph start: tolerance, iteration limit, iteration count
__global__ void loop_setup_kernel(double* __restrict__ scal, double tol, double max_iter) {
    scal[S_TOL] = tol;
    scal[S_MAXIT] = max_iter;
    scal[S_ITER] = 0.0;
}

// d = z + beta d, and its packed copy for the next near-field pass
template <typename R>
__global__ void pcg_direction_kernel(int64_t n, const double* __restrict__ scal, const double* __restrict__ z,
                                     double* __restrict__ d, void* __restrict__ packed, const int* __restrict__ slot) {
    pdl_wait();  // beta and z come from the update kernel before
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double beta = scal[S_BETA];
    double v[3];
    for (int k = 0; k < 3; k++) {
        v[k] = z[3 * i + k] + beta * d[3 * i + k];
        d[3 * i + k] = v[k];
    }
    store_packed<R>(packed, slot, i, v[0], v[1], v[2]);
}

// packed copy of d after the PCG start (d = z)
template <typename R>
__global__ void pack_vec_kernel(int64_t n, const double* __restrict__ v, void* __restrict__ packed,
                                const int* __restrict__ slot) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    store_packed<R>(packed, slot, i, v[3 * i], v[3 * i + 1], v[3 * i + 2]);
}

// Jacobi fixed point: r = E^q + T mu - mu/alpha (residual at the current mu),
// mu <- alpha (E^q + T mu); partial r.r
__global__ void jacobi_kernel(int64_t n, const double* __restrict__ alpha, const double* __restrict__ Eq,
                              const double* __restrict__ Tmu, double* __restrict__ mu, double* __restrict__ partial) {
    __shared__ double sh[kRedThreads];
    double rr = 0;
    RED_LOOP(i, 3 * n) {
        double a = alpha[i / 3];
        if (a > 0.0) {
            double e = Eq[i] + Tmu[i];
            double ri = e - mu[i] / a;
            rr += ri * ri;
            mu[i] = a * e;
        } else {
            mu[i] = 0.0;
        }
    }
    rr = block_sum(rr, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = rr;
}

__global__ void norm_b_kernel(int64_t n, const double* __restrict__ alpha, const double* __restrict__ Eq,
                              double* __restrict__ partial) {
    __shared__ double sh[kRedThreads];
    double bb = 0;
    RED_LOOP(i, 3 * n) {
        if (alpha[i / 3] > 0.0) bb += Eq[i] * Eq[i];
    }
    bb = block_sum(bb, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = bb;
}

// gather / scatter between caller order and sorted order
__global__ void gather_kernel(int64_t n, int comps, const int* __restrict__ perm, const double* __restrict__ src,
                              double* __restrict__ dst) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * comps) return;
    int64_t i = t / comps;
    int k = (int)(t - i * comps);
    dst[t] = src[(int64_t)perm[i] * comps + k];
}

__global__ void scatter_kernel(int64_t n, int comps, const int* __restrict__ perm, const double* __restrict__ src,
                               double* __restrict__ dst, double scale) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * comps) return;
    int64_t i = t / comps;
    int k = (int)(t - i * comps);
    dst[(int64_t)perm[i] * comps + k] = scale * src[t];
}

// forces, dU/dq, dU/dalpha (caller order) and energy partials, at the dipoles
// mu (Sec. II.A, Eq. upol_derivatives).  The last FMM pass had the field
// charges q^E (= q when none are set) and the dipoles as sources: phi, E, G;
// phiq, Eq are the potential and field of the Coulomb charges q, EqE, phiqE
// those of the field charges (null: the same as phiq, Eq).  With E^mu = E - EqE
// and Phi^mu = phi - phiqE:
//   F = q Eq + q^E E^mu + (grad E) mu;  U^pol terms use E^q = EqE and E^mu;
//   dU/dq = phiq + Phi^mu (= phi) without field charges, phiq with them, and
//   then dU/dq^E = Phi^mu (written to dqE, sorted order);
//   dU/dalpha = -|mu|^2 / (2 alpha^2) (-|E|^2/2 where alpha = 0);
// energies: 1/2 q Phi^q, mu.E^q, mu.E^mu, |mu|^2/(2 alpha)
__global__ void assemble_kernel(int64_t n, const int* __restrict__ perm, const double* __restrict__ q,
                                const double* __restrict__ qE, const double* __restrict__ alpha,
                                const double* __restrict__ mu, const double* __restrict__ phiq,
                                const double* __restrict__ Eq, const double* __restrict__ phiqE,
                                const double* __restrict__ EqE, const double* __restrict__ phi,
                                const double* __restrict__ E, const double* __restrict__ G,
                                const double* __restrict__ thE, const double* __restrict__ thF,
                                const double* __restrict__ thdA, double kc,
                                double* __restrict__ F, double* __restrict__ dq, double* __restrict__ dqE,
                                double* __restrict__ da, double* __restrict__ partial) {
    __shared__ double sh[kRedThreads];
    double uqq = 0, mueq = 0, muemu = 0, amu = 0;
    RED_LOOP(i, n) {
        const double qi = q[i], ai = alpha[i];
        const double m0 = mu[3 * i], m1 = mu[3 * i + 1], m2 = mu[3 * i + 2];
        const double e0 = E[3 * i], e1 = E[3 * i + 1], e2 = E[3 * i + 2];
        const double* g = G + 6 * i;
        const int o = perm[i];
        const double* ep = EqE ? EqE : Eq;  // the polarizing field E^q
        const double q0 = ep[3 * i], q1 = ep[3 * i + 1], q2 = ep[3 * i + 2];
        if (F) {
            double f0, f1, f2;
            if (qE) {
                const double qe = qE[i];
                f0 = qi * Eq[3 * i] + qe * (e0 - q0);
                f1 = qi * Eq[3 * i + 1] + qe * (e1 - q1);
                f2 = qi * Eq[3 * i + 2] + qe * (e2 - q2);
            } else {
                f0 = qi * e0;
                f1 = qi * e1;
                f2 = qi * e2;
            }
            if (thF) {  // Thole: the damped minus undamped dipole-dipole force
                f0 += thF[3 * i];
                f1 += thF[3 * i + 1];
                f2 += thF[3 * i + 2];
            }
            F[3 * (int64_t)o + 0] = kc * (f0 + g[0] * m0 + g[1] * m1 + g[2] * m2);
            F[3 * (int64_t)o + 1] = kc * (f1 + g[1] * m0 + g[3] * m1 + g[4] * m2);
            F[3 * (int64_t)o + 2] = kc * (f2 + g[2] * m0 + g[4] * m1 + g[5] * m2);
        }
        if (dq) dq[o] = kc * (qE ? phiq[i] : phi[i]);
        if (dqE) dqE[i] = kc * (phi[i] - (phiqE ? phiqE[i] : phiq[i]));
        const double mm = m0 * m0 + m1 * m1 + m2 * m2;
        if (da)
            da[o] = ai > 0.0 ? kc * (-mm / (2.0 * ai * ai) + (thdA ? thdA[i] : 0.0))
                             : -0.5 * kc * (e0 * e0 + e1 * e1 + e2 * e2);
        uqq += 0.5 * qi * phiq[i];
        mueq += m0 * q0 + m1 * q1 + m2 * q2;
        muemu += m0 * (e0 - q0) + m1 * (e1 - q1) + m2 * (e2 - q2);
        if (thE) muemu += m0 * thE[3 * i] + m1 * thE[3 * i + 1] + m2 * thE[3 * i + 2];  // the damped E^mu
        if (ai > 0.0) amu += mm / (2.0 * ai);
    }
    uqq = block_sum(uqq, sh);
    mueq = block_sum(mueq, sh);
    muemu = block_sum(muemu, sh);
    amu = block_sum(amu, sh);
    if (threadIdx.x == 0) {
        partial[0 * kRedBlocks + blockIdx.x] = uqq;
        partial[1 * kRedBlocks + blockIdx.x] = mueq;
        partial[2 * kRedBlocks + blockIdx.x] = muemu;
        partial[3 * kRedBlocks + blockIdx.x] = amu;
    }
}

// stationary energy terms (Sec. II.A): partials of 1/2 q Phi^q and mu.E^q (E^q
// the polarizing field); at a converged solve U^pol = -1/2 sum mu.E^q (Eq.
// upol_derivatives)
__global__ void energy_stationary_kernel(int64_t n, const double* __restrict__ q, const double* __restrict__ mu,
                                         const double* __restrict__ phiq, const double* __restrict__ Eq,
                                         double* __restrict__ partial) {
    __shared__ double sh[kRedThreads];
    double uqq = 0, mueq = 0;
    RED_LOOP(i, n) {
        uqq += 0.5 * q[i] * phiq[i];
        mueq += mu[3 * i] * Eq[3 * i] + mu[3 * i + 1] * Eq[3 * i + 1] + mu[3 * i + 2] * Eq[3 * i + 2];
    }
    uqq = block_sum(uqq, sh);
    mueq = block_sum(mueq, sh);
    if (threadIdx.x == 0) {
        partial[0 * kRedBlocks + blockIdx.x] = uqq;
        partial[1 * kRedBlocks + blockIdx.x] = mueq;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static void reduce(polfmm_ctx* c, int nslot, int s0, int s1, int s2, int s3, int post, int fam) {
    LaunchScope ls(c, fam);
    reduce_final_kernel<<<1, kRedThreads, 0, c->stream>>>(c->partial, nslot, s0, s1, s2, s3, c->scal, post);
}

void gather_sites(polfmm_ctx* c, const double* src, double* dst, int comps) {
    LaunchScope ls(c, F_ASSEMBLE);
    gather_kernel<<<grid_for(c->n * comps, 256), 256, 0, c->stream>>>(c->n, comps, c->perm, src, dst);
}

void scatter_sites(polfmm_ctx* c, const double* src, double* dst, int comps) {
    LaunchScope ls(c, F_ASSEMBLE);
    scatter_kernel<<<grid_for(c->n * comps, 256), 256, 0, c->stream>>>(c->n, comps, c->perm, src, dst, 1.0);
}

void mask_dipoles(polfmm_ctx* c, double* v) {
    LaunchScope ls(c, F_SOLVER);
    mask_kernel<<<grid_for(3 * c->n, 256), 256, 0, c->stream>>>(c->n, c->alpha_s, v);
}

// PCG start: mu (given or alpha E^q), one operator application, residual
void solver_init(polfmm_ctx* c, bool warm) {
    if (!warm) {
        LaunchScope ls(c, F_SOLVER);
        mu_init_kernel<<<grid_for(3 * c->n, 256), 256, 0, c->stream>>>(c->n, c->alpha_s, polarizing_field(c), c->mu);
    }
    if (c->opt.solver == POLFMM_SOLVER_JACOBI) {
        {
            LaunchScope ls(c, F_SOLVER);
            norm_b_kernel<<<kRedBlocks, kRedThreads, 0, c->stream>>>(c->n, c->alpha_s, polarizing_field(c), c->partial);
        }
        reduce(c, 1, S_BB, 0, 0, 0, 0, F_SOLVER);
        return;
    }
    fmm_pass(c, LEAF_DIPOLE_E, false, c->mu, nullptr, c->Td, nullptr);
    {
        LaunchScope ls(c, F_SOLVER);
        pcg_init_kernel<<<kRedBlocks, kRedThreads, 0, c->stream>>>(c->n, c->alpha_s, polarizing_field(c), c->mu, c->Td, c->r,
                                                                    c->z, c->d, c->partial);
    }
    reduce(c, 3, S_RZ, S_RR, S_BB, 0, 2, F_SOLVER);
    LaunchScope ls(c, F_SOLVER);
    if (c->mixed)
        pack_vec_kernel<float><<<grid_for(c->n, 256), 256, 0, c->stream>>>(c->n, c->d, c->near_pairs, c->near_slot);
    else
        pack_vec_kernel<double><<<grid_for(c->n, 256), 256, 0, c->stream>>>(c->n, c->d, c->srcB, nullptr);
}

// one PCG iteration: T d by the FMM (d already packed for the near field;
// the kernel completing the field also forms Ad and d.Ad when it can), then
// the fused update and direction kernels
void solver_pcg_step(polfmm_ctx* c) {
    const cudaGraphConditionalHandle cond = c->capturing_loop ? c->loop_cond : 0;
    if (!fmm_pass(c, LEAF_DIPOLE_E, false, c->d, nullptr, c->Td, nullptr, true, true)) {
        LaunchScope ls(c, F_SOLVER);
        pcg_ad_kernel<<<kRedBlocks, kRedThreads, 0, c->stream>>>(c->n, c->inv_alpha_s, c->d, c->Td, c->Ad, c->partial,
                                                                  c->scal, c->ticket, cond);
    }
    {
        LaunchScope ls(c, F_SOLVER);
        launch_pdl(!c->opt.no_pdl, pcg_update_kernel, dim3(kRedBlocks), dim3(kRedThreads), 0, c->stream, c->n,
                   c->alpha_s, c->scal, c->d, c->Ad, c->mu, c->r, c->z, c->partial, c->ticket, cond);
    }
    {
        LaunchScope ls(c, F_SOLVER);
        if (c->mixed)
            launch_pdl(!c->opt.no_pdl, pcg_direction_kernel<float>, dim3(grid_for(c->n, 256)), dim3(256), 0,
                       c->stream, c->n, c->scal, c->z, c->d, (void*)c->near_pairs, (const int*)c->near_slot);
        else
            launch_pdl(!c->opt.no_pdl, pcg_direction_kernel<double>, dim3(grid_for(c->n, 256)), dim3(256), 0,
                       c->stream, c->n, c->scal, c->z, c->d, (void*)c->srcB, (const int*)nullptr);
    }
}

void solver_loop_setup(polfmm_ctx* c, double tol, int max_iter) {
    LaunchScope ls(c, F_SOLVER);
    loop_setup_kernel<<<1, 1, 0, c->stream>>>(c->scal, tol, (double)max_iter);
}

void solver_jacobi_step(polfmm_ctx* c) {
    fmm_pass(c, LEAF_DIPOLE_E, false, c->mu, nullptr, c->Td, nullptr);
    {
        LaunchScope ls(c, F_SOLVER);
        jacobi_kernel<<<kRedBlocks, kRedThreads, 0, c->stream>>>(c->n, c->alpha_s, polarizing_field(c), c->Td, c->mu,
                                                                c->partial);
    }
    reduce(c, 1, S_RR, 0, 0, 0, 0, F_SOLVER);
}

void energy_and_gradients(polfmm_ctx* c, double* F, double* dq, double* da, bool want_f, bool want_dq,
                          bool want_da) {
    const bool th = c->th_npairs > 0;
    if (th) thole_forces(c);
    {
        LaunchScope ls(c, F_ASSEMBLE);
        assemble_kernel<<<kRedBlocks, kRedThreads, 0, c->stream>>>(
            c->n, c->perm, c->q_s, c->qE_s, c->alpha_s, c->mu, c->phiq, c->Eq, c->phiqE, c->EqE, c->phi_t, c->E_t,
            c->G_t, th ? c->thE : nullptr, th ? c->thF : nullptr, th ? c->thdA : nullptr, c->opt.coulomb_k,
            want_f ? F : nullptr, want_dq ? dq : nullptr, c->qE_s ? c->dqE : nullptr, want_da ? da : nullptr,
            c->partial);
    }
    reduce(c, 4, S_UQQ, S_MUEQ, S_MUEMU, S_AMU, 0, F_ASSEMBLE);
}

void energy_stationary(polfmm_ctx* c) {
    {
        LaunchScope ls(c, F_ASSEMBLE);
        energy_stationary_kernel<<<kRedBlocks, kRedThreads, 0, c->stream>>>(c->n, c->q_s, c->mu, c->phiq,
                                                                              polarizing_field(c), c->partial);
    }
    reduce(c, 2, S_UQQ, S_MUEQ, 0, 0, 0, F_ASSEMBLE);
}

}  // namespace polfmm
