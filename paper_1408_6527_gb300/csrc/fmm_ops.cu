// FMM operators on the GPU (Sec. II.B, II.C of Coles & Masella), in
// normalised Cartesian coefficients (m_n = M_n / h^|n|, f_n = F_n h^(|n|+1),
// h the box side of the level), templated on the arithmetic type R
// (double: FP64 mode, float: MIXED mode).
//
//   P2M   multipoles of the charges and point dipoles of each leaf
//         (Eq. multipole; a point dipole is the dl -> 0 limit of the +-q pair
//         of Sec. II.C, i.e. the derivative of a charge's multipole)
//   M2M   children -> parent shift (k <= n componentwise)
//   M2L   multipole -> local for the 189 well-separated offsets of each
//         octant class, grouped so that every thread of a warp applies the
//         same derivative table D_o (SIMT kernel here; the tensor-core kernel
//         is in m2l_tc.cu)
//   L2L   parent -> child shift (|k| <= p - |n|), plus the M2L partial sums
//   leaf  L2P evaluation of potential / field / field gradient fused with
//         the near-field pair sums over the 27 adjacent leaves
//         (Phi = Phi^direct + Phi^fmm, Sec. III)
#include <algorithm>

#include "internal.cuh"

namespace polfmm {

__device__ inline void decode_mi(int packed, int& nx, int& ny, int& nz) {
    nx = packed & 0xff;
    ny = (packed >> 8) & 0xff;
    nz = (packed >> 16) & 0xff;
}

// ---------------------------------------------------------------------------
// shared helpers of the upward and downward passes
// ---------------------------------------------------------------------------
// 2^-s for 0 <= s <= 2 kMaxP + 2, exact
template <typename R>
__device__ inline R pow2neg(int s);
template <>
__device__ inline float pow2neg<float>(int s) {
    return __int_as_float((127 - s) << 23);
}
template <>
__device__ inline double pow2neg<double>(int s) {
    return __longlong_as_double((long long)(1023 - s) << 52);
}

// table of the arithmetic type R from its double / float copies
template <typename R>
__host__ __device__ inline const R* pick(const double* d, const float* f);
template <>
__host__ __device__ inline const double* pick<double>(const double* d, const float*) {
    return d;
}
template <>
__host__ __device__ inline const float* pick<float>(const double*, const float* f) {
    return f;
}

// copies the first p + 1 entries of a small table into shared memory
template <typename R>
__device__ inline void stage_small(R* dst, const R* __restrict__ src, int p) {
    if ((int)threadIdx.x <= p) dst[threadIdx.x] = src[threadIdx.x];
}

// The index of the multi-index n +- k e_AX in the coefficient order, stepped
// term by term from idx(x, y, z) = T3(o) + T2(a) + z (o = |n|, a = o - x,
// T3(m) = m(m+1)(m+2)/6, T2(m) = m(m+1)/2): one step changes T3 by T2(o + k)
// (or -T2(o - k + 1)), T2(a) by a + k (or -(a - k + 1)) when AX >= 1, and z by
// 1 when AX = 2, so that no term evaluates the cubic.
//
// one L2L pass along axis AX: a_n = sum_{k <= p - |n|} W_k f_{n + k e_AX}, with
// sign (-1)^k where the shift is negative
template <int AX, typename R>
__device__ inline R shift_up_axis(const R* src, int cc, int pk, bool neg, const R* W, int p) {
    const int x = pk & 0xff, o = pk >> 24;
    const int kmax = p - o;
    int a1 = o - x;
    int t = (o + 1) * (o + 2) / 2;  // T2(o + 1)
    int idx = cc;
    R a = src[cc];
    for (int k = 1; k <= kmax; k++) {
        idx += t;
        t += o + k + 1;
        if (AX >= 1) {
            a1 += 1;
            idx += a1;
        }
        if (AX == 2) idx += 1;
        const R v = W[k] * src[idx];
        a += (neg && (k & 1)) ? -v : v;
    }
    return a;
}

// one M2M pass along axis AX: g_n = sum_{k <= n_AX} W_k m_{n - k e_AX}, with
// sign (-1)^k where the shift is negative
template <int AX, typename R>
__device__ inline R shift_down_axis(const R* src, int cc, int pk, bool neg, const R* W) {
    const int x = pk & 0xff, y = (pk >> 8) & 0xff, z = (pk >> 16) & 0xff, o = pk >> 24;
    const int kmax = AX == 0 ? x : (AX == 1 ? y : z);
    int a1 = o - x;
    int t = o * (o + 1) / 2;  // T2(o)
    int idx = cc;
    R a = src[cc];
    for (int k = 1; k <= kmax; k++) {
        idx -= t;
        t -= o - k + 1;
        if (AX >= 1) {
            idx -= a1;
            a1 -= 1;
        }
        if (AX == 2) idx -= 1;
        const R v = W[k] * src[idx];
        a += (neg && (k & 1)) ? -v : v;
    }
    return a;
}

// ---------------------------------------------------------------------------
// upward pass: P2M of every leaf, then M2M up to level 2 inside the same
// launch.  Each box shifts its own multipole to its parent's centre as soon as
// it is known; the block that completes the last child of a parent (counted
// with one atomic per parent) adds the children's shifted rows in Morton order
// whichever block does it, so the result does not depend on the schedule.
//
// P2M (Eq. multipole, normalised): m_n = sum_i q_i v_i^n/n! - sum_d
// (mu_i,d/h) v_i^(n-e_d)/(n-e_d)!, v_i = -(x_i - z)/h; a point dipole is the
// dl -> 0 limit of the +-q pair of Sec. II.C.
// M2M (Sec. II.B, shift of a multipole expansion): with child centre
// z_C = z_P + (b - 1/2) h_P / 2 per axis,
//   m^P_n = sum_{k <= n} prod_d (s_d/4)^k_d / k_d!  2^-|n-k| m^C_{n-k},
// s_d = -1 where the child bit b_d is 1.  The kernel applies it as three
// one-axis convolutions (exact: the truncation k <= n is a box).
// ---------------------------------------------------------------------------
constexpr int kP2MChunk = 64;
constexpr int kUpThreads = 128;
constexpr int kUpMaxSlices = 8;

struct UpPtrs {
    void* M[kMaxDepth + 1];
    const int* parent[kMaxDepth + 1];
    const int* child0[kMaxDepth + 1];
    const int* nchild[kMaxDepth + 1];
    const int* key[kMaxDepth + 1];
    int* arrive[kMaxDepth + 1];
    void* Msh[kMaxDepth + 1];  // multipoles shifted to the parent's centre
};

template <typename R>
__host__ __device__ inline size_t upward_smem_bytes(int ncoef) {
    return sizeof(R) * 9 * (size_t)ncoef + sizeof(int) * (size_t)ncoef;
}

template <typename R>
__device__ inline void store_multipole(const UpPtrs& up, int l, int box, int cc, R v, int ld) {
    reinterpret_cast<R*>(up.M[l])[(int64_t)box * ld + cc] = v;
}

// per-site factors of the P2M sum, axis a, order k (P_a[-1] = 0):
//   P_a[k] = v_a^k / k!,  D_a[k] = (mu_a / h) P_a[k-1],  A_x[k] = q P_x[k] - D_x[k]
// so that m_n = sum_i A_x[nx] P_y[ny] P_z[nz] - P_x[nx] (D_y[ny] P_z[nz] + P_y[ny] D_z[nz])
enum { F_PX = 0, F_PY, F_PZ, F_AX, F_DY, F_DZ, F_NUM };

template <typename R, bool PAIRS>
__global__ void __launch_bounds__(kUpThreads) upward_kernel(
    int nleaf, int depth, const int* __restrict__ lstart, const int* __restrict__ lcount,
    const R* __restrict__ ploc, const double* __restrict__ q, const double* __restrict__ mu, UpPtrs up, int ld,
    int ncoef, int p, const int* __restrict__ mi, const R* __restrict__ w4, const R* __restrict__ rinv, R inv_h,
    double dl) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* S = reinterpret_cast<R*>(smem_raw);         // [8][ncoef] slice partials of P2M, then shift rows
    R* Mrow = S + 8 * ncoef;                        // [ncoef] multipole of the current box
    int* smi = reinterpret_cast<int*>(Mrow + ncoef);  // [ncoef] packed multi-indices
    __shared__ R fac[kP2MChunk][F_NUM][kMaxP + 1];
    __shared__ R W[kMaxP + 1];
    __shared__ R RI[kMaxP + 1];
    __shared__ int s_next;
    const int b = blockIdx.x;
    if (b >= nleaf) return;
    const int tid = threadIdx.x;
    for (int cc = tid; cc < ncoef; cc += kUpThreads) smi[cc] = mi[cc];
    stage_small(W, w4, p);
    stage_small(RI, rinv, p);

    // P2M of leaf b: thread (coefficient c, slice sl) sums the sites sl, sl + slices, ...
    const int slices = ncoef <= kUpThreads ? min(kUpMaxSlices, kUpThreads / ncoef) : 1;
    const int sl = ncoef <= kUpThreads ? tid / ncoef : 0;
    const int c_first = ncoef <= kUpThreads ? tid - sl * ncoef : tid;
    const bool worker = sl < slices;
    constexpr int CPT = (286 + kUpThreads - 1) / kUpThreads;  // coefficients per thread (p <= 10)
    R acc[CPT];
    int nx[CPT], ny[CPT], nz[CPT];
#pragma unroll
    for (int k = 0; k < CPT; k++) {
        acc[k] = R(0);
        const int cc = c_first + k * kUpThreads;
        const int pk = worker && cc < ncoef ? mi[cc] : 0;
        nx[k] = pk & 0xff;
        ny[k] = (pk >> 8) & 0xff;
        nz[k] = (pk >> 16) & 0xff;
    }
    // P2M entries: one per site; with dipoles as +-q pairs (dl > 0, Sec. II.C)
    // three per site: the charge at x, +q^mu at x + dl mu/|mu|, -q^mu at x - dl mu/|mu|
    // (PAIRS is the dl > 0 form with dipoles; the plain form keeps its own instantiation)
    const int s0 = lstart[b], cnt = lcount[b];
    constexpr int per = PAIRS ? 3 : 1;
    for (int k0 = 0; k0 < cnt * per; k0 += kP2MChunk) {
        const int m = min(kP2MChunk, cnt * per - k0);
        __syncthreads();
        if (tid < m) {
            const int e = k0 + tid;
            const int i = s0 + e / per, which = e % per;
            R qi = which == 0 && q ? R(q[i]) : R(0);
            R off[3] = {R(0), R(0), R(0)};
            if (PAIRS && which > 0) {
                const double mx = mu[3 * i], my = mu[3 * i + 1], mz = mu[3 * i + 2];
                const double nm = sqrt(mx * mx + my * my + mz * mz);
                if (nm > 0.0) {
                    const double sgn = which == 1 ? 1.0 : -1.0;
                    qi = R(sgn * nm / (2.0 * dl));
                    off[0] = R(sgn * dl * mx / nm);
                    off[1] = R(sgn * dl * my / nm);
                    off[2] = R(sgn * dl * mz / nm);
                }
            }
            for (int a = 0; a < 3; a++) {
                const R v = PAIRS ? -(ploc[3 * i + a] + off[a]) * inv_h : -ploc[3 * i + a] * inv_h;
                const R ma = mu && !PAIRS ? R(mu[3 * i + a]) * inv_h : R(0);
                R t = R(1), prev = R(0);
                for (int k = 0; k <= p; k++) {
                    if (k > 0) t = t * v * RI[k];
                    const R dk = ma * prev;  // (mu_a / h) P_a[k-1]
                    fac[tid][F_PX + a][k] = t;
                    if (a == 0) fac[tid][F_AX][k] = qi * t - dk;
                    if (a == 1) fac[tid][F_DY][k] = dk;
                    if (a == 2) fac[tid][F_DZ][k] = dk;
                    prev = t;
                }
            }
        }
        __syncthreads();
        if (!worker) continue;
#pragma unroll
        for (int k = 0; k < CPT; k++) {
            if (c_first + k * kUpThreads >= ncoef) continue;
            const int x = nx[k], y = ny[k], z = nz[k];
            R a = acc[k];
            for (int s = sl; s < m; s += slices) {
                const R(*F)[kMaxP + 1] = fac[s];
                const R pz = F[F_PZ][z], py = F[F_PY][y];
                a += F[F_AX][x] * py * pz - F[F_PX][x] * (F[F_DY][y] * pz + py * F[F_DZ][z]);
            }
            acc[k] = a;
        }
    }
    // the leaf's multipole -> Mrow (shared) and global memory
    if (slices > 1) {
        // slice partials through shared memory, added in slice order
        if (worker && c_first < ncoef) S[sl * ncoef + c_first] = acc[0];
        __syncthreads();
        for (int cc = tid; cc < ncoef; cc += kUpThreads) {
            R a = R(0);
            for (int u = 0; u < slices; u++) a += S[u * ncoef + cc];
            Mrow[cc] = a;
            store_multipole(up, depth, b, cc, a, ld);
        }
    } else {
#pragma unroll
        for (int k = 0; k < CPT; k++) {
            const int cc = c_first + k * kUpThreads;
            if (worker && cc < ncoef) {
                Mrow[cc] = acc[k];
                store_multipole(up, depth, b, cc, acc[k], ld);
            }
        }
    }

    // M2M, split between the children and the parent: every box shifts its own
    // multipole to its parent's centre (Msh); the block that completes a
    // parent's last child adds the children's shifted rows in Morton order
    R* T0 = S;           // shift work rows
    R* T1 = S + ncoef;
    int box = b;
    for (int l = depth; l > 2; l--) {
        __syncthreads();  // Mrow complete
        const bool neg_x = (up.key[l][box] & 1) != 0, neg_y = (up.key[l][box] & 2) != 0,
                   neg_z = (up.key[l][box] & 4) != 0;
        for (int cc = tid; cc < ncoef; cc += kUpThreads) T0[cc] = Mrow[cc] * pow2neg<R>(smi[cc] >> 24);
        __syncthreads();
        // g_n = sum_{k <= n_d} (s/4)^k/k! m_{n - k e_d}, along x (T0 -> T1), y (T1 -> T0), z (T0 -> T1)
        for (int cc = tid; cc < ncoef; cc += kUpThreads) T1[cc] = shift_down_axis<0>(T0, cc, smi[cc], neg_x, W);
        __syncthreads();
        for (int cc = tid; cc < ncoef; cc += kUpThreads) T0[cc] = shift_down_axis<1>(T1, cc, smi[cc], neg_y, W);
        __syncthreads();
        for (int cc = tid; cc < ncoef; cc += kUpThreads) T1[cc] = shift_down_axis<2>(T0, cc, smi[cc], neg_z, W);
        __syncthreads();
        R* msh = reinterpret_cast<R*>(up.Msh[l]) + (int64_t)box * ld;
        for (int cc = tid; cc < ncoef; cc += kUpThreads) msh[cc] = T1[cc];
        __threadfence();  // the shifted row is visible before the count
        __syncthreads();
        if (tid == 0) {
            const int par = up.parent[l][box];
            const int old = atomicAdd(&up.arrive[l - 1][par], 1);
            int nxt = -1;
            if (old == up.nchild[l - 1][par] - 1) {
                up.arrive[l - 1][par] = 0;  // re-armed for the next pass
                nxt = par;
            }
            s_next = nxt;
        }
        __syncthreads();
        const int par = s_next;
        if (par < 0) {
            pdl_launch_dependents();
            return;
        }
        __threadfence();
        const int c0 = up.child0[l - 1][par], nc = up.nchild[l - 1][par];
        const R* shc = reinterpret_cast<const R*>(up.Msh[l]);
        for (int cc = tid; cc < ncoef; cc += kUpThreads) {
            R a = R(0);
            for (int j = 0; j < nc; j++) a += __ldcg(shc + (int64_t)(c0 + j) * ld + cc);
            Mrow[cc] = a;
            store_multipole(up, l - 1, par, cc, a, ld);
        }
        box = par;
    }
    pdl_launch_dependents();
}

// ---------------------------------------------------------------------------
// downward pass, inside the kernels that evaluate the leaves: the block of
// leaf b forms the locals of b's ancestors from level 2 down to b itself,
//   f^l = sum over offset chunks of the M2L partials of level l
//         + 2^-(|n|+1) sum_{|k| <= p-|n|} prod_d (t_d)^k_d / k_d!  f^(l-1)_{n+k},
// t_d = +1/4 where the child bit is 1, -1/4 where it is 0 (L2L, Sec. II.B,
// shift of a local expansion to the child centre z_P + (b - 1/2) h_P / 2).
// The shift runs as three one-axis passes (exact: |n + k| <= p is kept by each).
// cinfo[4 c .. 4 c + 3] = packed n, index of n + e_x, n + e_y, n + e_z.
// ---------------------------------------------------------------------------
struct DownPtrs {
    const void* Lp[kMaxDepth + 1];
    const int* map[kMaxDepth + 1];  // Morton key -> slot
    const int* key[kMaxDepth + 1];
    int cap[kMaxDepth + 1];
    int depth, nchunk, p;
};

// all threads of the block call it; f, t0, t1: ncoef each, psum: (depth - 1)
// x ncoef, all in shared memory; cinfo[4 c] = packed multi-index of c.  The
// ancestors come from the leaf's Morton key, the M2L partials of all of them
// are read first (independent loads), then the shifts run down the chain.
template <typename R, int NT>
__device__ void far_locals(const DownPtrs& dp, int b, R* f, R* t0, R* t1, R* psum, const int* cinfo, const R* W,
                           int ncoef, int ld) {
    __shared__ int chain[kMaxDepth + 1];
    __shared__ int coct[kMaxDepth + 1];
    const int tid = threadIdx.x;
    const int d = dp.depth;
    if (tid >= 2 && tid <= d) {
        const uint32_t k = (uint32_t)dp.key[d][b] >> (3 * (d - tid));
        chain[tid] = tid == d ? b : dp.map[tid][k];
        coct[tid] = k & 7;
    }
    __syncthreads();
    const int nchunk = dp.nchunk;
    for (int it = tid; it < (d - 1) * ncoef; it += NT) {
        const int li = it / ncoef, cc = it - li * ncoef;
        const R* lp = reinterpret_cast<const R*>(dp.Lp[2 + li]) + (int64_t)chain[2 + li] * ld + cc;
        const int64_t cs = (int64_t)dp.cap[2 + li] * ld;
        R a = R(0);
        int ch = 0;
        for (; ch + 8 <= nchunk; ch += 8) {
            R v[8];
#pragma unroll
            for (int k = 0; k < 8; k++) v[k] = lp[(ch + k) * cs];
#pragma unroll
            for (int k = 0; k < 8; k++) a += v[k];
        }
        for (; ch < nchunk; ch++) a += lp[ch * cs];
        psum[it] = a;
    }
    __syncthreads();
    for (int cc = tid; cc < ncoef; cc += NT) f[cc] = psum[cc];
    __syncthreads();
    for (int l = 3; l <= d; l++) {
        const int oct = coct[l];
        for (int cc = tid; cc < ncoef; cc += NT) t0[cc] = shift_up_axis<0>(f, cc, cinfo[4 * cc], !(oct & 1), W, dp.p);
        __syncthreads();
        for (int cc = tid; cc < ncoef; cc += NT) t1[cc] = shift_up_axis<1>(t0, cc, cinfo[4 * cc], !(oct & 2), W, dp.p);
        __syncthreads();
        const R* pl = psum + (l - 2) * ncoef;
        for (int cc = tid; cc < ncoef; cc += NT) {
            const int pk = cinfo[4 * cc];
            f[cc] = pl[cc] + pow2neg<R>((pk >> 24) + 1) * shift_up_axis<2>(t1, cc, pk, !(oct & 4), W, dp.p);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// M2L (SIMT): tiles of up to 32 same-level, same-octant-class target boxes;
// lane = target box, each warp owns a balanced set of output coefficients;
// the offsets of the class are split into `nchunk` ranges over blockIdx.y,
// each writing its own partial output (summed in fixed order by the downward
// pass in the leaf kernels).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) m2l_simt_kernel(const M2LTile* __restrict__ tiles, LevelPtrs lp,
                                                       const R* __restrict__ D, const int* __restrict__ class_off,
                                                       const short* __restrict__ add, const int* __restrict__ pre,
                                                       const int* __restrict__ wptr, const int* __restrict__ wout,
                                                       int ncoef, int ld, int nchunk) {
    extern __shared__ unsigned char smem_raw[];
    const int st = ncoef + 1;
    R* S = reinterpret_cast<R*>(smem_raw);  // [32][st] source coefficients
    R* A = S + 32 * st;                      // [32][st] accumulators
    R* Ds = A + 32 * st;                     // [ncoef] derivative table of the offset
    int* srcs = reinterpret_cast<int*>(Ds + ncoef);
    const M2LTile tile = tiles[blockIdx.x];
    const int chunk = blockIdx.y;
    const int l = tile.level;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nside = 1 << l;
    int slot = -1, bx = 0, by = 0, bz = 0;
    if (lane < tile.count) {
        slot = lp.by_class[l][tile.first + lane];
        uint32_t k = (uint32_t)lp.key[l][slot];
        bx = compact3(k);
        by = compact3(k >> 1);
        bz = compact3(k >> 2);
    }
    for (int idx = threadIdx.x; idx < 32 * st; idx += blockDim.x) A[idx] = R(0);
    const R* M = reinterpret_cast<const R*>(lp.M[l]);
    const int* map = lp.map[l];
    const int per = (kNumOffsets + nchunk - 1) / nchunk;
    const int t0 = chunk * per, t1 = min(kNumOffsets, t0 + per);
    const int w0 = wptr[warp], w1 = wptr[warp + 1];
    for (int t = t0; t < t1; t++) {
        const int o = class_off[tile.cls * kNumOffsets + t];
        const int ox = (o & 15) - 3, oy = ((o >> 4) & 15) - 3, oz = ((o >> 8) & 15) - 3;
        __syncthreads();
        if (warp == 0) {
            int s = -1;
            int ax = bx - ox, ay = by - oy, az = bz - oz;
            if (slot >= 0 && ax >= 0 && ay >= 0 && az >= 0 && ax < nside && ay < nside && az < nside)
                s = map[morton3(ax, ay, az)];
            srcs[lane] = s;
        }
        __syncthreads();
        if (!__syncthreads_or(srcs[lane] >= 0)) continue;
        for (int idx = threadIdx.x; idx < 32 * ncoef; idx += blockDim.x) {
            int r = idx / ncoef, j = idx - r * ncoef;
            int s = srcs[r];
            S[r * st + j] = s >= 0 ? M[(int64_t)s * ld + j] : R(0);
        }
        const int oidx = (ox + 3) + kOffsetGrid * ((oy + 3) + kOffsetGrid * (oz + 3));
        for (int j = threadIdx.x; j < ncoef; j += blockDim.x) Ds[j] = D[oidx * ncoef + j];
        __syncthreads();
        const R* Srow = S + lane * st;
        R* Arow = A + lane * st;
        for (int e = w0; e < w1; e++) {
            const int nn = wout[e];
            const int np = pre[nn];
            const short* ad = add + (int64_t)nn * ncoef;
            R a = Arow[nn];
            for (int j = 0; j < np; j++) a += Ds[ad[j]] * Srow[j];
            Arow[nn] = a;
        }
    }
    __syncthreads();
    if (slot >= 0) {
        R* Lp = reinterpret_cast<R*>(lp.Lp[l]) + ((int64_t)chunk * lp.cap[l] + slot) * ld;
        for (int e = w0; e < w1; e++) {
            int nn = wout[e];
            Lp[nn] = A[lane * st + nn];
        }
    }
}

// ---------------------------------------------------------------------------
// leaf evaluation: L2P + near field over the 27 adjacent leaves
//
// Sources are packed per site as two 4-vectors: (x, y, z, q) with x relative
// to the site's own leaf centre, and (mu_x, mu_y, mu_z, 0).  One block per
// work item (a leaf and up to leaf_targets of its sites) stages the sources
// of all 27 neighbour leaves (shifted into the target leaf's frame, exact
// small-integer multiples of the leaf side) into shared memory with one
// barrier pair per CAP sources; thread (t, s) owns target t and every
// slices-th source (the FP32 dipole field: every slices-th pair of sources),
// and the slices are added in a fixed order at the end.  The self pair has
// r = 0 exactly and is masked.
// ---------------------------------------------------------------------------
constexpr int kLeafThreads = 256;

template <typename R>
struct alignas(sizeof(R) == 4 ? 16 : 16) Q4 {
    R x, y, z, w;
};

template <typename R>
struct LeafCap;
template <>
struct LeafCap<float> {
    static constexpr int N = 1024;
};
template <>
struct LeafCap<double> {
    static constexpr int N = 128;
};

template <int MODE>
struct LeafOut {
    static constexpr int NC = MODE == LEAF_FULL ? 10 : (MODE == LEAF_CHARGE_PHI_E ? 4 : 3);
};

__device__ inline float rsqrt_pos(float r2) { return r2 > 0.f ? rsqrtf(r2) : 0.f; }
__device__ inline double rsqrt_pos(double r2) { return r2 > 0.0 ? rsqrt(r2) : 0.0; }

// two FP32 values in one 64-bit register for the packed f32x2 arithmetic of
// sm_100 and later (one instruction, two lanes; IEEE round to nearest)
typedef unsigned long long F2;
__device__ inline F2 f2_pack(float lo, float hi) {
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ inline void f2_unpack(F2 v, float& lo, float& hi) { asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v)); }
__device__ inline F2 f2_sub(F2 a, F2 b) {
    F2 d;
    asm("sub.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ inline F2 f2_mul(F2 a, F2 b) {
    F2 d;
    asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ inline F2 f2_fma(F2 a, F2 b, F2 c) {
    F2 d;
    asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// a padding source for an odd count: far away (|r|^-3 underflows to zero) and
// without dipole, so that it adds exactly zero
constexpr float kFarPad = 3.0e18f;

// dynamic shared memory of leaf_kernel<R, MODE>
template <typename R, int MODE>
__host__ __device__ inline size_t leaf_smem_bytes(int ncoef, int depth) {
    constexpr int CAP = LeafCap<R>::N;
    size_t b = sizeof(Q4<R>) * CAP;                          // positions + charge
    if (MODE != LEAF_CHARGE_PHI_E) b += sizeof(Q4<R>) * CAP;  // dipoles
    if (MODE == LEAF_CHARGE_PHI_E) b += sizeof(int) * CAP;    // source index (coincidence check)
    b += sizeof(R) * (4 + (size_t)(depth > 1 ? depth - 1 : 0)) * ncoef;  // locals, shift buffers, 1/n!, partials
    b += sizeof(int) * 4 * (size_t)ncoef;                     // packed n, n + e_d
    if (MODE == LEAF_FULL) b += sizeof(int) * 6 * (size_t)ncoef;
    return b;
}

template <typename R>
__global__ void pack_positions_kernel(int64_t n, const R* __restrict__ ploc, const double* __restrict__ q,
                                      Q4<R>* __restrict__ A) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    A[i] = Q4<R>{ploc[3 * i], ploc[3 * i + 1], ploc[3 * i + 2], R(q[i])};
}

template <typename R>
__global__ void pack_dipoles_kernel(int64_t n, const double* __restrict__ mu, Q4<R>* __restrict__ B) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    B[i] = Q4<R>{R(mu[3 * i]), R(mu[3 * i + 1]), R(mu[3 * i + 2]), R(0)};
}

template <typename R, int MODE>
__global__ void __launch_bounds__(kLeafThreads) leaf_kernel(
    const int2* __restrict__ items, const int* __restrict__ nitems, const int* __restrict__ lkey,
    const int* __restrict__ lstart, const int* __restrict__ lcount, const int* __restrict__ lmap, int depth,
    const Q4<R>* __restrict__ srcA,
    const Q4<R>* __restrict__ srcB, DownPtrs dp, int ld, int ncoef, int p, const int* __restrict__ mi,
    const double* __restrict__ inv_fact, const int* __restrict__ up1, const int* __restrict__ up2,
    const R* __restrict__ w4, R h,
    double* __restrict__ out_phi, double* __restrict__ out_E, double* __restrict__ out_G, int* __restrict__ err,
    int far) {
    constexpr int NC = LeafOut<MODE>::NC;
    constexpr int CAP = LeafCap<R>::N;
    constexpr bool HAS_PHI = MODE != LEAF_DIPOLE_E;
    constexpr bool HAS_G = MODE == LEAF_FULL;
    constexpr bool SRC_Q = MODE != LEAF_DIPOLE_E;
    constexpr bool SRC_MU = MODE != LEAF_CHARGE_PHI_E;
    constexpr bool CHECK = MODE == LEAF_CHARGE_PHI_E;
    constexpr int IE = HAS_PHI ? 1 : 0;  // component layout: [phi] E(3) [G(6)]
    constexpr int IG = IE + 3;
    // FP32 dipole field: two sources per thread step in packed f32x2 arithmetic;
    // the staged sources are then stored as pairs, 12 floats per pair
    // (x0 x1 y0 y1 | z0 z1 mx0 mx1 | my0 my1 mz0 mz1), over the sA/sB space
    constexpr bool PACKED = MODE == LEAF_DIPOLE_E && sizeof(R) == 4;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    Q4<R>* sA = reinterpret_cast<Q4<R>*>(smem_raw);
    Q4<R>* sB = sA + CAP;
    unsigned char* tail = reinterpret_cast<unsigned char*>(SRC_MU ? sB + CAP : sA + CAP);
    int* sidx = reinterpret_cast<int*>(tail);
    if (CHECK) tail += sizeof(int) * CAP;
    R* f = reinterpret_cast<R*>(tail);
    R* t0 = f + ncoef;
    R* t1 = t0 + ncoef;
    R* ifact = t1 + ncoef;
    int* cinfo = reinterpret_cast<int*>(ifact + ncoef);  // [ncoef][4]: packed n, n+e_x, n+e_y, n+e_z
    int* cup2 = cinfo + 4 * ncoef;                       // [ncoef][6] (FULL only)
    R* psum = reinterpret_cast<R*>(cup2 + (HAS_G ? 6 * ncoef : 0));  // [depth - 1][ncoef]
    __shared__ R W[kMaxP + 1];
    __shared__ int nb_start[27];
    __shared__ int nb_pre[28];
    __shared__ R nb_shift[27][3];
    __shared__ R part[NC][kLeafThreads];

    if ((int)blockIdx.x >= *nitems) return;
    const int2 item = items[blockIdx.x];
    const int b = item.x;
    const int s0 = lstart[b], cnt = lcount[b];
    const int t_lo = item.y, t_hi = min(cnt, item.y + leaf_targets(sizeof(R) == 4));  // this block's targets
    const int tid = threadIdx.x;
    if (tid < 32) {
        int c = 0;
        if (tid < 27) {
            const uint32_t key = (uint32_t)lkey[b];
            const int nside = 1 << depth;
            const int dx = tid % 3 - 1, dy = (tid / 3) % 3 - 1, dz = tid / 9 - 1;
            const int ax = (int)compact3(key) + dx, ay = (int)compact3(key >> 1) + dy, az = (int)compact3(key >> 2) + dz;
            int ns = -1;
            if (ax >= 0 && ay >= 0 && az >= 0 && ax < nside && ay < nside && az < nside) ns = lmap[morton3(ax, ay, az)];
            nb_start[tid] = ns >= 0 ? lstart[ns] : 0;
            c = ns >= 0 ? lcount[ns] : 0;
            nb_shift[tid][0] = R(dx) * h;
            nb_shift[tid][1] = R(dy) * h;
            nb_shift[tid][2] = R(dz) * h;
        }
        int incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (tid >= o) incl += v;
        }
        if (tid < 27) nb_pre[tid + 1] = incl;
        if (tid == 0) nb_pre[0] = 0;
    }
    for (int cc = tid; cc < ncoef; cc += blockDim.x) {
        ifact[cc] = R(inv_fact[cc]);
        cinfo[4 * cc] = mi[cc];
        cinfo[4 * cc + 1] = up1[3 * cc];
        cinfo[4 * cc + 2] = up1[3 * cc + 1];
        cinfo[4 * cc + 3] = up1[3 * cc + 2];
        if (HAS_G)
            for (int k = 0; k < 6; k++) cup2[6 * cc + k] = up2[6 * cc + k];
    }
    stage_small(W, w4, p);
    __syncthreads();
    if (far) far_locals<R, kLeafThreads>(dp, b, f, t0, t1, psum, cinfo, W, ncoef, ld);
    const int total = nb_pre[27];
    const R inv_h = R(1) / h;

    for (int tg = t_lo; tg < t_hi; tg += kLeafThreads) {
        const int nt = min(kLeafThreads, t_hi - tg);
        const int slices = kLeafThreads / nt;
        const int t = tid % nt, s = tid / nt;
        const bool active = s < slices;
        const int i = s0 + tg + t;
        R acc[NC], acc2[NC];
#pragma unroll
        for (int k = 0; k < NC; k++) acc[k] = acc2[k] = R(0);
        // dipole field of the sources, E = 3 er - em with er = sum (mu.r) r / r^5 and
        // em = sum mu / r^3 (two sets, like acc / acc2)
        R er[2][3], em[2][3];
#pragma unroll
        for (int k = 0; k < 3; k++) er[0][k] = er[1][k] = em[0][k] = em[1][k] = R(0);
        F2 per[3] = {0, 0, 0}, pem[3] = {0, 0, 0};  // packed er / em (PACKED)
        R xi = R(0), yi = R(0), zi = R(0);
        if (active) {
            const Q4<R> me = srcA[i];
            xi = me.x;
            yi = me.y;
            zi = me.z;
            // far field: L2P of this slice's share of the coefficients
            const R ux = xi * inv_h, uy = yi * inv_h, uz = zi * inv_h;
            R phi = R(0), d0 = R(0), d1 = R(0), d2 = R(0);
            R dd[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
            for (int cc = far ? s : ncoef; cc < ncoef; cc += slices) {
                const int pk = cinfo[4 * cc];
                R wgt = ifact[cc];
                for (int k = pk & 0xff; k > 0; k--) wgt *= ux;
                for (int k = (pk >> 8) & 0xff; k > 0; k--) wgt *= uy;
                for (int k = (pk >> 16) & 0xff; k > 0; k--) wgt *= uz;
                if (HAS_PHI) phi += wgt * f[cc];
                const int u0 = cinfo[4 * cc + 1];
                if (u0 >= 0) {
                    d0 += wgt * f[u0];
                    d1 += wgt * f[cinfo[4 * cc + 2]];
                    d2 += wgt * f[cinfo[4 * cc + 3]];
                }
                if (HAS_G) {
                    const int v0 = cup2[6 * cc];
                    if (v0 >= 0) {
                        dd[0] += wgt * f[v0];
#pragma unroll
                        for (int k = 1; k < 6; k++) dd[k] += wgt * f[cup2[6 * cc + k]];
                    }
                }
            }
            // Phi = phi / h, E = -dPhi / h^2, G = -ddPhi / h^3
            if (HAS_PHI) acc[0] = phi * inv_h;
            const R s2 = -inv_h * inv_h;
            acc[IE + 0] = d0 * s2;
            acc[IE + 1] = d1 * s2;
            acc[IE + 2] = d2 * s2;
            if (HAS_G) {
                const R s3 = s2 * inv_h;
#pragma unroll
                for (int k = 0; k < 6; k++) acc[IG + k] = dd[k] * s3;
            }
        }
        // near field
        for (int base = 0; base < total; base += CAP) {
            const int m = min(CAP, total - base);
            __syncthreads();
#pragma unroll 4
            for (int idx = tid; idx < m; idx += blockDim.x) {
                const int g = base + idx;
                int lo = 0, hi = 26;  // range r with nb_pre[r] <= g < nb_pre[r + 1]
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (nb_pre[mid] <= g) lo = mid; else hi = mid - 1;
                }
                const int j = nb_start[lo] + (g - nb_pre[lo]);
                Q4<R> a = srcA[j];
                a.x += nb_shift[lo][0];
                a.y += nb_shift[lo][1];
                a.z += nb_shift[lo][2];
                if constexpr (PACKED) {
                    const Q4<R> mv = srcB[j];
                    float* q = reinterpret_cast<float*>(sA) + 12 * (idx >> 1) + (idx & 1);
                    q[0] = a.x;
                    q[2] = a.y;
                    q[4] = a.z;
                    q[6] = mv.x;
                    q[8] = mv.y;
                    q[10] = mv.z;
                } else {
                    sA[idx] = a;
                    if (SRC_MU) sB[idx] = srcB[j];
                    if (CHECK) sidx[idx] = j;
                }
            }
            if constexpr (PACKED) {
                if ((m & 1) && tid == 0) {
                    float* q = reinterpret_cast<float*>(sA) + 12 * (m >> 1) + 1;
                    q[0] = q[2] = q[4] = kFarPad;
                    q[6] = q[8] = q[10] = 0.f;
                }
            }
            __syncthreads();
            if (!active) continue;
            if constexpr (PACKED) {
                // er += (mu.r) r / r^5, em += mu / r^3 for the sources 2 pp and 2 pp + 1
                const ulonglong2* sp = reinterpret_cast<const ulonglong2*>(sA);
                const F2 XI = f2_pack(xi, xi), YI = f2_pack(yi, yi), ZI = f2_pack(zi, zi);
                const int np = (m + 1) >> 1;
#pragma unroll 2
                for (int pp = s; pp < np; pp += slices) {
                    const ulonglong2 A = sp[3 * pp], B = sp[3 * pp + 1], C = sp[3 * pp + 2];
                    const F2 rx = f2_sub(XI, A.x), ry = f2_sub(YI, A.y), rz = f2_sub(ZI, B.x);
                    const F2 r2 = f2_fma(rz, rz, f2_fma(ry, ry, f2_mul(rx, rx)));
                    float r2a, r2b;
                    f2_unpack(r2, r2a, r2b);
                    const F2 ri = f2_pack(rsqrt_pos(r2a), rsqrt_pos(r2b));  // 0 for the self pair
                    const F2 ri2 = f2_mul(ri, ri);
                    const F2 ri3 = f2_mul(ri, ri2);
                    const F2 mr = f2_fma(C.y, rz, f2_fma(C.x, ry, f2_mul(B.y, rx)));
                    const F2 am = f2_mul(mr, f2_mul(ri3, ri2));
                    per[0] = f2_fma(am, rx, per[0]);
                    per[1] = f2_fma(am, ry, per[1]);
                    per[2] = f2_fma(am, rz, per[2]);
                    pem[0] = f2_fma(ri3, B.y, pem[0]);
                    pem[1] = f2_fma(ri3, C.x, pem[1]);
                    pem[2] = f2_fma(ri3, C.y, pem[2]);
                }
                continue;
            }
            // two independent accumulator sets (sources jj and jj + slices) for
            // instruction-level parallelism; added in fixed order after the loop
            auto pair = [&](R* ac, R* ar, R* am, const int jj) {
                const Q4<R> a = sA[jj];
                const R rx = xi - a.x, ry = yi - a.y, rz = zi - a.z;
                const R r2 = rx * rx + ry * ry + rz * rz;
                if (CHECK && r2 == R(0) && sidx[jj] != i) atomicOr(err, 2);
                const R ri = rsqrt_pos(r2);  // 0 for the self pair
                const R ri2 = ri * ri;
                const R ri3 = ri * ri2;
                if (SRC_Q) {
                    const R qj = a.w;
                    const R qr3 = qj * ri3;
                    if (HAS_PHI) ac[0] += qj * ri;
                    ac[IE + 0] += qr3 * rx;
                    ac[IE + 1] += qr3 * ry;
                    ac[IE + 2] += qr3 * rz;
                    if (HAS_G) {
                        const R t5 = R(3) * qr3 * ri2;
                        ac[IG + 0] += qr3 - t5 * rx * rx;
                        ac[IG + 1] -= t5 * rx * ry;
                        ac[IG + 2] -= t5 * rx * rz;
                        ac[IG + 3] += qr3 - t5 * ry * ry;
                        ac[IG + 4] -= t5 * ry * rz;
                        ac[IG + 5] += qr3 - t5 * rz * rz;
                    }
                }
                if (SRC_MU) {
                    const Q4<R> mv = sB[jj];
                    const R mr = mv.x * rx + mv.y * ry + mv.z * rz;
                    const R ri5 = ri3 * ri2;
                    const R a = mr * ri5;
                    if (HAS_PHI) ac[0] += mr * ri3;
                    ar[0] = fma(a, rx, ar[0]);
                    ar[1] = fma(a, ry, ar[1]);
                    ar[2] = fma(a, rz, ar[2]);
                    am[0] = fma(ri3, mv.x, am[0]);
                    am[1] = fma(ri3, mv.y, am[1]);
                    am[2] = fma(ri3, mv.z, am[2]);
                    if (HAS_G) {
                        const R a3 = R(3) * a;
                        // G_de = 3 (mu_d r_e + mu_e r_d + mr delta_de) / r^5 - 15 mr r_d r_e / r^7
                        const R t5 = R(3) * ri5;
                        const R t7 = R(5) * a3 * ri2;
                        ac[IG + 0] += t5 * (R(2) * mv.x * rx + mr) - t7 * rx * rx;
                        ac[IG + 1] += t5 * (mv.x * ry + mv.y * rx) - t7 * rx * ry;
                        ac[IG + 2] += t5 * (mv.x * rz + mv.z * rx) - t7 * rx * rz;
                        ac[IG + 3] += t5 * (R(2) * mv.y * ry + mr) - t7 * ry * ry;
                        ac[IG + 4] += t5 * (mv.y * rz + mv.z * ry) - t7 * ry * rz;
                        ac[IG + 5] += t5 * (R(2) * mv.z * rz + mr) - t7 * rz * rz;
                    }
                }
            };
            int jj = s;
#pragma unroll 2
            for (; jj + slices < m; jj += 2 * slices) {
                pair(acc, er[0], em[0], jj);
                pair(acc2, er[1], em[1], jj + slices);
            }
            if (jj < m) pair(acc, er[0], em[0], jj);
        }
#pragma unroll
        for (int k = 0; k < NC; k++) acc[k] += acc2[k];
        if constexpr (PACKED) {
#pragma unroll
            for (int k = 0; k < 3; k++) {
                float r0, r1, m0, m1;
                f2_unpack(per[k], r0, r1);
                f2_unpack(pem[k], m0, m1);
                er[0][k] = r0;
                er[1][k] = r1;
                em[0][k] = m0;
                em[1][k] = m1;
            }
        }
        if (SRC_MU) {
#pragma unroll
            for (int k = 0; k < 3; k++) acc[IE + k] += R(3) * (er[0][k] + er[1][k]) - (em[0][k] + em[1][k]);
        }
        // fixed-order reduction over slices
        __syncthreads();
#pragma unroll
        for (int k = 0; k < NC; k++) part[k][tid] = active ? acc[k] : R(0);
        __syncthreads();
        if (tid < nt) {
            const int ii = s0 + tg + tid;
            double o[NC];
#pragma unroll
            for (int k = 0; k < NC; k++) {
                R v = R(0);
                for (int u = 0; u < slices; u++) v += part[k][tid + u * nt];
                o[k] = (double)v;
            }
            if (HAS_PHI && out_phi) out_phi[ii] = o[0];
            if (out_E)
                for (int d = 0; d < 3; d++) out_E[3 * (int64_t)ii + d] = o[IE + d];
            if (HAS_G && out_G)
                for (int k = 0; k < 6; k++) out_G[6 * (int64_t)ii + k] = o[IG + k];
        }
    }
}

// ---------------------------------------------------------------------------
// FP32 near field of the dipole solve: E_i = sum_j [3 (mu_j.r) r / r^5 - mu_j / r^3]
// over the sites j != i of the 27 adjacent leaves (Sec. II.A, the field of the
// induced dipoles; the far field is added after the multipole passes).
//
// The sources are pair records in global memory (near_pairs: positions
// relative to their own leaf centre, written once per tree; dipoles, written
// once per pass), so that a leaf's sources are one contiguous range.  Each
// work item (a leaf and up to kNearTargets of its sites) has a 240-byte record
// with the 27 ranges of its adjacent leaves, its own leaf first.
//
// One block per item.  Staging: thread t copies records t, t + 256, ... of
// the item's concatenated ranges (three 16-byte loads and stores each),
// adding the neighbour leaf's offset to the positions.  Thread (w, s) owns targets 2w and 2w + 1 and every
// slices-th record: four pairs per step in packed f32x2 arithmetic, the three
// 16-byte loads of a record serving both targets; only the own leaf's
// records, which come first, test for the self pair.  The slices are added in
// a fixed order.
// ---------------------------------------------------------------------------
constexpr int kNearThreads = 256;
constexpr int kNearBlocksPerSM = 3;
constexpr int kNearPairCap = 512;  // pair records per chunk (1,024 sources, 24 KB)
constexpr int kNearTargets = 64;    // targets per near-field item
static_assert(kLeafTargetsF32 <= 2 * kNearTargets, "a leaf item makes at most two near-field items");

struct NearSmem {
    float4 pairs[kNearPairCap * 3];
    float part[3][2 * kNearThreads];
    float shift[27][3];
    int segx[28];    // item-relative first record of segment r; segx[27] = records of the item
    int segsrc[27];  // first pair record of segment r in near_pairs
    int nt, s0t;
};
static_assert(kNearBlocksPerSM * (sizeof(NearSmem) + 1024) <= 228 * 1024, "three blocks fit on one SM");

constexpr size_t near_dipole_smem_bytes() { return sizeof(NearSmem); }

// E += r^-3 [nu - 3 (nu.r) r / r^2] for the two sources of record pp, nu = -mu
// the stored (negated) dipole: the field 3 (mu.r) r / r^5 - mu / r^3 with one
// accumulator per component
template <bool SELF>
__device__ __forceinline__ void near_step(const ulonglong2* __restrict__ sp, int pp, const F2 (&X)[2][3],
                                          F2 (&E)[2][3]) {
    const ulonglong2 A = sp[3 * pp], B = sp[3 * pp + 1], C = sp[3 * pp + 2];
    const F2 M3 = f2_pack(-3.f, -3.f);
#pragma unroll
    for (int u = 0; u < 2; u++) {
        const F2 rx = f2_sub(X[u][0], A.x), ry = f2_sub(X[u][1], A.y), rz = f2_sub(X[u][2], B.x);
        const F2 r2 = f2_fma(rz, rz, f2_fma(ry, ry, f2_mul(rx, rx)));
        float r2a, r2b;
        f2_unpack(r2, r2a, r2b);
        const F2 ri = SELF ? f2_pack(rsqrt_pos(r2a), rsqrt_pos(r2b)) : f2_pack(rsqrtf(r2a), rsqrtf(r2b));
        const F2 ri2 = f2_mul(ri, ri);
        const F2 ri3 = f2_mul(ri, ri2);
        const F2 nr = f2_fma(C.y, rz, f2_fma(C.x, ry, f2_mul(B.y, rx)));  // nu.r
        const F2 a = f2_mul(nr, f2_mul(ri2, M3));                          // -3 (nu.r) / r^2
        E[u][0] = f2_fma(ri3, f2_fma(a, rx, B.y), E[u][0]);
        E[u][1] = f2_fma(ri3, f2_fma(a, ry, C.x), E[u][1]);
        E[u][2] = f2_fma(ri3, f2_fma(a, rz, C.y), E[u][2]);
    }
}

__global__ void __launch_bounds__(kNearThreads, kNearBlocksPerSM) near_dipole_f32_kernel(
    const NearItem* __restrict__ items, const int* __restrict__ nitems, const float4* __restrict__ P,
    const Q4<float>* __restrict__ srcA, float h, double* __restrict__ out_E) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    NearSmem& S = *reinterpret_cast<NearSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if ((int)blockIdx.x >= *nitems) return;
    const NearItem& R = items[blockIdx.x];
    if (tid < 27) {
        // segment r: the own leaf (offset 0), then the other 26 in a fixed order
        const int o = tid == 0 ? 13 : (tid <= 13 ? tid - 1 : tid);
        S.shift[tid][0] = float(o % 3 - 1) * h;
        S.shift[tid][1] = float((o / 3) % 3 - 1) * h;
        S.shift[tid][2] = float(o / 9 - 1) * h;
    }
    if (warp == 0) {
        const int2 e = lane < 27 ? R.seg[lane] : make_int2(0, 0);
        int incl = e.y;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane < 27) {
            S.segx[lane] = incl - e.y;
            S.segsrc[lane] = e.x;
        }
        if (lane == 26) S.segx[27] = incl;
        if (lane == 0) {
            S.nt = R.nt;
            S.s0t = R.s0 + R.t_lo;
        }
    }
    __syncthreads();
    const int nt = S.nt, s0t = S.s0t, total = S.segx[27];
    const int ntp = (nt + 1) >> 1;
    const int slices = kNearThreads / ntp;
    const int w = tid % ntp, s = tid / ntp;
    const bool active = s < slices;
    F2 X[2][3];
#pragma unroll
    for (int v = 0; v < 2; v++) {
        // a missing second target repeats the first (its sums are dropped)
        const Q4<float> t = srcA[s0t + min(2 * w + v, nt - 1)];
        X[v][0] = f2_pack(t.x, t.x);
        X[v][1] = f2_pack(t.y, t.y);
        X[v][2] = f2_pack(t.z, t.z);
    }
    F2 E[2][3];
#pragma unroll
    for (int v = 0; v < 2; v++)
#pragma unroll
        for (int k = 0; k < 3; k++) E[v][k] = 0ull;
    const ulonglong2* sp = reinterpret_cast<const ulonglong2*>(S.pairs);
    for (int lo = 0; lo < total; lo += kNearPairCap) {
        const int m = min(total - lo, kNearPairCap);
        if (lo > 0) __syncthreads();  // the previous chunk is consumed
        // record k of the chunk: segment r with segx[r] <= lo + k < segx[r + 1]
        // (a search instead of a loop over segments, so that every thread
        // issues its loads at once)
        for (int k = tid; k < m; k += kNearThreads) {
            const int g = lo + k;
            int r = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (r + step < 27 && S.segx[r + step] <= g) r += step;
            const float4* src = P + 3 * ((int64_t)S.segsrc[r] + (g - S.segx[r]));
            float4 p0 = src[0], p1 = src[1];
            const float4 p2 = src[2];
            const float sx = S.shift[r][0], sy = S.shift[r][1], sz = S.shift[r][2];
            p0.x += sx;
            p0.y += sx;
            p0.z += sy;
            p0.w += sy;
            p1.x += sz;
            p1.y += sz;
            float4* d = &S.pairs[3 * k];
            d[0] = p0;
            d[1] = p1;
            d[2] = p2;
        }
        __syncthreads();
        if (active) {
            const int own_end = min(max(S.segx[1] - lo, 0), m);
            int pp = s;
            for (; pp < own_end; pp += slices) near_step<true>(sp, pp, X, E);
            for (; pp < m; pp += slices) near_step<false>(sp, pp, X, E);
        }
    }
    // fixed-order reduction over slices: target t, slice s at part[.][s * 2 ntp + t]
    if (active) {
#pragma unroll
        for (int v = 0; v < 2; v++)
#pragma unroll
            for (int k = 0; k < 3; k++) {
                float e0, e1;
                f2_unpack(E[v][k], e0, e1);
                S.part[k][s * 2 * ntp + 2 * w + v] = e0 + e1;
            }
    }
    __syncthreads();
    if (tid < nt) {
        const int64_t ii = s0t + tid;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            float acc = 0.f;
            for (int q = 0; q < slices; q++) acc += S.part[k][q * 2 * ntp + tid];
            out_E[3 * ii + k] = (double)acc;
        }
    }
}

// per tree (MIXED): records of ceil(count / 2) per leaf, first record of each leaf
__global__ void near_pair_count_kernel(int nleaf, const int* __restrict__ lcount, int* __restrict__ npair) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nleaf) npair[b] = (lcount[b] + 1) >> 1;
}

// per tree: the positions of the pair records (dipoles zero until a pass packs
// them), the far padding source of odd leaves, and the record slot of each site
__global__ void near_records_kernel(int nleaf, const int* __restrict__ lstart, const int* __restrict__ lcount,
                                    const int* __restrict__ pbase, const Q4<float>* __restrict__ srcA,
                                    float* __restrict__ P, int* __restrict__ slot) {
    const int b = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (b >= nleaf) return;
    const int s0 = lstart[b], cnt = lcount[b], np = (cnt + 1) >> 1, pb = pbase[b];
    for (int k = lane; k < np; k += 32) {
        const int i0 = s0 + 2 * k;
        const bool two = 2 * k + 1 < cnt;
        const Q4<float> a = srcA[i0];
        const Q4<float> c = two ? srcA[i0 + 1] : Q4<float>{kFarPad, kFarPad, kFarPad, 0.f};
        float4* q = reinterpret_cast<float4*>(P + 12 * (int64_t)(pb + k));
        q[0] = make_float4(a.x, c.x, a.y, c.y);
        q[1] = make_float4(a.z, c.z, 0.f, 0.f);
        q[2] = make_float4(0.f, 0.f, 0.f, 0.f);
        slot[i0] = 2 * (pb + k);
        if (two) slot[i0 + 1] = 2 * (pb + k) + 1;
    }
}

// per tree: near-field items per leaf item (ceil(targets / 32)), 0 past the list
__global__ void near_item_count_kernel(const int2* __restrict__ litems, const int* __restrict__ nitems, int bound,
                                       const int* __restrict__ lcount, int* __restrict__ cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= bound) return;
    int c = 0;
    if (i < *nitems) {
        const int nt = min(lcount[litems[i].x] - litems[i].y, kLeafTargetsF32);
        c = (nt + kNearTargets - 1) / kNearTargets;
    }
    cnt[i] = c;
}

// per tree: the work-item records, in the order of the leaf items (heaviest
// first): own leaf first, then the other 26 adjacent leaves in a fixed order;
// absent leaves are empty ranges
__global__ void near_items_kernel(const int2* __restrict__ litems, const int* __restrict__ nitems,
                                  const int* __restrict__ first, int depth, const int* __restrict__ lkey,
                                  const int* __restrict__ lmap, const int* __restrict__ lstart,
                                  const int* __restrict__ lcount, const int* __restrict__ pbase,
                                  NearItem* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *nitems) return;
    const int b = litems[i].x, t0 = litems[i].y;
    const int nt_all = min(lcount[b] - t0, kLeafTargetsF32);
    int2 seg[27];
    const uint32_t key = (uint32_t)lkey[b];
    const int nside = 1 << depth;
    const int bx = (int)compact3(key), by = (int)compact3(key >> 1), bz = (int)compact3(key >> 2);
    for (int r = 0; r < 27; r++) {
        const int o = r == 0 ? 13 : (r <= 13 ? r - 1 : r);
        const int ax = bx + o % 3 - 1, ay = by + (o / 3) % 3 - 1, az = bz + o / 9 - 1;
        int ns = -1;
        if (ax >= 0 && ay >= 0 && az >= 0 && ax < nside && ay < nside && az < nside) ns = lmap[morton3(ax, ay, az)];
        seg[r] = ns >= 0 ? make_int2(pbase[ns], (lcount[ns] + 1) >> 1) : make_int2(0, 0);
    }
    int o = first[i];
    for (int t = 0; t < nt_all; t += kNearTargets, o++) {
        NearItem& R = out[o];
        R.b = b;
        R.s0 = lstart[b];
        R.t_lo = t0 + t;
        R.nt = min(nt_all - t, kNearTargets);
        R.pad[0] = R.pad[1] = 0;
        for (int r = 0; r < 27; r++) R.seg[r] = seg[r];
    }
}

// per pass: the dipoles into the pair records (negated: the kernel's form)
__global__ void near_pack_mu_kernel(int64_t n, const double* __restrict__ mu, const int* __restrict__ slot,
                                    float* __restrict__ P) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int sl = slot[i];
    float* q = P + 12 * (int64_t)(sl >> 1) + (sl & 1);
    q[6] = -(float)mu[3 * i];
    q[8] = -(float)mu[3 * i + 1];
    q[10] = -(float)mu[3 * i + 2];
}

int near_tables(polfmm_ctx* c) {
    if (!c->mixed) return POLFMM_OK;
    Level& L = c->lv[c->depth];
    const int nl = L.nbox;
    {
        LaunchScope ls(c, F_TREE);
        near_pair_count_kernel<<<grid_for(nl, 256), 256, 0, c->stream>>>(nl, c->lcount, c->flags);
    }
    scan_exclusive(c, c->flags, c->near_pbase, nl, nullptr);
    LaunchScope ls(c, F_TREE);
    near_records_kernel<<<grid_for((int64_t)nl * 32, 256), 256, 0, c->stream>>>(
        nl, c->lstart, c->lcount, c->near_pbase, reinterpret_cast<const Q4<float>*>(c->srcA), c->near_pairs,
        c->near_slot);
    // every leaf item has a target of its own: at most n items
    const int bound = (int)std::min<int64_t>(c->leaf_items_grid, c->n);
    near_item_count_kernel<<<grid_for(bound, 256), 256, 0, c->stream>>>(c->leaf_items, c->leaf_nitems, bound,
                                                                         c->lcount, c->flags);
    scan_exclusive(c, c->flags, c->val_a, bound, c->near_nitems);
    near_items_kernel<<<grid_for(bound, 128), 128, 0, c->stream>>>(c->leaf_items, c->leaf_nitems, c->val_a,
                                                                   c->depth, L.key, L.map, c->lstart, c->lcount,
                                                                   c->near_pbase, c->near_items);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? POLFMM_OK : cuda_fail(e, "near-field tables");
}

// far field of the solver pass, added to the near field already in out_E:
// E += -(1/h^2) sum_{|n| <= p-1} u^n/n! f_{n+e_d}, u = (x - z) / h (Sec. II.B).
// With pf.Ad set (PCG), the kernel also forms Ad = d/alpha - E of its sites
// and the leaf's partial of d.Ad; the last block to finish adds the partials
// of all leaves in leaf order into scal[S_DAD] (deterministic).
constexpr int kL2PThreads = 128;
constexpr int kPowStride = 3 * kMaxP + 1;  // odd: the per-thread rows hit distinct banks

struct PcgFuse {
    const double* inv_alpha;  // 1 / alpha, 0 where alpha = 0
    const double* d;
    double* Ad;
    double* partial;  // [nleaf]
    double* scal;
    int* ticket;
    cudaGraphConditionalHandle cond;  // inside the solve graph: cleared here, set by the update kernel
};

// f, t0, t1 and the partials of depth - 1 levels, each padded to ld (a
// multiple of 4) so that the int4 rows of cinfo after them stay 16-byte aligned
template <typename R>
__host__ __device__ inline size_t l2p_smem_bytes(int ld, int depth) {
    return sizeof(R) * (3 + (size_t)(depth > 1 ? depth - 1 : 0)) * ld + sizeof(int) * 4 * (size_t)ld;
}

// thread (site t, slice sl) of a block of sites evaluates the coefficients
// sl, sl + slices, ... of the field expansion with its own table of
// u_a^k / k! (k < p); the slices are added in fixed order
template <typename R>
__global__ void __launch_bounds__(kL2PThreads) l2p_field_add_kernel(
    int nleaf, const int* __restrict__ lstart, const int* __restrict__ lcount, const Q4<R>* __restrict__ srcA,
    DownPtrs dp, int ld, int ncoef, int p, const int* __restrict__ mi, const int* __restrict__ up1,
    const R* __restrict__ w4, const R* __restrict__ rinv, R h, double* __restrict__ out_E, PcgFuse pf) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* f = reinterpret_cast<R*>(smem_raw);
    R* t0 = f + ld;
    R* t1 = t0 + ld;
    R* psum = t1 + ld;                                               // [depth - 1][ncoef]
    int* cinfo = reinterpret_cast<int*>(psum + (dp.depth - 1) * ld);  // [ncoef][4], 16-byte aligned
    __shared__ R pw[kL2PThreads * kPowStride];
    __shared__ R part[3][kL2PThreads];
    __shared__ R W[kMaxP + 1];
    __shared__ R RI[kMaxP + 1];
    __shared__ double red[kL2PThreads / 32];
    __shared__ bool last;
    const int b = blockIdx.x;
    if (b >= nleaf) return;
    const int tid = threadIdx.x;
    if (pf.cond && b == 0 && tid == 0) cudaGraphSetConditional(pf.cond, 0u);
    for (int cc = tid; cc < ncoef; cc += kL2PThreads) {
        cinfo[4 * cc] = mi[cc];
        cinfo[4 * cc + 1] = up1[3 * cc];
        cinfo[4 * cc + 2] = up1[3 * cc + 1];
        cinfo[4 * cc + 3] = up1[3 * cc + 2];
    }
    stage_small(W, w4, p);
    stage_small(RI, rinv, p);
    // launched after the M2L with programmatic serialization: its partials and
    // the near field are complete from here on
    pdl_wait();
    // the first site group's near field, alpha and d, read now so that their
    // latency hides behind the downward pass
    const int s0 = lstart[b], cnt = lcount[b];
    double pre[7] = {0, 0, 0, 0, 0, 0, 0};
    if (tid < cnt) {
        const int64_t i = s0 + tid;
        for (int k = 0; k < 3; k++) pre[k] = out_E[3 * i + k];
        if (pf.Ad) {
            pre[3] = pf.inv_alpha[i];
            for (int k = 0; k < 3; k++) pre[4 + k] = pf.d[3 * i + k];
        }
    }
    __syncthreads();
    far_locals<R, kL2PThreads>(dp, b, f, t0, t1, psum, cinfo, W, ncoef, ld);
    const int nlow = p * (p + 1) * (p + 2) / 6;  // coefficients with |n| <= p - 1
    const R inv_h = R(1) / h;
    const R s2 = -inv_h * inv_h;
    double dot = 0.0;
    R* mypw = pw + tid * kPowStride;
    for (int tg = 0; tg < cnt; tg += kL2PThreads) {
        const int nt = min(kL2PThreads, cnt - tg);
        const int slices = kL2PThreads / nt;
        const int t = tid % nt, sl = tid / nt;
        R d0 = R(0), d1 = R(0), d2 = R(0);
        if (sl < slices) {
            const Q4<R> me = srcA[s0 + tg + t];
            const R u[3] = {me.x * inv_h, me.y * inv_h, me.z * inv_h};
            for (int a = 0; a < 3; a++) {
                R w = R(1);
                mypw[a * kMaxP] = w;
                for (int k = 1; k < p; k++) {
                    w = w * u[a] * RI[k];
                    mypw[a * kMaxP + k] = w;
                }
            }
            // E_d = -(1/h^2) sum_{|n| <= p-1} u^n/n! f_{n+e_d}
            for (int cc = sl; cc < nlow; cc += slices) {
                const int4 ci = *reinterpret_cast<const int4*>(cinfo + 4 * cc);
                const R wgt = mypw[ci.x & 0xff] * mypw[kMaxP + ((ci.x >> 8) & 0xff)] *
                              mypw[2 * kMaxP + ((ci.x >> 16) & 0xff)];
                d0 += wgt * f[ci.y];
                d1 += wgt * f[ci.z];
                d2 += wgt * f[ci.w];
            }
        }
        part[0][tid] = d0;
        part[1][tid] = d1;
        part[2][tid] = d2;
        __syncthreads();
        if (tid < nt) {
            const int i = s0 + tg + tid;
            R e0 = R(0), e1 = R(0), e2 = R(0);
            for (int u = 0; u < slices; u++) {
                e0 += part[0][tid + u * nt];
                e1 += part[1][tid + u * nt];
                e2 += part[2][tid + u * nt];
            }
            if (tg > 0) {
                for (int k = 0; k < 3; k++) pre[k] = out_E[3 * (int64_t)i + k];
                if (pf.Ad) {
                    pre[3] = pf.inv_alpha[i];
                    for (int k = 0; k < 3; k++) pre[4 + k] = pf.d[3 * (int64_t)i + k];
                }
            }
            double e[3];
            e[0] = pre[0] + (double)(e0 * s2);
            e[1] = pre[1] + (double)(e1 * s2);
            e[2] = pre[2] + (double)(e2 * s2);
            for (int k = 0; k < 3; k++) out_E[3 * (int64_t)i + k] = e[k];
            if (pf.Ad) {
                const double ia = pre[3];
                for (int k = 0; k < 3; k++) {
                    const double dk = pre[4 + k];
                    const double v = ia > 0.0 ? dk * ia - e[k] : 0.0;
                    pf.Ad[3 * (int64_t)i + k] = v;
                    dot += dk * v;
                }
            }
        }
        __syncthreads();
    }
    pdl_launch_dependents();
    if (!pf.Ad) return;
    // leaf partial, then the last block adds all leaves in order
    for (int o = 16; o > 0; o >>= 1) dot += __shfl_down_sync(0xffffffffu, dot, o);
    if ((tid & 31) == 0) red[tid >> 5] = dot;
    __syncthreads();
    if (tid == 0) {
        double v = 0.0;
        for (int w = 0; w < kL2PThreads / 32; w++) v += red[w];
        pf.partial[b] = v;
        __threadfence();
        last = atomicAdd(pf.ticket, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // four loads in flight per thread
    double v = 0.0;
    int k = tid;
    for (; k + 3 * kL2PThreads < nleaf; k += 4 * kL2PThreads) {
        const double a = __ldcg(pf.partial + k), b2 = __ldcg(pf.partial + k + kL2PThreads);
        const double c2 = __ldcg(pf.partial + k + 2 * kL2PThreads), d2 = __ldcg(pf.partial + k + 3 * kL2PThreads);
        v += a;
        v += b2;
        v += c2;
        v += d2;
    }
    for (; k < nleaf; k += kL2PThreads) v += __ldcg(pf.partial + k);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < kL2PThreads / 32; w++) t += red[w];
        pf.scal[S_DAD] = t;
        *pf.ticket = 0;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static LevelPtrs level_ptrs(polfmm_ctx* c) {
    LevelPtrs lp{};
    for (int l = 0; l <= c->depth; l++) {
        lp.key[l] = c->lv[l].key;
        lp.map[l] = c->lv[l].map;
        lp.by_class[l] = c->lv[l].by_class;
        lp.M[l] = c->lv[l].M;
        lp.Lp[l] = c->lv[l].Lp;
        lp.cap[l] = c->lv[l].cap;
    }
    return lp;
}

size_t m2l_simt_smem(int ncoef, size_t rsize) {
    return rsize * (2 * 32 * (size_t)(ncoef + 1) + ncoef) + 32 * sizeof(int) + 16;
}

int m2l_setup(polfmm_ctx* c) {
    // tiles of same-level, same-class boxes
    std::vector<M2LTile> t;
    for (int l = 2; l <= c->depth; l++)
        for (int k = 0; k < 8; k++) {
            int cnt = c->lv[l].class_count[k], st = c->lv[l].class_start[k];
            for (int f = 0; f < cnt; f += kM2LTileBoxes)
                t.push_back(M2LTile{l, k, st + f, std::min(kM2LTileBoxes, cnt - f)});
        }
    c->ntiles = (int)t.size();
    if (c->ntiles > c->ntiles_cap) {
        if (c->tiles) cudaFree(c->tiles);
        c->tiles = nullptr;
        c->ntiles_cap = std::max(c->ntiles, 64);
        if (dev_alloc(reinterpret_cast<void**>(&c->tiles), sizeof(M2LTile) * c->ntiles_cap) != cudaSuccess)
            return POLFMM_ERR_OUT_OF_MEMORY;
    }
    if (c->ntiles)
        if (cudaMemcpyAsync(c->tiles, t.data(), sizeof(M2LTile) * c->ntiles, cudaMemcpyHostToDevice, c->stream) !=
            cudaSuccess)
            return POLFMM_ERR_CUDA;
    // split the 189 offsets over enough blocks to cover the SMs twice
    int want = c->ntiles > 0 ? (2 * c->num_sms + c->ntiles - 1) / c->ntiles : 1;
    c->m2l_chunks = std::max(1, std::min(want, c->mixed ? 7 : 7));
    return POLFMM_OK;
}

static DownPtrs down_ptrs(polfmm_ctx* c) {
    DownPtrs dp{};
    for (int l = 0; l <= c->depth; l++) {
        dp.Lp[l] = c->lv[l].Lp;
        dp.map[l] = c->lv[l].map;
        dp.key[l] = c->lv[l].key;
        dp.cap[l] = c->lv[l].cap;
    }
    dp.depth = c->depth;
    dp.nchunk = c->m2l_chunks;
    dp.p = c->p;
    return dp;
}

template <typename R>
static void launch_leaf(polfmm_ctx* c, int mode, const double* mu_sorted, double* phi, double* E, double* G,
                        bool mu_packed, cudaStream_t st, int far) {
    Level& L = c->lv[c->depth];
    const R h = R(c->side / (double)(1 << c->depth));
    const Tables& T = c->tab;
    Q4<R>* A = reinterpret_cast<Q4<R>*>(c->srcA);
    Q4<R>* B = reinterpret_cast<Q4<R>*>(c->srcB);
    if (mode == LEAF_DIPOLE_E && sizeof(R) == 4 && !far) {
        // FP32 dipole near field from the pair records
        if (!mu_packed) {
            LaunchScope ls(c, F_P2M);
            near_pack_mu_kernel<<<grid_for(c->n, 256), 256, 0, st>>>(c->n, mu_sorted, c->near_slot, c->near_pairs);
        }
        LaunchScope ls(c, F_LEAF_DIPOLE);
        // one block per item; at most two items per leaf item (their count is on the device)
        const int grid = 2 * c->leaf_items_grid;
        near_dipole_f32_kernel<<<grid, kNearThreads, near_dipole_smem_bytes(), st>>>(
            c->near_items, c->near_nitems, reinterpret_cast<const float4*>(c->near_pairs),
            reinterpret_cast<const Q4<float>*>(c->srcA), float(h), E);
        return;
    }
    if (mode != LEAF_CHARGE_PHI_E && !mu_packed) {
        LaunchScope ls(c, F_P2M);
        pack_dipoles_kernel<R><<<grid_for(c->n, 256), 256, 0, st>>>(c->n, mu_sorted, B);
    }
    LaunchScope ls(c, mode == LEAF_DIPOLE_E ? F_LEAF_DIPOLE : (mode == LEAF_CHARGE_PHI_E ? F_LEAF_STATIC : F_LEAF_FULL));
    const DownPtrs dp = down_ptrs(c);
#define LEAF_ARGS                                                                                                \
    c->leaf_items, c->leaf_nitems, L.key, c->lstart, c->lcount, L.map, c->depth, A, B, dp, c->ld, c->ncoef, c->p, T.mi, \
        T.inv_fact, T.up1, T.up2, pick<R>(T.w4, T.w4f), h, phi, E, G, c->err, far
    const int grid = c->leaf_items_grid;
    const int dsm = far ? c->depth : 0;
    if (mode == LEAF_DIPOLE_E)
        leaf_kernel<R, LEAF_DIPOLE_E>
            <<<grid, kLeafThreads, leaf_smem_bytes<R, LEAF_DIPOLE_E>(c->ncoef, dsm), st>>>(LEAF_ARGS);
    else if (mode == LEAF_CHARGE_PHI_E)
        leaf_kernel<R, LEAF_CHARGE_PHI_E>
            <<<grid, kLeafThreads, leaf_smem_bytes<R, LEAF_CHARGE_PHI_E>(c->ncoef, dsm), st>>>(LEAF_ARGS);
    else
        leaf_kernel<R, LEAF_FULL><<<grid, kLeafThreads, leaf_smem_bytes<R, LEAF_FULL>(c->ncoef, dsm), st>>>(LEAF_ARGS);
#undef LEAF_ARGS
}

// positions + charges of the sorted sites, packed once per tree
void pack_positions(polfmm_ctx* c) {
    LaunchScope ls(c, F_TREE);
    if (c->mixed)
        pack_positions_kernel<float><<<grid_for(c->n, 256), 256, 0, c->stream>>>(
            c->n, (const float*)c->ploc, c->q_s, (Q4<float>*)c->srcA);
    else
        pack_positions_kernel<double><<<grid_for(c->n, 256), 256, 0, c->stream>>>(
            c->n, (const double*)c->ploc, c->q_s, (Q4<double>*)c->srcA);
}

size_t source_record_bytes(bool mixed) { return mixed ? sizeof(Q4<float>) : sizeof(Q4<double>); }

void m2l_tensor_launch(polfmm_ctx* c);  // m2l_tc.cu
bool m2l_tensor_enabled(polfmm_ctx* c);

static UpPtrs up_ptrs(polfmm_ctx* c) {
    UpPtrs up{};
    for (int l = 0; l <= c->depth; l++) {
        up.M[l] = c->lv[l].M;
        up.parent[l] = c->lv[l].parent;
        up.child0[l] = c->lv[l].child0;
        up.nchild[l] = c->lv[l].nchild;
        up.key[l] = c->lv[l].key;
        up.arrive[l] = c->lv[l].arrive;
        up.Msh[l] = c->lv[l].Msh;
    }
    return up;
}

template <typename R>
static bool pass_impl(polfmm_ctx* c, int mode, bool use_q, const double* mu_sorted, double* phi, double* E,
                      double* G, bool mu_packed, bool pcg) {
    const int d = c->depth;
    const Tables& T = c->tab;
    Level& Lf = c->lv[d];
    // solver passes: the near-field pair sums run on a second stream while the
    // far-field chain (upward pass, M2L) runs here; the far field is added after
    // the join.  Profiling keeps the same kernels on one stream.
    const bool split = mode == LEAF_DIPOLE_E && d >= 2;
    const bool overlap = split && c->side_stream && !c->opt.profile;
    if (split) {
        if (overlap) {
            cudaEventRecord(c->ev_fork, c->stream);
            cudaStreamWaitEvent(c->side_stream, c->ev_fork, 0);
        }
        launch_leaf<R>(c, mode, mu_sorted, phi, E, G, mu_packed, overlap ? c->side_stream : c->stream, 0);
        // excluded pairs off the near field, before the far field completes it
        exclusion_correct(c, mode, nullptr, mu_sorted, nullptr, E, nullptr, overlap ? c->side_stream : c->stream);
        thole_field(c, mu_sorted, E, overlap ? c->side_stream : c->stream);
        if (overlap) cudaEventRecord(c->ev_join, c->side_stream);
    }
    if (d >= 2) {
        // P2M and M2M up to level 2 (one launch)
        {
            LaunchScope ls(c, F_P2M);
            R inv_h = R((double)(1 << d) / c->side);
            auto kern = mu_sorted && c->opt.dipole_dl > 0.0 ? upward_kernel<R, true> : upward_kernel<R, false>;
            kern<<<Lf.nbox, kUpThreads, upward_smem_bytes<R>(c->ncoef), c->stream>>>(
                Lf.nbox, d, c->lstart, c->lcount, (const R*)c->ploc, use_q ? c->q_s : nullptr, mu_sorted,
                up_ptrs(c), c->ld, c->ncoef, c->p, T.mi, pick<R>(T.w4, T.w4f), pick<R>(T.rinv, T.rinvf), inv_h,
                c->opt.dipole_dl);
        }
        // M2L, all levels >= 2 in one launch
        if (m2l_ffma_enabled(c)) {
            m2l_ffma_launch(c);
        } else if (m2l_tensor_enabled(c)) {
            m2l_tensor_launch(c);
        } else {
            LaunchScope ls(c, F_M2L);
            dim3 grid(c->ntiles, c->m2l_chunks);
            size_t smem = m2l_simt_smem(c->ncoef, sizeof(R));
            m2l_simt_kernel<R><<<grid, 256, smem, c->stream>>>(
                c->tiles, level_ptrs(c), c->mixed ? (const R*)T.Df : (const R*)T.D, T.class_off, T.add, T.pre,
                T.warp_out_ptr, T.warp_out, c->ncoef, c->ld, c->m2l_chunks);
        }
    }
    // L2L runs inside the leaf kernels below
    if (split) {
        if (overlap) cudaStreamWaitEvent(c->stream, c->ev_join, 0);
        LaunchScope ls(c, F_L2P);
        const R h = R(c->side / (double)(1 << d));
        const size_t smem = l2p_smem_bytes<R>(c->ld, d);
        PcgFuse pf{};
        if (pcg)
            pf = PcgFuse{c->inv_alpha_s, c->d,      c->Ad, c->leaf_partial,
                         c->scal,    c->ticket, c->capturing_loop ? c->loop_cond : 0};
        launch_pdl(!c->opt.no_pdl, l2p_field_add_kernel<R>, dim3(Lf.nbox), dim3(kL2PThreads), smem, c->stream,
                   Lf.nbox, c->lstart, c->lcount, reinterpret_cast<const Q4<R>*>(c->srcA), down_ptrs(c), c->ld,
                   c->ncoef, c->p, T.mi, T.up1, pick<R>(T.w4, T.w4f), pick<R>(T.rinv, T.rinvf), h, E, pf);
        return pcg;
    }
    launch_leaf<R>(c, mode, mu_sorted, phi, E, G, mu_packed, c->stream, d >= 2 ? 1 : 0);
    exclusion_correct(c, mode, use_q ? c->q_s : nullptr, mu_sorted, phi, E, G, c->stream);
    if (mode == LEAF_DIPOLE_E) thole_field(c, mu_sorted, E, c->stream);
    return false;
}

bool fmm_pass(polfmm_ctx* c, int mode, bool use_q, const double* mu_sorted, double* phi, double* E, double* G,
              bool mu_packed, bool pcg) {
    if (c->mixed) return pass_impl<float>(c, mode, use_q, mu_sorted, phi, E, G, mu_packed, pcg);
    return pass_impl<double>(c, mode, use_q, mu_sorted, phi, E, G, mu_packed, pcg);
}

int fmm_ops_init_attributes(polfmm_ctx*) {
    // sized for the largest order so that contexts of different p coexist
    const int nc_max = ncoef_of(kMaxP);
    size_t need_d = m2l_simt_smem(nc_max, sizeof(double));
    size_t need_f = m2l_simt_smem(nc_max, sizeof(float));
    if (cudaFuncSetAttribute(m2l_simt_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need_d) !=
        cudaSuccess)
        return POLFMM_ERR_CUDA;
    if (cudaFuncSetAttribute(m2l_simt_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need_f) !=
        cudaSuccess)
        return POLFMM_ERR_CUDA;
    if (cudaFuncSetAttribute(upward_kernel<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)upward_smem_bytes<double>(nc_max)) != cudaSuccess ||
        cudaFuncSetAttribute(upward_kernel<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)upward_smem_bytes<double>(nc_max)) != cudaSuccess ||
        cudaFuncSetAttribute(upward_kernel<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)upward_smem_bytes<float>(nc_max)) != cudaSuccess ||
        cudaFuncSetAttribute(upward_kernel<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)upward_smem_bytes<float>(nc_max)) != cudaSuccess)
        return POLFMM_ERR_CUDA;
    if (cudaFuncSetAttribute(l2p_field_add_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)l2p_smem_bytes<double>((nc_max + 3) & ~3, kMaxDepth)) != cudaSuccess ||
        cudaFuncSetAttribute(l2p_field_add_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)l2p_smem_bytes<float>((nc_max + 3) & ~3, kMaxDepth)) != cudaSuccess)
        return POLFMM_ERR_CUDA;
#define LEAF_ATTR(R, M)                                                                                 \
    if (cudaFuncSetAttribute(leaf_kernel<R, M>, cudaFuncAttributeMaxDynamicSharedMemorySize,            \
                             (int)leaf_smem_bytes<R, M>(nc_max, kMaxDepth)) != cudaSuccess)                        \
        return POLFMM_ERR_CUDA;
    LEAF_ATTR(float, LEAF_DIPOLE_E)
    LEAF_ATTR(float, LEAF_CHARGE_PHI_E)
    LEAF_ATTR(float, LEAF_FULL)
    LEAF_ATTR(double, LEAF_DIPOLE_E)
    LEAF_ATTR(double, LEAF_CHARGE_PHI_E)
    LEAF_ATTR(double, LEAF_FULL)
#undef LEAF_ATTR
    if (cudaFuncSetAttribute(near_dipole_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)near_dipole_smem_bytes()) != cudaSuccess)
        return POLFMM_ERR_CUDA;
    return POLFMM_OK;
}

}  // namespace polfmm
