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
// P2M
// ---------------------------------------------------------------------------
constexpr int kP2MChunk = 64;
constexpr int kP2MThreads = 128;

template <typename R>
__global__ void __launch_bounds__(kP2MThreads) p2m_kernel(
    int nleaf, const int* __restrict__ lstart, const int* __restrict__ lcount, const R* __restrict__ ploc,
    const double* __restrict__ q, const double* __restrict__ mu, R* __restrict__ M, int ld, int ncoef, int p,
    const int* __restrict__ mi, R inv_h) {
    const int b = blockIdx.x;
    if (b >= nleaf) return;
    const int s0 = lstart[b], cnt = lcount[b];
    // P[site][axis][k + 1] = v^k / k!, v = -(x - z) / h, P[.][.][0] = 0
    __shared__ R P[kP2MChunk][3][kMaxP + 2];
    __shared__ R sq[kP2MChunk];
    __shared__ R sm[kP2MChunk][3];
    constexpr int CPT = (286 + kP2MThreads - 1) / kP2MThreads;  // coefficients per thread (p <= 10)
    R acc[CPT];
#pragma unroll
    for (int k = 0; k < CPT; k++) acc[k] = R(0);
    for (int k0 = 0; k0 < cnt; k0 += kP2MChunk) {
        int m = min(kP2MChunk, cnt - k0);
        __syncthreads();
        if (threadIdx.x < m) {
            int i = s0 + k0 + threadIdx.x;
            for (int a = 0; a < 3; a++) {
                R v = -ploc[3 * i + a] * inv_h;
                R t = R(1);
                P[threadIdx.x][a][0] = R(0);
                P[threadIdx.x][a][1] = t;
                for (int k = 1; k <= p; k++) {
                    t = t * v / R(k);
                    P[threadIdx.x][a][k + 1] = t;
                }
                sm[threadIdx.x][a] = mu ? R(mu[3 * i + a]) * inv_h : R(0);
            }
            sq[threadIdx.x] = q ? R(q[i]) : R(0);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < CPT; k++) {
            int cidx = threadIdx.x + k * kP2MThreads;
            if (cidx >= ncoef) continue;
            int nx, ny, nz;
            decode_mi(mi[cidx], nx, ny, nz);
            R a = acc[k];
            for (int s = 0; s < m; s++) {
                R px = P[s][0][nx + 1], py = P[s][1][ny + 1], pz = P[s][2][nz + 1];
                // m_n = q v^n/n! - sum_d (mu_d/h) v^(n-e_d)/(n-e_d)!
                a += sq[s] * px * py * pz;
                a -= sm[s][0] * P[s][0][nx] * py * pz + sm[s][1] * px * P[s][1][ny] * pz +
                     sm[s][2] * px * py * P[s][2][nz];
            }
            acc[k] = a;
        }
    }
#pragma unroll
    for (int k = 0; k < CPT; k++) {
        int cidx = threadIdx.x + k * kP2MThreads;
        if (cidx < ncoef) M[(int64_t)b * ld + cidx] = acc[k];
    }
}

// ---------------------------------------------------------------------------
// M2M: m^P_n = sum_children sum_{k <= n} (-1)^(b.k) 2^-(|n|+|k|)/k! m^C_{n-k}
// (child centre offset from the parent centre is (b - 1/2) h_P / 2 per axis)
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(128) m2m_kernel(int npar, const int* __restrict__ child0,
                                                  const int* __restrict__ nchild, const int* __restrict__ ckey,
                                                  const R* __restrict__ Mc, R* __restrict__ Mp, int ld, int ncoef,
                                                  const int* __restrict__ ptr, const int* __restrict__ src,
                                                  const int* __restrict__ par, const R* __restrict__ w) {
    extern __shared__ unsigned char smem_raw[];
    R* S = reinterpret_cast<R*>(smem_raw);  // [8][ld]
    __shared__ int oct[8];
    const int b = blockIdx.x;
    if (b >= npar) return;
    const int c0 = child0[b], nc = nchild[b];
    if (threadIdx.x < nc) oct[threadIdx.x] = ckey[c0 + threadIdx.x] & 7;
    for (int idx = threadIdx.x; idx < nc * ncoef; idx += blockDim.x) {
        int j = idx / ncoef, cc = idx - j * ncoef;
        S[j * ld + cc] = Mc[(int64_t)(c0 + j) * ld + cc];
    }
    __syncthreads();
    for (int cc = threadIdx.x; cc < ncoef; cc += blockDim.x) {
        R acc = R(0);
        for (int e = ptr[cc]; e < ptr[cc + 1]; e++) {
            int s = src[e], pb = par[e];
            R ww = w[e];
            for (int j = 0; j < nc; j++) {
                R v = ww * S[j * ld + s];
                acc += (__popc(pb & oct[j]) & 1) ? -v : v;
            }
        }
        Mp[(int64_t)b * ld + cc] = acc;
    }
}

// ---------------------------------------------------------------------------
// L2L: f^C_n = sum_chunks M2L partial + 2^-(|n|+1) sum_k (x/h_P)^k/k! f^P_{n+k},
// x/h_P = +-1/4 per axis (+ where the child bit is 1)
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(128) l2l_kernel(int nbox, int cap, int nchunk, const int* __restrict__ key,
                                                  const int* __restrict__ parent, const R* __restrict__ Lp,
                                                  const R* __restrict__ Lpar, R* __restrict__ L, int ld, int ncoef,
                                                  const int* __restrict__ ptr, const int* __restrict__ src,
                                                  const int* __restrict__ par, const R* __restrict__ w) {
    extern __shared__ unsigned char smem_raw[];
    R* F = reinterpret_cast<R*>(smem_raw);  // parent locals [ld]
    const int b = blockIdx.x;
    if (b >= nbox) return;
    const bool shift = Lpar != nullptr;
    int noct = 0;
    if (shift) {
        int ps = parent[b];
        noct = (~key[b]) & 7;
        for (int cc = threadIdx.x; cc < ncoef; cc += blockDim.x) F[cc] = Lpar[(int64_t)ps * ld + cc];
    }
    __syncthreads();
    for (int cc = threadIdx.x; cc < ncoef; cc += blockDim.x) {
        R acc = R(0);
        for (int k = 0; k < nchunk; k++) acc += Lp[((int64_t)k * cap + b) * ld + cc];
        if (shift) {
            for (int e = ptr[cc]; e < ptr[cc + 1]; e++) {
                R v = w[e] * F[src[e]];
                acc += (__popc(par[e] & noct) & 1) ? -v : v;
            }
        }
        L[(int64_t)b * ld + cc] = acc;
    }
}

// ---------------------------------------------------------------------------
// M2L (SIMT): tiles of up to 32 same-level, same-octant-class target boxes;
// lane = target box, each warp owns a balanced set of output coefficients;
// the offsets of the class are split into `nchunk` ranges over blockIdx.y,
// each writing its own partial output (summed in fixed order by l2l_kernel).
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
// target leaf stages the sources of all 27 neighbour leaves (shifted into the
// target leaf's frame, exact small-integer multiples of the leaf side) into
// shared memory with one barrier pair per CAP sources; thread (t, s) owns
// target t and every slices-th source, and the slices are added in a fixed
// order at the end.  The self pair has r = 0 exactly and is masked.
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
    static constexpr int N = 256;
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

// dynamic shared memory of leaf_kernel<R, MODE>
template <typename R, int MODE>
__host__ __device__ inline size_t leaf_smem_bytes(int ncoef) {
    constexpr int CAP = LeafCap<R>::N;
    size_t b = sizeof(Q4<R>) * CAP;                          // positions + charge
    if (MODE != LEAF_CHARGE_PHI_E) b += sizeof(Q4<R>) * CAP;  // dipoles
    if (MODE == LEAF_CHARGE_PHI_E) b += sizeof(int) * CAP;    // source index (coincidence check)
    b += sizeof(R) * 2 * (size_t)ncoef;                      // locals, 1/n!
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
    int nleaf, const int* __restrict__ lkey, const int* __restrict__ lstart, const int* __restrict__ lcount,
    const int* __restrict__ lmap, const int* __restrict__ order, int depth, const Q4<R>* __restrict__ srcA,
    const Q4<R>* __restrict__ srcB,
    const R* __restrict__ Lf, int ld, int ncoef, const int* __restrict__ mi, const double* __restrict__ inv_fact,
    const int* __restrict__ up1, const int* __restrict__ up2, R h, double* __restrict__ out_phi,
    double* __restrict__ out_E, double* __restrict__ out_G, int* __restrict__ err, int far) {
    constexpr int NC = LeafOut<MODE>::NC;
    constexpr int CAP = LeafCap<R>::N;
    constexpr bool HAS_PHI = MODE != LEAF_DIPOLE_E;
    constexpr bool HAS_G = MODE == LEAF_FULL;
    constexpr bool SRC_Q = MODE != LEAF_DIPOLE_E;
    constexpr bool SRC_MU = MODE != LEAF_CHARGE_PHI_E;
    constexpr bool CHECK = MODE == LEAF_CHARGE_PHI_E;
    constexpr int IE = HAS_PHI ? 1 : 0;  // component layout: [phi] E(3) [G(6)]
    constexpr int IG = IE + 3;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    Q4<R>* sA = reinterpret_cast<Q4<R>*>(smem_raw);
    Q4<R>* sB = sA + CAP;
    unsigned char* tail = reinterpret_cast<unsigned char*>(SRC_MU ? sB + CAP : sA + CAP);
    int* sidx = reinterpret_cast<int*>(tail);
    if (CHECK) tail += sizeof(int) * CAP;
    R* f = reinterpret_cast<R*>(tail);
    R* ifact = f + ncoef;
    int* cinfo = reinterpret_cast<int*>(ifact + ncoef);  // [ncoef][4]: packed n, n+e_x, n+e_y, n+e_z
    int* cup2 = cinfo + 4 * ncoef;                       // [ncoef][6] (FULL only)
    __shared__ int nb_start[27];
    __shared__ int nb_pre[28];
    __shared__ R nb_shift[27][3];
    __shared__ R part[NC][kLeafThreads];

    if ((int)blockIdx.x >= nleaf) return;
    const int b = order[blockIdx.x];
    const int s0 = lstart[b], cnt = lcount[b];
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
        f[cc] = far ? Lf[(int64_t)b * ld + cc] : R(0);
        ifact[cc] = R(inv_fact[cc]);
        cinfo[4 * cc] = mi[cc];
        cinfo[4 * cc + 1] = up1[3 * cc];
        cinfo[4 * cc + 2] = up1[3 * cc + 1];
        cinfo[4 * cc + 3] = up1[3 * cc + 2];
        if (HAS_G)
            for (int k = 0; k < 6; k++) cup2[6 * cc + k] = up2[6 * cc + k];
    }
    __syncthreads();
    const int total = nb_pre[27];
    const R inv_h = R(1) / h;

    for (int tg = 0; tg < cnt; tg += kLeafThreads) {
        const int nt = min(kLeafThreads, cnt - tg);
        const int slices = kLeafThreads / nt;
        const int t = tid % nt, s = tid / nt;
        const bool active = s < slices;
        const int i = s0 + tg + t;
        R acc[NC];
#pragma unroll
        for (int k = 0; k < NC; k++) acc[k] = R(0);
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
                sA[idx] = a;
                if (SRC_MU) sB[idx] = srcB[j];
                if (CHECK) sidx[idx] = j;
            }
            __syncthreads();
            if (!active) continue;
#pragma unroll 4
            for (int jj = s; jj < m; jj += slices) {
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
                    if (HAS_PHI) acc[0] += qj * ri;
                    acc[IE + 0] += qr3 * rx;
                    acc[IE + 1] += qr3 * ry;
                    acc[IE + 2] += qr3 * rz;
                    if (HAS_G) {
                        const R t5 = R(3) * qr3 * ri2;
                        acc[IG + 0] += qr3 - t5 * rx * rx;
                        acc[IG + 1] -= t5 * rx * ry;
                        acc[IG + 2] -= t5 * rx * rz;
                        acc[IG + 3] += qr3 - t5 * ry * ry;
                        acc[IG + 4] -= t5 * ry * rz;
                        acc[IG + 5] += qr3 - t5 * rz * rz;
                    }
                }
                if (SRC_MU) {
                    const Q4<R> mv = sB[jj];
                    const R mr = mv.x * rx + mv.y * ry + mv.z * rz;
                    const R ri5 = ri3 * ri2;
                    const R a3 = R(3) * mr * ri5;
                    if (HAS_PHI) acc[0] += mr * ri3;
                    acc[IE + 0] += a3 * rx - mv.x * ri3;
                    acc[IE + 1] += a3 * ry - mv.y * ri3;
                    acc[IE + 2] += a3 * rz - mv.z * ri3;
                    if (HAS_G) {
                        // G_de = 3 (mu_d r_e + mu_e r_d + mr delta_de) / r^5 - 15 mr r_d r_e / r^7
                        const R t5 = R(3) * ri5;
                        const R t7 = R(5) * a3 * ri2;
                        acc[IG + 0] += t5 * (R(2) * mv.x * rx + mr) - t7 * rx * rx;
                        acc[IG + 1] += t5 * (mv.x * ry + mv.y * rx) - t7 * rx * ry;
                        acc[IG + 2] += t5 * (mv.x * rz + mv.z * rx) - t7 * rx * rz;
                        acc[IG + 3] += t5 * (R(2) * mv.y * ry + mr) - t7 * ry * ry;
                        acc[IG + 4] += t5 * (mv.y * rz + mv.z * ry) - t7 * ry * rz;
                        acc[IG + 5] += t5 * (R(2) * mv.z * rz + mr) - t7 * rz * rz;
                    }
                }
            }
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

// far field of the solver pass, added to the near field already in out_E:
// E += -(1/h^2) sum_{|n| <= p-1} u^n/n! f_{n+e_d}, u = (x - z) / h (Sec. II.B)
template <typename R>
__global__ void __launch_bounds__(128) l2p_field_add_kernel(int nleaf, const int* __restrict__ lstart,
                                                            const int* __restrict__ lcount,
                                                            const Q4<R>* __restrict__ srcA, const R* __restrict__ Lf,
                                                            int ld, int ncoef, const int* __restrict__ mi,
                                                            const double* __restrict__ inv_fact,
                                                            const int* __restrict__ up1, R h,
                                                            double* __restrict__ out_E) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* f = reinterpret_cast<R*>(smem_raw);
    R* ifact = f + ncoef;
    int* cinfo = reinterpret_cast<int*>(ifact + ncoef);  // [ncoef][4]
    const int b = blockIdx.x;
    if (b >= nleaf) return;
    for (int cc = threadIdx.x; cc < ncoef; cc += blockDim.x) {
        f[cc] = Lf[(int64_t)b * ld + cc];
        ifact[cc] = R(inv_fact[cc]);
        cinfo[4 * cc] = mi[cc];
        cinfo[4 * cc + 1] = up1[3 * cc];
        cinfo[4 * cc + 2] = up1[3 * cc + 1];
        cinfo[4 * cc + 3] = up1[3 * cc + 2];
    }
    __syncthreads();
    const int s0 = lstart[b], cnt = lcount[b];
    const R inv_h = R(1) / h;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        const int i = s0 + t;
        const Q4<R> me = srcA[i];
        const R ux = me.x * inv_h, uy = me.y * inv_h, uz = me.z * inv_h;
        R d0 = R(0), d1 = R(0), d2 = R(0);
        for (int cc = 0; cc < ncoef; cc++) {
            const int u0 = cinfo[4 * cc + 1];
            if (u0 < 0) continue;
            const int pk = cinfo[4 * cc];
            R wgt = ifact[cc];
            for (int k = pk & 0xff; k > 0; k--) wgt *= ux;
            for (int k = (pk >> 8) & 0xff; k > 0; k--) wgt *= uy;
            for (int k = (pk >> 16) & 0xff; k > 0; k--) wgt *= uz;
            d0 += wgt * f[u0];
            d1 += wgt * f[cinfo[4 * cc + 2]];
            d2 += wgt * f[cinfo[4 * cc + 3]];
        }
        const R s2 = -inv_h * inv_h;
        out_E[3 * (int64_t)i] += (double)(d0 * s2);
        out_E[3 * (int64_t)i + 1] += (double)(d1 * s2);
        out_E[3 * (int64_t)i + 2] += (double)(d2 * s2);
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
        if (cudaMalloc(&c->tiles, sizeof(M2LTile) * c->ntiles_cap) != cudaSuccess) return POLFMM_ERR_OUT_OF_MEMORY;
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

template <typename R>
static void launch_leaf(polfmm_ctx* c, int mode, const double* mu_sorted, double* phi, double* E, double* G,
                        bool mu_packed, cudaStream_t st, int far) {
    Level& L = c->lv[c->depth];
    const R h = R(c->side / (double)(1 << c->depth));
    const Tables& T = c->tab;
    Q4<R>* A = reinterpret_cast<Q4<R>*>(c->srcA);
    Q4<R>* B = reinterpret_cast<Q4<R>*>(c->srcB);
    if (mode != LEAF_CHARGE_PHI_E && !mu_packed) {
        LaunchScope ls(c, F_P2M);
        pack_dipoles_kernel<R><<<grid_for(c->n, 256), 256, 0, st>>>(c->n, mu_sorted, B);
    }
    LaunchScope ls(c, mode == LEAF_DIPOLE_E ? F_LEAF_DIPOLE : (mode == LEAF_CHARGE_PHI_E ? F_LEAF_STATIC : F_LEAF_FULL));
#define LEAF_ARGS                                                                                                  \
    L.nbox, L.key, c->lstart, c->lcount, L.map, c->leaf_order, c->depth, A, B, (const R*)L.L, c->ld, c->ncoef,     \
        T.mi, T.inv_fact,                                                                                      \
        T.up1, T.up2, h, phi, E, G, c->err, far
    if (mode == LEAF_DIPOLE_E)
        leaf_kernel<R, LEAF_DIPOLE_E>
            <<<L.nbox, kLeafThreads, leaf_smem_bytes<R, LEAF_DIPOLE_E>(c->ncoef), st>>>(LEAF_ARGS);
    else if (mode == LEAF_CHARGE_PHI_E)
        leaf_kernel<R, LEAF_CHARGE_PHI_E>
            <<<L.nbox, kLeafThreads, leaf_smem_bytes<R, LEAF_CHARGE_PHI_E>(c->ncoef), st>>>(LEAF_ARGS);
    else
        leaf_kernel<R, LEAF_FULL><<<L.nbox, kLeafThreads, leaf_smem_bytes<R, LEAF_FULL>(c->ncoef), st>>>(
            LEAF_ARGS);
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

template <typename R>
static const R* weights(const double* wd, const float* wf);
template <>
const double* weights<double>(const double* wd, const float*) {
    return wd;
}
template <>
const float* weights<float>(const double*, const float* wf) {
    return wf;
}

template <typename R>
static void pass_impl(polfmm_ctx* c, int mode, bool use_q, const double* mu_sorted, double* phi, double* E,
                      double* G, bool mu_packed) {
    const int d = c->depth;
    const Tables& T = c->tab;
    Level& Lf = c->lv[d];
    // solver passes: the near-field pair sums run on a second stream while the
    // far-field chain (P2M .. L2L) runs here; the far field is added after the join
    const bool overlap = mode == LEAF_DIPOLE_E && d >= 2 && c->side_stream && !c->opt.profile;
    if (overlap) {
        cudaEventRecord(c->ev_fork, c->stream);
        cudaStreamWaitEvent(c->side_stream, c->ev_fork, 0);
        launch_leaf<R>(c, mode, mu_sorted, phi, E, G, mu_packed, c->side_stream, 0);
        cudaEventRecord(c->ev_join, c->side_stream);
    }
    // P2M
    {
        LaunchScope ls(c, F_P2M);
        R inv_h = R((double)(1 << d) / c->side);
        p2m_kernel<R><<<Lf.nbox, kP2MThreads, 0, c->stream>>>(Lf.nbox, c->lstart, c->lcount, (const R*)c->ploc,
                                                              use_q ? c->q_s : nullptr, mu_sorted, (R*)Lf.M, c->ld,
                                                              c->ncoef, c->p, T.mi, inv_h);
    }
    if (d >= 2) {
        // M2M up to level 2
        for (int l = d - 1; l >= 2; l--) {
            LaunchScope ls(c, F_M2M);
            Level& P = c->lv[l];
            Level& C = c->lv[l + 1];
            m2m_kernel<R><<<P.nbox, 128, sizeof(R) * 8 * c->ld, c->stream>>>(
                P.nbox, P.child0, P.nchild, C.key, (const R*)C.M, (R*)P.M, c->ld, c->ncoef, T.m2m_ptr, T.m2m_src,
                T.m2m_par, weights<R>(T.m2m_w, T.m2m_wf));
        }
        // M2L
        if (c->ntiles > 0) {
            if (m2l_tensor_enabled(c)) {
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
        // L2L (level 2: partial sums only)
        for (int l = 2; l <= d; l++) {
            LaunchScope ls(c, F_L2L);
            Level& B = c->lv[l];
            const R* Lpar = l >= 3 ? (const R*)c->lv[l - 1].L : nullptr;
            l2l_kernel<R><<<B.nbox, 128, sizeof(R) * c->ld, c->stream>>>(
                B.nbox, B.cap, c->m2l_chunks, B.key, B.parent, (const R*)B.Lp, Lpar, (R*)B.L, c->ld, c->ncoef,
                T.l2l_ptr, T.l2l_src, T.l2l_par, weights<R>(T.l2l_w, T.l2l_wf));
        }
    } else {
        cudaMemsetAsync(Lf.L, 0, sizeof(R) * (size_t)Lf.cap * c->ld, c->stream);
    }
    if (overlap) {
        cudaStreamWaitEvent(c->stream, c->ev_join, 0);
        LaunchScope ls(c, F_LEAF_DIPOLE);
        const R h = R(c->side / (double)(1 << d));
        size_t smem = (2 * sizeof(R) + 4 * sizeof(int)) * (size_t)c->ncoef;
        l2p_field_add_kernel<R><<<Lf.nbox, 128, smem, c->stream>>>(Lf.nbox, c->lstart, c->lcount,
                                                                   reinterpret_cast<const Q4<R>*>(c->srcA),
                                                                   (const R*)Lf.L, c->ld, c->ncoef, T.mi, T.inv_fact,
                                                                   T.up1, h, E);
        return;
    }
    launch_leaf<R>(c, mode, mu_sorted, phi, E, G, mu_packed, c->stream, 1);
}

void fmm_pass(polfmm_ctx* c, int mode, bool use_q, const double* mu_sorted, double* phi, double* E, double* G,
              bool mu_packed) {
    if (c->mixed)
        pass_impl<float>(c, mode, use_q, mu_sorted, phi, E, G, mu_packed);
    else
        pass_impl<double>(c, mode, use_q, mu_sorted, phi, E, G, mu_packed);
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
#define LEAF_ATTR(R, M)                                                                                 \
    if (cudaFuncSetAttribute(leaf_kernel<R, M>, cudaFuncAttributeMaxDynamicSharedMemorySize,            \
                             (int)leaf_smem_bytes<R, M>(nc_max)) != cudaSuccess)                        \
        return POLFMM_ERR_CUDA;
    LEAF_ATTR(float, LEAF_DIPOLE_E)
    LEAF_ATTR(float, LEAF_CHARGE_PHI_E)
    LEAF_ATTR(float, LEAF_FULL)
    LEAF_ATTR(double, LEAF_DIPOLE_E)
    LEAF_ATTR(double, LEAF_CHARGE_PHI_E)
    LEAF_ATTR(double, LEAF_FULL)
#undef LEAF_ATTR
    return POLFMM_OK;
}

}  // namespace polfmm
