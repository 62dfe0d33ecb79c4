// FP32 multipole-to-local translation on the CUDA cores (MIXED, p <= 6).
//
// For a target box A and a source box B = A - o of its interaction list
// (Sec. II.B; o one of the 189 offsets of A's octant class), the partial local
// expansion is
//     L_n(A) += sum_{|m| <= p - |n|} D_{n+m}(o) M_m(B),
// D the Cartesian derivatives of 1/r at the integer offset o (normalised
// coefficients, box side 1), the same contraction as the SIMT and tensor-core
// kernels.  At p <= 6 one box pair is 924 multiply-adds on 84 + 84 values, so a
// thread can hold its target's 84 accumulators and one source row in registers.
//
// Work decomposition.  The boxes of levels >= 2 are listed by octant class and
// cut into groups of 32 (one per lane).  When the tree is built, every group
// gets the list of offsets for which at least one of its 32 sources exists
// (in offset order), with the 32 source rows of each (a row of zeros for an
// empty box).  Per pass a CTA of kFfPairs warp pairs takes one group and one of
// nchunk contiguous ranges of that list; its pairs take every kFfPairs-th
// entry.  The two warps of a pair share a shared-memory stage per entry, filled
// with cp.async one entry ahead of the arithmetic (half the rows each, one
// contiguous row per instruction), and split the outputs by degree: at p = 6
// the first takes |n| <= 2 (10 accumulators, all 84 inputs), the second
// |n| >= 3 (74 accumulators, the 20 inputs of |m| <= 3), 462 FMAs each, so that
// both fit in 128 registers and four warps share each scheduler.  The FMAs run
// in an order fixed at compile time (by n + m, one float4 of D live at a time).
// At the end the pairs' accumulators are added in pair order and the CTA writes
// one partial local per box and chunk; the leaf kernels add the chunks in order.
// Every sum therefore has a fixed order.
#include <algorithm>
#include <utility>
#include <vector>

#include "internal.cuh"

namespace polfmm {

constexpr int kFfPairs = 4;  // warp pairs per CTA; the two warps of a pair share the staged entries
constexpr int kFfThreads = 64 * kFfPairs;
constexpr int kFfRows = 32;  // target boxes per group (one per lane)
constexpr int kFfMaxP = 6;
constexpr int kFfMaxChunks = 16;  // partial locals per box (the leaf kernels add them in order)

// ---------------------------------------------------------------------------
// compile-time schedule of the contraction
// ---------------------------------------------------------------------------
constexpr int ff_ncoef(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

// the library's coefficient order: degree ascending, then x descending, then z ascending
constexpr int ff_index(int x, int y, int z) {
    const int o = x + y + z, a = o - x;
    return o * (o + 1) * (o + 2) / 6 + a * (a + 1) / 2 + z;
}

// number of (n, m) with |n| + |m| <= p: sum over k = n + m of prod_d (k_d + 1)
constexpr int ff_terms(int p) {
    int s = 0;
    for (int o = 0; o <= p; o++)
        for (int x = o; x >= 0; x--)
            for (int z = 0; z <= o - x; z++) s += (x + 1) * (o - x - z + 1) * (z + 1);
    return s;
}

// terms of the outputs of degree s: (s + 1)(s + 2)/2 outputs of ncoef(p - s) terms
constexpr int ff_terms_of_degree(int p, int s) { return (s + 1) * (s + 2) / 2 * ff_ncoef(p - s); }

// the two warps of a pair split the outputs by degree: |n| <= split to the
// first, the rest to the second, with the term counts as equal as they come
constexpr int ff_split(int p) {
    const int tot = ff_terms(p);
    int best = 0, bestd = 1 << 30, run = 0;
    for (int s = 0; s < p; s++) {
        run += ff_terms_of_degree(p, s);
        const int d = 2 * run > tot ? 2 * run - tot : tot - 2 * run;
        if (d < bestd) {
            bestd = d;
            best = s;
        }
    }
    return best;
}

template <int P>
struct FfSplit {
    static constexpr int SA = ff_split(P);
    static constexpr int NA = ff_ncoef(SA);               // outputs of the first warp: 0 .. NA - 1
    static constexpr int NB = ff_ncoef(P) - NA;           // outputs of the second: NA .. ncoef - 1
    static constexpr int MB = ff_ncoef(P - SA - 1);       // inputs the second warp uses (|m| <= P - SA - 1)
};

constexpr int ff_part_terms(int p, int part) {
    int s = 0;
    for (int d = 0; d <= p; d++)
        if ((part == 0) == (d <= ff_split(p))) s += ff_terms_of_degree(p, d);
    return s;
}

// the terms of one part ordered by k = n + m (the D index), so that one float4
// of D is live at a time; n is relative to the part's first output
template <int P, int PART>
struct FfPlan {
    static constexpr int NT = ff_part_terms(P, PART);
    short n[NT] = {};
    short m[NT] = {};
    short k[NT] = {};
    bool load[NT] = {};  // first term of its D group 4 * (k / 4) in this part: load that float4
    constexpr FfPlan() {
        const int sa = ff_split(P), n0 = PART == 0 ? 0 : ff_ncoef(sa);
        int e = 0;
        for (int o = 0; o <= P; o++)
            for (int x = o; x >= 0; x--)
                for (int z = 0; z <= o - x; z++) {
                    const int y = o - x - z, kk = ff_index(x, y, z);
                    for (int nx = 0; nx <= x; nx++)
                        for (int ny = 0; ny <= y; ny++)
                            for (int nz = 0; nz <= z; nz++) {
                                if ((PART == 0) != (nx + ny + nz <= sa)) continue;
                                n[e] = (short)(ff_index(nx, ny, nz) - n0);
                                m[e] = (short)ff_index(x - nx, y - ny, z - nz);
                                k[e] = (short)kk;
                                load[e] = e == 0 || k[e - 1] / 4 != kk / 4;
                                e++;
                            }
                }
    }
};

template <int P, int PART>
inline constexpr FfPlan<P, PART> kFfPlan{};

template <int P>
struct FfDims {
    static constexpr int NC = ff_ncoef(P);
    static constexpr int NCP = (NC + 3) / 4 * 4;                  // = ld: floats per multipole row
    static constexpr int RS = (NCP / 4) % 2 ? NCP : NCP + 4;      // staged row stride: an odd number of
                                                                  // float4, so that lane-own rows are read
                                                                  // without bank conflicts
    static constexpr int STAGE = kFfRows * RS + NCP;              // 32 rows, then the offset's D
};

template <int J>
__device__ __forceinline__ float ff_lane(const float4& v) {
    if constexpr (J == 0) return v.x;
    else if constexpr (J == 1) return v.y;
    else if constexpr (J == 2) return v.z;
    else return v.w;
}

template <int P, int PART, int NL, int NM, int E>
__device__ __forceinline__ void ff_term(float (&L)[NL], const float4 (&M4)[NM], const float4* __restrict__ D4,
                                        float4& d4) {
    constexpr int n = kFfPlan<P, PART>.n[E], m = kFfPlan<P, PART>.m[E], k = kFfPlan<P, PART>.k[E];
    if constexpr (kFfPlan<P, PART>.load[E]) d4 = D4[k / 4];
    L[n] = fmaf(ff_lane<m % 4>(M4[m / 4]), ff_lane<k % 4>(d4), L[n]);
}

template <int P, int PART, int NL, int NM, int... E>
__device__ __forceinline__ void ff_contract(float (&L)[NL], const float4 (&M4)[NM], const float4* __restrict__ D4,
                                            std::integer_sequence<int, E...>) {
    float4 d4 = make_float4(0.f, 0.f, 0.f, 0.f);
    (ff_term<P, PART, NL, NM, E>(L, M4, D4, d4), ...);
}

// ---------------------------------------------------------------------------
// asynchronous 16-byte copies into shared memory, shared-memory loads
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ff_smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ float4 ff_lds4(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr));
    return v;
}

// a 16-byte copy issued only by the lanes with on != 0 (predicated, no branch)
__device__ __forceinline__ void ff_cp16_if(uint32_t dst, const void* src, int on) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %2, 0;\n @p cp.async.ca.shared.global [%0], [%1], 16;\n}\n" ::"r"(dst),
                 "l"(src), "r"(on)
                 : "memory");
}

__device__ __forceinline__ void ff_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void ff_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

struct FfOut {
    float* Lp[kMaxDepth + 1];  // [chunk][cap][ld] partial locals per level
    int cap[kMaxDepth + 1];
};

__device__ __forceinline__ void ff_bar(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(nthreads) : "memory");
}

// one warp of a pair: its entries, its half of the copies, its part of the
// outputs; at the end its accumulators go to red[pair][row][RS]
template <int P, int PART>
__device__ __forceinline__ void ff_warp(const int* __restrict__ eoff, const int* __restrict__ esrc, int e, int e_hi,
                                        float* stage0, const float* __restrict__ Mall, const float* __restrict__ Dpad,
                                        int ld, int pair, int lane, float* red) {
    using Dm = FfDims<P>;
    using Sp = FfSplit<P>;
    constexpr int NL = PART == 0 ? Sp::NA : Sp::NB;            // accumulators
    constexpr int NM = PART == 0 ? Dm::NCP / 4 : (Sp::MB + 3) / 4;  // float4 of the source row used
    constexpr int CH = Dm::NCP / 4;
    float L[NL];
#pragma unroll
    for (int i = 0; i < NL; i++) L[i] = 0.f;

    // this warp's copies of an entry: rows 16 PART .. 16 PART + 15, one row per
    // instruction by the first CH lanes (each instruction reads one contiguous
    // row), and by the first warp the offset's derivative row; lane i holds row
    // i's source index (an empty box's source is the zero row).
    const int copier = lane < CH;
    const float* mbase = Mall + 4 * (copier ? lane : 0);
    auto issue = [&](float* st, int src, int oi) {
        const uint32_t dst = ff_smem_addr(st) + 16u * (uint32_t)(copier ? lane : 0);
#pragma unroll
        for (int i = 16 * PART; i < 16 * PART + 16; i++) {
            const int s = __shfl_sync(0xffffffffu, src, i);
            ff_cp16_if(dst + 4u * (uint32_t)(i * Dm::RS), mbase + (size_t)s * ld, copier);
        }
        if (PART == 0)
            ff_cp16_if(dst + 4u * (uint32_t)(kFfRows * Dm::RS), Dpad + (size_t)(copier ? oi * Dm::NCP + 4 * lane : 0),
                       copier);
    };

    if (e < e_hi) issue(stage0, esrc[(size_t)e * kFfRows + lane], eoff[e]);
    ff_commit();
    int src_b = 0, oi_b = 0;  // the entry after the current one
    if (e + kFfPairs < e_hi) {
        src_b = esrc[(size_t)(e + kFfPairs) * kFfRows + lane];
        oi_b = eoff[e + kFfPairs];
    }
    for (int it = 0; e < e_hi; it++, e += kFfPairs) {
        float* cur = stage0 + (it & 1) * Dm::STAGE;
        float* nxt = stage0 + ((it + 1) & 1) * Dm::STAGE;
        ff_wait<0>();
        // both halves of this entry have landed, and both warps are done with nxt
        ff_bar(1 + pair, 64);
        if (e + kFfPairs < e_hi) issue(nxt, src_b, oi_b);
        ff_commit();
        // the lookups of the entry after next overlap this entry's arithmetic
        if (e + 2 * kFfPairs < e_hi) {
            src_b = esrc[(size_t)(e + 2 * kFfPairs) * kFfRows + lane];
            oi_b = eoff[e + 2 * kFfPairs];
        }
        // the source row, loaded once (volatile: not re-read from shared memory later)
        float4 M4[NM];
        const uint32_t rrow = ff_smem_addr(cur + lane * Dm::RS);
#pragma unroll
        for (int j = 0; j < NM; j++) M4[j] = ff_lds4(rrow + 16u * j);
        ff_contract<P, PART, NL, NM>(L, M4, reinterpret_cast<const float4*>(cur + kFfRows * Dm::RS),
                                     std::make_integer_sequence<int, FfPlan<P, PART>::NT>{});
    }
    ff_wait<0>();
    ff_bar(0, kFfThreads);  // every warp is done with its stages: reuse them for the pair sums
    float* row = red + ((size_t)pair * kFfRows + lane) * Dm::RS + (PART == 0 ? 0 : Sp::NA);
#pragma unroll
    for (int i = 0; i < NL; i++) row[i] = L[i];
}

// groups[g] = (first row, row count, octant class, 0); rows[r] = (level, slot)
template <int P>
__global__ void __launch_bounds__(kFfThreads, 2)
    m2l_ffma_kernel(const int4* __restrict__ groups, const int2* __restrict__ rows, const int* __restrict__ ent_cnt,
                    const int* __restrict__ ent_off, const int* __restrict__ ent_src, const float* __restrict__ Mall,
                    const float* __restrict__ Dpad, FfOut out, int ld, int nchunk) {
    using Dm = FfDims<P>;
    extern __shared__ __align__(16) float ff_smem[];
    __shared__ float* s_out[kFfRows];  // this chunk's partial-local row of each target
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, pair = warp >> 1;
    const int g = blockIdx.x, chunk = blockIdx.y;
    const int4 gr = groups[g];
    if (threadIdx.x < gr.y) {
        const int2 rs = rows[gr.x + threadIdx.x];
        float* base = nullptr;
        int cap = 0;
#pragma unroll
        for (int l = 2; l <= kMaxDepth; l++)
            if (rs.x == l) {
                base = out.Lp[l];
                cap = out.cap[l];
            }
        s_out[threadIdx.x] = base + ((size_t)chunk * cap + rs.y) * ld;
    }
    const int cnt = ent_cnt[g];
    const int e_lo = (int)((long long)chunk * cnt / nchunk), e_hi = (int)((long long)(chunk + 1) * cnt / nchunk);
    const int* eoff = ent_off + (size_t)g * kNumOffsets;
    const int* esrc = ent_src + (size_t)g * kNumOffsets * kFfRows;
    float* stage0 = ff_smem + (size_t)pair * 2 * Dm::STAGE;
    // launched after the upward pass with programmatic serialization: the
    // multipoles are complete from here on
    pdl_wait();
    // warp 2i takes the low-degree outputs of pair i, warp 2i + 1 the others
    if ((warp & 1) == 0)
        ff_warp<P, 0>(eoff, esrc, e_lo + pair, e_hi, stage0, Mall, Dpad, ld, pair, lane, ff_smem);
    else
        ff_warp<P, 1>(eoff, esrc, e_lo + pair, e_hi, stage0, Mall, Dpad, ld, pair, lane, ff_smem);
    ff_bar(0, kFfThreads);
    // the pairs' sums in pair order
    const float* red = ff_smem;
    for (int idx = threadIdx.x; idx < gr.y * Dm::NC; idx += kFfThreads) {
        const int r = idx / Dm::NC, nn = idx - r * Dm::NC;
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < kFfPairs; w++) s += red[((size_t)w * kFfRows + r) * Dm::RS + nn];
        s_out[r][nn] = s;
    }
    pdl_launch_dependents();
}

// ---------------------------------------------------------------------------
// per-tree tables
// ---------------------------------------------------------------------------
struct FfTree {
    const int* key[kMaxDepth + 1];
    const int* map[kMaxDepth + 1];
    int row0[kMaxDepth + 1];  // first row of level l in the all-level multipole array
    int zero_row;             // a row of zeros in that array: the source of an empty box
};

struct FfRowArgs {
    int off[8], start[8];
};

// rows of one level, grouped by octant class after those of the coarser levels
__global__ void ff_rows_kernel(int nbox, int level, const int* __restrict__ by_class, const int* __restrict__ key,
                               FfRowArgs ra, int2* __restrict__ rows) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nbox) return;
    const int slot = by_class[i];
    const int c = key[slot] & 7;
    rows[ra.off[c] + (i - ra.start[c])] = make_int2(level, slot);
}

// one block per group: the offsets with at least one source, in offset order,
// and per such entry the 32 source rows (the zero row where there is no box)
constexpr int kFfListThreads = 1024;  // 32 warps share a group's 189 offsets

__global__ void __launch_bounds__(kFfListThreads) ff_lists_kernel(const int4* __restrict__ groups, const int2* __restrict__ rows,
                                                       FfTree tp, const int* __restrict__ class_off,
                                                       int* __restrict__ ent_off, int* __restrict__ ent_src,
                                                       int* __restrict__ ent_cnt) {
    __shared__ int s_flag[kNumOffsets];
    __shared__ int s_pos[kNumOffsets];
    const int g = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const int4 gr = groups[g];
    const bool has = lane < gr.y;
    int level = 0, bx = 0, by = 0, bz = 0, nside = 0;
    if (has) {
        const int2 r = rows[gr.x + lane];
        level = r.x;
        const uint32_t k = (uint32_t)tp.key[level][r.y];
        bx = (int)compact3(k);
        by = (int)compact3(k >> 1);
        bz = (int)compact3(k >> 2);
        nside = 1 << level;
    }
    auto lookup = [&](int t, int& oi) {
        const int o = class_off[gr.z * kNumOffsets + t];
        const int ox = (o & 15) - 3, oy = ((o >> 4) & 15) - 3, oz = ((o >> 8) & 15) - 3;
        oi = (ox + 3) + 7 * ((oy + 3) + 7 * (oz + 3));
        const int ax = bx - ox, ay = by - oy, az = bz - oz;
        int s = -1;
        if (has && ax >= 0 && ay >= 0 && az >= 0 && ax < nside && ay < nside && az < nside) {
            const int slot = tp.map[level][morton3(ax, ay, az)];
            if (slot >= 0) s = tp.row0[level] + slot;
        }
        return s;
    };
    for (int t = warp; t < kNumOffsets; t += nwarp) {
        int oi;
        const int s = lookup(t, oi);
        const unsigned b = __ballot_sync(0xffffffffu, s >= 0);
        if (lane == 0) s_flag[t] = b != 0u;
    }
    __syncthreads();
    if (warp == 0) {
        // exclusive scan of the flags: lane owns offsets 6 lane .. 6 lane + 5
        constexpr int per = (kNumOffsets + 31) / 32;
        int v[per], tot = 0;
#pragma unroll
        for (int j = 0; j < per; j++) {
            const int t = per * lane + j;
            v[j] = t < kNumOffsets ? s_flag[t] : 0;
            tot += v[j];
        }
        int incl = tot;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += u;
        }
        int run = incl - tot;
#pragma unroll
        for (int j = 0; j < per; j++) {
            const int t = per * lane + j;
            if (t < kNumOffsets) s_pos[t] = run;
            run += v[j];
        }
        if (lane == 31) ent_cnt[g] = incl;
    }
    __syncthreads();
    for (int t = warp; t < kNumOffsets; t += nwarp) {
        if (!s_flag[t]) continue;
        int oi;
        const int s = lookup(t, oi);
        const size_t e = (size_t)g * kNumOffsets + s_pos[t];
        ent_src[e * kFfRows + lane] = s >= 0 ? s : tp.zero_row;
        if (lane == 0) ent_off[e] = oi;
    }
}

// derivative rows padded to NCP floats (16-byte aligned rows for cp.async)
__global__ void ff_pad_kernel(const float* __restrict__ Df, int nc, int ncp, float* __restrict__ Dpad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 343 * ncp) return;
    const int oi = i / ncp, k = i - oi * ncp;
    Dpad[i] = k < nc ? Df[(size_t)oi * nc + k] : 0.f;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct FfState {
    float* Dpad = nullptr;
    int2* rows = nullptr;
    size_t rows_cap = 0;
    int4* groups = nullptr;
    int* ent_off = nullptr;
    int* ent_src = nullptr;
    int* ent_cnt = nullptr;
    int groups_cap = 0;
    int ngroups = 0;
    size_t smem = 0;
    bool ready = false;
};

static FfState* ff_state(polfmm_ctx* c) { return reinterpret_cast<FfState*>(c->ff); }

bool m2l_ffma_wanted(const polfmm_ctx* c) {
    return c->mixed && c->p >= 1 && c->p <= kFfMaxP && c->depth >= 2 &&
           (c->opt.m2l_impl == POLFMM_M2L_AUTO || c->opt.m2l_impl == POLFMM_M2L_FFMA);
}

bool m2l_ffma_enabled(polfmm_ctx* c) {
    FfState* S = ff_state(c);
    return m2l_ffma_wanted(c) && S && S->ready && S->ngroups > 0;
}

template <int P>
static size_t ff_smem_bytes() {
    return sizeof(float) * (size_t)kFfPairs * 2 * FfDims<P>::STAGE;
}

template <int P>
static cudaError_t ff_set_attr(size_t& smem) {
    smem = ff_smem_bytes<P>();
    return cudaFuncSetAttribute(m2l_ffma_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int m2l_ffma_prepare(polfmm_ctx* c) {
    if (!m2l_ffma_wanted(c)) return POLFMM_OK;
    FfState* S = ff_state(c);
    if (!S) {
        S = new FfState();
        c->ff = S;
        const int nc = c->ncoef, ncp = c->ld;
        if (ncp != (nc + 3) / 4 * 4) return POLFMM_ERR_INVALID_ARG;
        if (dev_alloc(reinterpret_cast<void**>(&S->Dpad), sizeof(float) * 343 * (size_t)ncp) != cudaSuccess)
            return POLFMM_ERR_OUT_OF_MEMORY;
        {
            LaunchScope ls(c, F_TREE);
            ff_pad_kernel<<<grid_for(343 * ncp, 256), 256, 0, c->stream>>>(c->tab.Df, nc, ncp, S->Dpad);
        }
        cudaError_t e = cudaSuccess;
        switch (c->p) {
            case 1: e = ff_set_attr<1>(S->smem); break;
            case 2: e = ff_set_attr<2>(S->smem); break;
            case 3: e = ff_set_attr<3>(S->smem); break;
            case 4: e = ff_set_attr<4>(S->smem); break;
            case 5: e = ff_set_attr<5>(S->smem); break;
            default: e = ff_set_attr<6>(S->smem); break;
        }
        if (e != cudaSuccess) return cuda_fail(e, "FP32 M2L shared-memory attribute");
        S->ready = true;
    }
    // rows of all levels >= 2 grouped by octant class, coarse levels first
    int total[8] = {0};
    size_t nrows = 0;
    for (int l = 2; l <= c->depth; l++)
        for (int k = 0; k < 8; k++) total[k] += c->lv[l].class_count[k];
    int cls_first[8];
    for (int k = 0; k < 8; k++) {
        cls_first[k] = (int)nrows;
        nrows += total[k];
    }
    if (nrows > S->rows_cap) {
        if (S->rows) cudaFree(S->rows);
        S->rows = nullptr;
        S->rows_cap = std::max<size_t>(nrows, 64);
        if (dev_alloc(reinterpret_cast<void**>(&S->rows), sizeof(int2) * S->rows_cap) != cudaSuccess)
            return POLFMM_ERR_OUT_OF_MEMORY;
    }
    int fill[8];
    for (int k = 0; k < 8; k++) fill[k] = cls_first[k];
    for (int l = 2; l <= c->depth; l++) {
        Level& B = c->lv[l];
        FfRowArgs ra;
        for (int k = 0; k < 8; k++) {
            ra.off[k] = fill[k];
            ra.start[k] = B.class_start[k];
            fill[k] += B.class_count[k];
        }
        if (B.nbox > 0) {
            LaunchScope ls(c, F_TREE);
            ff_rows_kernel<<<grid_for(B.nbox, 256), 256, 0, c->stream>>>(B.nbox, l, B.by_class, B.key, ra, S->rows);
        }
    }
    std::vector<int4> gl;
    for (int k = 0; k < 8; k++)
        for (int f = 0; f < total[k]; f += kFfRows)
            gl.push_back(make_int4(cls_first[k] + f, std::min(kFfRows, total[k] - f), k, 0));
    S->ngroups = (int)gl.size();
    if (S->ngroups == 0) return POLFMM_OK;
    if (S->ngroups > S->groups_cap) {
        for (void* p : {(void*)S->groups, (void*)S->ent_off, (void*)S->ent_src, (void*)S->ent_cnt})
            if (p) cudaFree(p);
        S->groups = nullptr;
        S->ent_off = S->ent_src = S->ent_cnt = nullptr;
        S->groups_cap = std::max(S->ngroups, 16);
        const size_t G = (size_t)S->groups_cap;
        if (dev_alloc(reinterpret_cast<void**>(&S->groups), sizeof(int4) * G) != cudaSuccess ||
            dev_alloc(reinterpret_cast<void**>(&S->ent_off), sizeof(int) * G * kNumOffsets) != cudaSuccess ||
            dev_alloc(reinterpret_cast<void**>(&S->ent_src), sizeof(int) * G * kNumOffsets * kFfRows) != cudaSuccess ||
            dev_alloc(reinterpret_cast<void**>(&S->ent_cnt), sizeof(int) * G) != cudaSuccess)
            return POLFMM_ERR_OUT_OF_MEMORY;
    }
    if (cudaMemcpyAsync(S->groups, gl.data(), sizeof(int4) * gl.size(), cudaMemcpyHostToDevice, c->stream) !=
        cudaSuccess)
        return POLFMM_ERR_CUDA;
    FfTree tp{};
    tp.zero_row = (int)c->mrow_zero;
    if (cudaMemsetAsync(static_cast<float*>(c->Mall) + (size_t)c->mrow_zero * c->ld, 0, sizeof(float) * c->ld,
                        c->stream) != cudaSuccess)
        return POLFMM_ERR_CUDA;
    for (int l = 2; l <= c->depth; l++) {
        tp.key[l] = c->lv[l].key;
        tp.map[l] = c->lv[l].map;
        tp.row0[l] = (int)c->mrow0[l];
    }
    {
        LaunchScope ls(c, F_TREE);
        ff_lists_kernel<<<S->ngroups, kFfListThreads, 0, c->stream>>>(S->groups, S->rows, tp, c->tab.class_off, S->ent_off,
                                                           S->ent_src, S->ent_cnt);
    }
    // chunks of each group's list so that the CTAs (two per SM) fill the SMs once
    const int slots = 2 * c->num_sms;
    c->m2l_chunks = std::max(1, std::min(kFfMaxChunks, slots / S->ngroups));
    return POLFMM_OK;
}

template <int P>
static void ff_launch(polfmm_ctx* c, FfState* S, const FfOut& out) {
    launch_pdl(!c->opt.no_pdl, m2l_ffma_kernel<P>, dim3(S->ngroups, c->m2l_chunks), dim3(kFfThreads), S->smem,
               c->stream, S->groups, S->rows, S->ent_cnt, S->ent_off, S->ent_src, (const float*)c->Mall, S->Dpad,
               out, c->ld, c->m2l_chunks);
}

void m2l_ffma_launch(polfmm_ctx* c) {
    FfState* S = ff_state(c);
    FfOut out{};
    for (int l = 2; l <= c->depth; l++) {
        out.Lp[l] = (float*)c->lv[l].Lp;
        out.cap[l] = c->lv[l].cap;
    }
    LaunchScope ls(c, F_M2L);
    switch (c->p) {
        case 1: ff_launch<1>(c, S, out); break;
        case 2: ff_launch<2>(c, S, out); break;
        case 3: ff_launch<3>(c, S, out); break;
        case 4: ff_launch<4>(c, S, out); break;
        case 5: ff_launch<5>(c, S, out); break;
        default: ff_launch<6>(c, S, out); break;
    }
}

void m2l_ffma_release(polfmm_ctx* c) {
    FfState* S = ff_state(c);
    if (!S) return;
    for (void* p : {(void*)S->Dpad, (void*)S->rows, (void*)S->groups, (void*)S->ent_off, (void*)S->ent_src,
                    (void*)S->ent_cnt})
        if (p) cudaFree(p);
    delete S;
    c->ff = nullptr;
}

}  // namespace polfmm

// ---------------------------------------------------------------------------
// the compiled schedule, for checks on the CPU
// ---------------------------------------------------------------------------
namespace {
template <int P, int PART>
int ff_plan_copy(int cap, int* n, int* m, int* k, int* load) {
    constexpr const polfmm::FfPlan<P, PART>& pl = polfmm::kFfPlan<P, PART>;
    const int nt = polfmm::FfPlan<P, PART>::NT;
    for (int e = 0; e < nt && e < cap; e++) {
        if (n) n[e] = pl.n[e];
        if (m) m[e] = pl.m[e];
        if (k) k[e] = pl.k[e];
        if (load) load[e] = pl.load[e] ? 1 : 0;
    }
    return nt;
}

template <int P>
int ff_plan_part(int part, int cap, int* n, int* m, int* k, int* load) {
    return part == 0 ? ff_plan_copy<P, 0>(cap, n, m, k, load) : ff_plan_copy<P, 1>(cap, n, m, k, load);
}
}  // namespace

extern "C" POLFMM_API int fmm_testing_m2l_plan(int p, int part, int cap, int* n, int* m, int* k, int* load,
                                                int* split_out) {
    if (p < 1 || p > polfmm::kFfMaxP || (part != 0 && part != 1)) return -1;
    if (split_out) *split_out = polfmm::ff_split(p);
    switch (p) {
        case 1: return ff_plan_part<1>(part, cap, n, m, k, load);
        case 2: return ff_plan_part<2>(part, cap, n, m, k, load);
        case 3: return ff_plan_part<3>(part, cap, n, m, k, load);
        case 4: return ff_plan_part<4>(part, cap, n, m, k, load);
        case 5: return ff_plan_part<5>(part, cap, n, m, k, load);
        default: return ff_plan_part<6>(part, cap, n, m, k, load);
    }
}
