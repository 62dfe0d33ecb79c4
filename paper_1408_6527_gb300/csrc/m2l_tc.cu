// Multipole-to-local translation on the 5th-generation tensor cores (MIXED
// mode).  Sec. II.B: F_n(z_B) = sum_{|m| <= p-|n|} M_m(z_A) d^{n+m} phi(z_B - z_A).
// In normalised coefficients and for a fixed integer offset o = B - A the
// operator is one matrix K_o[n][m] = D_o[n+m] (zero where |n| + |m| > p), so all
// target boxes of one level and one octant class that share the offset form a
// dense contraction  C[box][n] += sum_m A[box][m] K_o[n][m].
//
// One CTA = one tile of up to 128 same-class target boxes (the M = 128 rows of
// the MMA) and a range of the class's 189 offsets.  Per offset:
//   * the warps gather the FP32 multipole row of every box's source B - o
//     (zero where the source box is empty or outside the tree) with 16-byte
//     cp.async copies into the no-swizzle K-major core-matrix layout, eight
//     rows x 64 contiguous bytes per instruction; one thread bulk-copies the
//     pre-split image of K_o with cp.async.bulk completing on an mbarrier;
//   * the threads split the gathered rows into a TF32 high part and the
//     residual in shared memory;
//   * one thread issues tcgen05.mma kind::tf32 for A_hi B_lo + A_lo B_hi +
//     A_hi B_hi (FP32-level accuracy from TF32 inputs).  Inputs come in steps
//     of 8; step k only feeds the outputs n with |n| + (degree of input 8k) <= p,
//     a prefix of the outputs, so each step is ONE MMA whose N is that prefix
//     (rounded to 16): the image of K_o is stored as one slab per step;
//   * every thread waits for the commit, then folds the offset's accumulator
//     into a running sum held in TMEM with round-to-nearest FP32 additions.
// At the end each warp reads its 32 TMEM lanes (tcgen05.ld) and writes the
// partial locals of its boxes; partials of different offset ranges are summed
// in fixed order by the downward pass of the leaf kernels.  Every wait is
// bounded: on timeout the CTA raises an error bit, stops issuing and still
// frees its TMEM.
#include <math.h>
#include <string.h>

#include <vector>

#include "async_copy.cuh"
#include "internal.cuh"

namespace polfmm {

constexpr int kTcRows = 128;
constexpr int kTcThreads = 128;
constexpr int kTcMaxSteps = 24;  // input steps of 8 (p <= 8: KP <= 168)
constexpr uint64_t kTcWaitNs = kAsyncWaitNs;  // 2 s bound on every wait

struct TcSchedule {
    int nks;                   // input steps of 8 (KP / 8)
    int width[kTcMaxSteps];    // outputs fed by step k (multiple of 16, non-increasing)
    int soff[kTcMaxSteps];     // float offset of step k's slab inside one image part
    int KP;                    // padded input count (multiple of 8)
    int NP;                    // padded output count (multiple of 16) = width[0]
    int bpart;                 // floats per image part (hi or lo) per offset
    int tmem_cols;             // power of two >= 2 NP
    int nmma;                  // MMAs per offset: 3 products x nks
    int tab_off;               // byte offset of the MMA table in dynamic shared memory
};

// one tcgen05.mma of the per-offset sequence: the stage buffers sit at fixed
// shared addresses, so the descriptors are the same for every offset
struct TcMma {
    uint64_t a, b;      // shared-memory matrix descriptors
    uint32_t idesc;     // instruction descriptor
    uint32_t acc;       // 0: overwrite the accumulator, 1: add
};

struct TcTile {
    int cls;
    int first;  // into the class-ordered row list
    int count;  // <= kTcRows
};

constexpr int kWsWorkerWarps = 12;
constexpr int kWsSlots = kWsWorkerWarps / 4;  // worker threads per row
constexpr int kWsWorkers = kWsWorkerWarps * 32;
constexpr int kWsIssuerWarp = kWsWorkerWarps;
constexpr int kWsLoaderWarp = kWsWorkerWarps + 1;
constexpr int kWsThreads = kWsWorkers + 64;
constexpr int kWsMaxKT = 40;
constexpr int kWsMaxSteps = kWsMaxKT / 8;
constexpr int kWsMaxNP = 96;
constexpr int kWsFoldChunks = 2;      // 16-column accumulator chunks per thread (NP / 16 <= 6 over 3 slots)
constexpr int kWsRowStages = 4;       // gathered-row stages
constexpr int kWsBStages = 3;         // K_o image stages
constexpr int kWsSrcStages = 4;       // source-row lists

struct WsSchedule {
    int KT;                       // inputs on the tensor cores (multiple of 8)
    int nks;                      // KT / 8
    int NP;                       // accumulator columns (multiple of 16)
    int nmma;                     // 3 nks
    int width[kWsMaxSteps];       // outputs fed by input step k (multiple of 16)
    int soff[kWsMaxSteps];        // float offset of step k's slab in one image part
    int bpart;                    // floats per image part
    int rs;                       // floats per gathered row in a stage (multiple of 4, rs / 4 odd)
    int dsw;                      // floats of the CUDA-core derivative block of an offset (multiple of 4)
    int stage_floats;             // 128 rs + dsw: one gathered-row stage
    int nsim;                     // outputs with a CUDA-core part (<= 4)
    int sim_out[4];               // their coefficient indices (< 16)
    int nchk;                     // 4-input chunks of the CUDA-core part (inputs KT .. ncoef - 1)
};

struct TcState {
    TcSchedule sch;                          // m2l_tc_kernel (A in shared memory; p = 7, 8)
    WsSchedule ws;                           // m2l_ws_kernel (A in tensor memory; p <= 6)
    bool use_ws = false;
    float* Bimg = nullptr;                   // [343][2][bpart] of the kernel in use
    float* Dsim = nullptr;                   // [343][dsw]: derivative blocks of the CUDA-core part (ws)
    int2* rows = nullptr;                    // (level, slot) of every box of levels >= 2, by class
    TcTile* tiles = nullptr;
    int ntiles = 0, tiles_cap = 0;
    size_t stage_bytes = 0;
    size_t smem = 0;
    bool ready = false;
};

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}


__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
        "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
        "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
        : "memory");
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
}

// D (TMEM) (+)= A (TMEM, lane = row, column = input) x B (shared-memory descriptor)
__device__ __forceinline__ void mma_tf32_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// TF32 high part (round to nearest, ties away) and FP32 residual of v
__device__ __forceinline__ void tf32_split(float v, float& hi, float& lo) {
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
    hi = __uint_as_float(h);
    lo = v - hi;
}

// shared-memory matrix descriptor, K-major, no swizzle: core matrices of
// 8 rows x 16 bytes; lbo = byte step between core matrices along K, sbo =
// byte step between 8-row groups along M / N.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of this architecture
    return d;                // base offset 0, layout type 0 (no swizzle)
}

// instruction descriptor: kind::tf32, FP32 accumulator, both operands K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4)                         // D format F32
           | (2u << 7)                       // A format TF32
           | (2u << 10)                      // B format TF32
           | ((uint32_t)(N >> 3) << 17)      // N / 8
           | ((uint32_t)(M >> 4) << 24);     // M / 16
}

// (level, slot) rows of every box of one level, placed by octant class
struct TcRowArgs {
    int off[8];    // first row of (class, this level) in the class-ordered list
    int start[8];  // first index of the class in the level's by_class list
};

__global__ void tc_rows_kernel(int nbox, int level, const int* __restrict__ by_class, const int* __restrict__ key,
                               TcRowArgs ra, int2* __restrict__ rows) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nbox) return;
    const int slot = by_class[i];
    const int c = key[slot] & 7;
    rows[ra.off[c] + (i - ra.start[c])] = make_int2(level, slot);
}

// ---------------------------------------------------------------------------
// the tensor-core M2L kernel
// ---------------------------------------------------------------------------
struct TcLevelPtrs {
    const int* key[kMaxDepth + 1];
    const int* map[kMaxDepth + 1];
    const float* M[kMaxDepth + 1];  // multipoles [cap][ld]
    float* Lp[kMaxDepth + 1];
    int cap[kMaxDepth + 1];
    int row0[kMaxDepth + 1];        // first row of level l in the all-level multipole array
    const float* Mall;              // that array
};

// One stage per CTA: gather, split, multiply, fold; two CTAs per SM overlap
// one CTA's gather with the other's MMAs.
__global__ void __launch_bounds__(kTcThreads, 1) m2l_tc_kernel(const TcTile* __restrict__ tiles,
                                                               const int2* __restrict__ rows, TcLevelPtrs lp,
                                                               const float* __restrict__ Bimg,
                                                               const int* __restrict__ class_off, TcSchedule sch,
                                                               int ncoef, int ld, int nchunk,
                                                               int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int KP = sch.KP;
    // A_hi [KP/4][16][8][4] floats, A_lo (same), K_o image hi, K_o image lo, MMA table
    float* const Ahi = reinterpret_cast<float*>(smem_raw);
    float* const Alo = Ahi + kTcRows * KP;
    float* const Bhi = Alo + kTcRows * KP;
    float* const Blo = Bhi + sch.bpart;
    __shared__ __align__(8) uint64_t bar_b;  // K_o image landed
    __shared__ __align__(8) uint64_t bar_m;  // MMAs of the offset done
    __shared__ uint32_t tmem_base_sh;
    __shared__ int fail_sh;
    __shared__ int s_src[2][kTcRows];
    __shared__ int s_lvl[kTcRows];

    const TcTile tile = tiles[blockIdx.x];
    const int chunk = blockIdx.y;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;

    if (warp == 0) tmem_alloc(&tmem_base_sh, (uint32_t)sch.tmem_cols);
    if (tid == 0) {
        mbar_init(&bar_b, 1);
        mbar_init(&bar_m, 1);
        fail_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    // this thread's target box: row `tid` of the tile, any level >= 2
    int level = 0, slot = -1, bx = 0, by = 0, bz = 0;
    if (tid < tile.count) {
        const int2 r = rows[tile.first + tid];
        level = r.x;
        slot = r.y;
        const uint32_t k = (uint32_t)lp.key[level][slot];
        bx = (int)compact3(k);
        by = (int)compact3(k >> 1);
        bz = (int)compact3(k >> 2);
    }
    const int nside = 1 << level;
    const int* map = slot >= 0 ? lp.map[level] : nullptr;
    s_lvl[tid] = level;

    const int per = (kNumOffsets + nchunk - 1) / nchunk;
    const int t0 = min(kNumOffsets, chunk * per), t1 = min(kNumOffsets, t0 + per);
    const int nt = t1 - t0;
    const uint32_t a_lbo = kTcRows / 8 * 128;  // bytes between K chunks of A
    const uint32_t bbytes = (uint32_t)sch.bpart * 4u;
    uint32_t pb = 0, pm = 0;  // mbarrier phases
    // thread 0: an image copy armed and not yet seen to land, MMAs committed and
    // not yet seen to finish (waited for before the tensor memory is freed)
    bool b_pending = false, m_pending = false;

    // the MMA sequence of one offset, built once: product (A_hi B_lo, A_lo B_hi,
    // A_hi B_hi: the two small correction products first) x input step k, one
    // MMA of N = width[k] at accumulator column 0; the first one overwrites
    TcMma* mtab = reinterpret_cast<TcMma*>(smem_raw + sch.tab_off);
    {
        const uint32_t a_hi = smem_u32(Ahi), a_lo = smem_u32(Alo);
        const uint32_t b_hi = smem_u32(Bhi), b_lo = smem_u32(Blo);
        for (int j = tid; j < sch.nmma; j += kTcThreads) {
            const int prod = j / sch.nks, k = j - prod * sch.nks;
            const int w = sch.width[k];
            const uint32_t b_lbo = (uint32_t)(w / 8) * 128u;
            const uint32_t a_base = prod == 1 ? a_lo : a_hi;
            const uint32_t b_base = (prod == 0 ? b_lo : b_hi) + (uint32_t)sch.soff[k] * 4u;
            TcMma m;
            m.a = smem_desc(a_base + 2u * (uint32_t)k * a_lbo, a_lbo, 128u);
            m.b = smem_desc(b_base, b_lbo, 128u);
            m.idesc = idesc_tf32(kTcRows, w);
            m.acc = j == 0 ? 0u : 1u;
            mtab[j] = m;
        }
    }

    // source row of this thread's box for offset t (-1: empty or outside), one
    // offset ahead of the gather that uses it; the gather reads it from shared memory
    auto lookup = [&](int t) {
        int src = -1;
        if (slot >= 0) {
            const int o = class_off[tile.cls * kNumOffsets + t];
            const int ox = (o & 15) - 3, oy = ((o >> 4) & 15) - 3, oz = ((o >> 8) & 15) - 3;
            const int ax = bx - ox, ay = by - oy, az = bz - oz;
            if (ax >= 0 && ay >= 0 && az >= 0 && ax < nside && ay < nside && az < nside)
                src = map[morton3(ax, ay, az)];
        }
        s_src[(t - t0) & 1][tid] = src;
    };

    // gather of offset t: warp w copies the 8-row groups w, w + 4, .. with lane =
    // (row in group) + 8 (chunk in a group of 4 chunks): each instruction moves
    // 8 rows x 64 contiguous bytes and its shared stores hit distinct banks.
    // Inputs ncoef .. KP - 1 are zero-filled.  The K_o image by thread 0.
    const int lane = tid & 31;
    const int rr = lane & 7, cq = lane >> 3;
    const int nch = KP / 4;
    auto issue = [&](int t) {
        if (tid == 0) {
            const int o = class_off[tile.cls * kNumOffsets + t];
            const int ox = (o & 15) - 3, oy = ((o >> 4) & 15) - 3, oz = ((o >> 8) & 15) - 3;
            const int oidx = (ox + 3) + kOffsetGrid * ((oy + 3) + kOffsetGrid * (oz + 3));
            const float* img = Bimg + (size_t)oidx * 2 * sch.bpart;
            mbar_arrive_expect_tx(&bar_b, 2 * bbytes);
            bulk_g2s(Bhi, img, bbytes, &bar_b);
            bulk_g2s(Blo, img + sch.bpart, bbytes, &bar_b);
            b_pending = true;
        }
        const int* srcs = s_src[(t - t0) & 1];
        for (int rg = warp; rg < kTcRows / 8; rg += kTcThreads / 32) {
            const int row = rg * 8 + rr;
            const int src = srcs[row];
            const float* g = src >= 0 ? lp.M[s_lvl[row]] + (size_t)src * ld : Bimg;  // any valid address when nothing is read
            const int off0 = rg * 32 + rr * 4;
            for (int c = cq; c < nch; c += 4) {
                const int valid = src >= 0 ? min(4, max(0, ncoef - 4 * c)) : 0;
                cp_async16(Ahi + c * (kTcRows / 8) * 32 + off0, valid ? g + 4 * c : Bimg, (uint32_t)(4 * valid));
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };

    if (nt > 0) lookup(t0);
    __syncthreads();
    if (nt > 0) issue(t0);
    if (nt > 1) lookup(t0 + 1);
    float4* const ah4 = reinterpret_cast<float4*>(Ahi);
    float4* const al4 = reinterpret_cast<float4*>(Alo);
    for (int i = 0; i < nt; i++) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        // FP32 rows -> TF32 high part (round to nearest, ties away) + residual
        for (int q = tid; q < kTcRows * KP / 4; q += kTcThreads) {
            const float4 v = ah4[q];
            float4 h, l;
            tf32_split(v.x, h.x, l.x);
            tf32_split(v.y, h.y, l.y);
            tf32_split(v.z, h.z, l.z);
            tf32_split(v.w, h.w, l.w);
            ah4[q] = h;
            al4[q] = l;
        }
        fence_proxy_async();
        __syncthreads();
        if (fail_sh) break;
        if (tid == 0) {
            if (!mbar_wait_bounded(&bar_b, pb)) {
                atomicOr(err, 4);
                fail_sh = 1;
            } else {
                b_pending = false;
                tc_fence_after();
                for (int j = 0; j < sch.nmma; j++) {
                    const TcMma m = mtab[j];
                    mma_tf32(tmem, m.a, m.b, m.idesc, m.acc);
                }
                mma_commit(&bar_m);
                m_pending = true;
            }
        }
        if (!fail_sh) pb ^= 1;
        // wait for this offset's MMAs, then fold the accumulator into the running
        // sum with round-to-nearest FP32 additions (warp w: TMEM lanes 32 w ..)
        __syncthreads();
        if (fail_sh) break;
        if (!mbar_wait_bounded(&bar_m, pm)) atomicOr(err, 4), fail_sh = 1;
        __syncthreads();
        if (fail_sh) break;
        if (tid == 0) m_pending = false;
        pm ^= 1;
        tc_fence_after();
        {
            const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
            for (int c0 = 0; c0 < sch.NP; c0 += 16) {
                float a[16], b[16];
                tmem_ld16(lane_base + (uint32_t)c0, a);
                if (i > 0) {
                    tmem_ld16(lane_base + (uint32_t)(sch.NP + c0), b);
#pragma unroll
                    for (int k = 0; k < 16; k++) a[k] += b[k];
                }
                tmem_st16(lane_base + (uint32_t)(sch.NP + c0), a);
            }
            tmem_wait_st();
        }
        tc_fence_before();
        __syncthreads();
        if (fail_sh) break;
        if (i + 1 < nt) {
            issue(t0 + i + 1);  // the stage is free again
            if (i + 2 < nt) lookup(t0 + i + 2);
        }
    }
    __syncthreads();
    // on failure the image copy and the MMAs already issued finish (bounded
    // waits) before the tensor memory is freed
    if (fail_sh && tid == 0) {
        if (b_pending) mbar_wait_bounded(&bar_b, pb);
        if (m_pending) mbar_wait_bounded(&bar_m, pm);
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();

    // epilogue: TMEM lanes 32 w .. 32 w + 31 hold the rows of warp w; the loads
    // are warp-collective, so every lane takes part and only rows with a box store
    tc_fence_after();
    if (!fail_sh) {
        float* out = slot >= 0 ? lp.Lp[level] + ((size_t)chunk * lp.cap[level] + slot) * ld : nullptr;
        for (int c0 = 0; c0 < sch.NP; c0 += 16) {
            float v[16];
            if (nt > 0) {
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(sch.NP + c0), v);
            } else {
#pragma unroll
                for (int k = 0; k < 16; k++) v[k] = 0.f;
            }
            if (out)
                for (int k = 0; k < 16; k++)
                    if (c0 + k < ncoef) out[c0 + k] = v[k];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, (uint32_t)sch.tmem_cols);
}

// ---------------------------------------------------------------------------
// the warp-specialised tensor-core M2L kernel (one CTA per SM, p <= 6)
//
// Same contraction as m2l_tc_kernel, split in two by input degree.  The first
// KT inputs (multiple of 8) go through the tensor cores; the remaining inputs,
// of degree >= d_KT (the degree of input KT), only feed the outputs of degree
// <= p - d_KT (at p = 6 and KT = 40: inputs of degree 5 and 6 feed the outputs
// of degree <= 1), so their few terms per row are FP32 FMAs on the CUDA cores
// instead of narrow MMAs of at least 16 outputs.  Roles:
//   * a loader warp: per offset, looks up the source box of each row (one
//     dependent load of the level's key -> slot map), writes the list of
//     source rows to a small ring, arms the row stage's mbarrier with the byte
//     count of the existing rows and bulk-copies (cp.async.bulk) the block of
//     derivatives of the CUDA-core part into it; bulk-copies the K_o image of
//     the offset (TF32 high part and residual) into an image stage;
//   * 12 worker warps, three threads per row: issue the bulk copies of the
//     source rows two offsets ahead -- one FP32 multipole row of ld floats
//     per lane, one instruction per warp, counted by the stage's barrier --
//     so that the copies stream in while the warps work; split the first KT
//     inputs of the current offset into TF32 high part and residual in tensor
//     memory (the A operand, double-buffered); evaluate the CUDA-core part;
//     and fold the previous offset's accumulator into running sums in
//     registers with round-to-nearest FP32 additions;
//   * an issuing warp: one thread issues the 3 x KT/8 MMAs of an offset
//     (A_hi B_lo, A_lo B_hi, A_hi B_hi; A from tensor memory, B from the
//     image stage) into the accumulator buffer of the offset's parity, then
//     commits to that buffer's "done" barrier and to the image stage's "empty"
//     barrier.
// Stages, A buffers and accumulators are handed over with mbarriers, so the
// gather of offset t + 1, the split of offset t, the MMAs of offset t - 1 and
// the fold of offset t - 2 can all be in flight at once.  Every wait is
// bounded; a role that times out raises the error bit and the shared failure
// flag, every role stops, the MMAs and copies already issued are waited for
// (bounded), and the tensor memory is freed.
// TMEM columns: accumulator b at b NP, A buffer b at 2 NP + 2 KT b (high
// part) and 2 NP + 2 KT b + KT (residual).  Worker warp w owns TMEM lanes
// 32 (w % 4) .. + 31 (its rows) and the column chunks of slot w / 4.
// ---------------------------------------------------------------------------
struct WsBars {
    uint64_t full[kWsRowStages];    // rows and derivative block of the stage's offset landed (bytes)
    uint64_t rempty[kWsRowStages];  // stage read by every worker warp
    uint64_t sfull[kWsSrcStages];   // source-row list written (loader)
    uint64_t sempty[kWsSrcStages];  // source-row list used (every worker warp)
    uint64_t bfull[kWsBStages];     // K_o image landed (loader, bytes)
    uint64_t bempty[kWsBStages];    // K_o image read by the offset's MMAs (commit)
    uint64_t a_full[2];             // A buffer written (every worker warp)
    uint64_t acc_empty[2];          // accumulator buffer read (every worker warp)
    uint64_t done[2];               // MMAs of the buffer's latest offset complete (commit)
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// bounded wait that gives up as soon as another role has failed:
// 1 = phase complete, 0 = another role failed, -1 = this wait timed out
__device__ __forceinline__ int ws_wait(uint64_t* bar, uint32_t parity, volatile int* fail) {
    if (mbar_try_wait(bar, parity)) return 1;
    const uint64_t t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return 1;
        if (*fail) return 0;
        if (global_ns() - t0 >= kTcWaitNs) {
            *fail = 1;
            return -1;
        }
    }
}

// the same wait taken by all lanes of a warp, with one outcome for the whole
// warp (every lane observes the phase itself; the lanes agree on the result)
__device__ __forceinline__ int ws_wait_warp(uint64_t* bar, uint32_t parity, volatile int* fail) {
    const int r = ws_wait(bar, parity, fail);
    return __reduce_min_sync(0xffffffffu, r);
}

__device__ __forceinline__ void workers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kWsWorkers) : "memory"); }

struct TcaMma {
    uint64_t b;         // B descriptor (image stage 0)
    uint32_t a_tmem;    // column of the A operand relative to the A buffer
    uint32_t idesc;
};

__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__global__ void __launch_bounds__(kWsThreads, 1) m2l_ws_kernel(const TcTile* __restrict__ tiles,
                                                               const int2* __restrict__ rows, TcLevelPtrs lp,
                                                               const float* __restrict__ Bimg,
                                                               const float* __restrict__ Dsim,
                                                               const int* __restrict__ class_off, WsSchedule sch,
                                                               int ncoef, int ld, int nchunk, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float* const ring = reinterpret_cast<float*>(smem_raw);  // [row stages][128 rs | dsw]
    float* const bring = ring + (size_t)kWsRowStages * sch.stage_floats;  // [image stages][B hi | B lo]
    TcaMma* const mtab = reinterpret_cast<TcaMma*>(bring + (size_t)kWsBStages * 2 * sch.bpart);  // [nmma]
    int* const s_src = reinterpret_cast<int*>(mtab + sch.nmma);            // [src stages][128]
    float* const xs = reinterpret_cast<float*>(s_src + kWsSrcStages * kTcRows);  // [128 rows][4 (slots)][4 outputs]
    __shared__ __align__(8) WsBars bars;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int fail_sh;
    __shared__ int s_off[kNumOffsets];

    const TcTile tile = tiles[blockIdx.x];
    const int chunk = blockIdx.y;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int per = (kNumOffsets + nchunk - 1) / nchunk;
    const int t0 = min(kNumOffsets, chunk * per), t1 = min(kNumOffsets, t0 + per);
    const int nt = t1 - t0;
    const int KT = sch.KT, NP = sch.NP, rs = sch.rs;
    const uint32_t bstage_bytes = (uint32_t)sch.bpart * 8u;
    volatile int* const fail = &fail_sh;

    if (warp == 0) tmem_alloc(&tmem_base_sh, 512u);
    if (tid == 0) {
        for (int s = 0; s < kWsRowStages; s++) {
            mbar_init(&bars.full[s], 1);
            mbar_init(&bars.rempty[s], kWsWorkerWarps);
        }
        for (int s = 0; s < kWsSrcStages; s++) {
            mbar_init(&bars.sfull[s], 1);
            mbar_init(&bars.sempty[s], kWsWorkerWarps);
        }
        for (int s = 0; s < kWsBStages; s++) {
            mbar_init(&bars.bfull[s], 1);
            mbar_init(&bars.bempty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&bars.a_full[b], kWsWorkerWarps);
            mbar_init(&bars.acc_empty[b], kWsWorkerWarps);
            mbar_init(&bars.done[b], 1);
        }
        fail_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the per-offset MMA sequence for image stage 0 and A buffer 0: product x input step
    {
        const uint32_t b_hi = smem_u32(bring), b_lo = b_hi + (uint32_t)sch.bpart * 4u;
        for (int j = tid; j < sch.nmma; j += kWsThreads) {
            const int prod = j / sch.nks, k = j - prod * sch.nks;
            const int w = sch.width[k];
            TcaMma m;
            m.b = smem_desc((prod == 0 ? b_lo : b_hi) + (uint32_t)sch.soff[k] * 4u, (uint32_t)(w / 8) * 128u, 128u);
            m.a_tmem = (prod == 1 ? (uint32_t)KT : 0u) + 8u * (uint32_t)k;
            m.idesc = idesc_tf32(kTcRows, w);
            mtab[j] = m;
        }
    }
    for (int t = t0 + tid; t < t1; t += kWsThreads) s_off[t - t0] = class_off[tile.cls * kNumOffsets + t];
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    if (warp == kWsIssuerWarp) {
        // ------------------------------------------------------------ MMAs
        if (lane == 0) {
            // the whole per-offset sequence in registers, issued unrolled: a table load
            // between two MMAs would cost more than the MMA itself
            constexpr int kMaxMma = 3 * kWsMaxSteps;
            uint64_t bd[kMaxMma];
            uint32_t ad[kMaxMma], id[kMaxMma];
#pragma unroll
            for (int j = 0; j < kMaxMma; j++) {
                const TcaMma m = mtab[j < sch.nmma ? j : 0];
                bd[j] = m.b;
                ad[j] = m.a_tmem;
                id[j] = m.idesc;
            }
            const int nm = sch.nmma;
            int last = -1;
            for (int i = 0; i < nt; i++) {
                const int bs = i % kWsBStages, b = i & 1;
                const uint32_t pb = (uint32_t)(i >> 1) & 1u;
                int r = ws_wait(&bars.bfull[bs], (uint32_t)(i / kWsBStages) & 1u, fail);
                if (r > 0) r = ws_wait(&bars.a_full[b], pb, fail);
                if (r > 0 && i >= 2) r = ws_wait(&bars.acc_empty[b], pb ^ 1u, fail);  // fold of offset i - 2
                if (r <= 0) {
                    if (r < 0) atomicOr(err, 4);
                    break;
                }
                tc_fence_after();
                const uint64_t boff = (uint64_t)(((uint32_t)bs * bstage_bytes) >> 4);
                const uint32_t dcol = tmem + (uint32_t)(b * NP);
                const uint32_t acol = tmem + (uint32_t)(2 * NP + 2 * KT * b);
#pragma unroll
                for (int j = 0; j < kMaxMma; j++)
                    if (j < nm) mma_tf32_ta(dcol, acol + ad[j], bd[j] + boff, id[j], j == 0 ? 0u : 1u);
                mma_commit(&bars.done[b]);
                mma_commit(&bars.bempty[bs]);
                last = i;
            }
            // on failure the MMAs already issued finish before the tensor memory is freed
            if (*fail && last >= 0) mbar_wait_bounded(&bars.done[last & 1], (uint32_t)(last >> 1) & 1u);
        }
    } else if (warp == kWsLoaderWarp) {
        // ------------------------------------------- source lookups, K_o images
        // this lane's rows: lane + 32 k
        int bxyz[4], nside[4], row0[4];
        const int* mmap[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int r = lane + 32 * k;
            bxyz[k] = -1;
            nside[k] = 0;
            row0[k] = 0;
            mmap[k] = nullptr;
            if (r < tile.count) {
                const int2 rr = rows[tile.first + r];
                const uint32_t key = (uint32_t)lp.key[rr.x][rr.y];
                bxyz[k] = (int)(compact3(key) | (compact3(key >> 1) << 10) | (compact3(key >> 2) << 20));
                nside[k] = 1 << rr.x;
                row0[k] = lp.row0[rr.x];
                mmap[k] = lp.map[rr.x];
            }
        }
        int barmed[kWsBStages], rarmed[kWsRowStages];
#pragma unroll
        for (int s = 0; s < kWsBStages; s++) barmed[s] = -1;
#pragma unroll
        for (int s = 0; s < kWsRowStages; s++) rarmed[s] = -1;
        for (int i = 0; i < nt; i++) {
            const int ss = i % kWsSrcStages, bs = i % kWsBStages;
            const int o = s_off[i];
            const int ox = (o & 15) - 3, oy = ((o >> 4) & 15) - 3, oz = ((o >> 8) & 15) - 3;
            // source rows of offset i (row index into the all-level array; -1: none)
            int src[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                src[k] = -1;
                if (bxyz[k] >= 0) {
                    const int ax = (bxyz[k] & 1023) - ox, ay = ((bxyz[k] >> 10) & 1023) - oy,
                              az = ((bxyz[k] >> 20) & 1023) - oz;
                    if (ax >= 0 && ay >= 0 && az >= 0 && ax < nside[k] && ay < nside[k] && az < nside[k]) {
                        const int sl = mmap[k][morton3(ax, ay, az)];
                        src[k] = sl >= 0 ? row0[k] + sl : -1;
                    }
                }
            }
            const int rsg = i % kWsRowStages;
            int r = 1;
            if (i >= kWsSrcStages) r = ws_wait_warp(&bars.sempty[ss], (uint32_t)(i / kWsSrcStages - 1) & 1u, fail);
            // the row stage of offset i is free once every worker warp has read offset i - stages
            if (r > 0 && i >= kWsRowStages)
                r = ws_wait_warp(&bars.rempty[rsg], (uint32_t)(i / kWsRowStages - 1) & 1u, fail);
            if (r <= 0) {
                if (r < 0 && lane == 0) atomicOr(err, 4);
                break;
            }
            int nvalid = 0;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                s_src[ss * kTcRows + lane + 32 * k] = src[k];
                nvalid += __popc(__ballot_sync(0xffffffffu, src[k] >= 0));
            }
            __syncwarp();
            __threadfence_block();
            if (lane == 0) {
                // the stage's byte count (existing rows and the derivative block) is armed
                // before any worker may copy into it (they wait for sfull)
                const int oidx = (o & 15) + kOffsetGrid * (((o >> 4) & 15) + kOffsetGrid * ((o >> 8) & 15));
                float* st = ring + (size_t)rsg * sch.stage_floats;
                mbar_arrive_expect_tx(&bars.full[rsg], (uint32_t)nvalid * (uint32_t)ld * 4u + (uint32_t)sch.dsw * 4u);
                bulk_g2s(st + (size_t)kTcRows * rs, Dsim + (size_t)oidx * sch.dsw, (uint32_t)sch.dsw * 4u,
                         &bars.full[rsg]);
                rarmed[rsg] = i;
                mbar_arrive(&bars.sfull[ss]);
            }
            // K_o image of offset i, once the MMAs of offset i - stages are done with its stage
            if (i >= kWsBStages) {
                r = ws_wait_warp(&bars.bempty[bs], (uint32_t)(i / kWsBStages - 1) & 1u, fail);
                if (r <= 0) {
                    if (r < 0 && lane == 0) atomicOr(err, 4);
                    break;
                }
            }
            if (lane == 0) {
                const int oidx = (o & 15) + kOffsetGrid * (((o >> 4) & 15) + kOffsetGrid * ((o >> 8) & 15));
                float* bst = bring + (size_t)bs * 2 * sch.bpart;
                mbar_arrive_expect_tx(&bars.bfull[bs], bstage_bytes);
                bulk_g2s(bst, Bimg + (size_t)oidx * 2 * sch.bpart, bstage_bytes, &bars.bfull[bs]);
            }
            barmed[bs] = i;
        }
        // on failure every copy issued lands before the CTA may exit: the images, and the
        // rows of every armed stage (whose copies the workers may have issued)
        if (*fail && lane == 0) {
            for (int s = 0; s < kWsBStages; s++)
                if (barmed[s] >= 0) mbar_wait_bounded(&bars.bfull[s], (uint32_t)(barmed[s] / kWsBStages) & 1u);
            for (int s = 0; s < kWsRowStages; s++)
                if (rarmed[s] >= 0) mbar_wait_bounded(&bars.full[s], (uint32_t)(rarmed[s] / kWsRowStages) & 1u);
        }
    } else {
        // ------------------------------------------------------------ workers
        const int q = warp & 3, slot = warp >> 2, row = 32 * q + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
        float sum[kWsFoldChunks][16];
#pragma unroll
        for (int cc = 0; cc < kWsFoldChunks; cc++)
#pragma unroll
            for (int k = 0; k < 16; k++) sum[cc][k] = 0.f;
        float sa[4] = {0.f, 0.f, 0.f, 0.f};  // CUDA-core sums of the outputs sim_out[0..3]
        // fold of offset i: accumulator buffer i & 1 into the running sums
        auto fold = [&](int i) -> bool {
            const int b = i & 1;
            const int r = ws_wait_warp(&bars.done[b], (uint32_t)(i >> 1) & 1u, fail);
            if (r <= 0) {
                if (r < 0 && lane == 0) atomicOr(err, 4);
                return false;
            }
            tc_fence_after();
            uint32_t a[kWsFoldChunks][16];
#pragma unroll
            for (int cc = 0; cc < kWsFoldChunks; cc++) {
                const int c0 = 16 * (slot + kWsSlots * cc);
                if (c0 < NP) tmem_ld16_nowait(lane_base + (uint32_t)(b * NP + c0), a[cc]);
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int cc = 0; cc < kWsFoldChunks; cc++) {
                const int c0 = 16 * (slot + kWsSlots * cc);
                if (c0 < NP)
#pragma unroll
                    for (int k = 0; k < 16; k++) sum[cc][k] += __uint_as_float(a[cc][k]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars.acc_empty[b]);
            return true;
        };
        // rows of offset i: row r is copied by lane r / 12 of worker warp r % 12, one
        // bulk copy (cp.async.bulk) per existing source row, counted by the stage's
        // barrier that the loader armed
        auto issue_rows = [&](int i) -> bool {
            const int ss = i % kWsSrcStages;
            const int r = ws_wait_warp(&bars.sfull[ss], (uint32_t)(i / kWsSrcStages) & 1u, fail);
            if (r <= 0) {
                if (r < 0 && lane == 0) atomicOr(err, 4);
                return false;
            }
            const int rr = lane * kWsWorkerWarps + warp;
            if (rr < kTcRows) {
                const int sr = s_src[ss * kTcRows + rr];
                if (sr >= 0)
                    bulk_g2s(ring + (size_t)(i % kWsRowStages) * sch.stage_floats + (size_t)rr * rs,
                             lp.Mall + (size_t)sr * ld, (uint32_t)ld * 4u, &bars.full[i % kWsRowStages]);
            }
            return true;
        };
        bool ok = (nt < 1 || issue_rows(0)) && (nt < 2 || issue_rows(1));
        for (int i = 0; ok && i < nt; i++) {
            const int s = i % kWsRowStages, ss = i % kWsSrcStages, b = i & 1;
            if (i + 2 < nt && !issue_rows(i + 2)) break;  // two offsets ahead
            const int r = ws_wait_warp(&bars.full[s], (uint32_t)(i / kWsRowStages) & 1u, fail);
            if (r <= 0) {
                if (r < 0 && lane == 0) atomicOr(err, 4);
                break;
            }
            const float* st = ring + (size_t)s * sch.stage_floats;
            const bool valid = s_src[ss * kTcRows + row] >= 0;
            const float* src = st + (size_t)row * rs;
            // split of the first KT inputs (chunks of 8: slot and slot + kWsSlots) into A buffer b;
            // the A buffer was last read by the MMAs of offset i - 2, folded already
            const uint32_t acol = lane_base + (uint32_t)(2 * NP + 2 * KT * b);
            {
                const int c1 = slot + kWsSlots;
                const bool two = c1 < sch.nks;
                float4 v[4];
#pragma unroll
                for (int k = 0; k < 4; k++) v[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (valid && slot < sch.nks) {
                    v[0] = *reinterpret_cast<const float4*>(src + 8 * slot);
                    v[1] = *reinterpret_cast<const float4*>(src + 8 * slot + 4);
                    if (two) {
                        v[2] = *reinterpret_cast<const float4*>(src + 8 * c1);
                        v[3] = *reinterpret_cast<const float4*>(src + 8 * c1 + 4);
                    }
                }
                if (slot < sch.nks) {
                    float h[8], l[8];
                    const float x0[8] = {v[0].x, v[0].y, v[0].z, v[0].w, v[1].x, v[1].y, v[1].z, v[1].w};
#pragma unroll
                    for (int k = 0; k < 8; k++) tf32_split(8 * slot + k < ncoef ? x0[k] : 0.f, h[k], l[k]);
                    tmem_st8(acol + (uint32_t)(8 * slot), h);
                    tmem_st8(acol + (uint32_t)(KT + 8 * slot), l);
                    if (two) {
                        const float x1[8] = {v[2].x, v[2].y, v[2].z, v[2].w, v[3].x, v[3].y, v[3].z, v[3].w};
#pragma unroll
                        for (int k = 0; k < 8; k++) tf32_split(8 * c1 + k < ncoef ? x1[k] : 0.f, h[k], l[k]);
                        tmem_st8(acol + (uint32_t)(8 * c1), h);
                        tmem_st8(acol + (uint32_t)(KT + 8 * c1), l);
                    }
                }
            }
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars.a_full[b]);
            // CUDA-core part: chunks slot, slot + kWsSlots, .. of inputs KT .. ncoef - 1,
            // four outputs each (a dense 4 x 4 block of derivatives per chunk)
            if (valid) {
                const float* ds = st + (size_t)kTcRows * rs;
                for (int ch = slot; ch < sch.nchk; ch += kWsSlots) {
                    const float4 v = *reinterpret_cast<const float4*>(src + KT + 4 * ch);
                    const float4* dk = reinterpret_cast<const float4*>(ds + 16 * ch);
#pragma unroll
                    for (int o = 0; o < 4; o++) {
                        const float4 d = dk[o];
                        float t = d.x * v.x;
                        t = fmaf(d.y, v.y, t);
                        t = fmaf(d.z, v.z, t);
                        t = fmaf(d.w, v.w, t);
                        sa[o] += t;
                    }
                }
            }
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&bars.rempty[s]);
                mbar_arrive(&bars.sempty[ss]);
            }
            if (i > 0 && !fold(i - 1)) break;
        }
        if (nt > 0 && __all_sync(0xffffffffu, *fail == 0)) fold(nt - 1);
        // epilogue: the CUDA-core sums join slot 0's first chunk, slots and outputs in order
#pragma unroll
        for (int k = 0; k < 4; k++) xs[(row * 4 + slot) * 4 + k] = sa[k];
        workers_sync();
        if (!*fail && row < tile.count) {
            const int2 rr = rows[tile.first + row];
            float* out = lp.Lp[rr.x] + ((size_t)chunk * lp.cap[rr.x] + rr.y) * ld;
            if (slot == 0) {
#pragma unroll
                for (int k = 0; k < 16; k++) {
                    float v = sum[0][k];
                    for (int j = 0; j < 4; j++)
                        if (j < sch.nsim && sch.sim_out[j] == k)
                            for (int u = 0; u < kWsSlots; u++) v += xs[(row * 4 + u) * 4 + j];
                    sum[0][k] = v;
                }
            }
#pragma unroll
            for (int cc = 0; cc < kWsFoldChunks; cc++) {
                const int c0 = 16 * (slot + kWsSlots * cc);
                if (c0 < NP)
                    for (int k = 0; k < 16; k++)
                        if (c0 + k < ncoef) out[c0 + k] = sum[cc][k];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 512u);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static TcState* state(polfmm_ctx* c) { return reinterpret_cast<TcState*>(c->tc); }

bool m2l_tensor_enabled(polfmm_ctx* c) {
    TcState* S = state(c);
    return c->mixed && c->opt.m2l_impl != POLFMM_M2L_SIMT && !m2l_ffma_wanted(c) && S && S->ready && S->ntiles > 0;
}

static int degree_of(int idx, int p) {
    for (int s = 0; s <= p; s++)
        if (idx < ncoef_of(s)) return s;
    return p + 1;
}

// rounding to TF32 (10 explicit mantissa bits), nearest with ties away
static float tf32_round(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;
    float r;
    memcpy(&r, &u, 4);
    return r;
}

// schedule of m2l_ws_kernel for order p (false: the kernel does not apply)
static bool ws_schedule(int p, int nc, int ld, WsSchedule& w) {
    memset(&w, 0, sizeof(w));
    const int KP = (nc + 7) / 8 * 8;
    w.KT = std::min(KP, kWsMaxKT);
    w.nks = w.KT / 8;
    w.NP = (nc + 15) / 16 * 16;
    if (w.NP > kWsMaxNP || 2 * w.NP + 4 * w.KT > 512) return false;
    w.nmma = 3 * w.nks;
    int off = 0;
    for (int k = 0; k < w.nks; k++) {
        const int dmax = p - degree_of(8 * k, p);
        const int nout = dmax >= 0 ? ncoef_of(dmax) : 0;
        w.width[k] = std::max(16, (nout + 15) / 16 * 16);
        w.soff[k] = off;
        off += w.width[k] * 8;
    }
    w.bpart = off;
    w.rs = ld;
    if ((w.rs / 4) % 2 == 0) w.rs += 4;  // odd number of float4 per row: conflict-free row reads
    // CUDA-core part: the inputs m >= KT feed the outputs n with |n| + |m| <= p;
    // per offset a dense block D[chunk of 4 inputs][output][input] (zero where
    // |n| + |m| > p), the outputs being those reached by any input >= KT
    w.nsim = 0;
    for (int j = 0; j < 4; j++) w.sim_out[j] = -1;
    for (int n = 0; n < nc && w.KT < nc; n++) {
        if (ncoef_of(p - degree_of(n, p)) <= w.KT) continue;
        if (w.nsim == 4 || n >= 16) return false;
        w.sim_out[w.nsim++] = n;
    }
    w.nchk = w.KT < nc ? (nc - w.KT + 3) / 4 : 0;
    // at least 4 floats: the split of a short row may read up to 4 floats past the last row
    w.dsw = std::max(4, 16 * w.nchk);
    w.stage_floats = kTcRows * w.rs + w.dsw;
    return true;
}

static size_t ws_smem_bytes(const WsSchedule& w) {
    return sizeof(float) * ((size_t)kWsRowStages * w.stage_floats + (size_t)kWsBStages * 2 * w.bpart) +
           sizeof(TcaMma) * (size_t)w.nmma + sizeof(int) * kWsSrcStages * kTcRows + sizeof(float) * kTcRows * 16;
}

int m2l_tensor_prepare(polfmm_ctx* c) {
    if (!c->mixed || c->opt.m2l_impl == POLFMM_M2L_SIMT || c->p > 8 || c->depth < 2 || m2l_ffma_wanted(c))
        return POLFMM_OK;
    TcState* S = state(c);
    if (!S) {
        S = new TcState();
        c->tc = S;
        const int p = c->p, nc = c->ncoef;
        const size_t limit = 227 * 1024;
        std::vector<int> lut((p + 1) * (p + 1) * (p + 1), -1);
        std::vector<int> mx(nc), my(nc), mz(nc);
        for (int k = 0; k < nc; k++) {
            int v = c->tab.h_mi[k];
            mx[k] = v & 0xff;
            my[k] = (v >> 8) & 0xff;
            mz[k] = (v >> 16) & 0xff;
            lut[(mx[k] * (p + 1) + my[k]) * (p + 1) + mz[k]] = k;
        }
        auto sum_index = [&](int n, int m) {
            return lut[((mx[n] + mx[m]) * (p + 1) + my[n] + my[m]) * (p + 1) + mz[n] + mz[m]];
        };
        std::vector<double> Dd((size_t)343 * nc);
        if (cudaMemcpy(Dd.data(), c->tab.D, sizeof(double) * Dd.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
            return POLFMM_ERR_CUDA;
        // K_o images, one slab per input step: slab k holds outputs 0 .. width[k] - 1
        // x inputs 8k .. 8k + 7 in the core-matrix layout, element (n, kk) at
        // (kk/4)*(width/8)*32 + (n/8)*32 + (n%8)*4 + kk%4; split into a TF32 part and residual
        auto make_image = [&](int nks, const int* width, const int* soff, int bpart, std::vector<float>& img) {
            img.assign((size_t)343 * 2 * bpart, 0.f);
            for (int oi = 0; oi < 343; oi++) {
                float* hi = &img[(size_t)oi * 2 * bpart];
                float* lo = hi + bpart;
                for (int k = 0; k < nks; k++) {
                    const int w = width[k];
                    for (int n = 0; n < w; n++)
                        for (int kk = 0; kk < 8; kk++) {
                            const int m = 8 * k + kk;
                            float v = 0.f;
                            if (n < nc && m < nc && degree_of(n, p) + degree_of(m, p) <= p)
                                v = (float)Dd[(size_t)oi * nc + sum_index(n, m)];
                            const size_t pos =
                                soff[k] + (size_t)(kk / 4) * (w / 8) * 32 + (n / 8) * 32 + (n % 8) * 4 + kk % 4;
                            const float h = tf32_round(v);
                            hi[pos] = h;
                            lo[pos] = v - h;
                        }
                }
            }
        };
        std::vector<float> img;
        S->use_ws = ws_schedule(p, nc, c->ld, S->ws) && ws_smem_bytes(S->ws) <= limit;
        if (S->use_ws) {
            const WsSchedule& w = S->ws;
            S->smem = ws_smem_bytes(w);
            make_image(w.nks, w.width, w.soff, w.bpart, img);
            // derivative blocks of the CUDA-core part
            std::vector<float> ds((size_t)343 * w.dsw, 0.f);
            for (int oi = 0; oi < 343; oi++)
                for (int ch = 0; ch < w.nchk; ch++)
                    for (int o = 0; o < w.nsim; o++) {
                        const int n = w.sim_out[o];
                        const int mend = ncoef_of(p - degree_of(n, p));
                        for (int kk = 0; kk < 4; kk++) {
                            const int m = w.KT + 4 * ch + kk;
                            if (m < mend && m < nc)
                                ds[(size_t)oi * w.dsw + (ch * 4 + o) * 4 + kk] =
                                    (float)Dd[(size_t)oi * nc + sum_index(n, m)];
                        }
                    }
            if (dev_alloc(reinterpret_cast<void**>(&S->Dsim), sizeof(float) * ds.size()) != cudaSuccess)
                return POLFMM_ERR_OUT_OF_MEMORY;
            if (cudaMemcpy(S->Dsim, ds.data(), sizeof(float) * ds.size(), cudaMemcpyHostToDevice) != cudaSuccess)
                return POLFMM_ERR_CUDA;
        } else {
            TcSchedule& sch = S->sch;
            memset(&sch, 0, sizeof(sch));
            sch.KP = (nc + 7) / 8 * 8;
            sch.NP = (nc + 15) / 16 * 16;
            sch.nks = sch.KP / 8;
            if (sch.nks > kTcMaxSteps) {
                delete S;
                c->tc = nullptr;
                return POLFMM_OK;  // the SIMT kernel stays in use
            }
            // input step k (inputs 8k .. 8k + 7, lowest degree that of input 8k) feeds
            // the outputs n with |n| <= p - degree(8k): a prefix of the outputs
            int off = 0;
            for (int k = 0; k < sch.nks; k++) {
                const int dmax = p - degree_of(8 * k, p);
                const int nout = dmax >= 0 ? ncoef_of(dmax) : 0;
                sch.width[k] = std::max(16, (nout + 15) / 16 * 16);
                sch.soff[k] = off;
                off += sch.width[k] * 8;
            }
            sch.bpart = off;
            // TMEM: one accumulator for the current offset and one running sum (NP columns each)
            sch.tmem_cols = 32;
            while (sch.tmem_cols < 2 * sch.NP) sch.tmem_cols *= 2;
            if (sch.tmem_cols > 512) {
                delete S;
                c->tc = nullptr;
                return POLFMM_OK;  // the SIMT kernel stays in use
            }
            S->stage_bytes = sizeof(float) * (2 * (size_t)kTcRows * sch.KP + 2 * (size_t)sch.bpart);
            sch.nmma = 3 * sch.nks;
            sch.tab_off = (int)((S->stage_bytes + 15) / 16 * 16);
            // one shared-memory stage per CTA and two CTAs per SM
            S->smem = (size_t)sch.tab_off + sizeof(TcMma) * (size_t)sch.nmma;
            if (S->smem > limit) {
                delete S;
                c->tc = nullptr;
                return POLFMM_OK;  // does not fit: the SIMT kernel stays in use
            }
            make_image(sch.nks, sch.width, sch.soff, sch.bpart, img);
        }
        if (dev_alloc(reinterpret_cast<void**>(&S->Bimg), sizeof(float) * img.size()) != cudaSuccess)
            return POLFMM_ERR_OUT_OF_MEMORY;
        if (cudaMemcpy(S->Bimg, img.data(), sizeof(float) * img.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return POLFMM_ERR_CUDA;
        size_t rows_cap = 0;
        for (int l = 2; l <= c->depth; l++) rows_cap += c->lv[l].cap;
        if (dev_alloc(reinterpret_cast<void**>(&S->rows), sizeof(int2) * std::max<size_t>(rows_cap, 1)) != cudaSuccess)
            return POLFMM_ERR_OUT_OF_MEMORY;
        cudaError_t e1 = S->use_ws ? cudaFuncSetAttribute(m2l_ws_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          (int)S->smem)
                                   : cudaFuncSetAttribute(m2l_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          (int)S->smem);
        if (e1 != cudaSuccess) {
            cudaGetLastError();
            return POLFMM_ERR_CUDA;
        }
        S->ready = true;
    }
    // rows of all levels >= 2 grouped by octant class, and tiles of 128 rows
    int total[8] = {0};
    for (int l = 2; l <= c->depth; l++)
        for (int k = 0; k < 8; k++) total[k] += c->lv[l].class_count[k];
    int cls_first[8];
    int run = 0;
    for (int k = 0; k < 8; k++) {
        cls_first[k] = run;
        run += total[k];
    }
    int fill[8];
    for (int k = 0; k < 8; k++) fill[k] = cls_first[k];
    for (int l = 2; l <= c->depth; l++) {
        Level& B = c->lv[l];
        TcRowArgs ra;
        for (int k = 0; k < 8; k++) {
            ra.off[k] = fill[k];
            ra.start[k] = B.class_start[k];
            fill[k] += B.class_count[k];
        }
        if (B.nbox > 0) {
            LaunchScope ls(c, F_TREE);
            tc_rows_kernel<<<grid_for(B.nbox, 256), 256, 0, c->stream>>>(B.nbox, l, B.by_class, B.key, ra, S->rows);
        }
    }
    std::vector<TcTile> tl;
    for (int k = 0; k < 8; k++)
        for (int f = 0; f < total[k]; f += kTcRows) tl.push_back(TcTile{k, cls_first[k] + f, std::min(kTcRows, total[k] - f)});
    S->ntiles = (int)tl.size();
    if (S->ntiles > S->tiles_cap) {
        if (S->tiles) cudaFree(S->tiles);
        S->tiles = nullptr;
        S->tiles_cap = std::max(S->ntiles, 16);
        if (dev_alloc(reinterpret_cast<void**>(&S->tiles), sizeof(TcTile) * S->tiles_cap) != cudaSuccess)
            return POLFMM_ERR_OUT_OF_MEMORY;
    }
    if (S->ntiles &&
        cudaMemcpyAsync(S->tiles, tl.data(), sizeof(TcTile) * S->ntiles, cudaMemcpyHostToDevice, c->stream) !=
            cudaSuccess)
        return POLFMM_ERR_CUDA;
    // split the offsets so that the CTAs fill the SMs in one wave: one CTA per
    // SM with A in TMEM, two otherwise
    if (S->ntiles > 0) {
        int want = S->use_ws ? c->num_sms / S->ntiles : (2 * c->num_sms + S->ntiles - 1) / S->ntiles;
        c->m2l_chunks = std::max(1, std::min(want, 27));
    }
    return POLFMM_OK;
}

void m2l_tensor_launch(polfmm_ctx* c) {
    TcState* S = state(c);
    const TcSchedule& sch = S->sch;
    TcLevelPtrs lp{};
    for (int l = 2; l <= c->depth; l++) {
        Level& B = c->lv[l];
        lp.key[l] = B.key;
        lp.map[l] = B.map;
        lp.M[l] = (const float*)B.M;
        lp.Lp[l] = (float*)B.Lp;
        lp.cap[l] = B.cap;
        lp.row0[l] = (int)c->mrow0[l];
    }
    lp.Mall = (const float*)c->Mall;
    LaunchScope ls(c, F_M2L);
    dim3 grid(S->ntiles, c->m2l_chunks);
    if (S->use_ws)
        m2l_ws_kernel<<<grid, kWsThreads, S->smem, c->stream>>>(S->tiles, S->rows, lp, S->Bimg, S->Dsim,
                                                                c->tab.class_off, S->ws, c->ncoef, c->ld,
                                                                c->m2l_chunks, c->err);
    else
        m2l_tc_kernel<<<grid, kTcThreads, S->smem, c->stream>>>(S->tiles, S->rows, lp, S->Bimg, c->tab.class_off, sch,
                                                                c->ncoef, c->ld, c->m2l_chunks, c->err);
}

void m2l_tensor_release(polfmm_ctx* c) {
    TcState* S = state(c);
    if (!S) return;
    if (S->Bimg) cudaFree(S->Bimg);
    if (S->Dsim) cudaFree(S->Dsim);
    if (S->rows) cudaFree(S->rows);
    if (S->tiles) cudaFree(S->tiles);
    delete S;
    c->tc = nullptr;
}

}  // namespace polfmm
