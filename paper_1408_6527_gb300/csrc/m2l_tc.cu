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

#include "internal.cuh"

namespace polfmm {

constexpr int kTcRows = 128;
constexpr int kTcThreads = 128;
constexpr int kTcMaxSteps = 24;  // input steps of 8 (p <= 8: KP <= 168)
constexpr uint64_t kTcWaitNs = 2000000000ull;  // 2 s bound on every wait

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

struct TcState {
    TcSchedule sch;
    bool tmem_a = false;                     // A operands in TMEM (m2l_tca_kernel), else in shared memory
    size_t row_stride = 0;                   // m2l_tca_kernel: floats per gathered row
    float* Bimg = nullptr;                   // [343][2][bpart]
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
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// try_wait that lets the hardware suspend the thread for up to hint_ns
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t* bar, uint32_t phase, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// bounded wait of threads that have nothing else to do: suspended between polls
__device__ __forceinline__ bool mbar_wait_bounded_idle(uint64_t* bar, uint32_t phase) {
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait_hint(bar, phase, 1000u))
        if (global_ns() - t0 >= kTcWaitNs) return false;
    return true;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase) {
    if (mbar_try_wait(bar, phase)) return true;
    const uint64_t t0 = global_ns();
    while (global_ns() - t0 < kTcWaitNs)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

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
                tc_fence_after();
                for (int j = 0; j < sch.nmma; j++) {
                    const TcMma m = mtab[j];
                    mma_tf32(tmem, m.a, m.b, m.idesc, m.acc);
                }
                mma_commit(&bar_m);
            }
        }
        pb ^= 1;
        // wait for this offset's MMAs, then fold the accumulator into the running
        // sum with round-to-nearest FP32 additions (warp w: TMEM lanes 32 w ..)
        __syncthreads();
        if (fail_sh) break;
        if (!mbar_wait_bounded(&bar_m, pm)) atomicOr(err, 4), fail_sh = 1;
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
// the tensor-core M2L kernel with A in tensor memory (one CTA per SM, p <= 6)
//
// Same contraction and MMA schedule as m2l_tc_kernel.  Eight worker warps
// gather FP32 rows two offsets ahead through a two-stage shared-memory ring,
// split them into TF32 high / low parts written straight into TMEM (lane =
// box, column = input) and fold each offset's accumulator into a running sum
// held in registers; a ninth warp issues the MMAs, which read A from TMEM and
// only the K_o image (double-buffered) from shared memory.  A is
// double-buffered in TMEM, so the split of offset t + 1 runs while the MMAs of
// offset t execute.  TMEM columns: accumulator [0, NP), A buffer b at
// NP + 2 KP b (high part) and NP + 2 KP b + KP (low part).
// Worker warp w owns TMEM lanes 32 (w % 4) .. + 31 and the 16-column chunks
// of parity w / 4.
// ---------------------------------------------------------------------------
constexpr int kTcaWorkers = 256;
constexpr int kTcaThreads = kTcaWorkers + 32;
constexpr int kTcaMaxNP = 128;  // running sum: NP / 2 registers per thread

struct TcaMma {
    uint64_t b;         // B descriptor
    uint32_t a_tmem;    // TMEM address of the A operand
    uint32_t idesc;
};

__device__ __forceinline__ void workers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kTcaWorkers) : "memory"); }

__global__ void __launch_bounds__(kTcaThreads, 1) m2l_tca_kernel(const TcTile* __restrict__ tiles,
                                                                 const int2* __restrict__ rows, TcLevelPtrs lp,
                                                                 const float* __restrict__ Bimg,
                                                                 const int* __restrict__ class_off, TcSchedule sch,
                                                                 int ncoef, int ld, int nchunk, int rs,
                                                                 int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int KP = sch.KP, NP = sch.NP;
    // gather ring [2][kTcRows][rs] floats, K_o images [2][hi | lo], MMA table
    float* const ring = reinterpret_cast<float*>(smem_raw);
    float* const Bbuf = ring + 2 * (size_t)kTcRows * rs;
    TcaMma* const mtab = reinterpret_cast<TcaMma*>(Bbuf + 4 * (size_t)sch.bpart);  // [2][nmma]
    __shared__ __align__(8) uint64_t bar_b[2];  // K_o image landed
    __shared__ __align__(8) uint64_t bar_m;     // MMAs of an offset done
    __shared__ uint32_t tmem_base_sh;
    __shared__ int fail_sh;
    __shared__ int s_src[4][kTcRows];
    __shared__ int s_lvl[kTcRows];
    __shared__ int s_off[kNumOffsets];  // this CTA's offsets (packed)

    const TcTile tile = tiles[blockIdx.x];
    const int chunk = blockIdx.y;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const bool worker = warp < kTcaWorkers / 32;
    const int quarter = warp & 3, half = (warp >> 2) & 1;
    const int myrow = quarter * 32 + lane;

    if (warp == 0) tmem_alloc(&tmem_base_sh, 512u);
    if (tid == 0) {
        mbar_init(&bar_b[0], 1);
        mbar_init(&bar_b[1], 1);
        mbar_init(&bar_m, 1);
        fail_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    const uint32_t abuf_cols = 2u * (uint32_t)KP;

    // target box of row tid (threads 0..127), any level >= 2
    int level = 0, slot = -1, bx = 0, by = 0, bz = 0;
    if (tid < kTcRows && tid < tile.count) {
        const int2 r = rows[tile.first + tid];
        level = r.x;
        slot = r.y;
        const uint32_t k = (uint32_t)lp.key[level][slot];
        bx = (int)compact3(k);
        by = (int)compact3(k >> 1);
        bz = (int)compact3(k >> 2);
    }
    if (tid < kTcRows) s_lvl[tid] = level;
    const int nside = 1 << level;
    const int* map = slot >= 0 ? lp.map[level] : nullptr;

    const int per = (kNumOffsets + nchunk - 1) / nchunk;
    const int t0 = min(kNumOffsets, chunk * per), t1 = min(kNumOffsets, t0 + per);
    const int nt = t1 - t0;
    const uint32_t bbytes = (uint32_t)sch.bpart * 4u;

    // MMA table for each buffer pair (A buffer b, image buffer b): product
    // (A_hi B_lo, A_lo B_hi, A_hi B_hi) x input step k, complete descriptors so
    // that the issuing thread does one shared load per MMA
    for (int jb = tid; jb < 2 * sch.nmma; jb += kTcaThreads) {
        const int bi = jb / sch.nmma, j = jb - bi * sch.nmma;
        const int prod = j / sch.nks, k = j - prod * sch.nks;
        const int w = sch.width[k];
        const uint32_t b_hi = smem_u32(Bbuf) + (uint32_t)bi * 2u * bbytes, b_lo = b_hi + bbytes;
        TcaMma m;
        m.b = smem_desc((prod == 0 ? b_lo : b_hi) + (uint32_t)sch.soff[k] * 4u, (uint32_t)(w / 8) * 128u, 128u);
        m.a_tmem = tmem + (uint32_t)NP + abuf_cols * (uint32_t)bi + (prod == 1 ? (uint32_t)KP : 0u) + 8u * (uint32_t)k;
        m.idesc = idesc_tf32(kTcRows, w);
        mtab[jb] = m;
    }

    // source row of this thread's box (threads 0..127) for offset t: the map load
    // is issued one iteration before its value is stored (lookup_load, then the
    // store of the previous result), so its latency stays off the worker path
    for (int t = t0 + tid; t < t1; t += kTcaThreads) s_off[t - t0] = class_off[tile.cls * kNumOffsets + t];
    __syncthreads();
    auto lookup_load = [&](int t) -> int {
        int src = -1;
        if (tid < kTcRows && t < t1 && slot >= 0) {
            const int o = s_off[t - t0];
            const int ox = (o & 15) - 3, oy = ((o >> 4) & 15) - 3, oz = ((o >> 8) & 15) - 3;
            const int ax = bx - ox, ay = by - oy, az = bz - oz;
            if (ax >= 0 && ay >= 0 && az >= 0 && ax < nside && ay < nside && az < nside)
                src = map[morton3(ax, ay, az)];
        }
        return src;
    };
    auto lookup_store = [&](int t, int src) {
        if (tid < kTcRows && t < t1) s_src[(t - t0) & 3][tid] = src;
    };
    // workers: FP32 rows of offset t into ring stage (t - t0) & 1, 8 rows x 64
    // contiguous bytes per instruction; inputs ncoef .. KP - 1 are zero; always
    // commits one group
    const int rr = lane & 7, cq = lane >> 3;
    const int nch = KP / 4;
    auto gather = [&](int t) {
        if (t < t1) {
            const int* srcs = s_src[(t - t0) & 3];
            float* dst = ring + (size_t)((t - t0) & 1) * kTcRows * rs;
            for (int rg = warp; rg < kTcRows / 8; rg += kTcaWorkers / 32) {
                const int row = rg * 8 + rr;
                const int src = srcs[row];
                const float* g = src >= 0 ? lp.M[s_lvl[row]] + (size_t)src * ld : Bimg;
                float* drow = dst + (size_t)row * rs;
                for (int c = cq; c < nch; c += 4) {
                    const int valid = src >= 0 ? min(4, max(0, ncoef - 4 * c)) : 0;
                    cp_async16(drow + 4 * c, valid ? g + 4 * c : Bimg, (uint32_t)(4 * valid));
                }
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    // workers: ring stage of offset t -> TMEM A buffer (t - t0) & 1 (row myrow)
    auto split = [&](int t) {
        const float* src = ring + (size_t)((t - t0) & 1) * kTcRows * rs + (size_t)myrow * rs;
        const uint32_t col = (uint32_t)NP + abuf_cols * (uint32_t)((t - t0) & 1);
        for (int c0 = 8 * half; c0 < KP; c0 += 16) {
            const float4 v0 = *reinterpret_cast<const float4*>(src + c0);
            const float4 v1 = *reinterpret_cast<const float4*>(src + c0 + 4);
            float h[8], l[8];
            tf32_split(v0.x, h[0], l[0]);
            tf32_split(v0.y, h[1], l[1]);
            tf32_split(v0.z, h[2], l[2]);
            tf32_split(v0.w, h[3], l[3]);
            tf32_split(v1.x, h[4], l[4]);
            tf32_split(v1.y, h[5], l[5]);
            tf32_split(v1.z, h[6], l[6]);
            tf32_split(v1.w, h[7], l[7]);
            tmem_st8(lane_base + col + (uint32_t)c0, h);
            tmem_st8(lane_base + col + (uint32_t)KP + (uint32_t)c0, l);
        }
        tmem_wait_st();
    };
    auto load_b = [&](int t) {  // issuer: K_o image of offset t into buffer (t - t0) & 1
        const int o = class_off[tile.cls * kNumOffsets + t];
        const int ox = (o & 15) - 3, oy = ((o >> 4) & 15) - 3, oz = ((o >> 8) & 15) - 3;
        const int oidx = (ox + 3) + kOffsetGrid * ((oy + 3) + kOffsetGrid * (oz + 3));
        const float* img = Bimg + (size_t)oidx * 2 * sch.bpart;
        const int bi = (t - t0) & 1;
        float* bh = Bbuf + (size_t)bi * 2 * sch.bpart;
        mbar_arrive_expect_tx(&bar_b[bi], 2 * bbytes);
        bulk_g2s(bh, img, bbytes, &bar_b[bi]);
        bulk_g2s(bh + sch.bpart, img + sch.bpart, bbytes, &bar_b[bi]);
    };

    // running sum of this thread's row and column chunks c0 = 16 half + 32 j
    float sum[kTcaMaxNP / 32][16];
#pragma unroll
    for (int j = 0; j < kTcaMaxNP / 32; j++)
#pragma unroll
        for (int k = 0; k < 16; k++) sum[j][k] = 0.f;

    // prologue: lookups of four offsets, gathers of two, split of the first, images of two
    for (int t = t0; t < t0 + 4; t++) lookup_store(t, lookup_load(t));
    int pend = lookup_load(t0 + 4);  // in flight until the first iteration stores it
    __syncthreads();
    const bool issuer = warp == kTcaWorkers / 32 && lane == 0;
    uint32_t pbits = 0, pm = 0;  // phases: image buffers (bit b), MMA barrier
    if (worker) {
        gather(t0);
        gather(t0 + 1);
        if (nt > 0) {
            asm volatile("cp.async.wait_group 1;" ::: "memory");
            workers_sync();
            split(t0);
            workers_sync();
        }
        gather(t0 + 2);
    } else if (issuer) {
        if (nt > 0) load_b(t0);
        if (nt > 1) load_b(t0 + 1);
    }
    tc_fence_before();
    __syncthreads();

    for (int i = 0; i < nt; i++) {
        const int t = t0 + i;
        tc_fence_after();
        if (issuer) {
            const int bi = i & 1;
            if (!mbar_wait_bounded(&bar_b[bi], (pbits >> bi) & 1u)) {
                atomicOr(err, 4);
                fail_sh = 1;
            } else {
                const TcaMma* tb = mtab + bi * sch.nmma;
                const int nm = sch.nmma;
                mma_tf32_ta(tmem, tb[0].a_tmem, tb[0].b, tb[0].idesc, 0u);
                int j = 1;
                for (; j + 4 <= nm; j += 4) {  // table entries loaded ahead of their MMAs
                    const TcaMma m0 = tb[j], m1 = tb[j + 1], m2 = tb[j + 2], m3 = tb[j + 3];
                    mma_tf32_ta(tmem, m0.a_tmem, m0.b, m0.idesc, 1u);
                    mma_tf32_ta(tmem, m1.a_tmem, m1.b, m1.idesc, 1u);
                    mma_tf32_ta(tmem, m2.a_tmem, m2.b, m2.idesc, 1u);
                    mma_tf32_ta(tmem, m3.a_tmem, m3.b, m3.idesc, 1u);
                }
                for (; j < nm; j++) {
                    const TcaMma m = tb[j];
                    mma_tf32_ta(tmem, m.a_tmem, m.b, m.idesc, 1u);
                }
                mma_commit(&bar_m);
            }
            pbits ^= 1u << bi;
            // the image buffer of offset t is free once its MMAs are done
            if (!mbar_wait_bounded(&bar_m, pm)) atomicOr(err, 4), fail_sh = 1;
            if (i + 2 < nt) load_b(t + 2);
        } else if (worker) {
            // while the MMAs of offset t run: split offset t + 1 into the other A buffer
            if (i + 1 < nt) {
                asm volatile("cp.async.wait_group 1;" ::: "memory");
                workers_sync();
                split(t + 1);
                workers_sync();  // every row of the stage is read: refill it
                gather(t + 3);
                lookup_store(t + 4, pend);
                pend = lookup_load(t + 5);
            }
            // fold offset t into the running sum (suspended while the MMAs run, so
            // that the issuing warp keeps its issue slots)
            if (!mbar_wait_bounded_idle(&bar_m, pm)) atomicOr(err, 4), fail_sh = 1;
            tc_fence_after();
#pragma unroll
            for (int j = 0; j < kTcaMaxNP / 32; j++) {
                const int c0 = 16 * half + 32 * j;
                if (c0 < NP) {
                    float a[16];
                    tmem_ld16(lane_base + (uint32_t)c0, a);
#pragma unroll
                    for (int k = 0; k < 16; k++) sum[j][k] += a[k];
                }
            }
        }
        pm ^= 1;
        tc_fence_before();
        __syncthreads();  // A buffer of t + 1 written, accumulator read: the next MMAs may start
        if (fail_sh) break;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    // epilogue: row myrow, this warp's column chunks
    if (worker && !fail_sh && myrow < tile.count) {
        const int2 r = rows[tile.first + myrow];
        float* out = lp.Lp[r.x] + ((size_t)chunk * lp.cap[r.x] + r.y) * ld;
#pragma unroll
        for (int j = 0; j < kTcaMaxNP / 32; j++) {
            const int c0 = 16 * half + 32 * j;
            if (c0 < NP)
                for (int k = 0; k < 16; k++)
                    if (c0 + k < ncoef) out[c0 + k] = sum[j][k];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512u);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static TcState* state(polfmm_ctx* c) { return reinterpret_cast<TcState*>(c->tc); }

bool m2l_tensor_enabled(polfmm_ctx* c) {
    TcState* S = state(c);
    return c->mixed && c->opt.m2l_impl != POLFMM_M2L_SIMT && S && S->ready && S->ntiles > 0;
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

int m2l_tensor_prepare(polfmm_ctx* c) {
    if (!c->mixed || c->opt.m2l_impl == POLFMM_M2L_SIMT || c->p > 8 || c->depth < 2) return POLFMM_OK;
    TcState* S = state(c);
    if (!S) {
        S = new TcState();
        c->tc = S;
        const int p = c->p, nc = c->ncoef;
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
        const size_t limit = 227 * 1024;
        // A in TMEM (accumulator, running sum, A_hi, A_lo within the 512 columns of
        // an SM) with a two-stage gather ring and double-buffered images; else one
        // shared-memory stage per CTA and two CTAs per SM
        S->row_stride = (size_t)sch.KP + 4;  // odd multiple of 4 floats: conflict-free row reads
        const size_t tca_smem = sizeof(float) * (2 * (size_t)kTcRows * S->row_stride + 4 * (size_t)sch.bpart) +
                                2 * sizeof(TcaMma) * (size_t)sch.nmma;
        S->tmem_a = sch.NP + 4 * sch.KP <= 512 && sch.NP <= kTcaMaxNP && tca_smem <= limit;
        S->smem = S->tmem_a ? tca_smem : (size_t)sch.tab_off + sizeof(TcMma) * (size_t)sch.nmma;
        if (S->smem > limit) {
            delete S;
            c->tc = nullptr;
            return POLFMM_OK;  // does not fit: the SIMT kernel stays in use
        }
        // K_o images, one slab per input step: slab k holds outputs 0 .. width[k] - 1
        // x inputs 8k .. 8k + 7 in the core-matrix layout, element (n, kk) at
        // (kk/4)*(width/8)*32 + (n/8)*32 + (n%8)*4 + kk%4; split into a TF32 part and residual
        std::vector<double> Dd((size_t)343 * nc);
        if (cudaMemcpy(Dd.data(), c->tab.D, sizeof(double) * Dd.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
            return POLFMM_ERR_CUDA;
        std::vector<int> lut((p + 1) * (p + 1) * (p + 1), -1);
        std::vector<int> mx(nc), my(nc), mz(nc);
        for (int k = 0; k < nc; k++) {
            int v = c->tab.h_mi[k];
            mx[k] = v & 0xff;
            my[k] = (v >> 8) & 0xff;
            mz[k] = (v >> 16) & 0xff;
            lut[(mx[k] * (p + 1) + my[k]) * (p + 1) + mz[k]] = k;
        }
        std::vector<float> img((size_t)343 * 2 * sch.bpart, 0.f);
        for (int oi = 0; oi < 343; oi++) {
            float* hi = &img[(size_t)oi * 2 * sch.bpart];
            float* lo = hi + sch.bpart;
            for (int k = 0; k < sch.nks; k++) {
                const int w = sch.width[k];
                for (int n = 0; n < w; n++)
                    for (int kk = 0; kk < 8; kk++) {
                        const int m = 8 * k + kk;
                        float v = 0.f;
                        if (n < nc && m < nc && degree_of(n, p) + degree_of(m, p) <= p) {
                            int s2 = lut[((mx[n] + mx[m]) * (p + 1) + my[n] + my[m]) * (p + 1) + mz[n] + mz[m]];
                            v = (float)Dd[(size_t)oi * nc + s2];
                        }
                        const size_t pos = sch.soff[k] + (size_t)(kk / 4) * (w / 8) * 32 + (n / 8) * 32 + (n % 8) * 4 + kk % 4;
                        const float h = tf32_round(v);
                        hi[pos] = h;
                        lo[pos] = v - h;
                    }
            }
        }
        if (dev_alloc(reinterpret_cast<void**>(&S->Bimg), sizeof(float) * img.size()) != cudaSuccess)
            return POLFMM_ERR_OUT_OF_MEMORY;
        if (cudaMemcpy(S->Bimg, img.data(), sizeof(float) * img.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return POLFMM_ERR_CUDA;
        size_t rows_cap = 0;
        for (int l = 2; l <= c->depth; l++) rows_cap += c->lv[l].cap;
        if (dev_alloc(reinterpret_cast<void**>(&S->rows), sizeof(int2) * std::max<size_t>(rows_cap, 1)) != cudaSuccess)
            return POLFMM_ERR_OUT_OF_MEMORY;
        cudaError_t e1 = S->tmem_a ? cudaFuncSetAttribute(m2l_tca_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
        int want = S->tmem_a ? c->num_sms / S->ntiles : (2 * c->num_sms + S->ntiles - 1) / S->ntiles;
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
    }
    LaunchScope ls(c, F_M2L);
    dim3 grid(S->ntiles, c->m2l_chunks);
    if (S->tmem_a)
        m2l_tca_kernel<<<grid, kTcaThreads, S->smem, c->stream>>>(S->tiles, S->rows, lp, S->Bimg, c->tab.class_off,
                                                                  sch, c->ncoef, c->ld, c->m2l_chunks,
                                                                  (int)S->row_stride, c->err);
    else
        m2l_tc_kernel<<<grid, kTcThreads, S->smem, c->stream>>>(S->tiles, S->rows, lp, S->Bimg, c->tab.class_off, sch,
                                                                c->ncoef, c->ld, c->m2l_chunks, c->err);
}

void m2l_tensor_release(polfmm_ctx* c) {
    TcState* S = state(c);
    if (!S) return;
    if (S->Bimg) cudaFree(S->Bimg);
    if (S->rows) cudaFree(S->rows);
    if (S->tiles) cudaFree(S->tiles);
    delete S;
    c->tc = nullptr;
}

}  // namespace polfmm
