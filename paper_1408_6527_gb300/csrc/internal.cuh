// Internal declarations of the polfmm CUDA library (not part of the C ABI).
//
// Data layout in HBM (all per-site arrays are in Morton-sorted site order):
//   pos_s  double[3n]   sorted positions             q_s, alpha_s double[n]
//   perm   int[n]       sorted index -> caller index
//   ploc   R[3n]        position minus its leaf centre (Angstrom), R = double
//                       (FP64 mode) or float (MIXED mode)
//   per level l = 0..depth: occupied boxes in Morton order (key, parent,
//   first child, child count), a dense Morton-key -> slot map of 8^l int32,
//   the boxes regrouped by octant class (key & 7), and the normalised
//   multipole / local coefficients m (nbox x ld) and f (nbox x ld):
//       m_n = M_n / h^|n|,  f_n = F_n h^(|n|+1),  h = box side at that level,
//   so that every stored coefficient is O(1) and one table of normalised
//   derivatives per integer offset serves every level.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/polfmm.h"

namespace polfmm {

constexpr int kMaxP = 10;
constexpr int kMaxDepth = 8;
constexpr int kNumOffsets = 189;    // interaction-list offsets per octant class
constexpr int kOffsetGrid = 7;      // offsets live in [-3, 3]^3
constexpr int kM2LTileBoxes = 32;   // target boxes per multipole-to-local tile
// targets per near-field block (heavy leaves span several blocks): the FP32
// kernel stages up to 1,024 sources per chunk and gains from serving more
// targets with each; the FP64 kernel stages 128 and is fastest at 16
constexpr int kLeafTargetsF32 = 64;
constexpr int kLeafTargetsF64 = 16;
constexpr int kLeafTargetsMin = 16;  // bound of the work-list length
__host__ __device__ constexpr int leaf_targets(bool fp32) { return fp32 ? kLeafTargetsF32 : kLeafTargetsF64; }

inline int ncoef_of(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

// position of the multi-index (x, y, z) in the coefficient order: degree
// o = x + y + z ascending, then x descending, then y descending (z ascending)
__host__ __device__ inline int mi_index(int x, int y, int z) {
    const int o = x + y + z, a = o - x;
    return o * (o + 1) * (o + 2) / 6 + a * (a + 1) / 2 + z;
}

// ---------------------------------------------------------------------------
// index tables for one expansion order p (device copies)
// ---------------------------------------------------------------------------
struct Tables {
    int p = 0, ncoef = 0, ld = 0;
    // multi-index of coefficient c packed as nx | ny << 8 | nz << 16 | |n| << 24
    int* mi = nullptr;
    double* inv_fact = nullptr;       // 1 / n!
    float* inv_fact_f = nullptr;
    int* up1 = nullptr;               // [ncoef][3]: index of n + e_d or -1
    int* up2 = nullptr;               // [ncoef][6]: index of n + e_d + e_e (xx xy xz yy yz zz) or -1
    int* pre = nullptr;               // [ncoef]: number of m with |m| <= p - |n| (a prefix)
    short* add = nullptr;             // [ncoef][ncoef]: index of n + m (valid for m < pre[n])
    int* dn1 = nullptr;               // [ncoef][3]: index of n - e_d or -1
    double* w4 = nullptr;             // [kMaxP + 1]: 4^-k / k!, 1-D weights of a quarter-side shift
    float* w4f = nullptr;
    double* rinv = nullptr;           // [kMaxP + 1]: 1 / k (0 at k = 0)
    float* rinvf = nullptr;
    double* D = nullptr;              // [343][ncoef] normalised derivatives of 1/r at integer offsets
    float* Df = nullptr;
    int* class_off = nullptr;         // [8][189] packed offsets (ox+3) | (oy+3)<<4 | (oz+3)<<8
    int* warp_out_ptr = nullptr;      // M2L output lists per warp (CSR, 8 warps)
    int* warp_out = nullptr;
    std::vector<int> h_mi;            // host copies used by the host code
};

// one tile of same-level, same-octant-class target boxes for the M2L kernel
// FP32 near field of the dipole solve, one work item: its leaf b, the leaf's
// first sorted site s0, the item's first target t_lo (relative to s0) and its
// target count, and the 27 source segments (first pair record, records) of
// the adjacent leaves, the leaf itself first (240 bytes, one bulk copy)
struct NearItem {
    int b, s0, t_lo, nt;
    int2 seg[27];
    int pad[2];
};
static_assert(sizeof(NearItem) == 240, "NearItem is copied as 15 x 16 bytes");

struct M2LTile {
    int level;
    int cls;
    int first;   // index into the level's by_class list
    int count;   // <= kM2LTileBoxes
};

struct LevelPtrs {
    int* key[kMaxDepth + 1];
    int* map[kMaxDepth + 1];
    int* by_class[kMaxDepth + 1];
    void* M[kMaxDepth + 1];
    void* Lp[kMaxDepth + 1];   // M2L partial outputs [chunk][cap][ld]
    int cap[kMaxDepth + 1];
};

struct Level {
    int nbox = 0, cap = 0;
    int* key = nullptr;
    int* map = nullptr;
    int* parent = nullptr;
    int* child0 = nullptr;
    int* nchild = nullptr;
    int* by_class = nullptr;
    int class_count[8] = {0};
    int class_start[8] = {0};
    void* M = nullptr;    // [cap][ld]
    void* Lp = nullptr;   // [m2l_chunks][cap][ld] M2L partial locals
    int* arrive = nullptr;  // [cap] children whose multipoles are done (0 between passes)
    void* Msh = nullptr;    // [cap][ld] multipoles shifted to the parent's centre (levels >= 3)
};

// profiling families
enum Family { F_TREE = 0, F_P2M, F_M2M, F_M2L, F_L2L, F_LEAF_DIPOLE, F_LEAF_STATIC, F_LEAF_FULL, F_SOLVER, F_ASSEMBLE, F_L2P, F_COUNT };

// leaf evaluation modes
enum LeafMode { LEAF_DIPOLE_E = 0, LEAF_CHARGE_PHI_E = 1, LEAF_FULL = 2 };

}  // namespace polfmm

struct polfmm_ctx {
    polfmm_options opt;
    int64_t n = 0;
    int p = 0, depth = 0, ncoef = 0, ld = 0;
    bool mixed = false;
    double lo[3] = {0, 0, 0};
    double side = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;

    // sorted site data
    double* pos_s = nullptr;
    double* q_s = nullptr;
    double* alpha_s = nullptr;
    double* inv_alpha_s = nullptr;  // 1 / alpha (0 where alpha = 0), sorted
    int* perm = nullptr;
    uint32_t* key_s = nullptr;
    void* ploc = nullptr;
    void* srcA = nullptr;         // packed (x, y, z, q) per sorted site, R4
    void* srcB = nullptr;         // packed (mu_x, mu_y, mu_z, 0) per sorted site, R4
    // leaves
    int* lstart = nullptr;
    int* lcount = nullptr;
    int* leaf_order = nullptr;    // leaves by descending near-field work
    int2* leaf_items = nullptr;   // near-field blocks: (leaf, first target), heaviest leaves first
    int* leaf_nitems = nullptr;   // device count of leaf_items
    // MIXED: sources of the dipole near field as pair records of 12 floats
    // (x0 x1 y0 y1 | z0 z1 nx0 nx1 | ny0 ny1 nz0 nz1, nu = -mu), each leaf padded to an
    // even count with a far, dipole-free source; positions once per tree,
    // dipoles once per pass
    float* near_pairs = nullptr;
    int* near_pbase = nullptr;     // first pair record of each leaf
    int* near_slot = nullptr;      // pair slot (2 record + half) of each sorted site
    polfmm::NearItem* near_items = nullptr;  // up to 2 per leaf item (32 targets each)
    int* near_nitems = nullptr;               // device count of near_items
    int leaf_items_cap = 0;       // capacity of leaf_items
    int leaf_items_grid = 0;      // launch bound of the current tree: leaves + n / leaf_targets + 1
    polfmm::Level lv[polfmm::kMaxDepth + 1];
    void* Mall = nullptr;                      // multipoles of all levels; level l from row mrow0[l]
    int64_t mrow0[polfmm::kMaxDepth + 1] = {0};
    int64_t mrow_zero = 0;                     // row after the last level's: all zeros
    polfmm::Tables tab;
    // M2L work list
    polfmm::M2LTile* tiles = nullptr;
    int ntiles = 0;
    int m2l_chunks = 1;
    int ntiles_cap = 0;

    // caller-order staging
    double* in_buf = nullptr;     // 6n doubles
    double* out_buf = nullptr;    // 10n doubles
    // static pass
    double* phiq = nullptr;
    double* Eq = nullptr;
    // solver vectors (3n each)
    double *mu = nullptr, *r = nullptr, *z = nullptr, *d = nullptr, *Ad = nullptr, *Td = nullptr;
    // full pass outputs
    double *phi_t = nullptr, *E_t = nullptr, *G_t = nullptr;
    // reductions
    double* partial = nullptr;    // [kRedSlots][kRedBlocks]
    double* scal = nullptr;       // device scalars
    double* h_scal = nullptr;     // pinned host mirror
    int* err = nullptr;           // device error word
    int* ticket = nullptr;        // last-block counter of the fused reductions (0 between kernels)
    double* leaf_partial = nullptr;  // [leaves] per-leaf partial sums of the fused d.Ad reduction
    // sort / scan scratch
    uint32_t* key_tmp = nullptr;
    int* val_tmp = nullptr;
    int* val_a = nullptr;
    int* counts = nullptr;
    int* scan_tmp = nullptr;
    int* flags = nullptr;
    size_t counts_cap = 0, scan_tmp_cap = 0;
    int* tree_cnt = nullptr;      // device tree counts ((kMaxDepth + 1) * 9 ints)
    int* h_counts = nullptr;      // pinned host copy of tree counts
    double* h_bbox = nullptr;     // pinned host bounding box

    // field charges and excluded pairs (Sec. II.A, III); see polaris.cu
    double* qE_s = nullptr;       // field charges q^E (sorted); null: q^E = q
    void* srcAE = nullptr;        // packed (x, y, z, q^E) per sorted site
    double* phiqE = nullptr;      // potential and field of the field charges (null: phiq, Eq)
    double* EqE = nullptr;
    double* dqE = nullptr;        // dU/dq^E of the last force pass (sorted)
    int64_t n_excl = 0;           // excluded pairs
    int n_excl_targets = 0;       // sites with at least one excluded partner
    int* excl_targets = nullptr;  // their caller indices
    int* excl_ptr = nullptr;      // [n_excl_targets + 1] offsets into excl_idx
    int* excl_idx = nullptr;      // [2 n_excl] partners, caller indices, ascending per site
    int* inv_perm = nullptr;      // [n] sorted index of each caller index
    size_t excl_cap = 0, excl_targets_cap = 0;
    int* excl_row = nullptr;      // [n] caller index -> row of excl_targets, -1 if none
    // Thole damping: parameter (0 = off), the damped pairs of the current tree
    // (CSR over sorted sites, partners in sorted order), alpha^(1/6) per sorted
    // site, the hash scratch, and the force-pass corrections (sorted order)
    double thole_a = 0.0;
    int predictor = 0;            // dipole predictor order for fmm_update_positions
    double* mu_hist = nullptr;    // [3n] caller order: the dipoles of the update before
    bool have_hist = false;
    int* th_ptr = nullptr;        // [n + 1]
    int* th_idx = nullptr;        // [th_cap]
    int64_t th_cap = 0, th_npairs = 0;
    double* a16 = nullptr;        // [n]
    float4* th_xa = nullptr;      // [n] position and alpha^(1/6) in FP32 (the pair search)
    float4* th_r = nullptr;       // [th_cap] MIXED: r_ij and 3 (lambda5 - 1) / r^5 per pair
    float* th_t3 = nullptr;       // [th_cap] MIXED: (lambda3 - 1) / r^3 per pair
    int* th_bucket = nullptr;     // [th_nb + 1] bucket starts
    int* th_count = nullptr;      // [th_nb] bucket counts
    int* th_member = nullptr;     // [n] sites grouped by bucket
    int4* th_cell = nullptr;      // [n] cell coordinates and bucket
    int* th_cnt = nullptr;        // [n + 64] pairs per site
    double* th_max = nullptr;     // device max of alpha^(1/6)
    int th_nb = 0;
    double* thE = nullptr;        // [3n] damped minus undamped dipole field
    double* thF = nullptr;        // [3n] damped minus undamped dipole-dipole force
    double* thdA = nullptr;       // [n] damping part of dU/dalpha
    bool have_dqE = false;        // dqE holds the last force pass's dU/dq^E

    bool have_mu = false;
    int64_t launches = 0;
    void* extra = nullptr;        // host-side bookkeeping of device allocations
    cudaStream_t cap_stream = nullptr;     // private stream for graph capture
    cudaStream_t side_stream = nullptr;    // near-field pairs concurrent with the far-field chain
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaGraphExec_t pcg_graph = nullptr;   // one PCG iteration of the current tree
    bool pcg_graph_dirty = true;
    int64_t pcg_graph_launches = 0;
    // PCG iterations until convergence as one graph: a while node whose body is
    // one iteration; the last kernel of the body sets the loop condition
    cudaGraph_t loop_g = nullptr;
    cudaGraph_t loop_body = nullptr;
    cudaGraphExec_t loop_exec = nullptr;
    cudaGraphConditionalHandle loop_cond = 0;
    bool loop_dirty = true;
    bool loop_failed = false;              // set-up refused: per-iteration graphs instead
    bool capturing_loop = false;           // kernels captured now take loop_cond
    int64_t loop_launches = 0;             // kernel launches per iteration of the body
    void* tc = nullptr;           // tensor-core M2L state
    void* ff = nullptr;           // FP32 CUDA-core M2L state
    // the dipole solve's own tree over the polarizable sites (T^mu, Sec. III)
    polfmm_ctx* tmu = nullptr;
    int64_t nmu = 0;              // its sites
    int* mu_rows = nullptr;       // [nmu] caller index of each of them (device)
    double* tmu_caller = nullptr; // [3 n] scratch in caller order
    double* tmu_rows = nullptr;   // [3 nmu] scratch in the second tree's caller order
    bool dipole_only = false;     // this context is such a tree: no charges, no static passes
    // profiling
    cudaEvent_t ev_pool[2 * 4096];
    int ev_used = 0;
    int ev_family[4096];
    bool ev_created = false;
    double prof_ms[polfmm::F_COUNT] = {0};
    int64_t prof_n[polfmm::F_COUNT] = {0};
};

namespace polfmm {

// every device or pinned-host allocation of the library goes through these two,
// so that fmm_testing_alloc_hook can make the k-th one fail
cudaError_t dev_alloc(void** p, size_t bytes);
// records the CUDA error for fmm_last_error and returns POLFMM_ERR_CUDA
int cuda_fail(cudaError_t e, const char* where);
cudaError_t host_alloc(void** p, size_t bytes);

// launch bookkeeping / profiling around one kernel launch
struct LaunchScope {
    polfmm_ctx* c;
    int fam;
    int slot;
    LaunchScope(polfmm_ctx* ctx, int family);
    ~LaunchScope();
};
void profile_flush(polfmm_ctx* c);

// tree.cu
int tree_root_box(polfmm_ctx* c, const double* x_dev, double* part_dev, double* h_pinned);
int tree_build(polfmm_ctx* c, const double* x_in);
int tree_tables(polfmm_ctx* c, const double* x_in, const double* q_in, const double* a_in);
size_t tree_scan_scratch(int64_t n);
size_t tree_count_scratch(int64_t n);
int scan_exclusive(polfmm_ctx* c, const int* in, int* out, int n, int* total_dev);

// fmm_ops.cu
// pcg: when non-null in a solver pass, the kernel that completes the field
// also forms Ad = d/alpha - T d and the sum d.Ad (scal[S_DAD]); returns true
// if it did (false: the caller runs the separate kernel)
bool fmm_pass(polfmm_ctx* c, int mode, bool use_q, const double* mu_sorted, double* phi, double* E,
              double* G, bool mu_packed = false, bool pcg = false);
int m2l_setup(polfmm_ctx* c);
// m2l_ffma.cu: the FP32 CUDA-core M2L (MIXED, p <= 6): per-tree lists, launch
bool m2l_ffma_wanted(const polfmm_ctx* c);
bool m2l_ffma_enabled(polfmm_ctx* c);
int m2l_ffma_prepare(polfmm_ctx* c);
void m2l_ffma_launch(polfmm_ctx* c);
void m2l_ffma_release(polfmm_ctx* c);
void pack_positions(polfmm_ctx* c);
// MIXED: per-tree tables of the FP32 dipole near field (pair records, work items)
int near_tables(polfmm_ctx* c);
size_t source_record_bytes(bool mixed);

// solver.cu
void gather_sites(polfmm_ctx* c, const double* src_caller, double* dst_sorted, int comps);
void scatter_sites(polfmm_ctx* c, const double* src_sorted, double* dst_caller, int comps);
void solver_init(polfmm_ctx* c, bool warm);
void solver_pcg_step(polfmm_ctx* c);
void solver_loop_setup(polfmm_ctx* c, double tol, int max_iter);
void solver_jacobi_step(polfmm_ctx* c);
void energy_and_gradients(polfmm_ctx* c, double* forces_caller, double* dq_caller,
                          double* dalpha_caller, bool want_f, bool want_dq, bool want_da);
void energy_stationary(polfmm_ctx* c);
// residual growths in a row after which a solve stops as not converged
constexpr int kStagnationIters = 3;
void mask_dipoles(polfmm_ctx* c, double* v);

// polaris.cu: subtract the excluded pairs' direct terms from the outputs of a
// pass (leaf_mode: the pass's sources), and the caller -> sorted map they use
void exclusion_correct(polfmm_ctx* c, int leaf_mode, const double* w_sorted, const double* mu_sorted, double* phi,
                       double* E, double* G, cudaStream_t st);
void exclusion_inv_perm(polfmm_ctx* c);
// Thole damping (polaris.cu): the pair list of the current tree, the solve's
// field correction (E += (T^damp - T) mu, after the near field), and the
// force-pass corrections into thE, thF, thdA
int thole_pairs(polfmm_ctx* c);
void thole_field(polfmm_ctx* c, const double* mu_sorted, double* E, cudaStream_t st);
void thole_forces(polfmm_ctx* c);
// the field that polarizes the sites: that of the field charges when set
inline const double* polarizing_field(const polfmm_ctx* c) { return c->EqE ? c->EqE : c->Eq; }

// device scalar slots
enum Scal {
    S_RZ = 0, S_RZ_NEW, S_DAD, S_RR, S_BB, S_UQQ, S_MUEQ, S_MUEMU, S_AMU, S_BETA, S_TOL, S_MAXIT, S_ITER,
    S_GROW,  // consecutive iterations whose residual grew (stagnation / divergence test)
    S_COUNT
};
constexpr int kRedBlocks = 256;
constexpr int kRedSlots = 8;

// helpers
__host__ __device__ inline uint32_t spread3(uint32_t v) {
    v &= 0x3ff;
    v = (v | (v << 16)) & 0x030000FF;
    v = (v | (v << 8)) & 0x0300F00F;
    v = (v | (v << 4)) & 0x030C30C3;
    v = (v | (v << 2)) & 0x09249249;
    return v;
}
__host__ __device__ inline uint32_t compact3(uint32_t v) {
    v &= 0x09249249;
    v = (v ^ (v >> 2)) & 0x030C30C3;
    v = (v ^ (v >> 4)) & 0x0300F00F;
    v = (v ^ (v >> 8)) & 0x030000FF;
    v = (v ^ (v >> 16)) & 0x000003FF;
    return v;
}
__host__ __device__ inline uint32_t morton3(uint32_t i, uint32_t j, uint32_t k) {
    return spread3(i) | (spread3(j) << 1) | (spread3(k) << 2);
}

inline int grid_for(int64_t n, int block) { return (int)((n + block - 1) / block); }

// Programmatic dependent launch (the solver iteration's chain of kernels).
// pdl_wait: a kernel launched with programmatic stream serialization waits here
// until the previous kernel of its stream has completed and its writes are
// visible (without the attribute it returns at once); nothing that kernel
// writes may be read, and nothing it reads may be written, before this call.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
// lets the next kernel of the stream be scheduled; called by each block when
// its work is done, so that waiting blocks never hold an SM this grid needs
__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// launch with programmatic stream serialization when pdl is set (the kernel
// calls pdl_wait before touching its predecessor's output)
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

}  // namespace polfmm

#define POLFMM_CUDA_TRY(expr)                         \
    do {                                              \
        cudaError_t e_ = (expr);                      \
        if (e_ != cudaSuccess) return POLFMM_ERR_CUDA; \
    } while (0)
