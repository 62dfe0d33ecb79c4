// C ABI of the polfmm library (declared in include/polfmm.h): context
// lifetime, the three calls of the paper's force procedure (Sec. III: static
// pass in fmm_build, iterative dipoles in fmm_solve_induced_dipoles, energy
// and forces in fmm_energy_forces), and the index / derivative tables.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <utility>
#include <new>
#include <string>
#include <vector>

#include "internal.cuh"

namespace polfmm {

thread_local char g_last_error[256] = "";

int cuda_fail(cudaError_t e, const char* where) {
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
    return POLFMM_ERR_CUDA;
}
// linear dipole prediction: cur <- 2 cur - hist, hist <- old cur
__global__ void extrapolate_kernel(int64_t n3, double* __restrict__ cur, double* __restrict__ hist) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n3) return;
    const double v = cur[k];
    cur[k] = 2.0 * v - hist[k];
    hist[k] = v;
}
// rows of a caller-order array: dst[k] = src[rows[k]] (take) or dst[rows[k]] = src[k] (put),
// comps values per row
__global__ void take_rows_kernel(int64_t m, int comps, const int* __restrict__ rows, const double* __restrict__ src,
                                 double* __restrict__ dst) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= m * comps) return;
    const int64_t r = k / comps, c = k - r * comps;
    dst[k] = src[(int64_t)rows[r] * comps + c];
}
__global__ void put_rows_kernel(int64_t m, int comps, const int* __restrict__ rows, const double* __restrict__ src,
                                double* __restrict__ dst) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= m * comps) return;
    const int64_t r = k / comps, c = k - r * comps;
    dst[(int64_t)rows[r] * comps + c] = src[k];
}
int fmm_ops_init_attributes(polfmm_ctx* c);
size_t m2l_simt_smem(int ncoef, size_t rsize);
int m2l_tensor_prepare(polfmm_ctx* c);
void m2l_tensor_release(polfmm_ctx* c);
}  // namespace polfmm

using namespace polfmm;

// ---------------------------------------------------------------------------
// launch bookkeeping and profiling
// ---------------------------------------------------------------------------
namespace polfmm {

// allocation counter and the planted failure of fmm_testing_alloc_hook
static std::atomic<int64_t> g_alloc_count{0};
static std::atomic<int64_t> g_alloc_fail_at{-1};

static bool alloc_should_fail() {
    const int64_t k = g_alloc_count.fetch_add(1);
    int64_t at = g_alloc_fail_at.load();
    return at >= 0 && k == at && g_alloc_fail_at.compare_exchange_strong(at, -1);
}

cudaError_t dev_alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (alloc_should_fail()) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
    }
    return e;
}

cudaError_t host_alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (alloc_should_fail()) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMallocHost(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
    }
    return e;
}

LaunchScope::LaunchScope(polfmm_ctx* ctx, int family) : c(ctx), fam(family), slot(-1) {
    c->launches++;
    if (c->opt.profile && c->ev_created) {
        if (c->ev_used >= 4096) profile_flush(c);
        slot = c->ev_used++;
        c->ev_family[slot] = fam;
        cudaEventRecord(c->ev_pool[2 * slot], c->stream);
    }
}

LaunchScope::~LaunchScope() {
    if (slot >= 0) cudaEventRecord(c->ev_pool[2 * slot + 1], c->stream);
}

void profile_flush(polfmm_ctx* c) {
    if (!c->ev_created || c->ev_used == 0) return;
    cudaStreamSynchronize(c->stream);
    for (int s = 0; s < c->ev_used; s++) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev_pool[2 * s], c->ev_pool[2 * s + 1]) == cudaSuccess) {
            c->prof_ms[c->ev_family[s]] += ms;
            c->prof_n[c->ev_family[s]]++;
        }
    }
    c->ev_used = 0;
}

}  // namespace polfmm

// ---------------------------------------------------------------------------
// tables
// ---------------------------------------------------------------------------
namespace {

double factorial(int k) {
    double f = 1.0;
    for (int i = 2; i <= k; i++) f *= i;
    return f;
}

struct HostMI {
    int p, nc;
    std::vector<int> nx, ny, nz, s;
    std::vector<int> lut;  // (p+1)^3
    explicit HostMI(int p_) : p(p_) {
        nc = ncoef_of(p);
        lut.assign((p + 1) * (p + 1) * (p + 1), -1);
        for (int o = 0; o <= p; o++)
            for (int x = o; x >= 0; x--)
                for (int y = o - x; y >= 0; y--) {
                    int z = o - x - y;
                    lut[(x * (p + 1) + y) * (p + 1) + z] = (int)nx.size();
                    nx.push_back(x);
                    ny.push_back(y);
                    nz.push_back(z);
                    s.push_back(o);
                }
    }
    int at(int x, int y, int z) const {
        if (x < 0 || y < 0 || z < 0 || x + y + z > p) return -1;
        return lut[(x * (p + 1) + y) * (p + 1) + z];
    }
};

// d^n (1/r) at integer offsets for |n| <= p.  Recurrence from the Euler
// identity of the degree -1 homogeneous function 1/r and its harmonicity:
//   |n| r^2 a_n = -(2|n|-1) sum_d n_d R_d a_{n-e_d} - (|n|-1) sum_d n_d (n_d-1) a_{n-2e_d}
void derivative_table(const HostMI& t, const double R[3], double* a) {
    double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
    a[0] = 1.0 / sqrt(r2);
    for (int c = 1; c < t.nc; c++) {
        int n[3] = {t.nx[c], t.ny[c], t.nz[c]};
        int s = t.s[c];
        double acc = 0.0;
        for (int d = 0; d < 3; d++) {
            int m[3] = {n[0], n[1], n[2]};
            if (n[d] >= 1) {
                m[d] = n[d] - 1;
                acc += (2.0 * s - 1.0) * n[d] * R[d] * a[t.at(m[0], m[1], m[2])];
            }
            if (n[d] >= 2) {
                m[d] = n[d] - 2;
                acc += (s - 1.0) * n[d] * (n[d] - 1.0) * a[t.at(m[0], m[1], m[2])];
            }
        }
        a[c] = -acc / (s * r2);
    }
}

template <typename T>
int upload(const std::vector<T>& h, T** d, cudaStream_t st) {
    if (h.empty()) {
        *d = nullptr;
        return POLFMM_OK;
    }
    if (dev_alloc(reinterpret_cast<void**>(d), sizeof(T) * h.size()) != cudaSuccess) return POLFMM_ERR_OUT_OF_MEMORY;
    if (cudaMemcpyAsync(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return POLFMM_ERR_CUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? POLFMM_OK : POLFMM_ERR_CUDA;
}

int build_tables(polfmm_ctx* c) {
    const int p = c->p;
    HostMI t(p);
    Tables& T = c->tab;
    T.p = p;
    T.ncoef = t.nc;
    T.ld = c->ld;
    const int nc = t.nc;
    std::vector<int> mi(nc), pre(nc), up1(3 * nc), dn1(3 * nc), up2(6 * nc);
    std::vector<double> inv_fact(nc);
    std::vector<float> inv_fact_f(nc);
    std::vector<short> add((size_t)nc * nc, (short)-1);
    static const int hd[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    for (int k = 0; k < nc; k++) {
        mi[k] = t.nx[k] | (t.ny[k] << 8) | (t.nz[k] << 16) | (t.s[k] << 24);
        inv_fact[k] = 1.0 / (factorial(t.nx[k]) * factorial(t.ny[k]) * factorial(t.nz[k]));
        inv_fact_f[k] = (float)inv_fact[k];
        pre[k] = ncoef_of(p - t.s[k]);
        for (int d = 0; d < 3; d++) {
            int m[3] = {t.nx[k], t.ny[k], t.nz[k]};
            m[d]++;
            up1[3 * k + d] = t.at(m[0], m[1], m[2]);
            m[d] -= 2;
            dn1[3 * k + d] = m[d] >= 0 ? t.at(m[0], m[1], m[2]) : -1;
        }
        for (int e = 0; e < 6; e++) {
            int m[3] = {t.nx[k], t.ny[k], t.nz[k]};
            m[hd[e][0]]++;
            m[hd[e][1]]++;
            up2[6 * k + e] = t.at(m[0], m[1], m[2]);
        }
        for (int j = 0; j < pre[k]; j++) add[(size_t)k * nc + j] = (short)t.at(t.nx[k] + t.nx[j], t.ny[k] + t.ny[j], t.nz[k] + t.nz[j]);
    }
    // the device code locates multi-indices by formula; the order must agree
    for (int k = 0; k < nc; k++)
        if (mi_index(t.nx[k], t.ny[k], t.nz[k]) != k) return POLFMM_ERR_INVALID_ARG;
    std::vector<double> w4(kMaxP + 1), rinv(kMaxP + 1, 0.0);
    for (int k = 0; k <= kMaxP; k++) {
        w4[k] = ldexp(1.0, -2 * k) / factorial(k);
        if (k > 0) rinv[k] = 1.0 / k;
    }
    std::vector<float> w4f(w4.begin(), w4.end()), rinvf(rinv.begin(), rinv.end());
    // derivative tables at the integer offsets of [-3, 3]^3
    std::vector<double> D((size_t)343 * nc, 0.0);
    std::vector<float> Df((size_t)343 * nc, 0.f);
    for (int oz = -3; oz <= 3; oz++)
        for (int oy = -3; oy <= 3; oy++)
            for (int ox = -3; ox <= 3; ox++) {
                if (!ox && !oy && !oz) continue;
                int oi = (ox + 3) + 7 * ((oy + 3) + 7 * (oz + 3));
                double R[3] = {(double)ox, (double)oy, (double)oz};
                derivative_table(t, R, &D[(size_t)oi * nc]);
                for (int k = 0; k < nc; k++) Df[(size_t)oi * nc + k] = (float)D[(size_t)oi * nc + k];
            }
    // interaction offsets per octant class: o = B - A with o_d in [b_d - 3, b_d + 2], not adjacent
    std::vector<int> class_off(8 * kNumOffsets);
    for (int cls = 0; cls < 8; cls++) {
        int b[3] = {cls & 1, (cls >> 1) & 1, (cls >> 2) & 1};
        int k = 0;
        for (int oz = b[2] - 3; oz <= b[2] + 2; oz++)
            for (int oy = b[1] - 3; oy <= b[1] + 2; oy++)
                for (int ox = b[0] - 3; ox <= b[0] + 2; ox++) {
                    if (std::max(abs(ox), std::max(abs(oy), abs(oz))) <= 1) continue;
                    class_off[cls * kNumOffsets + k++] = (ox + 3) | ((oy + 3) << 4) | ((oz + 3) << 8);
                }
        if (k != kNumOffsets) return POLFMM_ERR_INVALID_ARG;
    }
    // balanced output lists for the 8 warps of the SIMT M2L kernel (longest first)
    std::vector<int> order(nc);
    for (int k = 0; k < nc; k++) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return pre[a] > pre[b]; });
    std::vector<std::vector<int>> lists(8);
    std::vector<long> load(8, 0);
    for (int k : order) {
        int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        lists[w].push_back(k);
        load[w] += pre[k] + 4;
    }
    std::vector<int> wptr(9, 0), wout;
    for (int w = 0; w < 8; w++) {
        for (int k : lists[w]) wout.push_back(k);
        wptr[w + 1] = (int)wout.size();
    }
    cudaStream_t st = c->stream;
    int rc;
#define UP(h, d) \
    if ((rc = upload(h, &d, st)) != POLFMM_OK) return rc
    UP(mi, T.mi);
    UP(inv_fact, T.inv_fact);
    UP(inv_fact_f, T.inv_fact_f);
    UP(up1, T.up1);
    UP(up2, T.up2);
    UP(pre, T.pre);
    UP(add, T.add);
    UP(dn1, T.dn1);
    UP(w4, T.w4);
    UP(w4f, T.w4f);
    UP(rinv, T.rinv);
    UP(rinvf, T.rinvf);
    UP(D, T.D);
    UP(Df, T.Df);
    UP(class_off, T.class_off);
    UP(wptr, T.warp_out_ptr);
    UP(wout, T.warp_out);
#undef UP
    T.h_mi = mi;
    return POLFMM_OK;
}

void free_tables(Tables& T) {
    void* ptrs[] = {T.mi,   T.inv_fact, T.inv_fact_f, T.up1,  T.dn1, T.w4,        T.w4f,        T.rinv,
                    T.rinvf, T.up2,     T.pre,        T.add,  T.D,   T.Df,        T.class_off,  T.warp_out_ptr,
                    T.warp_out};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    T = Tables();
}

// ---------------------------------------------------------------------------
// allocation
// ---------------------------------------------------------------------------
struct Alloc {
    std::vector<void*> ptrs;
    bool ok = true;
    template <typename T>
    T* get(size_t count) {
        if (!ok) return nullptr;
        void* p = nullptr;
        if (count == 0) count = 1;
        if (dev_alloc(&p, sizeof(T) * count) != cudaSuccess) {
            ok = false;
            return nullptr;
        }
        ptrs.push_back(p);
        return (T*)p;
    }
};

// device allocations owned by one context
struct CtxExtra {
    Alloc alloc;
    std::vector<void*> lp_bufs;
    size_t lp_cap_chunks = 0;
    std::vector<int> tmu_index;  // caller index -> index in the dipole tree (-1: not polarizable)
};

CtxExtra* extra_of(polfmm_ctx* c) { return reinterpret_cast<CtxExtra*>(c->extra); }

int allocate(polfmm_ctx* c) {
    Alloc& A = extra_of(c)->alloc;
    const int64_t n = c->n;
    const size_t rsz = c->mixed ? sizeof(float) : sizeof(double);
    c->pos_s = A.get<double>(3 * n);
    c->q_s = A.get<double>(n);
    c->alpha_s = A.get<double>(n);
    c->inv_alpha_s = A.get<double>(n);
    c->perm = A.get<int>(n);
    c->key_s = A.get<uint32_t>(n);
    c->ploc = A.get<unsigned char>(3 * n * rsz);
    c->srcA = A.get<unsigned char>(n * source_record_bytes(c->mixed));
    c->srcB = A.get<unsigned char>(n * source_record_bytes(c->mixed));
    c->in_buf = A.get<double>(9 * n);  // positions, q, alpha, mu, q^E (caller order)
    c->out_buf = A.get<double>(10 * n);
    c->phiq = A.get<double>(n);
    c->Eq = A.get<double>(3 * n);
    c->mu = A.get<double>(3 * n);
    c->r = A.get<double>(3 * n);
    c->z = A.get<double>(3 * n);
    c->d = A.get<double>(3 * n);
    c->Ad = A.get<double>(3 * n);
    c->Td = A.get<double>(3 * n);
    c->phi_t = A.get<double>(n);
    c->E_t = A.get<double>(3 * n);
    c->G_t = A.get<double>(6 * n);
    c->partial = A.get<double>((size_t)kRedSlots * kRedBlocks);
    c->scal = A.get<double>(S_COUNT + 8);
    c->err = A.get<int>(4);
    c->ticket = A.get<int>(4);
    c->key_tmp = A.get<uint32_t>(n);
    c->val_tmp = A.get<int>(n);
    c->val_a = A.get<int>(n);
    c->flags = A.get<int>(n + 64);
    c->counts_cap = tree_count_scratch(n);
    c->counts = A.get<int>(c->counts_cap);
    c->scan_tmp_cap = tree_scan_scratch(n);
    c->scan_tmp = A.get<int>(c->scan_tmp_cap);
    c->tree_cnt = A.get<int>((kMaxDepth + 1) * 9);
    // the multipoles of all levels in one array (level l from row mrow0[l]), so
    // that a row of any level is addressed by one index
    int64_t mrows = 0;
    for (int l = 0; l <= c->depth; l++) {
        c->mrow0[l] = mrows;
        mrows += std::min<int64_t>((int64_t)1 << (3 * l), n);
    }
    c->mrow_zero = mrows;  // one more row, kept at zero: the source of an empty box
    c->Mall = A.get<unsigned char>((size_t)(mrows + 1) * c->ld * rsz);
    for (int l = 0; l <= c->depth; l++) {
        Level& B = c->lv[l];
        int64_t full = (int64_t)1 << (3 * l);
        B.cap = (int)std::min<int64_t>(full, n);
        B.key = A.get<int>(B.cap);
        B.map = A.get<int>(full);
        B.parent = A.get<int>(B.cap);
        B.child0 = A.get<int>(B.cap);
        B.nchild = A.get<int>(B.cap);
        B.by_class = A.get<int>(B.cap);
        B.M = c->Mall ? static_cast<unsigned char*>(c->Mall) + (size_t)c->mrow0[l] * c->ld * rsz : nullptr;
        B.arrive = A.get<int>(B.cap);
        if (l >= 3) B.Msh = A.get<unsigned char>((size_t)B.cap * c->ld * rsz);
    }
    c->lstart = A.get<int>(c->lv[c->depth].cap);
    c->leaf_partial = A.get<double>(c->lv[c->depth].cap);
    c->lcount = A.get<int>(c->lv[c->depth].cap);
    c->leaf_order = A.get<int>(c->lv[c->depth].cap);
    c->leaf_items_cap = (int)std::min<int64_t>((int64_t)c->lv[c->depth].cap + n / kLeafTargetsMin + 1, 2 * n + 1);
    c->leaf_items = A.get<int2>(c->leaf_items_cap);
    c->leaf_nitems = A.get<int>(4);
    if (c->mixed) {
        // sum over leaves of ceil(count / 2) <= (n + leaves) / 2 <= n records
        c->near_pairs = A.get<float>(12 * (size_t)n);
        c->near_pbase = A.get<int>(c->lv[c->depth].cap + 1);
        c->near_slot = A.get<int>(n);
        c->near_items = A.get<NearItem>(2 * (size_t)c->leaf_items_cap);
        c->near_nitems = A.get<int>(4);
    }
    if (!A.ok) return POLFMM_ERR_OUT_OF_MEMORY;
    if (host_alloc(reinterpret_cast<void**>(&c->h_scal), sizeof(double) * (S_COUNT + 8)) != cudaSuccess ||
        host_alloc(reinterpret_cast<void**>(&c->h_counts), sizeof(int) * (kMaxDepth + 1) * 9) != cudaSuccess ||
        host_alloc(reinterpret_cast<void**>(&c->h_bbox), sizeof(double) * 8) != cudaSuccess)
        return POLFMM_ERR_OUT_OF_MEMORY;
    cudaMemsetAsync(c->err, 0, sizeof(int) * 4, c->stream);
    cudaMemsetAsync(c->ticket, 0, sizeof(int) * 4, c->stream);
    cudaMemsetAsync(c->scal, 0, sizeof(double) * (S_COUNT + 8), c->stream);
    for (int l = 0; l <= c->depth; l++) cudaMemsetAsync(c->lv[l].arrive, 0, sizeof(int) * c->lv[l].cap, c->stream);
    return POLFMM_OK;
}

// M2L partial-output buffers: chunks x cap x ld per level (grown on demand)
int ensure_lp(polfmm_ctx* c) {
    CtxExtra* X = extra_of(c);
    if ((size_t)c->m2l_chunks <= X->lp_cap_chunks) return POLFMM_OK;
    for (void* p : X->lp_bufs) cudaFree(p);
    X->lp_bufs.clear();
    const size_t rsz = c->mixed ? sizeof(float) : sizeof(double);
    for (int l = 0; l <= c->depth; l++) {
        void* p = nullptr;
        size_t bytes = (size_t)c->m2l_chunks * c->lv[l].cap * c->ld * rsz;
        if (dev_alloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) return POLFMM_ERR_OUT_OF_MEMORY;
        X->lp_bufs.push_back(p);
        c->lv[l].Lp = p;
    }
    X->lp_cap_chunks = c->m2l_chunks;
    return POLFMM_OK;
}


int read_err(polfmm_ctx* c) {
    int h[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(h, c->err, sizeof(int) * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "copy of the error word");
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(e, "stream synchronize");
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "kernel launch");
    if (h[0] & 1) return POLFMM_ERR_INVALID_ARG;
    if (h[0] & 2) return POLFMM_ERR_COINCIDENT;
    if (h[0] & 4) {
        snprintf(g_last_error, sizeof(g_last_error), "a bounded wait of the tensor-core M2L kernel timed out");
        return POLFMM_ERR_CUDA;
    }
    if (h[0] & 8) {
        snprintf(g_last_error, sizeof(g_last_error), "a bounded wait of the near-field kernel timed out");
        return POLFMM_ERR_CUDA;
    }
    return POLFMM_OK;
}

int copy_in(polfmm_ctx* c, double* dst, const double* src, size_t count, int on_device) {
    cudaError_t e = cudaMemcpyAsync(dst, src, sizeof(double) * count,
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream);
    return e == cudaSuccess ? POLFMM_OK : POLFMM_ERR_CUDA;
}

// sorted -> caller order, into a device pointer or through out_buf to the host
int scatter_out(polfmm_ctx* c, const double* src_sorted, double* dst, int comps, int on_device) {
    if (!dst) return POLFMM_OK;
    if (on_device) {
        scatter_sites(c, src_sorted, dst, comps);
        return POLFMM_OK;
    }
    scatter_sites(c, src_sorted, c->out_buf, comps);
    if (cudaMemcpyAsync(dst, c->out_buf, sizeof(double) * comps * c->n, cudaMemcpyDeviceToHost, c->stream) !=
        cudaSuccess)
        return POLFMM_ERR_CUDA;
    return cudaStreamSynchronize(c->stream) == cudaSuccess ? POLFMM_OK : POLFMM_ERR_CUDA;
}

__global__ void leaf_cells_kernel(int64_t n, const uint32_t* __restrict__ key, const int* __restrict__ perm,
                                  int32_t* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t k = key[i];
    int o = perm[i];
    out[3 * (int64_t)o] = (int32_t)compact3(k);
    out[3 * (int64_t)o + 1] = (int32_t)compact3(k >> 1);
    out[3 * (int64_t)o + 2] = (int32_t)compact3(k >> 2);
}

// The field charges q^E stand in for the charges q as the sources of one pass
// (the packed near-field records and the P2M read c->q_s and c->srcA).
struct FieldChargeSources {
    polfmm_ctx* c;
    double* q;
    void* a;
    explicit FieldChargeSources(polfmm_ctx* ctx) : c(ctx), q(ctx->q_s), a(ctx->srcA) {
        if (c->qE_s) {
            c->q_s = c->qE_s;
            c->srcA = c->srcAE;
        }
    }
    ~FieldChargeSources() {
        c->q_s = q;
        c->srcA = a;
    }
};

// static passes (Sec. III, first stage): potential and field of the Coulomb
// charges q, and with field charges set those of the q^E, which polarize the
// sites; every pass without the excluded pairs
void static_passes(polfmm_ctx* c) {
    if (c->dipole_only) return;  // a dipole tree: its field comes from the full tree
    fmm_pass(c, LEAF_CHARGE_PHI_E, true, nullptr, c->phiq, c->Eq, nullptr);
    if (c->qE_s) {
        FieldChargeSources fc(c);
        pack_positions(c);  // (x, y, z, q^E) records
        fmm_pass(c, LEAF_CHARGE_PHI_E, true, nullptr, c->phiqE, c->EqE, nullptr);
    }
}

// build the tree from caller-order inputs staged in in_buf and run the static pass
int rebuild(polfmm_ctx* c) {
    const int64_t n = c->n;
    double* x_in = c->in_buf;
    double* q_in = c->in_buf + 3 * n;
    double* a_in = c->in_buf + 4 * n;
    int rc;
    if (c->opt.use_root_box) {
        for (int d = 0; d < 3; d++) c->lo[d] = c->opt.root_lo[d];
        c->side = c->opt.root_side;
    } else if ((rc = tree_root_box(c, x_in, c->partial, c->h_bbox)) != POLFMM_OK) {
        return rc;
    }
    // the pair +-dl mu/|mu| stays well inside its leaf's expansion
    if (c->opt.dipole_dl > 0.25 * c->side / (double)(1 << c->depth)) return POLFMM_ERR_INVALID_ARG;
    if ((rc = tree_build(c, x_in)) != POLFMM_OK) return rc;
    if ((rc = tree_tables(c, x_in, q_in, a_in)) != POLFMM_OK) return rc;
    if ((rc = read_err(c)) != POLFMM_OK) return rc;
    if ((rc = m2l_setup(c)) != POLFMM_OK) return rc;
    if ((rc = m2l_tensor_prepare(c)) != POLFMM_OK) {  // may raise the offset-chunk count
        if (rc == POLFMM_ERR_CUDA) cuda_fail(cudaGetLastError(), "tensor-core M2L set-up");
        return rc;
    }
    if ((rc = m2l_ffma_prepare(c)) != POLFMM_OK) return rc;  // sets the chunk count when it runs
    if ((rc = ensure_lp(c)) != POLFMM_OK) return rc;
    if (c->qE_s) gather_sites(c, c->in_buf + 8 * n, c->qE_s, 1);
    exclusion_inv_perm(c);
    pack_positions(c);
    if ((rc = near_tables(c)) != POLFMM_OK) return rc;
    if ((rc = thole_pairs(c)) != POLFMM_OK) return rc;
    static_passes(c);
    c->pcg_graph_dirty = true;  // launch sizes of the solver iteration changed
    c->loop_dirty = true;
    return read_err(c);
}

// Capture one PCG iteration (FMM dipole-field pass + vector updates) as a CUDA
// graph on a private stream; later trees update the executable in place.
// graphs are captured on a private stream of the highest priority; captured
// kernels keep their stream's priority and the graphs are instantiated to use it
cudaError_t create_capture_stream(polfmm_ctx* c) {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    return cudaStreamCreateWithPriority(&c->cap_stream, cudaStreamNonBlocking, hi);
}

int capture_pcg_graph(polfmm_ctx* c) {
    if (!c->cap_stream &&
        create_capture_stream(c) != cudaSuccess)
        return POLFMM_ERR_CUDA;
    cudaStream_t orig = c->stream;
    const int64_t l0 = c->launches;
    c->stream = c->cap_stream;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        solver_pcg_step(c);
        e = cudaStreamEndCapture(c->cap_stream, &g);
    }
    c->stream = orig;
    c->pcg_graph_launches = c->launches - l0;
    c->launches = l0;
    if (e != cudaSuccess || !g) {
        cudaGetLastError();
        return POLFMM_ERR_CUDA;
    }
    if (c->pcg_graph) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(c->pcg_graph, g, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(c->pcg_graph);
            c->pcg_graph = nullptr;
        }
    }
    if (!c->pcg_graph && cudaGraphInstantiate(&c->pcg_graph, g, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess) {
        cudaGetLastError();
        c->pcg_graph = nullptr;
        cudaGraphDestroy(g);
        return POLFMM_ERR_CUDA;
    }
    cudaGraphDestroy(g);
    c->pcg_graph_dirty = false;
    return POLFMM_OK;
}

// The solve loop as one graph: a while node whose body is one PCG iteration.
// Graph and condition handle live as long as the context; after a new tree the
// body is emptied, captured again and the executable graph updated.  The body
// clears the condition in its first solver kernel and only the update kernel
// sets it again, so a body that fails to finish ends the loop.
int prepare_loop_graph(polfmm_ctx* c) {
    auto fail = [&](void) {
        cudaGetLastError();
        if (c->loop_exec) cudaGraphExecDestroy(c->loop_exec);
        if (c->loop_g) cudaGraphDestroy(c->loop_g);
        c->loop_exec = nullptr;
        c->loop_g = nullptr;
        c->loop_body = nullptr;
        c->loop_cond = 0;
        c->loop_failed = true;
        return POLFMM_ERR_CUDA;
    };
    if (!c->cap_stream && create_capture_stream(c) != cudaSuccess) return fail();
    if (!c->loop_g) {
        if (cudaGraphCreate(&c->loop_g, 0) != cudaSuccess) return fail();
        if (cudaGraphConditionalHandleCreate(&c->loop_cond, c->loop_g, 1, cudaGraphCondAssignDefault) != cudaSuccess)
            return fail();
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = c->loop_cond;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        if (cudaGraphAddNode(&node, c->loop_g, nullptr, nullptr, 0, &np) != cudaSuccess) return fail();
        c->loop_body = np.conditional.phGraph_out[0];
    } else {
        size_t nn = 0;
        if (cudaGraphGetNodes(c->loop_body, nullptr, &nn) != cudaSuccess) return fail();
        std::vector<cudaGraphNode_t> nodes(nn);
        if (nn && cudaGraphGetNodes(c->loop_body, nodes.data(), &nn) != cudaSuccess) return fail();
        for (cudaGraphNode_t nd : nodes)
            if (cudaGraphDestroyNode(nd) != cudaSuccess) return fail();
    }
    cudaStream_t orig = c->stream;
    const int64_t l0 = c->launches;
    c->stream = c->cap_stream;
    c->capturing_loop = true;
    cudaError_t e = cudaStreamBeginCaptureToGraph(c->cap_stream, c->loop_body, nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        solver_pcg_step(c);
        cudaGraph_t out = nullptr;
        e = cudaStreamEndCapture(c->cap_stream, &out);
    }
    c->capturing_loop = false;
    c->stream = orig;
    c->loop_launches = c->launches - l0;
    c->launches = l0;
    if (e != cudaSuccess) return fail();
    if (c->loop_exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(c->loop_exec, c->loop_g, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(c->loop_exec);
            c->loop_exec = nullptr;
        }
    }
    if (!c->loop_exec &&
        cudaGraphInstantiate(&c->loop_exec, c->loop_g, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess)
        return fail();
    c->loop_dirty = false;
    return POLFMM_OK;
}

int pcg_iteration(polfmm_ctx* c) {
    if (c->opt.no_graphs || c->opt.profile) {
        solver_pcg_step(c);
        return POLFMM_OK;
    }
    if (c->pcg_graph_dirty || !c->pcg_graph) {
        int rc = capture_pcg_graph(c);
        if (rc != POLFMM_OK) return rc;
    }
    if (cudaGraphLaunch(c->pcg_graph, c->stream) != cudaSuccess) return POLFMM_ERR_CUDA;
    c->launches += c->pcg_graph_launches;
    return POLFMM_OK;
}

void destroy_impl(polfmm_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    if (c->tmu) destroy_impl(c->tmu);
    c->tmu = nullptr;
    CtxExtra* X = extra_of(c);
    if (X) {
        for (void* p : X->alloc.ptrs) cudaFree(p);
        for (void* p : X->lp_bufs) cudaFree(p);
    }
    m2l_tensor_release(c);
    m2l_ffma_release(c);
    free_tables(c->tab);
    if (c->tiles) cudaFree(c->tiles);
    if (c->th_idx) cudaFree(c->th_idx);
    if (c->th_r) cudaFree(c->th_r);
    if (c->th_t3) cudaFree(c->th_t3);
    if (c->h_scal) cudaFreeHost(c->h_scal);
    if (c->h_counts) cudaFreeHost(c->h_counts);
    if (c->h_bbox) cudaFreeHost(c->h_bbox);
    if (c->ev_created)
        for (int i = 0; i < 2 * 4096; i++) cudaEventDestroy(c->ev_pool[i]);
    if (c->pcg_graph) cudaGraphExecDestroy(c->pcg_graph);
    if (c->loop_exec) cudaGraphExecDestroy(c->loop_exec);
    if (c->loop_g) cudaGraphDestroy(c->loop_g);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->side_stream) cudaStreamDestroy(c->side_stream);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    delete X;
    delete c;
}

bool finite_host(const double* v, size_t count) {
    for (size_t i = 0; i < count; i++)
        if (!isfinite(v[i])) return false;
    return true;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void fmm_default_options(polfmm_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->mode = POLFMM_FP64;
    o->solver = POLFMM_SOLVER_PCG;
    o->max_iter = 100;
    o->coulomb_k = 1.0;
    o->m2l_impl = POLFMM_M2L_AUTO;
}

static int build_impl(polfmm_ctx** out, int64_t n, const double* positions, const double* charges,
                      const double* polarizabilities, int order_p, int tree_depth, const polfmm_options* opt,
                      int inputs_on_device, bool dipole_only) {
    if (!out) return POLFMM_ERR_INVALID_ARG;
    *out = nullptr;
    // 3 n must fit the 32-bit indices of the per-component solver loops
    if (n < 1 || n > (int64_t)1 << 28 || !positions || !charges || !polarizabilities) return POLFMM_ERR_INVALID_ARG;
    if (order_p < 1 || order_p > kMaxP || tree_depth < 1 || tree_depth > kMaxDepth) return POLFMM_ERR_INVALID_ARG;
    polfmm_options o;
    if (opt)
        o = *opt;
    else
        fmm_default_options(&o);
    if (o.mode != POLFMM_FP64 && o.mode != POLFMM_MIXED) return POLFMM_ERR_INVALID_ARG;
    if (o.solver != POLFMM_SOLVER_PCG && o.solver != POLFMM_SOLVER_JACOBI) return POLFMM_ERR_INVALID_ARG;
    if (o.max_iter < 0) return POLFMM_ERR_INVALID_ARG;
    // the +-q pair form of the dipoles: FP64 only, finite, non-negative
    if (!(o.dipole_dl >= 0.0) || !isfinite(o.dipole_dl) || (o.dipole_dl > 0.0 && o.mode != POLFMM_FP64))
        return POLFMM_ERR_INVALID_ARG;
    if (!(o.coulomb_k == o.coulomb_k) || !isfinite(o.coulomb_k)) return POLFMM_ERR_INVALID_ARG;
    if (o.use_root_box && (!(o.root_side > 0.0) || !isfinite(o.root_side) || !finite_host(o.root_lo, 3)))
        return POLFMM_ERR_INVALID_ARG;
    if (!inputs_on_device) {
        if (!finite_host(positions, 3 * (size_t)n) || !finite_host(charges, n) || !finite_host(polarizabilities, n))
            return POLFMM_ERR_INVALID_ARG;
        for (int64_t i = 0; i < n; i++)
            if (polarizabilities[i] < 0.0) return POLFMM_ERR_INVALID_ARG;
    }
    polfmm_ctx* c = new (std::nothrow) polfmm_ctx();
    if (!c) return POLFMM_ERR_OUT_OF_MEMORY;
    c->extra = new (std::nothrow) CtxExtra();
    if (!c->extra) {
        delete c;
        return POLFMM_ERR_OUT_OF_MEMORY;
    }
    c->opt = o;
    c->dipole_only = dipole_only;
    c->n = n;
    c->p = order_p;
    c->depth = tree_depth;
    c->ncoef = ncoef_of(order_p);
    c->ld = (c->ncoef + 3) & ~3;
    c->mixed = o.mode == POLFMM_MIXED;
    c->stream = (cudaStream_t)o.cuda_stream;
    int dev = 0, rc;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        destroy_impl(c);
        return POLFMM_ERR_CUDA;
    }
    if (o.profile) {
        for (int i = 0; i < 2 * 4096; i++) cudaEventCreate(&c->ev_pool[i]);
        c->ev_created = true;
    }
    // the near-field pairs run at the lowest priority: their blocks fill the SMs
    // that the far-field chain (the critical path) leaves free
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (cudaStreamCreateWithPriority(&c->side_stream, cudaStreamNonBlocking, prio_lo) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        c->side_stream = nullptr;
    }
    if ((rc = allocate(c)) != POLFMM_OK || (rc = build_tables(c)) != POLFMM_OK ||
        (rc = fmm_ops_init_attributes(c)) != POLFMM_OK) {
        if (rc == POLFMM_ERR_CUDA) cuda_fail(cudaGetLastError(), "set-up (tables or kernel attributes)");
        destroy_impl(c);
        return rc;
    }
    if ((rc = copy_in(c, c->in_buf, positions, 3 * (size_t)n, inputs_on_device)) != POLFMM_OK ||
        (rc = copy_in(c, c->in_buf + 3 * n, charges, n, inputs_on_device)) != POLFMM_OK ||
        (rc = copy_in(c, c->in_buf + 4 * n, polarizabilities, n, inputs_on_device)) != POLFMM_OK ||
        (rc = rebuild(c)) != POLFMM_OK) {
        destroy_impl(c);
        return rc;
    }
    *out = c;
    return POLFMM_OK;
}

// the dipole solve's tree over the polarizable sites (T^mu of Sec. III)
static int build_dipole_tree(polfmm_ctx* c) {
    const int64_t n = c->n;
    std::vector<double> a((size_t)n);
    if (cudaMemcpyAsync(a.data(), c->in_buf + 4 * n, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "copy of the polarizabilities");
    CtxExtra* X = extra_of(c);
    X->tmu_index.assign((size_t)n, -1);
    std::vector<int> rows;
    for (int64_t i = 0; i < n; i++)
        if (a[i] > 0.0) {
            X->tmu_index[i] = (int)rows.size();
            rows.push_back((int)i);
        }
    const int64_t m = (int64_t)rows.size();
    if (m == 0 || m == n) return POLFMM_OK;  // the two trees would coincide (or there is nothing to solve)
    Alloc& A = X->alloc;
    c->mu_rows = A.get<int>(m);
    c->tmu_caller = A.get<double>(std::max(3 * n, 5 * m));
    c->tmu_rows = A.get<double>(3 * m);
    if (!A.ok) return POLFMM_ERR_OUT_OF_MEMORY;
    if (cudaMemcpyAsync(c->mu_rows, rows.data(), sizeof(int) * m, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "upload of the polarizable sites");
    c->nmu = m;
    // positions and polarizabilities of those sites; no charges
    double* xq = c->tmu_caller;  // 3 m positions, then m zeros, then m polarizabilities (m <= n - 1)
    {
        LaunchScope ls(c, F_TREE);
        take_rows_kernel<<<grid_for(3 * m, 256), 256, 0, c->stream>>>(m, 3, c->mu_rows, c->in_buf, xq);
        take_rows_kernel<<<grid_for(m, 256), 256, 0, c->stream>>>(m, 1, c->mu_rows, c->in_buf + 4 * n, xq + 4 * m);
    }
    cudaMemsetAsync(xq + 3 * m, 0, sizeof(double) * m, c->stream);
    // depth less log8(n / m), rounded down
    int depth = c->depth;
    for (int64_t r = n / m; r >= 8 && depth > 1; r /= 8) depth--;
    polfmm_options o = c->opt;
    o.dipole_tree = 0;
    polfmm_ctx* t = nullptr;
    int rc = build_impl(&t, m, xq, xq + 3 * m, xq + 4 * m, c->p, depth, &o, 1, true);
    if (rc != POLFMM_OK) return rc;
    c->tmu = t;
    return POLFMM_OK;
}

int fmm_build(polfmm_ctx** out, int64_t n, const double* positions, const double* charges,
              const double* polarizabilities, int order_p, int tree_depth, const polfmm_options* opt,
              int inputs_on_device) {
    int rc = build_impl(out, n, positions, charges, polarizabilities, order_p, tree_depth, opt, inputs_on_device,
                        false);
    if (rc != POLFMM_OK || !(*out)->opt.dipole_tree) return rc;
    if ((rc = build_dipole_tree(*out)) != POLFMM_OK) {
        destroy_impl(*out);
        *out = nullptr;
    }
    return rc;
}

// the solve on the dipole tree: its polarizing field from this tree, its dipoles
// back to this tree (zero at the sites that are not polarizable)
static int solve_on_dipole_tree(polfmm_ctx* c, double tol, int* iters_out, double* res_out) {
    polfmm_ctx* t = c->tmu;
    const int64_t m = c->nmu;
    scatter_sites(c, polarizing_field(c), c->tmu_caller, 3);
    {
        LaunchScope ls(c, F_SOLVER);
        take_rows_kernel<<<grid_for(3 * m, 256), 256, 0, c->stream>>>(m, 3, c->mu_rows, c->tmu_caller, c->tmu_rows);
    }
    gather_sites(t, c->tmu_rows, t->Eq, 3);
    const int status = fmm_solve_induced_dipoles(t, tol, iters_out, res_out);
    if (status != POLFMM_OK && status != POLFMM_ERR_NOT_CONVERGED) return status;
    // dipoles back (the last good iterate when the solve did not converge)
    scatter_sites(t, t->mu, c->tmu_rows, 3);
    cudaMemsetAsync(c->tmu_caller, 0, sizeof(double) * 3 * c->n, c->stream);
    {
        LaunchScope ls(c, F_SOLVER);
        put_rows_kernel<<<grid_for(3 * m, 256), 256, 0, c->stream>>>(m, 3, c->mu_rows, c->tmu_rows, c->tmu_caller);
    }
    gather_sites(c, c->tmu_caller, c->mu, 3);
    c->have_mu = true;
    int rc = read_err(c);
    return rc != POLFMM_OK ? rc : status;
}

int fmm_solve_induced_dipoles(polfmm_ctx* c, double tol, int* iters_out, double* res_out) {
    if (!c || !(tol >= 0.0)) return POLFMM_ERR_INVALID_ARG;
    if (c->tmu) return solve_on_dipole_tree(c, tol, iters_out, res_out);
    const bool jacobi = c->opt.solver == POLFMM_SOLVER_JACOBI;
    solver_init(c, c->have_mu);
    c->have_mu = true;
    int it = 0;
    double res = 0.0;
    int status = POLFMM_OK;
    auto fetch = [&](void) -> int {
        if (cudaMemcpyAsync(c->h_scal, c->scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess)
            return POLFMM_ERR_CUDA;
        return cudaStreamSynchronize(c->stream) == cudaSuccess ? POLFMM_OK : POLFMM_ERR_CUDA;
    };
    int rc;
    if ((rc = fetch()) != POLFMM_OK) return rc;
    const double bb = c->h_scal[S_BB];
    if (!(bb > 0.0)) {
        // no field at any polarizable site: the dipoles vanish
        cudaMemsetAsync(c->mu, 0, sizeof(double) * 3 * c->n, c->stream);
        if (iters_out) *iters_out = 0;
        if (res_out) *res_out = 0.0;
        return read_err(c);
    }
    const bool use_loop = !jacobi && !c->opt.no_graphs && !c->opt.profile && !c->loop_failed;
    if (use_loop && (res = sqrt(c->h_scal[S_RR] / bb)) > tol && c->opt.max_iter > 0 &&
        ((!c->loop_dirty && c->loop_exec) || prepare_loop_graph(c) == POLFMM_OK)) {
        // all iterations in one graph launch; the device decides when to stop
        solver_loop_setup(c, tol, c->opt.max_iter);
        cudaError_t e = cudaGraphLaunch(c->loop_exec, c->stream);
        if (e != cudaSuccess) return cuda_fail(e, "solve graph launch");
        if ((rc = fetch()) != POLFMM_OK) return rc;
        it = (int)c->h_scal[S_ITER];
        c->launches += c->loop_launches * it;
        // a direction of non-positive curvature (polarization catastrophe) was not
        // applied: the dipoles and residual are those of the last good iterate
        res = sqrt(fabs(c->h_scal[S_RR] / bb));
        if (!(c->h_scal[S_DAD] > 0.0) || !isfinite(res) || c->h_scal[S_GROW] >= kStagnationIters)
            status = POLFMM_ERR_NOT_CONVERGED;
    } else if (!jacobi) {
        res = sqrt(c->h_scal[S_RR] / bb);
        while (res > tol && it < c->opt.max_iter) {
            if ((rc = pcg_iteration(c)) != POLFMM_OK) return rc;
            it++;
            if ((rc = fetch()) != POLFMM_OK) return rc;
            res = sqrt(fabs(c->h_scal[S_RR] / bb));
            if (!(c->h_scal[S_DAD] > 0.0) || !isfinite(res) || c->h_scal[S_GROW] >= kStagnationIters) {
                status = POLFMM_ERR_NOT_CONVERGED;
                break;
            }
        }
    } else {
        res = INFINITY;
        int grow = 0;
        while (it < c->opt.max_iter) {
            solver_jacobi_step(c);
            it++;
            if ((rc = fetch()) != POLFMM_OK) return rc;
            const double r_new = sqrt(c->h_scal[S_RR] / bb);
            grow = it > 1 && r_new > res ? grow + 1 : 0;
            res = r_new;
            // a fixed point whose residual keeps growing diverges (spectral radius of alpha T >= 1)
            if (!isfinite(res) || grow >= kStagnationIters) {
                status = POLFMM_ERR_NOT_CONVERGED;
                break;
            }
            if (res <= tol) break;
        }
    }
    if (status == POLFMM_OK && res > tol) status = POLFMM_ERR_NOT_CONVERGED;
    if (iters_out) *iters_out = it;
    if (res_out) *res_out = res;
    rc = read_err(c);
    return rc != POLFMM_OK ? rc : status;
}

int fmm_energy_forces(polfmm_ctx* c, double* energy_out, double* forces, double* dU_dq, double* dU_dalpha,
                      int on_device) {
    if (!c) return POLFMM_ERR_INVALID_ARG;
    if (!c->have_mu) return POLFMM_ERR_STATE;
    const int64_t n = c->n;
    {
        FieldChargeSources fc(c);  // sources: the field charges (or q) and the dipoles
        fmm_pass(c, LEAF_FULL, true, c->mu, c->phi_t, c->E_t, c->G_t);
    }
    double* F = forces;
    double* dq = dU_dq;
    double* da = dU_dalpha;
    if (!on_device) {
        F = forces ? c->out_buf : nullptr;
        dq = dU_dq ? c->out_buf + 3 * n : nullptr;
        da = dU_dalpha ? c->out_buf + 4 * n : nullptr;
    }
    energy_and_gradients(c, F, dq, da, F != nullptr, dq != nullptr, da != nullptr);
    cudaMemcpyAsync(c->h_scal, c->scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, c->stream);
    if (!on_device) {
        if (forces) cudaMemcpyAsync(forces, F, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->stream);
        if (dU_dq) cudaMemcpyAsync(dU_dq, dq, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream);
        if (dU_dalpha) cudaMemcpyAsync(dU_dalpha, da, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream);
    }
    int rc = read_err(c);
    if (rc != POLFMM_OK) return rc;
    const double k = c->opt.coulomb_k;
    const double uqq = k * c->h_scal[S_UQQ];
    const double upol = k * (c->h_scal[S_AMU] - c->h_scal[S_MUEQ] - 0.5 * c->h_scal[S_MUEMU]);
    c->have_dqE = c->qE_s != nullptr;
    if (energy_out) {
        energy_out[0] = uqq + upol;
        energy_out[1] = uqq;
        energy_out[2] = upol;
    }
    return POLFMM_OK;
}

int fmm_energy(polfmm_ctx* c, double* energy_out) {
    if (!c || !energy_out) return POLFMM_ERR_INVALID_ARG;
    if (!c->have_mu) return POLFMM_ERR_STATE;
    energy_stationary(c);
    cudaMemcpyAsync(c->h_scal, c->scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, c->stream);
    int rc = read_err(c);
    if (rc != POLFMM_OK) return rc;
    const double k = c->opt.coulomb_k;
    const double uqq = k * c->h_scal[S_UQQ];
    const double upol = -0.5 * k * c->h_scal[S_MUEQ];
    energy_out[0] = uqq + upol;
    energy_out[1] = uqq;
    energy_out[2] = upol;
    return POLFMM_OK;
}

int fmm_get_dipoles(polfmm_ctx* c, double* mu, int on_device) {
    if (!c || !mu) return POLFMM_ERR_INVALID_ARG;
    if (!c->have_mu) return POLFMM_ERR_STATE;
    int rc = scatter_out(c, c->mu, mu, 3, on_device);
    return rc != POLFMM_OK ? rc : read_err(c);
}

int fmm_set_dipoles(polfmm_ctx* c, const double* mu, int on_device) {
    if (!c || !mu) return POLFMM_ERR_INVALID_ARG;
    if (!on_device && !finite_host(mu, 3 * (size_t)c->n)) return POLFMM_ERR_INVALID_ARG;
    int rc = copy_in(c, c->in_buf + 5 * c->n, mu, 3 * (size_t)c->n, on_device);
    if (rc != POLFMM_OK) return rc;
    gather_sites(c, c->in_buf + 5 * c->n, c->mu, 3);
    mask_dipoles(c, c->mu);
    c->have_mu = true;
    c->have_hist = false;  // the predictor's history restarts
    if (c->tmu) {
        LaunchScope ls(c, F_SOLVER);
        take_rows_kernel<<<grid_for(3 * c->nmu, 256), 256, 0, c->stream>>>(c->nmu, 3, c->mu_rows, c->in_buf + 5 * c->n,
                                                                           c->tmu_rows);
        if ((rc = fmm_set_dipoles(c->tmu, c->tmu_rows, 1)) != POLFMM_OK) return rc;
    }
    return read_err(c);
}

int fmm_reset_dipoles(polfmm_ctx* c) {
    if (!c) return POLFMM_ERR_INVALID_ARG;
    c->have_mu = false;
    c->have_hist = false;
    return c->tmu ? fmm_reset_dipoles(c->tmu) : POLFMM_OK;
}

int fmm_set_field_charges(polfmm_ctx* c, const double* qE, int on_device) {
    if (!c || !qE) return POLFMM_ERR_INVALID_ARG;
    const int64_t n = c->n;
    if (!on_device && !finite_host(qE, (size_t)n)) return POLFMM_ERR_INVALID_ARG;
    if (!c->qE_s) {
        Alloc& A = extra_of(c)->alloc;
        c->qE_s = A.get<double>(n);
        c->srcAE = A.get<unsigned char>(n * source_record_bytes(c->mixed));
        c->phiqE = A.get<double>(n);
        c->EqE = A.get<double>(3 * n);
        c->dqE = A.get<double>(n);
        if (!A.ok) return POLFMM_ERR_OUT_OF_MEMORY;
    }
    int rc = copy_in(c, c->in_buf + 8 * n, qE, (size_t)n, on_device);
    if (rc != POLFMM_OK) return rc;
    gather_sites(c, c->in_buf + 8 * n, c->qE_s, 1);
    {
        FieldChargeSources fc(c);
        pack_positions(c);
        fmm_pass(c, LEAF_CHARGE_PHI_E, true, nullptr, c->phiqE, c->EqE, nullptr);
    }
    c->have_dqE = false;
    return read_err(c);
}

int fmm_set_exclusions(polfmm_ctx* c, int64_t npairs, const int32_t* pairs, int on_device) {
    if (!c || npairs < 0 || (npairs > 0 && !pairs) || npairs > (int64_t)1 << 30) return POLFMM_ERR_INVALID_ARG;
    const int64_t n = c->n;
    std::vector<int32_t> h((size_t)2 * npairs);
    if (npairs > 0) {
        if (on_device) {
            if (cudaMemcpy(h.data(), pairs, sizeof(int32_t) * h.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
                return cuda_fail(cudaGetLastError(), "copy of the excluded pairs");
        } else {
            memcpy(h.data(), pairs, sizeof(int32_t) * h.size());
        }
    }
    // both directions of every pair, sorted by site then partner, duplicates dropped
    std::vector<std::pair<int, int>> e;
    e.reserve(h.size());
    for (int64_t k = 0; k < npairs; k++) {
        const int32_t i = h[2 * k], j = h[2 * k + 1];
        if (i < 0 || j < 0 || i >= n || j >= n || i == j) return POLFMM_ERR_INVALID_ARG;
        e.emplace_back(i, j);
        e.emplace_back(j, i);
    }
    std::sort(e.begin(), e.end());
    e.erase(std::unique(e.begin(), e.end()), e.end());
    std::vector<int> targets, ptr(1, 0), idx;
    for (size_t k = 0; k < e.size(); k++) {
        if (k == 0 || e[k].first != e[k - 1].first) {
            if (k) ptr.push_back((int)k);
            targets.push_back(e[k].first);
        }
        idx.push_back(e[k].second);
    }
    if (!e.empty()) ptr.push_back((int)e.size());
    Alloc& A = extra_of(c)->alloc;
    if (!c->inv_perm) c->inv_perm = A.get<int>(n);
    if (targets.size() > c->excl_targets_cap) {
        c->excl_targets_cap = targets.size();
        c->excl_targets = A.get<int>(targets.size());
        c->excl_ptr = A.get<int>(targets.size() + 1);
    }
    if (idx.size() > c->excl_cap) {
        c->excl_cap = idx.size();
        c->excl_idx = A.get<int>(idx.size());
    }
    if (!c->excl_row) c->excl_row = A.get<int>(n);
    if (!A.ok) return POLFMM_ERR_OUT_OF_MEMORY;
    {
        // caller index -> row of the target list (the Thole pair list skips excluded pairs)
        std::vector<int> row((size_t)n, -1);
        for (size_t t = 0; t < targets.size(); t++) row[targets[t]] = (int)t;
        if (cudaMemcpy(c->excl_row, row.data(), sizeof(int) * row.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "upload of the excluded pairs");
    }
    if (!targets.empty() &&
        (cudaMemcpy(c->excl_targets, targets.data(), sizeof(int) * targets.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(c->excl_ptr, ptr.data(), sizeof(int) * ptr.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(c->excl_idx, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice) != cudaSuccess))
        return cuda_fail(cudaGetLastError(), "upload of the excluded pairs");
    c->n_excl = (int64_t)(e.size() / 2);
    c->n_excl_targets = (int)targets.size();
    exclusion_inv_perm(c);
    int rc = thole_pairs(c);
    if (rc != POLFMM_OK) return rc;
    static_passes(c);
    c->pcg_graph_dirty = true;  // the solver pass gains (or loses) the correction kernel
    c->loop_dirty = true;
    c->have_dqE = false;
    if (c->tmu) {
        // the dipole tree excludes the pairs of polarizable sites, in its own indices
        const std::vector<int>& ix = extra_of(c)->tmu_index;
        std::vector<int32_t> sub;
        for (int64_t k = 0; k < npairs; k++) {
            const int a = ix[h[2 * k]], b = ix[h[2 * k + 1]];
            if (a >= 0 && b >= 0) {
                sub.push_back(a);
                sub.push_back(b);
            }
        }
        if ((rc = fmm_set_exclusions(c->tmu, (int64_t)sub.size() / 2, sub.data(), 0)) != POLFMM_OK) return rc;
    }
    return read_err(c);
}

int fmm_set_dipole_predictor(polfmm_ctx* c, int order) {
    if (!c || order < 0 || order > 1) return POLFMM_ERR_INVALID_ARG;
    if (order == 1 && !c->mu_hist) {
        Alloc& A = extra_of(c)->alloc;
        c->mu_hist = A.get<double>(3 * c->n);
        if (!A.ok) {
            c->mu_hist = nullptr;
            return POLFMM_ERR_OUT_OF_MEMORY;
        }
    }
    c->predictor = order;
    c->have_hist = false;
    return c->tmu ? fmm_set_dipole_predictor(c->tmu, order) : POLFMM_OK;
}

int fmm_set_thole(polfmm_ctx* c, double a) {
    if (!c || !(a >= 0.0) || !isfinite(a)) return POLFMM_ERR_INVALID_ARG;
    if (a > 0.0 && !c->a16) {
        const int64_t n = c->n;
        int nb = 1024;  // a power of two <= max(n, 4096): the tree's scan scratch holds it
        while ((int64_t)nb * 2 <= std::max<int64_t>(n, 4096)) nb *= 2;
        Alloc& A = extra_of(c)->alloc;
        c->th_nb = nb;
        c->a16 = A.get<double>(n);
        c->th_xa = A.get<float4>(n);
        c->th_bucket = A.get<int>(nb + 1);
        c->th_count = A.get<int>(nb);
        c->th_member = A.get<int>(n);
        c->th_cell = A.get<int4>(n);
        c->th_cnt = A.get<int>(n + 64);
        c->th_ptr = A.get<int>(n + 1);
        c->th_max = A.get<double>(2);
        c->thE = A.get<double>(3 * n);
        c->thF = A.get<double>(3 * n);
        c->thdA = A.get<double>(n);
        if (!A.ok) {
            c->a16 = nullptr;
            return POLFMM_ERR_OUT_OF_MEMORY;
        }
    }
    c->thole_a = a;
    int rc = thole_pairs(c);
    if (rc != POLFMM_OK) return rc;
    c->pcg_graph_dirty = true;  // the solver pass gains (or loses) the correction kernel
    c->loop_dirty = true;
    if (c->tmu && (rc = fmm_set_thole(c->tmu, a)) != POLFMM_OK) return rc;
    return read_err(c);
}

int fmm_field_charge_gradient(polfmm_ctx* c, double* dU_dqE, int on_device) {
    if (!c || !dU_dqE) return POLFMM_ERR_INVALID_ARG;
    if (!c->have_dqE) return POLFMM_ERR_STATE;
    int rc = scatter_out(c, c->dqE, dU_dqE, 1, on_device);
    return rc != POLFMM_OK ? rc : read_err(c);
}

int fmm_update_positions(polfmm_ctx* c, const double* positions, int on_device) {
    if (!c || !positions) return POLFMM_ERR_INVALID_ARG;
    const int64_t n = c->n;
    if (!on_device && !finite_host(positions, 3 * (size_t)n)) return POLFMM_ERR_INVALID_ARG;
    // current q, alpha and dipoles back to caller order, then the new positions
    scatter_sites(c, c->q_s, c->in_buf + 3 * n, 1);
    scatter_sites(c, c->alpha_s, c->in_buf + 4 * n, 1);
    if (c->have_mu) {
        scatter_sites(c, c->mu, c->in_buf + 5 * n, 3);
        if (c->predictor == 1) {
            if (c->have_hist) {
                LaunchScope ls(c, F_SOLVER);
                extrapolate_kernel<<<grid_for(3 * n, 256), 256, 0, c->stream>>>(3 * n, c->in_buf + 5 * n, c->mu_hist);
            } else {
                cudaMemcpyAsync(c->mu_hist, c->in_buf + 5 * n, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice,
                                c->stream);
                c->have_hist = true;
            }
        }
    }
    if (c->qE_s) scatter_sites(c, c->qE_s, c->in_buf + 8 * n, 1);
    c->have_dqE = false;
    int rc = copy_in(c, c->in_buf, positions, 3 * (size_t)n, on_device);
    if (rc != POLFMM_OK) return rc;
    if ((rc = rebuild(c)) != POLFMM_OK) return rc;
    if (c->have_mu) {
        gather_sites(c, c->in_buf + 5 * n, c->mu, 3);
        mask_dipoles(c, c->mu);
    }
    if (c->tmu) {
        {
            LaunchScope ls(c, F_TREE);
            take_rows_kernel<<<grid_for(3 * c->nmu, 256), 256, 0, c->stream>>>(c->nmu, 3, c->mu_rows, c->in_buf,
                                                                               c->tmu_rows);
        }
        if ((rc = fmm_update_positions(c->tmu, c->tmu_rows, 1)) != POLFMM_OK) return rc;
    }
    return read_err(c);
}

int fmm_static_field(polfmm_ctx* c, double* phi, double* E, int on_device) {
    if (!c) return POLFMM_ERR_INVALID_ARG;
    int rc = scatter_out(c, c->phiq, phi, 1, on_device);
    if (rc == POLFMM_OK) rc = scatter_out(c, c->Eq, E, 3, on_device);
    return rc != POLFMM_OK ? rc : read_err(c);
}

int fmm_dipole_field(polfmm_ctx* c, const double* mu, double* E, int on_device) {
    if (!c || !mu || !E) return POLFMM_ERR_INVALID_ARG;
    int rc = copy_in(c, c->in_buf + 5 * c->n, mu, 3 * (size_t)c->n, on_device);
    if (rc != POLFMM_OK) return rc;
    gather_sites(c, c->in_buf + 5 * c->n, c->d, 3);
    fmm_pass(c, LEAF_DIPOLE_E, false, c->d, nullptr, c->Td, nullptr);
    rc = scatter_out(c, c->Td, E, 3, on_device);
    return rc != POLFMM_OK ? rc : read_err(c);
}

int fmm_total_field(polfmm_ctx* c, const double* mu, double* phi, double* E, double* G, int on_device) {
    if (!c) return POLFMM_ERR_INVALID_ARG;
    int rc;
    if (mu) {
        if ((rc = copy_in(c, c->in_buf + 5 * c->n, mu, 3 * (size_t)c->n, on_device)) != POLFMM_OK) return rc;
        gather_sites(c, c->in_buf + 5 * c->n, c->d, 3);
    } else {
        cudaMemsetAsync(c->d, 0, sizeof(double) * 3 * c->n, c->stream);
    }
    fmm_pass(c, LEAF_FULL, true, c->d, c->phi_t, c->E_t, c->G_t);
    if ((rc = scatter_out(c, c->phi_t, phi, 1, on_device)) != POLFMM_OK) return rc;
    if ((rc = scatter_out(c, c->E_t, E, 3, on_device)) != POLFMM_OK) return rc;
    if ((rc = scatter_out(c, c->G_t, G, 6, on_device)) != POLFMM_OK) return rc;
    return read_err(c);
}

int fmm_leaf_cells(polfmm_ctx* c, int32_t* cells, int on_device) {
    if (!c || !cells) return POLFMM_ERR_INVALID_ARG;
    int32_t* dst = on_device ? cells : (int32_t*)c->out_buf;
    {
        LaunchScope ls(c, F_TREE);
        leaf_cells_kernel<<<grid_for(c->n, 256), 256, 0, c->stream>>>(c->n, c->key_s, c->perm, dst);
    }
    if (!on_device &&
        cudaMemcpyAsync(cells, dst, sizeof(int32_t) * 3 * c->n, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return POLFMM_ERR_CUDA;
    return read_err(c);
}

int fmm_tree_info(polfmm_ctx* c, int64_t* info) {
    if (!c || !info) return POLFMM_ERR_INVALID_ARG;
    info[0] = c->depth;
    info[1] = c->p;
    for (int l = 0; l <= c->depth; l++) info[2 + l] = c->lv[l].nbox;
    return POLFMM_OK;
}

int fmm_root_box(polfmm_ctx* c, double* lo, double* side) {
    if (!c || !lo || !side) return POLFMM_ERR_INVALID_ARG;
    for (int d = 0; d < 3; d++) lo[d] = c->lo[d];
    *side = c->side;
    return POLFMM_OK;
}

int fmm_profile_get(polfmm_ctx* c, const char* family, double* total_ms, int64_t* launches) {
    static const char* names[F_COUNT] = {"tree",      "p2m",       "m2m",    "m2l",      "l2l", "leaf_dipole",
                                         "leaf_static", "leaf_full", "solver", "assemble", "l2p"};
    if (!c || !family) return POLFMM_ERR_INVALID_ARG;
    profile_flush(c);
    for (int f = 0; f < F_COUNT; f++)
        if (!strcmp(family, names[f])) {
            // with a dipole tree, its kernels count with the context's
            double t_ms = 0.0;
            int64_t t_n = 0;
            if (c->tmu) fmm_profile_get(c->tmu, family, &t_ms, &t_n);
            if (total_ms) *total_ms = c->prof_ms[f] + t_ms;
            if (launches) *launches = c->prof_n[f] + t_n;
            return POLFMM_OK;
        }
    return POLFMM_ERR_INVALID_ARG;
}

int fmm_profile_reset(polfmm_ctx* c) {
    if (!c) return POLFMM_ERR_INVALID_ARG;
    profile_flush(c);
    for (int f = 0; f < F_COUNT; f++) {
        c->prof_ms[f] = 0;
        c->prof_n[f] = 0;
    }
    return c->tmu ? fmm_profile_reset(c->tmu) : POLFMM_OK;
}

int64_t fmm_launch_count(polfmm_ctx* c) { return c ? c->launches + fmm_launch_count(c->tmu) : 0; }

int64_t fmm_testing_alloc_hook(int64_t fail_at) {
    const int64_t made = g_alloc_count.exchange(0);
    g_alloc_fail_at.store(fail_at >= 0 ? fail_at : -1);
    return made;
}

void fmm_destroy(polfmm_ctx* c) { destroy_impl(c); }

const char* fmm_last_error(void) { return g_last_error; }

const char* fmm_status_string(int s) {
    switch (s) {
        case POLFMM_OK: return "ok";
        case POLFMM_ERR_INVALID_ARG: return "invalid argument";
        case POLFMM_ERR_COINCIDENT: return "coincident sites";
        case POLFMM_ERR_NOT_CONVERGED: return "dipole solve not converged";
        case POLFMM_ERR_OUT_OF_MEMORY: return "out of device memory";
        case POLFMM_ERR_CUDA: return "CUDA error";
        case POLFMM_ERR_STATE: return "call out of order";
        default: return "unknown status";
    }
}

}  // extern "C"
