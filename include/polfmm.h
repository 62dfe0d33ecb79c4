/*
 * polfmm -- polarizable fast multipole method on one GB300 GPU (sm_103a).
 *
 * C ABI of the hot path of Coles & Masella, "The Fast Multipole Method and
 * Point Dipole Moment Polarizable Force Fields" (arXiv:1408.6527): the FMM
 * evaluation of potential, field and field gradient produced by point charges
 * plus induced point dipoles (Sec. II.B, II.C), called once per iteration of
 * the self-consistent dipole solve mu_i = alpha_i (E^q_i + E^mu_i) (Sec. II.A,
 * Eq. dipole moment) and once more for energy and forces (Sec. III, the three
 * stages).
 *
 * Units and conventions (used by every call):
 *   - lengths in Angstrom, charges in e, polarizabilities in Angstrom^3
 *     (isotropic scalars, Sec. III); the field is computed with Coulomb
 *     constant 1 so that mu = alpha E holds directly; energies, forces and
 *     parameter gradients are multiplied by options.coulomb_k.
 *   - positions, forces, dipoles and fields are n x 3 row-major float64
 *     (AoS: x0 y0 z0 x1 ...); potentials, charges and gradients are n float64.
 *   - field gradients are n x 6 float64 in the order xx xy xz yy yz zz.
 *   - every per-site output is in the caller's site order.
 *   - a pointer flagged "on_device" must be a device pointer valid on the
 *     context's stream; otherwise it is host memory.  The library copies all
 *     inputs into its own device buffers; the caller keeps ownership of every
 *     pointer it passes and the library keeps none after a call returns.
 *   - no call traps, aborts or prints; every int-returning call returns one
 *     of the POLFMM_* status codes below.
 *   - calls on one context must not overlap; distinct contexts are independent.
 *   - every reduction (energies, dot products of the solver, the partial sums of
 *     the multipole-to-local pass) adds its terms in a fixed order, so the same
 *     inputs give bitwise identical outputs on every run; there is no
 *     non-deterministic fast path to switch off.
 */
#ifndef POLFMM_H
#define POLFMM_H

#include <stdint.h>

#if defined(__GNUC__)
#define POLFMM_API __attribute__((visibility("default")))
#else
#define POLFMM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define POLFMM_OK 0
#define POLFMM_ERR_INVALID_ARG 1   /* n outside [1, 2^28], p outside [1,10], depth outside [1,8], alpha < 0, non-finite input */
#define POLFMM_ERR_COINCIDENT 2    /* two distinct sites at the same position */
#define POLFMM_ERR_NOT_CONVERGED 3 /* dipole solve stopped at max_iter or diverged; dipoles stay readable */
#define POLFMM_ERR_OUT_OF_MEMORY 4
#define POLFMM_ERR_CUDA 5
#define POLFMM_ERR_STATE 6         /* call out of order, e.g. energy before a solve */

/* Precision of the FMM arithmetic.  FP64: everything in float64.  MIXED:
 * expansions, translations and near-field pairs in float32 (the
 * multipole-to-local translation on tensor cores), while the dipole solver
 * vectors, its dot products and convergence test, and the energy sums stay in
 * float64. */
#define POLFMM_FP64 0
#define POLFMM_MIXED 1

/* Dipole solver. */
#define POLFMM_SOLVER_PCG 0    /* conjugate gradients on (diag(1/alpha) - T) mu = E^q, Jacobi preconditioner */
#define POLFMM_SOLVER_JACOBI 1 /* fixed point mu <- alpha (E^q + T mu) */

/* Multipole-to-local implementation (MIXED only; FP64 always uses the SIMT kernel).
 * AUTO: FFMA for p <= 6, TENSOR for p = 7, 8.
 * SIMT: the generic kernel (32-box tiles, accumulators in shared memory).
 * TENSOR: tcgen05 TF32 tensor cores with three products (FP32-level accuracy).
 * FFMA (p <= 6; otherwise as AUTO): FP32 on the CUDA cores, one target box per lane
 * with its coefficients in registers. */
#define POLFMM_M2L_AUTO 0
#define POLFMM_M2L_SIMT 1
#define POLFMM_M2L_TENSOR 2
#define POLFMM_M2L_FFMA 3

typedef struct polfmm_ctx polfmm_ctx; /* opaque; owned by the library */

typedef struct {
    int mode;            /* POLFMM_FP64 or POLFMM_MIXED */
    int solver;          /* POLFMM_SOLVER_* */
    int max_iter;        /* dipole-solve iteration cap (default 100) */
    double coulomb_k;    /* energy / force scale (default 1.0) */
    int use_root_box;    /* 1: use root_lo / root_side instead of the bounding cube */
    double root_lo[3];   /* lower corner of the root cube (Angstrom) */
    double root_side;    /* side of the root cube (Angstrom) */
    int m2l_impl;        /* POLFMM_M2L_* */
    int profile;         /* 1: time kernels with CUDA events (see fmm_profile_get) */
    void* cuda_stream;   /* cudaStream_t for all work; NULL = the legacy default stream */
    int no_graphs;       /* 1: launch every solver iteration kernel by kernel instead of replaying a
                            CUDA graph of one iteration (graphs are also off while profiling) */
    double dipole_dl;    /* 0 (default): a point dipole enters the multipoles analytically (the
                            limit of Sec. II.C).  > 0: as the pair of charges +-q^mu at
                            x +- dl mu/|mu|, q^mu = |mu| / (2 dl) (Sec. II.C, mu = 2 |q^mu| dl);
                            the near-field pairs and the field at the sites keep the explicit
                            dipole.  FP64 mode only (in FP32 the pair's multipole cancels
                            catastrophically); dl must not exceed a quarter of the leaf side:
                            POLFMM_ERR_INVALID_ARG otherwise, at fmm_build or at a rebuild. */
    int no_pdl;          /* 1: launch the kernels of a solver iteration with plain stream order
                            instead of programmatic dependent launch (0, the default: each of
                            them may be scheduled while its predecessor drains; it waits for the
                            predecessor's completion before it reads that kernel's output) */
    int dipole_tree;     /* 0 (default): one tree for everything.  1: the dipole solve runs on a
                            second tree over the polarizable sites only (alpha > 0), T^mu of
                            Sec. III: its depth is the given depth less log8(n / n_mu), rounded
                            down; the field that polarizes the sites comes from the full tree,
                            and the converged dipoles go back to it for the energy and forces.
                            Exclusions (pairs of polarizable sites), Thole damping, the dipole
                            predictor and set dipoles are passed on to it.  When every site (or
                            none) is polarizable the two trees coincide and one is used. */
} polfmm_options;

/* Fill *opt with the defaults: FP64, PCG, max_iter 100, coulomb_k 1, bounding
 * root cube, automatic M2L choice, no profiling, default stream, analytic
 * point-dipole multipoles (dipole_dl = 0). */
POLFMM_API void fmm_default_options(polfmm_options* opt);

/*
 * Build the octree and run the static pass (first stage of Sec. III).
 *
 * positions      n x 3 site positions.
 * charges        n static charges q_i (Sec. II.A, Eq. equ:Uqq).
 * polarizabilities n isotropic alpha_i >= 0; alpha_i = 0 marks a site without
 *                an induced dipole.
 * order_p        expansion order p in [1, 10]: terms with |n| + |m| <= p of the
 *                two-centre Taylor expansion of Sec. II.B are kept.
 * tree_depth     leaf level of the uniform octree in [1, 8] (root = level 0).
 * opt            options (NULL = defaults).
 * inputs_on_device 1 if the three arrays are device pointers.
 *
 * The root cube is the bounding box of the sites, centred, with side equal to
 * the largest extent times (1 + 1e-6) (1 Angstrom if all coincide), unless
 * opt->use_root_box.  A site's leaf is floor((x - lo) / h), h = side / 2^depth,
 * clamped into the cube.  Boxes interact through multipoles when they are not
 * adjacent but their parents are (or coincide); adjacent leaves interact
 * directly.  On success *ctx owns all device state and the static field E^q
 * and potential Phi^q of the charges are available.  On failure *ctx is NULL.
 */
POLFMM_API int fmm_build(polfmm_ctx** ctx, int64_t n, const double* positions, const double* charges,
              const double* polarizabilities, int order_p, int tree_depth,
              const polfmm_options* opt, int inputs_on_device);

/*
 * Solve mu_i = alpha_i (E^q_i + E^mu_i) (Sec. II.A, Eq. dipole moment; second
 * stage of Sec. III) with the FMM dipole-field operator, starting from the
 * previous dipoles if any (fmm_set_dipoles, fmm_update_positions), else from
 * mu = alpha E^q.  Stops when ||r||_2 / ||E^q||_2 <= tolerance, r the residual
 * of (diag(1/alpha) - T) mu = E^q, or after max_iter iterations.
 * iterations_out / residual_out (nullable) receive the count and final
 * relative residual.  Returns POLFMM_ERR_NOT_CONVERGED, with the dipoles and
 * residual of the last good iterate readable, when
 *   - the cap is hit;
 *   - the residual turns non-finite;
 *   - a conjugate direction has d.(diag(1/alpha) - T) d <= 0: the operator is
 *     not positive definite (the polarization catastrophe of point dipoles);
 *     that direction is not applied;
 *   - the residual grew in 3 consecutive iterations (stagnation, or a
 *     diverging fixed-point iteration).
 */
POLFMM_API int fmm_solve_induced_dipoles(polfmm_ctx* ctx, double tolerance, int* iterations_out,
                              double* residual_out);

/*
 * Energy and gradients at the current dipoles (third stage of Sec. III).
 * One FMM pass with charges and dipoles as sources gives the total potential
 * Phi, field E and field gradient G at every site; then
 *   energy_out[0] = U = U^qq' + U^pol, energy_out[1] = U^qq' = 1/2 sum q Phi^q,
 *   energy_out[2] = U^pol = sum |mu|^2/(2 alpha) - sum mu.E^q - 1/2 sum mu.E^mu
 *   (Sec. II.A), all host float64, times coulomb_k;
 *   forces = -dU/dx = q E + (grad E) mu (n x 3), valid at a converged solve
 *   because dU^pol/dmu = 0 (Eq. upol_derivatives);
 *   dU_dq = Phi (total potential, n), dU_dalpha = -|mu|^2/(2 alpha^2) (n;
 *   -|E|^2/2 where alpha = 0).
 * forces, dU_dq, dU_dalpha are nullable.  Requires a prior
 * fmm_solve_induced_dipoles or fmm_set_dipoles (else POLFMM_ERR_STATE).
 */
POLFMM_API int fmm_energy_forces(polfmm_ctx* ctx, double* energy_out, double* forces, double* dU_dq,
                      double* dU_dalpha, int outputs_on_device);

/*
 * Stationary energy without the force pass: energy_out (host, 3 doubles) =
 * [U, U^qq', U^pol] with U^qq' = 1/2 sum q Phi^q (Sec. II.A, Eq. equ:Uqq) and
 * U^pol = -1/2 sum mu.E^q, the value of the polarization energy at the solution
 * of the dipole equations (Sec. II.A, Eq. upol_derivatives), both times
 * coulomb_k.  Uses the static pass of the tree and the current dipoles, summed
 * in float64 in a fixed order.  Valid after a converged
 * fmm_solve_induced_dipoles; for arbitrary dipoles (fmm_set_dipoles) use
 * fmm_energy_forces, whose U^pol is the full expression.  POLFMM_ERR_STATE
 * before any dipoles exist.
 */
POLFMM_API int fmm_energy(polfmm_ctx* ctx, double* energy_out);

/* Copy the current induced dipoles (n x 3) out; POLFMM_ERR_STATE before any. */
POLFMM_API int fmm_get_dipoles(polfmm_ctx* ctx, double* mu, int on_device);

/* Set the induced dipoles (n x 3), e.g. a warm start or a fixed set for an
 * energy evaluation; entries at sites with alpha = 0 are ignored (set to 0). */
POLFMM_API int fmm_set_dipoles(polfmm_ctx* ctx, const double* mu, int on_device);

/* Forget the current dipoles: the next solve starts again from mu = alpha E^q. */
POLFMM_API int fmm_reset_dipoles(polfmm_ctx* ctx);

/*
 * Field charges (Sec. III: the set of charges q^E that generate the field
 * polarizing the sites, which the force field may choose apart from the
 * Coulomb charges q; Sec. II.A, E^q).  qE: n float64 in caller order.  After
 * this call the static field that polarizes the sites is that of the q^E, the
 * Coulomb energy U^qq' and its field stay those of the q, and
 * fmm_energy_forces returns
 *   U^pol = sum |mu|^2/(2 alpha) - sum mu.E^qE - 1/2 sum mu.E^mu,
 *   F = q E^q + q^E E^mu + (grad E^qE + grad E^mu) mu,
 *   dU/dq = Phi^q (potential of the Coulomb charges),
 * with dU/dq^E = Phi^mu (potential of the dipoles) from
 * fmm_field_charge_gradient.  Without this call q^E = q and dU/dq = Phi^q +
 * Phi^mu.  Runs the field charges' static pass; kept across
 * fmm_update_positions.  The dipoles are kept as the next solve's guess.
 */
POLFMM_API int fmm_set_field_charges(polfmm_ctx* ctx, const double* qE, int on_device);

/*
 * Excluded pairs (Sec. II.A: the starred sums skip a list of pairs, e.g. atoms
 * less than two chemical bonds apart).  pairs: npairs x 2 int32 caller indices
 * (i != j, each in [0, n); duplicates and both orders allowed); npairs = 0
 * clears the list.  Every pair is removed from all three sums -- the Coulomb
 * energy and potential, the static field, and the dipole field of every
 * solver iteration and of the force pass -- by subtracting its direct terms
 * from the FMM result over all pairs (one thread per site, partners in
 * ascending order: deterministic).  Reruns the static passes; kept across
 * fmm_update_positions.  fmm_static_field, fmm_dipole_field and
 * fmm_total_field honour the list too.  POLFMM_ERR_INVALID_ARG for an index
 * out of range or i == j.
 */
POLFMM_API int fmm_set_exclusions(polfmm_ctx* ctx, int64_t npairs, const int32_t* pairs, int on_device);

/* dU/dq^E = Phi^mu (n, caller order) from the last fmm_energy_forces with field
 * charges set; POLFMM_ERR_STATE before one. */
POLFMM_API int fmm_field_charge_gradient(polfmm_ctx* ctx, double* dU_dqE, int on_device);

/*
 * Thole damping of the dipole-dipole interaction (Sec. II.A names Thole's
 * model as part of the force field without printing it; the form is Thole's
 * exponential model as used by the AMOEBA force field: B. T. Thole, Chem.
 * Phys. 59, 341 (1981); P. Ren and J. W. Ponder, J. Phys. Chem. B 107, 5933
 * (2003)).  Between two polarizable sites the field of a dipole,
 * 3 (mu.r) r / r^5 - mu / r^3, becomes
 *   lambda5 3 (mu.r) r / r^5 - lambda3 mu / r^3,  u = r / (alpha_i alpha_j)^(1/6),
 *   lambda3 = 1 - exp(-a u^3),  lambda5 = 1 - (1 + a u^3) exp(-a u^3).
 * Charge-dipole terms and pairs with a non-polarizable site stay undamped;
 * excluded pairs stay excluded.  The damping changes the dipole solve, the
 * energy, the forces (the derivatives of lambda3 and lambda5 included) and
 * dU/dalpha; fmm_static_field, fmm_dipole_field and fmm_total_field keep
 * returning the undamped FMM fields.  The pairs with a u^3 < 40 (beyond,
 * exp(-a u^3) < 5e-18) are listed per tree with a spatial hash and corrected
 * with direct pair terms (damped minus undamped), in the mode's precision
 * (FP32 in MIXED).  a = 0 switches it off;
 * a < 0 or non-finite: POLFMM_ERR_INVALID_ARG.  Kept across
 * fmm_update_positions; the next solve starts from the current dipoles.
 */
POLFMM_API int fmm_set_thole(polfmm_ctx* ctx, double a);

/*
 * Start of the next dipole solve after fmm_update_positions (a dipole
 * predictor for molecular dynamics, Sec. IV.B warm-starts each step's solve
 * from earlier dipoles): order 0 (default) starts from the last dipoles;
 * order 1 extrapolates linearly from the last two updates,
 * mu_start = 2 mu(t) - mu(t - dt), once two updates have been seen.
 * fmm_set_dipoles and fmm_reset_dipoles restart the history.  Other orders:
 * POLFMM_ERR_INVALID_ARG.
 */
POLFMM_API int fmm_set_dipole_predictor(polfmm_ctx* ctx, int order);

/* New positions for the same sites: rebuild the tree and the static pass,
 * keeping the current dipoles as the next solve's starting guess. */
POLFMM_API int fmm_update_positions(polfmm_ctx* ctx, const double* positions, int on_device);

/* Static potential Phi^q (n) and field E^q (n x 3) of the charges at every
 * site, from the build's FMM pass (Sec. III, first stage).  Either nullable. */
POLFMM_API int fmm_static_field(polfmm_ctx* ctx, double* phi, double* E, int on_device);

/* One application of the FMM dipole-field operator: E = T mu, the field at
 * every site of the point dipoles mu (n x 3) at the other sites (Sec. II.A,
 * E^mu; Sec. II.C).  This is the matrix-vector product of every solver
 * iteration. */
POLFMM_API int fmm_dipole_field(polfmm_ctx* ctx, const double* mu, double* E, int on_device);

/* One full FMM pass with the build's charges and the given dipoles mu (n x 3,
 * nullable = none) as sources: total potential (n), field (n x 3) and field
 * gradient (n x 6) at every site.  Outputs nullable. */
POLFMM_API int fmm_total_field(polfmm_ctx* ctx, const double* mu, double* phi, double* E, double* G,
                    int on_device);

/* Leaf cell (integer coordinates in [0, 2^depth)^3, n x 3 int32) of every site. */
POLFMM_API int fmm_leaf_cells(polfmm_ctx* ctx, int32_t* cells, int on_device);

/* Tree summary: info[0] = depth, info[1] = p, info[2 + l] = occupied boxes at
 * level l for l = 0..depth.  info must hold depth + 3 entries (at most 11). */
POLFMM_API int fmm_tree_info(polfmm_ctx* ctx, int64_t* info);

/* Root cube actually used: lo[3] and side. */
POLFMM_API int fmm_root_box(polfmm_ctx* ctx, double* lo, double* side);

/* Profiling (options.profile = 1): total CUDA-event milliseconds and launch
 * count of one kernel family since the last reset.  Families: "tree", "p2m"
 * (the upward pass: P2M and every M2M level in one launch), "m2l",
 * "leaf_dipole" (near field of the solver's dipole-field pass), "l2p" (L2L +
 * L2P of that pass, with the d.Ad reduction), "leaf_static" (L2L + L2P + near
 * field, static pass), "leaf_full" (same, energy / force pass), "solver",
 * "assemble"; "m2m" and "l2l" are accepted and stay at zero (those steps run
 * inside the "p2m", "l2p" and "leaf_*" kernels).
 * Unknown names return POLFMM_ERR_INVALID_ARG. */
POLFMM_API int fmm_profile_get(polfmm_ctx* ctx, const char* family, double* total_ms, int64_t* launches);
POLFMM_API int fmm_profile_reset(polfmm_ctx* ctx);

/* Count of the library's own kernel launches on this context since creation
 * (with polfmm_options.dipole_tree, those of its dipole tree included; the
 * same holds for fmm_profile_get and fmm_profile_reset). */
POLFMM_API int64_t fmm_launch_count(polfmm_ctx* ctx);

/*
 * Testing hook for the out-of-memory paths (the paper has no counterpart).
 * Returns how many device or pinned-host allocations the library made since
 * the previous call, and arms a planted failure: the fail_at-th allocation
 * from now (0 = the next one) reports out of memory, once; fail_at < 0
 * disarms it.  Process-wide, not thread-safe against concurrent builds.
 */
POLFMM_API int64_t fmm_testing_alloc_hook(int64_t fail_at);

/*
 * Testing: the schedule the FP32 CUDA-core M2L (MIXED, p <= 6) is compiled
 * with, for checks on the CPU.  For order p and part (0: the warp with the
 * outputs of degree <= split, 1: the warp with the others) it writes up to cap
 * terms of L_n += D_k M_m in execution order: n (relative to the part's first
 * output), m and k = index of n + m in the coefficient order, and load = 1
 * where the term's float4 of D is loaded.  Returns the part's term count, and
 * through split_out (if not NULL) the degree split; -1 for p outside 1..6 or
 * a part other than 0, 1.  Host only, no device work.
 */
POLFMM_API int fmm_testing_m2l_plan(int p, int part, int cap, int* n, int* m, int* k, int* load, int* split_out);

/*
 * Allocation-free tree set-up.  The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc -- code whose host framework
 * owns all device memory through its own pool, or a time-critical loop that
 * cannot afford the device-wide synchronisation that cudaMalloc and cudaFree
 * imply.  It computes, without allocating anything (no cudaMalloc, cudaFree or
 * allocating library routine), what fmm_build computes first: the root cube
 * (same rule as fmm_build), the leaf cell of every site, the Morton keys of
 * the cells and the stable sort of the sites by key.
 *
 * n              sites, 1 <= n <= POLFMM_NOALLOC_MAX_SITES (larger n: the call
 *                returns POLFMM_ERR_INVALID_ARG and does nothing).
 * positions      device, n x 3 float64 (caller order).
 * tree_depth     leaf level in [1, 8].
 * root_lo, root_side  host outputs: lower corner (3) and side of the root cube.
 * cells          device output, n x 3 int32: leaf cell of each site (caller order).
 * keys           device output, n uint32: Morton keys of the leaf cells in
 *                ascending order.
 * perm           device output, n int32: perm[k] = caller index of the site
 *                with the k-th key; sites with equal keys keep caller order.
 * cuda_stream    cudaStream_t (NULL = legacy default stream); the call returns
 *                after the stream has finished its work.
 *
 * All temporaries live in one static device array of about 2.3 MB that every
 * device which loads the library holds until the process exits.  The first
 * call on a device looks up that array's device address (cudaGetSymbolAddress,
 * with that device current), so that first call should come before any stream
 * capture.  The address is kept for the life of the process: a
 * cudaDeviceReset unloads the module and makes it stale, so a process that
 * resets a device must not call this entry point on that device afterwards.  Every call shares the array and it keeps the previous call's
 * contents: calls that overlap on the GPU (several streams, threads or
 * devices sharing a context) race and must be serialised by the caller.
 * Non-finite positions return POLFMM_ERR_INVALID_ARG.
 */
#define POLFMM_NOALLOC_MAX_SITES 262144
POLFMM_API int fmm_sort_sites_noalloc(int64_t n, const double* positions, int tree_depth, double* root_lo,
                                      double* root_side, int32_t* cells, uint32_t* keys, int32_t* perm,
                                      void* cuda_stream);

/*
 * The paper's own tree and walk (Sec. III), in FP64: potential, field and
 * field gradient at every site from charges and point dipoles, by an FMM on
 * an adaptive kd-tree.  A cell's particles split across the longest dimension
 * of their box, at their geometric centre along it, until a cell holds at most
 * n_bucket particles (8 in the paper); every cell expands about the centre of
 * its particles, with r_enc the distance to the farthest corner of its box
 * (padded by `pad` Angstrom on every side below three particles).  A mutual
 * dual-tree walk from (root, root) sums a pair directly when it holds fewer
 * than n_direct particles (about 64 in the paper) or both cells are leaves,
 * through multipoles when theta |z_A - z_B| > r_enc,A + r_enc,B (Eq. mac), and
 * otherwise splits the cell with the larger r_enc (a self pair pushes its
 * three child combinations).  Expansions keep |n| + |m| <= order_p (1..7);
 * dipole_dl > 0 builds the dipoles' multipoles from the +-q pairs of Sec.
 * II.C.  charges, dipoles and any output may be NULL.  stats (nullable)
 * receives 5 counts: cells, leaves, levels, multipole pairs, direct pairs.
 * Deterministic; allocates and frees its own device memory; synchronises
 * cuda_stream.  Each site's own term is excluded (Sec. II.A).  0 <= theta < 1
 * (0: every pair direct),
 * n_bucket >= 1: POLFMM_ERR_INVALID_ARG otherwise.
 */
POLFMM_API int fmm_kdtree_fields(int64_t n, const double* positions, const double* charges, const double* dipoles,
                                 int order_p, double theta, int n_bucket, int n_direct, double pad, double dipole_dl,
                                 double* phi, double* E, double* G, int64_t* stats, void* cuda_stream,
                                 int on_device);

/*
 * Dynamics around the FMM (Sec. IV.B runs molecular dynamics on these forces,
 * with the long-range part on a longer time step than the short-range part).
 * The paper's force field has short-range terms of its own, which are not part
 * of this library; the calls below give the purely repulsive wall that keeps
 * undamped point dipoles apart during a run, and the kicks and drifts of
 * velocity Verlet and of the reversible multiple-time-step integrator, so that
 * a step runs in device kernels only.  All pointers are device pointers on the
 * stream named at creation (or given); all arrays are float64, positions,
 * velocities and forces n x 3 row-major, masses n.
 *
 * fmm_wall_create: scratch for up to max_sites sites (1 <= max_sites <= 2^28;
 * about 40 bytes per site plus a hash table of 8 bytes per bucket, with at
 * least 2 max_sites buckets).  POLFMM_ERR_OUT_OF_MEMORY leaves *out NULL.
 */
typedef struct polfmm_wall polfmm_wall;
POLFMM_API int fmm_wall_create(polfmm_wall** out, int64_t max_sites, void* cuda_stream);

/*
 * The wall U = sum over pairs i < j with r_ij < r_c = 2^(1/6) sigma of
 * 4 eps [(sigma/r_ij)^12 - (sigma/r_ij)^6] + eps (zero and with zero slope at
 * r_c) and its forces F_i = -dU/dx_i, in FP64.  energy: one double, written on
 * the device (the caller reads it when it needs it); forces: n x 3,
 * overwritten.  Pairs come from a spatial hash of cells of side r_c; every sum
 * runs in a fixed order, so that the outputs are bitwise reproducible.
 * POLFMM_ERR_INVALID_ARG for n > max_sites, eps < 0 or sigma <= 0.  Coincident
 * sites give non-finite values (the FMM rejects them at fmm_build).
 */
POLFMM_API int fmm_wall_forces(polfmm_wall* wall, const double* positions, int64_t n, double eps, double sigma,
                               double* energy, double* forces);

/* Kinetic energy scale * sum_i 1/2 m_i |v_i|^2 into one device double (fixed
 * summation order), on the wall's stream and scratch. */
POLFMM_API int fmm_md_kinetic(polfmm_wall* wall, const double* velocities, const double* masses, int64_t n,
                              double scale, double* energy);

/* Kick v_i += coef * F_i / m_i (coef = the time step share times the unit
 * conversion from force / mass to acceleration). */
POLFMM_API int fmm_md_kick(double* velocities, const double* forces, const double* masses, double coef, int64_t n,
                           void* cuda_stream);

/* Total momentum sum_i m_i v_i (three device doubles, fixed summation order),
 * on the wall's stream and scratch. */
POLFMM_API int fmm_md_momentum(polfmm_wall* wall, const double* velocities, const double* masses, int64_t n,
                               double* momentum);

/* Drift x_i += dt * v_i. */
POLFMM_API int fmm_md_drift(double* positions, const double* velocities, double dt, int64_t n, void* cuda_stream);

/* Release the wall's scratch (after its stream has finished); NULL is a no-op. */
POLFMM_API void fmm_wall_destroy(polfmm_wall* wall);

/*
 * Measured peak rate of one arithmetic unit of the current device, for
 * roofline fractions (the paper has no counterpart): what = 0 -> FP32 fused
 * multiply-add, 1 -> FP64 fused multiply-add, in TFLOP/s (FMA = 2 flops), from
 * the fastest of three timed launches of independent FMA chains on every SM
 * (CUDA events on cuda_stream, NULL = legacy default stream).  Allocates and
 * frees a few bytes of device memory.
 */
POLFMM_API int fmm_measure_peak(int what, void* cuda_stream, double* tflops);

/* Release every device buffer of the context; NULL is a no-op. */
POLFMM_API void fmm_destroy(polfmm_ctx* ctx);

/* Description of the CUDA failure behind the last POLFMM_ERR_CUDA returned on
 * the calling thread ("" if none): the CUDA error name and string, or which
 * bounded device wait timed out. */
POLFMM_API const char* fmm_last_error(void);

/* Static description of a status code. */
POLFMM_API const char* fmm_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* POLFMM_H */
