/*
 * CPU oracle for the polarizable fast multipole method of Coles & Masella,
 * "The Fast Multipole Method and Point Dipole Moment Polarizable Force Fields"
 * (arXiv:1408.6527).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain FP64 reference the
 * CUDA path is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table
 * or constant generator with the CUDA library.
 *
 * Contents (each function cites the passage it follows):
 *   orc_direct       O(N^2) potential, field and field gradient from point
 *                    charges and point dipoles (Sec. II.A, Eqs. for U^qq',
 *                    E^q, E^mu and the dipolar tensor T_ij).
 *   orc_derivatives  Cartesian derivatives of 1/r up to a total order.
 *   orc_p2m / orc_m2m / orc_m2l / orc_l2l / orc_l2p
 *                    single-box FMM operators of Sec. II.B (multipole
 *                    expansion, shift, multipole-to-local, local shift,
 *                    evaluation), un-normalised, in FP64.
 *   orc_fmm          a complete CPU FMM on a uniform octree: leaves at a
 *                    fixed depth, the well-separated rule "not adjacent but
 *                    parents adjacent", per-pair derivative evaluation, and
 *                    near-field direct sums over the 27 adjacent leaves
 *                    (Sec. II.B and Sec. III, Phi = Phi^direct + Phi^fmm).
 *   orc_fmm_ex       orc_fmm with two options: the dipoles' multipoles from
 *                    the +-q^mu pairs of Sec. II.C at separation dipole_dl
 *                    (0: the analytic point dipole), and a measurement knob
 *                    that does the multipole shifts into levels 2..fp32_top
 *                    and the local shifts out of them in single precision
 *                    (arithmetic and stored result), everything else in FP64,
 *                    to measure what single precision at the top of the
 *                    tree costs.
 *
 * Conventions: positions AoS (n x 3); the field gradient G = grad E is
 * stored as (xx, xy, xz, yy, yz, zz); Coulomb constant 1; r_ij = x_i - x_j.
 * Point dipoles enter the multipoles through the limit dl -> 0 of the +-q
 * pair of Sec. II.C, which is the derivative of the charge multipole.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ECOINCIDENT 2
#define ORC_ENOMEM 4
#define ORC_MAXP 16

/* ---------------------------------------------------------------------- */
/* multi-indices n = (nx, ny, nz) with |n| <= p (App. D)                    */
/* ---------------------------------------------------------------------- */

typedef struct {
    int p;
    int ncoef;
    int (*n)[3];   /* ncoef entries, ordered by total order */
    int* lookup;   /* (p+1)^3 table, -1 where |n| > p */
} orc_mi;

static int mi_init(orc_mi* t, int p) {
    t->p = p;
    t->ncoef = (p + 1) * (p + 2) * (p + 3) / 6;
    t->n = malloc(sizeof(int[3]) * (size_t)t->ncoef);
    t->lookup = malloc(sizeof(int) * (size_t)(p + 1) * (p + 1) * (p + 1));
    if (!t->n || !t->lookup) return ORC_ENOMEM;
    for (int i = 0; i < (p + 1) * (p + 1) * (p + 1); i++) t->lookup[i] = -1;
    int c = 0;
    for (int s = 0; s <= p; s++)
        for (int x = s; x >= 0; x--)
            for (int y = s - x; y >= 0; y--) {
                int z = s - x - y;
                t->n[c][0] = x;
                t->n[c][1] = y;
                t->n[c][2] = z;
                t->lookup[(x * (p + 1) + y) * (p + 1) + z] = c;
                c++;
            }
    return ORC_OK;
}

static void mi_free(orc_mi* t) {
    free(t->n);
    free(t->lookup);
}

static inline int mi_at(const orc_mi* t, int x, int y, int z) {
    if (x < 0 || y < 0 || z < 0 || x + y + z > t->p) return -1;
    return t->lookup[(x * (t->p + 1) + y) * (t->p + 1) + z];
}

static double fact(int k) {
    double f = 1.0;
    for (int i = 2; i <= k; i++) f *= i;
    return f;
}

static double ipow(double x, int k) {
    double r = 1.0;
    for (int i = 0; i < k; i++) r *= x;
    return r;
}

/* n! = nx! ny! nz! and x^n = x^nx y^ny z^nz (App. D) */
static double mi_fact(const int n[3]) { return fact(n[0]) * fact(n[1]) * fact(n[2]); }
static double mi_pow(const double x[3], const int n[3]) {
    return ipow(x[0], n[0]) * ipow(x[1], n[1]) * ipow(x[2], n[2]);
}

int orc_ncoef(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

/* Export the multi-index order used by the operator functions below. */
int orc_multi_indices(int p, int* out /* ncoef x 3 */) {
    orc_mi t;
    if (p < 0 || p > ORC_MAXP || mi_init(&t, p)) return ORC_EINVAL;
    memcpy(out, t.n, sizeof(int[3]) * (size_t)t.ncoef);
    mi_free(&t);
    return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* derivatives of the Green's function phi(r) = 1/r                        */
/* ---------------------------------------------------------------------- */

/*
 * a_n = d^n (1/r) at R for all |n| <= p.  1/r is homogeneous of degree -1
 * (Euler: sum_d R_d d_d f = -f) and harmonic; differentiating both
 * identities gives, for s = |n| >= 1,
 *   s r^2 a_n = -(2s-1) sum_d n_d R_d a_{n-e_d} - (s-1) sum_d n_d (n_d-1) a_{n-2e_d}.
 */
static void derivs(const orc_mi* t, const double R[3], double* a) {
    double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
    a[0] = 1.0 / sqrt(r2);
    for (int i = 1; i < t->ncoef; i++) {
        const int* n = t->n[i];
        int s = n[0] + n[1] + n[2];
        double acc = 0.0;
        for (int d = 0; d < 3; d++) {
            int m1[3] = {n[0], n[1], n[2]};
            if (n[d] >= 1) {
                m1[d] -= 1;
                acc += (2.0 * s - 1.0) * n[d] * R[d] * a[mi_at(t, m1[0], m1[1], m1[2])];
                m1[d] += 1;
            }
            if (n[d] >= 2) {
                m1[d] -= 2;
                acc += (s - 1.0) * n[d] * (n[d] - 1.0) * a[mi_at(t, m1[0], m1[1], m1[2])];
            }
        }
        a[i] = -acc / (s * r2);
    }
}

int orc_derivatives(int p, const double R[3], double* out) {
    orc_mi t;
    if (p < 0 || p > ORC_MAXP || mi_init(&t, p)) return ORC_EINVAL;
    derivs(&t, R, out);
    mi_free(&t);
    return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* single-box operators, Sec. II.B                                          */
/* ---------------------------------------------------------------------- */

/*
 * Multipole expansion (Eq. multipole): M_n(z) = sum_a q_a (-1)^|n| r_a^n / n!,
 * r_a = x_a - z.  A point dipole mu_a is the dl -> 0 limit of the +-q pair of
 * Sec. II.C: M_n += (-1)^|n| sum_d mu_{a,d} n_d r_a^{n-e_d} / n!.
 * Accumulates into M.
 */
static void p2m_accum(const orc_mi* t, const double z[3], int64_t na, const double* x,
                      const double* q, const double* mu, double* M) {
    for (int64_t a = 0; a < na; a++) {
        double r[3] = {x[3 * a] - z[0], x[3 * a + 1] - z[1], x[3 * a + 2] - z[2]};
        for (int i = 0; i < t->ncoef; i++) {
            const int* n = t->n[i];
            int s = n[0] + n[1] + n[2];
            double sign = (s & 1) ? -1.0 : 1.0;
            double nf = mi_fact(n);
            double v = 0.0;
            if (q) v += q[a] * mi_pow(r, n);
            if (mu) {
                for (int d = 0; d < 3; d++) {
                    if (n[d] == 0) continue;
                    int m[3] = {n[0], n[1], n[2]};
                    m[d] -= 1;
                    v += mu[3 * a + d] * n[d] * mi_pow(r, m);
                }
            }
            M[i] += sign * v / nf;
        }
    }
}

int orc_p2m(int p, const double z[3], int64_t na, const double* x, const double* q,
            const double* mu, double* M) {
    orc_mi t;
    if (p < 0 || p > ORC_MAXP || mi_init(&t, p)) return ORC_EINVAL;
    memset(M, 0, sizeof(double) * (size_t)t.ncoef);
    p2m_accum(&t, z, na, x, q, mu, M);
    mi_free(&t);
    return ORC_OK;
}

/* Shift of multipoles (Sec. II.B): M_n(z + s) = sum_{k <= n} s^k/k! M_{n-k}(z),
 * k <= n componentwise.  Accumulates into Mout. */
static void m2m_accum(const orc_mi* t, const double s[3], const double* Min, double* Mout) {
    for (int i = 0; i < t->ncoef; i++) {
        const int* n = t->n[i];
        double acc = 0.0;
        for (int kx = 0; kx <= n[0]; kx++)
            for (int ky = 0; ky <= n[1]; ky++)
                for (int kz = 0; kz <= n[2]; kz++) {
                    int k[3] = {kx, ky, kz};
                    acc += mi_pow(s, k) / mi_fact(k) * Min[mi_at(t, n[0] - kx, n[1] - ky, n[2] - kz)];
                }
        Mout[i] += acc;
    }
}

/* m2m_accum in single precision: terms, sum and the stored result rounded to
 * float (the measurement knob of orc_fmm_ex). */
static void m2m_accum_f32(const orc_mi* t, const double s[3], const double* Min, double* Mout) {
    for (int i = 0; i < t->ncoef; i++) {
        const int* n = t->n[i];
        float acc = 0.0f;
        for (int kx = 0; kx <= n[0]; kx++)
            for (int ky = 0; ky <= n[1]; ky++)
                for (int kz = 0; kz <= n[2]; kz++) {
                    int k[3] = {kx, ky, kz};
                    acc += (float)(mi_pow(s, k) / mi_fact(k)) * (float)Min[mi_at(t, n[0] - kx, n[1] - ky, n[2] - kz)];
                }
        Mout[i] = (double)((float)Mout[i] + acc);
    }
}

int orc_m2m(int p, const double s[3], const double* Min, double* Mout) {
    orc_mi t;
    if (p < 0 || p > ORC_MAXP || mi_init(&t, p)) return ORC_EINVAL;
    memset(Mout, 0, sizeof(double) * (size_t)t.ncoef);
    m2m_accum(&t, s, Min, Mout);
    mi_free(&t);
    return ORC_OK;
}

/* Multipole to local (Sec. II.B): F_n(z_B) = sum_{|m| <= p-|n|} M_m(z_A) d^{n+m} phi(z_B - z_A).
 * `a` holds the derivatives at R = z_B - z_A.  Accumulates into F. */
static void m2l_accum(const orc_mi* t, const double* a, const double* M, double* F) {
    for (int i = 0; i < t->ncoef; i++) {
        const int* n = t->n[i];
        int sn = n[0] + n[1] + n[2];
        double acc = 0.0;
        for (int j = 0; j < t->ncoef; j++) {
            const int* m = t->n[j];
            if (m[0] + m[1] + m[2] > t->p - sn) continue;
            acc += M[j] * a[mi_at(t, n[0] + m[0], n[1] + m[1], n[2] + m[2])];
        }
        F[i] += acc;
    }
}

int orc_m2l(int p, const double R[3], const double* M, double* F) {
    orc_mi t;
    if (p < 0 || p > ORC_MAXP || mi_init(&t, p)) return ORC_EINVAL;
    double* a = malloc(sizeof(double) * (size_t)t.ncoef);
    derivs(&t, R, a);
    memset(F, 0, sizeof(double) * (size_t)t.ncoef);
    m2l_accum(&t, a, M, F);
    free(a);
    mi_free(&t);
    return ORC_OK;
}

/* Shift of locals (Sec. II.B): F_n(z + s) = sum_{|k| <= p-|n|} s^k/k! F_{n+k}(z).
 * Accumulates into Fout. */
static void l2l_accum(const orc_mi* t, const double s[3], const double* Fin, double* Fout) {
    for (int i = 0; i < t->ncoef; i++) {
        const int* n = t->n[i];
        int sn = n[0] + n[1] + n[2];
        double acc = 0.0;
        for (int j = 0; j < t->ncoef; j++) {
            const int* k = t->n[j];
            if (k[0] + k[1] + k[2] > t->p - sn) continue;
            acc += mi_pow(s, k) / mi_fact(k) * Fin[mi_at(t, n[0] + k[0], n[1] + k[1], n[2] + k[2])];
        }
        Fout[i] += acc;
    }
}

/* l2l_accum in single precision (the measurement knob of orc_fmm_ex). */
static void l2l_accum_f32(const orc_mi* t, const double s[3], const double* Fin, double* Fout) {
    for (int i = 0; i < t->ncoef; i++) {
        const int* n = t->n[i];
        int sn = n[0] + n[1] + n[2];
        float acc = 0.0f;
        for (int j = 0; j < t->ncoef; j++) {
            const int* k = t->n[j];
            if (k[0] + k[1] + k[2] > t->p - sn) continue;
            acc += (float)(mi_pow(s, k) / mi_fact(k)) * (float)Fin[mi_at(t, n[0] + k[0], n[1] + k[1], n[2] + k[2])];
        }
        Fout[i] = (double)((float)Fout[i] + acc);
    }
}

int orc_l2l(int p, const double s[3], const double* Fin, double* Fout) {
    orc_mi t;
    if (p < 0 || p > ORC_MAXP || mi_init(&t, p)) return ORC_EINVAL;
    memset(Fout, 0, sizeof(double) * (size_t)t.ncoef);
    l2l_accum(&t, s, Fin, Fout);
    mi_free(&t);
    return ORC_OK;
}

/*
 * Local evaluation (Sec. II.B, last equation, read without the stray q_b):
 *   d^k Phi(x) = sum_{|n| <= p-|k|} (x - z)^n / n! F_{n+k}.
 * Returns Phi, its gradient dPhi (3) and Hessian ddPhi (6: xx xy xz yy yz zz);
 * the field is E = -dPhi and its gradient G = -ddPhi.  Accumulates.
 */
static void l2p_accum(const orc_mi* t, const double r[3], const double* F, double* phi,
                      double* dphi, double* ddphi) {
    static const int hd[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    for (int i = 0; i < t->ncoef; i++) {
        const int* n = t->n[i];
        int sn = n[0] + n[1] + n[2];
        double w = mi_pow(r, n) / mi_fact(n);
        if (phi) *phi += w * F[i];
        if (dphi && sn <= t->p - 1)
            for (int d = 0; d < 3; d++) {
                int m[3] = {n[0], n[1], n[2]};
                m[d] += 1;
                dphi[d] += w * F[mi_at(t, m[0], m[1], m[2])];
            }
        if (ddphi && sn <= t->p - 2)
            for (int c = 0; c < 6; c++) {
                int m[3] = {n[0], n[1], n[2]};
                m[hd[c][0]] += 1;
                m[hd[c][1]] += 1;
                ddphi[c] += w * F[mi_at(t, m[0], m[1], m[2])];
            }
    }
}

int orc_l2p(int p, const double r[3], const double* F, double* phi, double* dphi, double* ddphi) {
    orc_mi t;
    if (p < 0 || p > ORC_MAXP || mi_init(&t, p)) return ORC_EINVAL;
    if (phi) *phi = 0.0;
    if (dphi) memset(dphi, 0, sizeof(double) * 3);
    if (ddphi) memset(ddphi, 0, sizeof(double) * 6);
    l2p_accum(&t, r, F, phi, dphi, ddphi);
    mi_free(&t);
    return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* direct pair interaction                                                  */
/* ---------------------------------------------------------------------- */

/*
 * Potential, field and field gradient at x_i from a charge q_j and a point
 * dipole mu_j at x_j, r = x_i - x_j (Sec. II.A):
 *   charge: phi = q/r, E = q r/r^3, G_de = q (delta_de/r^3 - 3 r_d r_e/r^5)
 *   dipole: phi = mu.r/r^3, E = 3(mu.r) r/r^5 - mu/r^3 (the physical dipole
 *           field; the printed T_ij carries the opposite sign),
 *           G_de = 3(mu_d r_e + mu_e r_d + (mu.r) delta_de)/r^5 - 15 (mu.r) r_d r_e/r^7
 */
static void pair_accum(const double r[3], double qj, const double* muj, double* phi, double* E,
                       double* G) {
    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    double ri = 1.0 / sqrt(r2);
    double ri2 = ri * ri;
    double ri3 = ri * ri2;
    double ri5 = ri3 * ri2;
    double ri7 = ri5 * ri2;
    static const int hd[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    if (qj != 0.0) {
        if (phi) *phi += qj * ri;
        if (E)
            for (int d = 0; d < 3; d++) E[d] += qj * r[d] * ri3;
        if (G)
            for (int c = 0; c < 6; c++) {
                int d = hd[c][0], e = hd[c][1];
                G[c] += qj * ((d == e ? ri3 : 0.0) - 3.0 * r[d] * r[e] * ri5);
            }
    }
    if (muj) {
        double mr = muj[0] * r[0] + muj[1] * r[1] + muj[2] * r[2];
        if (phi) *phi += mr * ri3;
        if (E)
            for (int d = 0; d < 3; d++) E[d] += 3.0 * mr * r[d] * ri5 - muj[d] * ri3;
        if (G)
            for (int c = 0; c < 6; c++) {
                int d = hd[c][0], e = hd[c][1];
                G[c] += 3.0 * (muj[d] * r[e] + muj[e] * r[d] + (d == e ? mr : 0.0)) * ri5 -
                        15.0 * mr * r[d] * r[e] * ri7;
            }
    }
}

/*
 * O(N^2) sums over all j != i of the pair terms above.  q or mu may be NULL
 * (that source kind absent); phi, E, G may be NULL (not wanted).  If targets
 * is non-NULL only those nt sites are evaluated (outputs indexed 0..nt-1).
 * Returns ORC_ECOINCIDENT if two distinct sites coincide.
 */
int orc_direct(int64_t n, const double* x, const double* q, const double* mu, int64_t nt,
               const int64_t* targets, double* phi, double* E, double* G) {
    if (n < 1) return ORC_EINVAL;
    if (!targets) nt = n;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
    for (int64_t t = 0; t < nt; t++) {
        int64_t i = targets ? targets[t] : t;
        double ph = 0.0, e[3] = {0, 0, 0}, g[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double r[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1], x[3 * i + 2] - x[3 * j + 2]};
            if (r[0] == 0.0 && r[1] == 0.0 && r[2] == 0.0) {
                bad = 1;
                continue;
            }
            pair_accum(r, q ? q[j] : 0.0, mu ? mu + 3 * j : NULL, phi ? &ph : NULL, E ? e : NULL,
                       G ? g : NULL);
        }
        if (phi) phi[t] = ph;
        if (E)
            for (int d = 0; d < 3; d++) E[3 * t + d] = e[d];
        if (G)
            for (int c = 0; c < 6; c++) G[6 * t + c] = g[c];
    }
    return bad ? ORC_ECOINCIDENT : ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* CPU FMM on a uniform octree                                              */
/* ---------------------------------------------------------------------- */

/*
 * Root cube: the bounding box of the sites, centred, side = largest extent
 * times (1 + 1e-6) (1 A if all sites coincide), unless given.  Leaf cell of
 * a site: floor((x - lo) / h), h = side / 2^depth, clamped to [0, 2^depth).
 */
int orc_root_box(int64_t n, const double* x, double* lo, double* side) {
    if (n < 1) return ORC_EINVAL;
    double mn[3], mx[3];
    for (int d = 0; d < 3; d++) mn[d] = mx[d] = x[d];
    for (int64_t i = 1; i < n; i++)
        for (int d = 0; d < 3; d++) {
            double v = x[3 * i + d];
            if (v < mn[d]) mn[d] = v;
            if (v > mx[d]) mx[d] = v;
        }
    double ext = 0.0;
    for (int d = 0; d < 3; d++)
        if (mx[d] - mn[d] > ext) ext = mx[d] - mn[d];
    double s = ext > 0.0 ? ext * (1.0 + 1e-6) : 1.0;
    for (int d = 0; d < 3; d++) {
        double c = 0.5 * (mn[d] + mx[d]);
        double half = 0.5 * s;
        lo[d] = c - half;
    }
    *side = s;
    return ORC_OK;
}

int orc_leaf_cells(int64_t n, const double* x, int depth, const double* lo, double side, int* cells) {
    if (depth < 0 || depth > 10) return ORC_EINVAL;
    int nside = 1 << depth;
    double h = side / (double)nside;
    for (int64_t i = 0; i < n; i++)
        for (int d = 0; d < 3; d++) {
            double u = (x[3 * i + d] - lo[d]) / h;
            double f = floor(u);
            int c = f < 0.0 ? 0 : (f > nside - 1 ? nside - 1 : (int)f);
            cells[3 * i + d] = c;
        }
    return ORC_OK;
}

typedef struct {
    int nside;
    int64_t nocc;
    int* slot;      /* nside^3, -1 if empty */
    int* cell;      /* nocc x 3 integer coordinates */
    double* M;      /* nocc x ncoef */
    double* F;      /* nocc x ncoef */
} orc_level;

static inline int64_t lin3(int nside, int i, int j, int k) {
    return (int64_t)i + (int64_t)nside * ((int64_t)j + (int64_t)nside * k);
}

/*
 * Full FMM evaluation: outputs Phi, E = -grad Phi and G = grad E at every site
 * from sources q (may be NULL) and mu (may be NULL), excluding self terms.
 * p: expansion order (|n| + |m| <= p); depth: leaf level (root = level 0).
 * Interaction rule at level l >= 2: boxes A, B with parents adjacent
 * (or equal) and A, B not adjacent interact through multipoles; adjacent
 * leaves interact directly.  Each multipole-to-local derivative tensor is
 * evaluated per pair by the recurrence above.
 */
int orc_fmm_ex(int64_t n, const double* x, const double* q, const double* mu, int p, int depth,
               const double* root_lo, double root_side, double* phi, double* E, double* G, int fp32_top,
               double dipole_dl) {
    if (n < 1 || p < 1 || p > ORC_MAXP || depth < 1 || depth > 8 || !(dipole_dl >= 0.0)) return ORC_EINVAL;
    orc_mi t;
    if (mi_init(&t, p)) return ORC_ENOMEM;
    const int nc = t.ncoef;
    double lo[3], side;
    if (root_lo) {
        for (int d = 0; d < 3; d++) lo[d] = root_lo[d];
        side = root_side;
    } else {
        orc_root_box(n, x, lo, &side);
    }
    int status = ORC_OK;
    int* cells = malloc(sizeof(int) * 3 * (size_t)n);
    orc_leaf_cells(n, x, depth, lo, side, cells);

    /* levels 0..depth; boxes present where they contain sites */
    orc_level* lv = calloc((size_t)depth + 1, sizeof(orc_level));
    for (int l = 0; l <= depth; l++) {
        int ns = 1 << l;
        lv[l].nside = ns;
        lv[l].slot = malloc(sizeof(int) * (size_t)ns * ns * ns);
        for (int64_t b = 0; b < (int64_t)ns * ns * ns; b++) lv[l].slot[b] = -1;
    }
    /* mark occupied boxes, then number them in increasing linear index */
    for (int64_t i = 0; i < n; i++)
        for (int l = 0; l <= depth; l++) {
            int sh = depth - l;
            lv[l].slot[lin3(lv[l].nside, cells[3 * i] >> sh, cells[3 * i + 1] >> sh, cells[3 * i + 2] >> sh)] = 0;
        }
    for (int l = 0; l <= depth; l++) {
        int ns = lv[l].nside;
        int64_t c = 0;
        for (int64_t b = 0; b < (int64_t)ns * ns * ns; b++)
            if (lv[l].slot[b] == 0) c++;
        lv[l].nocc = c;
        lv[l].cell = malloc(sizeof(int) * 3 * (size_t)c);
        lv[l].M = calloc((size_t)c * nc, sizeof(double));
        lv[l].F = calloc((size_t)c * nc, sizeof(double));
        c = 0;
        for (int k = 0; k < ns; k++)
            for (int j = 0; j < ns; j++)
                for (int i = 0; i < ns; i++) {
                    int64_t b = lin3(ns, i, j, k);
                    if (lv[l].slot[b] == 0) {
                        lv[l].slot[b] = (int)c;
                        lv[l].cell[3 * c] = i;
                        lv[l].cell[3 * c + 1] = j;
                        lv[l].cell[3 * c + 2] = k;
                        c++;
                    }
                }
    }
    /* sites of each leaf (counting sort on the leaf slot, stable) */
    orc_level* L = &lv[depth];
    int64_t* start = calloc((size_t)L->nocc + 1, sizeof(int64_t));
    int64_t* order = malloc(sizeof(int64_t) * (size_t)n);
    int* leaf_of = malloc(sizeof(int) * (size_t)n);
    for (int64_t i = 0; i < n; i++) {
        leaf_of[i] = L->slot[lin3(L->nside, cells[3 * i], cells[3 * i + 1], cells[3 * i + 2])];
        start[leaf_of[i] + 1]++;
    }
    for (int64_t b = 0; b < L->nocc; b++) start[b + 1] += start[b];
    {
        int64_t* fill = malloc(sizeof(int64_t) * (size_t)L->nocc);
        for (int64_t b = 0; b < L->nocc; b++) fill[b] = start[b];
        for (int64_t i = 0; i < n; i++) order[fill[leaf_of[i]]++] = i;
        free(fill);
    }

#define BOX_CENTRE(l, c, z)                                                    \
    do {                                                                       \
        double hl_ = side / (double)lv[l].nside;                               \
        for (int d_ = 0; d_ < 3; d_++) (z)[d_] = lo[d_] + (lv[l].cell[3 * (c) + d_] + 0.5) * hl_; \
    } while (0)

    /* P2M at the leaves */
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t b = 0; b < L->nocc; b++) {
        double z[3];
        BOX_CENTRE(depth, b, z);
        for (int64_t k = start[b]; k < start[b + 1]; k++) {
            int64_t a = order[k];
            if (mu && dipole_dl > 0.0) {
                /* the dipole as the charges +-q^mu at x +- dl mu/|mu|, q^mu = |mu|/(2 dl) (Sec. II.C) */
                if (q) p2m_accum(&t, z, 1, x + 3 * a, q + a, NULL, L->M + b * nc);
                const double* m = mu + 3 * a;
                double nm = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
                if (nm > 0.0) {
                    for (int sgn = -1; sgn <= 1; sgn += 2) {
                        double y[3], qq = sgn * nm / (2.0 * dipole_dl);
                        for (int d = 0; d < 3; d++) y[d] = x[3 * a + d] + sgn * dipole_dl * m[d] / nm;
                        p2m_accum(&t, z, 1, y, &qq, NULL, L->M + b * nc);
                    }
                }
            } else {
                p2m_accum(&t, z, 1, x + 3 * a, q ? q + a : NULL, mu ? mu + 3 * a : NULL, L->M + b * nc);
            }
        }
    }
    /* M2M up to level 2 */
    for (int l = depth - 1; l >= 2; l--) {
        orc_level* P = &lv[l];
        orc_level* C = &lv[l + 1];
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t b = 0; b < P->nocc; b++) {
            double zp[3];
            BOX_CENTRE(l, b, zp);
            for (int o = 0; o < 8; o++) {
                int ci = 2 * P->cell[3 * b] + (o & 1);
                int cj = 2 * P->cell[3 * b + 1] + ((o >> 1) & 1);
                int ck = 2 * P->cell[3 * b + 2] + ((o >> 2) & 1);
                int cs = C->slot[lin3(C->nside, ci, cj, ck)];
                if (cs < 0) continue;
                double zc[3];
                BOX_CENTRE(l + 1, cs, zc);
                double s[3] = {zp[0] - zc[0], zp[1] - zc[1], zp[2] - zc[2]};
                if (l <= fp32_top)
                    m2m_accum_f32(&t, s, C->M + (int64_t)cs * nc, P->M + b * nc);
                else
                    m2m_accum(&t, s, C->M + (int64_t)cs * nc, P->M + b * nc);
            }
        }
    }
    /* M2L at every level l >= 2 */
    for (int l = 2; l <= depth; l++) {
        orc_level* B = &lv[l];
        int ns = B->nside;
#pragma omp parallel
        {
            double* a = malloc(sizeof(double) * (size_t)nc);
#pragma omp for schedule(dynamic, 4)
            for (int64_t b = 0; b < B->nocc; b++) {
                int bi = B->cell[3 * b], bj = B->cell[3 * b + 1], bk = B->cell[3 * b + 2];
                int pi = bi >> 1, pj = bj >> 1, pk = bk >> 1;
                double zb[3];
                BOX_CENTRE(l, b, zb);
                for (int ak = 2 * (pk - 1); ak < 2 * (pk + 2); ak++)
                    for (int aj = 2 * (pj - 1); aj < 2 * (pj + 2); aj++)
                        for (int ai = 2 * (pi - 1); ai < 2 * (pi + 2); ai++) {
                            if (ai < 0 || aj < 0 || ak < 0 || ai >= ns || aj >= ns || ak >= ns) continue;
                            if (abs(ai - bi) <= 1 && abs(aj - bj) <= 1 && abs(ak - bk) <= 1) continue;
                            int as = B->slot[lin3(ns, ai, aj, ak)];
                            if (as < 0) continue;
                            double za[3];
                            BOX_CENTRE(l, as, za);
                            double R[3] = {zb[0] - za[0], zb[1] - za[1], zb[2] - za[2]};
                            derivs(&t, R, a);
                            m2l_accum(&t, a, B->M + (int64_t)as * nc, B->F + b * nc);
                        }
            }
            free(a);
        }
    }
    /* L2L from level 2 down to the leaves */
    for (int l = 3; l <= depth; l++) {
        orc_level* C = &lv[l];
        orc_level* P = &lv[l - 1];
#pragma omp parallel for schedule(dynamic, 8)
        for (int64_t b = 0; b < C->nocc; b++) {
            int ps = P->slot[lin3(P->nside, C->cell[3 * b] >> 1, C->cell[3 * b + 1] >> 1, C->cell[3 * b + 2] >> 1)];
            double zc[3], zp[3];
            BOX_CENTRE(l, b, zc);
            BOX_CENTRE(l - 1, ps, zp);
            double s[3] = {zc[0] - zp[0], zc[1] - zp[1], zc[2] - zp[2]};
            if (l - 1 <= fp32_top)
                l2l_accum_f32(&t, s, P->F + (int64_t)ps * nc, C->F + b * nc);
            else
                l2l_accum(&t, s, P->F + (int64_t)ps * nc, C->F + b * nc);
        }
    }
    /* L2P + near field over the 27 adjacent leaves */
    int bad = 0;
    int ns = L->nside;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
    for (int64_t b = 0; b < L->nocc; b++) {
        double zb[3];
        BOX_CENTRE(depth, b, zb);
        int bi = L->cell[3 * b], bj = L->cell[3 * b + 1], bk = L->cell[3 * b + 2];
        for (int64_t k = start[b]; k < start[b + 1]; k++) {
            int64_t i = order[k];
            double ph = 0.0, dph[3] = {0, 0, 0}, ddph[6] = {0, 0, 0, 0, 0, 0};
            double r[3] = {x[3 * i] - zb[0], x[3 * i + 1] - zb[1], x[3 * i + 2] - zb[2]};
            l2p_accum(&t, r, L->F + b * nc, &ph, dph, ddph);
            double e[3], g[6];
            for (int d = 0; d < 3; d++) e[d] = -dph[d];
            for (int c = 0; c < 6; c++) g[c] = -ddph[c];
            for (int ak = bk - 1; ak <= bk + 1; ak++)
                for (int aj = bj - 1; aj <= bj + 1; aj++)
                    for (int ai = bi - 1; ai <= bi + 1; ai++) {
                        if (ai < 0 || aj < 0 || ak < 0 || ai >= ns || aj >= ns || ak >= ns) continue;
                        int as = L->slot[lin3(ns, ai, aj, ak)];
                        if (as < 0) continue;
                        for (int64_t kk = start[as]; kk < start[as + 1]; kk++) {
                            int64_t j = order[kk];
                            if (j == i) continue;
                            double rr[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1], x[3 * i + 2] - x[3 * j + 2]};
                            if (rr[0] == 0.0 && rr[1] == 0.0 && rr[2] == 0.0) {
                                bad = 1;
                                continue;
                            }
                            pair_accum(rr, q ? q[j] : 0.0, mu ? mu + 3 * j : NULL, &ph, e, g);
                        }
                    }
            if (phi) phi[i] = ph;
            if (E)
                for (int d = 0; d < 3; d++) E[3 * i + d] = e[d];
            if (G)
                for (int c = 0; c < 6; c++) G[6 * i + c] = g[c];
        }
    }
    if (bad) status = ORC_ECOINCIDENT;
#undef BOX_CENTRE
    for (int l = 0; l <= depth; l++) {
        free(lv[l].slot);
        free(lv[l].cell);
        free(lv[l].M);
        free(lv[l].F);
    }
    free(lv);
    free(start);
    free(order);
    free(leaf_of);
    free(cells);
    mi_free(&t);
    return status;
}

int orc_fmm(int64_t n, const double* x, const double* q, const double* mu, int p, int depth,
            const double* root_lo, double root_side, double* phi, double* E, double* G) {
    return orc_fmm_ex(n, x, q, mu, p, depth, root_lo, root_side, phi, E, G, -1, 0.0);
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int k) {
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
#else
    (void)k;
#endif
}
