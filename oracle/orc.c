/*
 * orc.c -- plain FP64 CPU oracle for the tree-gravity path.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do. It shares no code, header or table with the CUDA library.
 *
 * What it computes (G = 1, Sect. 3; Plummer softening, Sect. 3):
 *   - the direct O(N^2) sum, the exact quantity the tree approximates;
 *   - Morton keys, a stable sort, the octree topology, the cell multipoles
 *     (monopole + traceless quadrupole about the centre of mass, the
 *     expansion of Sect. 1), walk groups and the tree walk under a box-box
 *     opening-angle test, each step written from its definition, slow and
 *     obvious, in FP64 on the FP32 input values;
 *   - the unsoftened FP64 chain/perturber couplings of Sect. 2 and Eq. 3;
 *   - k-nearest / radius perturber selection.
 *
 * Readings where the paper is silent (octree instead of VINE's binary tree,
 * key quantisation, leaf rule, group rule, MAC geometry, quadrupole form) are
 * the ones stated at each function. Build with -ffp-contract=off: the key
 * quantisation and the FP32 selection distances must round every operation
 * separately.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_BITS 21
#define ORC_MAXLEVEL 21
#define ORC_GRID 2097152.0 /* 2^21 */

/* ------------------------------------------------------------------ */
/* Neumaier compensated sum (order-independent to ~1e-16)              */
/* ------------------------------------------------------------------ */
typedef struct { double s, c; } nsum;
static void nadd(nsum *a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static double nval(const nsum *a) { return a->s + a->c; }

/* Pair softening (Sect. 3): stars and SMBHs have their own Plummer lengths,
 * interactions with the chain centre-of-mass particle are not softened.
 * Reading: eps_ij = max(eps_i, eps_j), and 0 if either particle is marked
 * unsoftened (eps = 0). */
static double pair_eps(double ei, double ej) {
    if (ei == 0.0 || ej == 0.0) return 0.0;
    return ei > ej ? ei : ej;
}

/* Spline softening (the "spline" option of Sect. 2; reading: the point mass
 * smoothed by the cubic spline kernel of compact support h, W(r) = 8/(pi h^3)
 * (1 - 6u^2 + 6u^3) for u = r/h < 1/2, 16/(pi h^3) (1 - u)^3 for 1/2 <= u < 1,
 * 0 beyond, with h = 2.8 e, so that the potential at r = 0 is -m/e as for
 * Plummer softening of length e). Integrating the kernel's enclosed mass
 * gives a = m r f(u) / h^3 toward the mass and phi = (m/h) P(u):
 *   u < 1/2:      f = 32/3 - 192/5 u^2 + 32 u^3,
 *                 P = -14/5 + 16/3 u^2 - 48/5 u^4 + 32/5 u^5,
 *   1/2 <= u < 1: f = 64/3 - 48 u + 192/5 u^2 - 32/3 u^3 - 1/(15 u^3),
 *                 P = -16/5 + 1/(15 u) + 32/3 u^2 - 16 u^3 + 48/5 u^4 - 32/15 u^5,
 *   u >= 1:       f = 1/u^3, P = -1/u (Newton). */
#define ORC_SPLINE_H 2.8
static void spline_fp(double u, double *f, double *p) {
    if (u < 0.5) {
        *f = 32.0 / 3.0 + u * u * (-192.0 / 5.0 + 32.0 * u);
        *p = -14.0 / 5.0 + u * u * (16.0 / 3.0 + u * u * (-48.0 / 5.0 + 32.0 / 5.0 * u));
    } else {
        *f = 64.0 / 3.0 - 48.0 * u + u * u * (192.0 / 5.0 - 32.0 / 3.0 * u) - 1.0 / (15.0 * u * u * u);
        *p = -16.0 / 5.0 + 1.0 / (15.0 * u) + u * u * (32.0 / 3.0 + u * (-16.0 + u * (48.0 / 5.0 - 32.0 / 15.0 * u)));
    }
}

/* Softened point-mass acceleration on i from j and potential (G = 1),
 * r = x_j - x_i. kind 0 (Plummer, Sect. 3): a = m_j r / (r^2+e^2)^{3/2},
 * phi = -m_j / (r^2+e^2)^{1/2}; a pair at zero softened distance contributes
 * nothing. kind 1: the spline field above with h = 2.8 e (Newton for e = 0). */
static void p2p_k(int kind, double xi, double yi, double zi, double xj, double yj, double zj,
                  double mj, double e, nsum *ax, nsum *ay, nsum *az, nsum *ph) {
    double dx = xj - xi, dy = yj - yi, dz = zj - zi;
    if (kind == 1 && e > 0.0) {
        const double h = ORC_SPLINE_H * e;
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        if (r < h) {
            double f, p;
            spline_fp(r / h, &f, &p);
            const double s = mj * f / (h * h * h);
            nadd(ax, s * dx); nadd(ay, s * dy); nadd(az, s * dz);
            nadd(ph, mj * p / h);
            return;
        }
        e = 0.0;
    }
    double r2 = dx * dx + dy * dy + dz * dz + e * e;
    if (r2 <= 0.0) return;
    double rinv = 1.0 / sqrt(r2);
    double mr3 = mj * rinv * rinv * rinv;
    nadd(ax, mr3 * dx); nadd(ay, mr3 * dy); nadd(az, mr3 * dz);
    nadd(ph, -mj * rinv);
}
static void p2p(double xi, double yi, double zi, double xj, double yj, double zj,
                double mj, double e, nsum *ax, nsum *ay, nsum *az, nsum *ph) {
    p2p_k(0, xi, yi, zi, xj, yj, zj, mj, e, ax, ay, az, ph);
}

/* Quadrupole part of the field of a particle that carries a traceless moment
 * q = (xx, yy, zz, xy, xz, yz) about its own position (a chain seen from
 * outside: its members' second moment about their centre of mass), at the
 * offset r = x_target - x_source, with the Plummer length e of the pair. Same
 * two-term expansion about the centre of mass as the cells' (Sect. 1):
 *   a = Q r / rho^5 - 5 (r.Q.r) r / (2 rho^7),  phi = -(r.Q.r) / (2 rho^5),
 * rho^2 = r.r + e^2 (the monopole is the point-mass pair term). */
static void quad_term(double rx, double ry, double rz, double e, const double *q,
                      nsum *ax, nsum *ay, nsum *az, nsum *ph) {
    double r2 = rx * rx + ry * ry + rz * rz + e * e;
    if (r2 <= 0.0) return;
    double rinv = 1.0 / sqrt(r2), rinv2 = rinv * rinv, rinv5 = rinv * rinv2 * rinv2, rinv7 = rinv5 * rinv2;
    double qx = q[0] * rx + q[3] * ry + q[4] * rz;
    double qy = q[3] * rx + q[1] * ry + q[5] * rz;
    double qz = q[4] * rx + q[5] * ry + q[2] * rz;
    double rqr = rx * qx + ry * qy + rz * qz;
    nadd(ax, qx * rinv5 - 2.5 * rqr * rx * rinv7);
    nadd(ay, qy * rinv5 - 2.5 * rqr * ry * rinv7);
    nadd(az, qz * rinv5 - 2.5 * rqr * rz * rinv7);
    nadd(ph, -0.5 * rqr * rinv5);
}

/* Total mass, centre of mass and traceless quadrupole of a chain of nch
 * members (masses cm, positions cx[3k..]) about its centre of mass:
 *   Q_ab = sum_k m_k (3 d_a d_b - |d|^2 delta_ab),  d = x_k - com,
 * out = (M, com x, y, z, Qxx, Qyy, Qzz, Qxy, Qxz, Qyz); com = 0 if M = 0. */
void orc_chain_moments(int32_t nch, const double *cm, const double *cx, double out[10]) {
    double M = 0.0, c[3] = {0.0, 0.0, 0.0};
    for (int32_t k = 0; k < nch; k++) {
        M += cm[k];
        for (int a = 0; a < 3; a++) c[a] += cm[k] * cx[3 * k + a];
    }
    for (int a = 0; a < 3; a++) c[a] = (M > 0.0) ? c[a] / M : 0.0;
    double q[6] = {0, 0, 0, 0, 0, 0};
    for (int32_t k = 0; k < nch; k++) {
        double d[3] = {cx[3 * k] - c[0], cx[3 * k + 1] - c[1], cx[3 * k + 2] - c[2]};
        double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        q[0] += cm[k] * (3.0 * d[0] * d[0] - d2);
        q[1] += cm[k] * (3.0 * d[1] * d[1] - d2);
        q[2] += cm[k] * (3.0 * d[2] * d[2] - d2);
        q[3] += cm[k] * 3.0 * d[0] * d[1];
        q[4] += cm[k] * 3.0 * d[0] * d[2];
        q[5] += cm[k] * 3.0 * d[1] * d[2];
    }
    out[0] = M;
    for (int a = 0; a < 3; a++) out[1 + a] = c[a];
    for (int a = 0; a < 6; a++) out[4 + a] = q[a];
}

/* ------------------------------------------------------------------ */
/* 1. Direct sum                                                        */
/* ------------------------------------------------------------------ */
/* Acceleration and potential on targets tidx[0..nt) from all n particles,
 * skipping j == i. eps[j] = 0 marks an unsoftened particle; kind 0 Plummer,
 * 1 spline softening (see p2p_k). */
void orc_direct(int64_t n, const double *x, const double *y, const double *z,
                const double *m, const double *eps, int64_t nt, const int64_t *tidx,
                double *ax, double *ay, double *az, double *pot, int32_t kind) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; t++) {
        int64_t i = tidx[t];
        nsum sx = {0, 0}, sy = {0, 0}, sz = {0, 0}, sp = {0, 0};
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            p2p_k(kind, x[i], y[i], z[i], x[j], y[j], z[j], m[j], pair_eps(eps[i], eps[j]), &sx, &sy, &sz, &sp);
        }
        ax[t] = nval(&sx); ay[t] = nval(&sy); az[t] = nval(&sz); pot[t] = nval(&sp);
    }
}

/* ------------------------------------------------------------------ */
/* 2. Morton keys                                                       */
/* ------------------------------------------------------------------ */
/* Bounding cube of FP32 positions: per axis min (exact FP32 compare), side
 * L = max_a (max_a - min_a) with each difference one FP64 subtraction, and
 * scale = 2^21 / L as one FP64 division (0 when L = 0). */
void orc_bounds(int64_t n, const float *x, const float *y, const float *z,
                double out_min[3], double *out_L, double *out_scale) {
    const float *c[3] = {x, y, z};
    double L = 0.0;
    for (int a = 0; a < 3; a++) {
        float lo = 0.0f, hi = 0.0f;
        for (int64_t i = 0; i < n; i++) {
            float v = c[a][i];
            if (i == 0 || v < lo) lo = v;
            if (i == 0 || v > hi) hi = v;
        }
        out_min[a] = (double)lo;
        double ext = (double)hi - (double)lo;
        if (ext > L) L = ext;
    }
    *out_L = L;
    *out_scale = (L > 0.0) ? ORC_GRID / L : 0.0;
}

/* Integer grid coordinate: q = min(floor((x - min) * scale), 2^21 - 1), the
 * subtraction and the product each rounded once in FP64. */
static uint64_t grid_coord(float v, double lo, double scale) {
    double d = (double)v - lo;
    double t = d * scale;
    double f = floor(t);
    if (f >= ORC_GRID - 1.0) return (uint64_t)(ORC_GRID - 1.0);
    if (f < 0.0) return 0;
    return (uint64_t)f;
}

/* 63-bit key: bit 3k = x_k, 3k+1 = y_k, 3k+2 = z_k (k = 0 least significant). */
static uint64_t interleave(uint64_t qx, uint64_t qy, uint64_t qz) {
    uint64_t key = 0;
    for (int k = 0; k < ORC_BITS; k++) {
        key |= ((qx >> k) & 1ull) << (3 * k);
        key |= ((qy >> k) & 1ull) << (3 * k + 1);
        key |= ((qz >> k) & 1ull) << (3 * k + 2);
    }
    return key;
}

static void deinterleave(uint64_t key, int64_t *qx, int64_t *qy, int64_t *qz) {
    int64_t a = 0, b = 0, c = 0;
    for (int k = 0; k < ORC_BITS; k++) {
        a |= (int64_t)((key >> (3 * k)) & 1ull) << k;
        b |= (int64_t)((key >> (3 * k + 1)) & 1ull) << k;
        c |= (int64_t)((key >> (3 * k + 2)) & 1ull) << k;
    }
    *qx = a; *qy = b; *qz = c;
}

void orc_keys(int64_t n, const float *x, const float *y, const float *z,
              const double lo[3], double scale, uint64_t *key) {
    for (int64_t i = 0; i < n; i++)
        key[i] = interleave(grid_coord(x[i], lo[0], scale), grid_coord(y[i], lo[1], scale),
                            grid_coord(z[i], lo[2], scale));
}

/* ------------------------------------------------------------------ */
/* 3. Stable sort of (key, index): equal keys keep ascending index       */
/* ------------------------------------------------------------------ */
typedef struct { uint64_t key; int64_t idx; } kv;
static int kv_cmp(const void *a, const void *b) {
    const kv *p = (const kv *)a, *q = (const kv *)b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    return (p->idx > q->idx) - (p->idx < q->idx);
}
void orc_sort(int64_t n, const uint64_t *key, uint64_t *skey, int64_t *perm) {
    kv *t = (kv *)malloc(sizeof(kv) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; i++) { t[i].key = key[i]; t[i].idx = i; }
    qsort(t, (size_t)n, sizeof(kv), kv_cmp);
    for (int64_t i = 0; i < n; i++) { skey[i] = t[i].key; perm[i] = t[i].idx; }
    free(t);
}

/* ------------------------------------------------------------------ */
/* 4. Octree                                                            */
/* ------------------------------------------------------------------ */
typedef struct {
    int64_t n, ncell, cap, ngroup, gcap;
    int32_t n_leaf, group_max;
    double lo[3], L, scale;
    uint64_t *key;        /* sorted keys */
    int64_t *perm;        /* sorted slot -> caller index */
    double *x, *y, *z, *m;/* sorted, FP64 copies of the FP32 inputs */
    /* cells in breadth-first order: ascending level, then ascending first */
    int32_t *level;
    int64_t *first, *count, *child, *nchild, *parent;
    int64_t *ox, *oy, *oz;          /* integer-grid origin of the cell box */
    double *cm, *cx, *cy, *cz, *cq; /* mass, centre of mass, Q (xx,yy,zz,xy,xz,yz) */
    /* walk groups: first star, count, integer-grid box [glo, ghi) per axis */
    int64_t *gfirst, *gcount, *glo, *ghi;
} orc_tree;

static void tree_push_cell(orc_tree *t, int32_t lev, int64_t first, int64_t count, int64_t parent) {
    if (t->ncell == t->cap) {
        t->cap = t->cap ? 2 * t->cap : 64;
#define GROW(p, ty) t->p = (ty *)realloc(t->p, sizeof(ty) * (size_t)t->cap)
        GROW(level, int32_t); GROW(first, int64_t); GROW(count, int64_t); GROW(child, int64_t);
        GROW(nchild, int64_t); GROW(parent, int64_t); GROW(ox, int64_t); GROW(oy, int64_t); GROW(oz, int64_t);
#undef GROW
    }
    int64_t c = t->ncell++;
    t->level[c] = lev; t->first[c] = first; t->count[c] = count;
    t->child[c] = -1; t->nchild[c] = 0; t->parent[c] = parent;
    /* box origin: the key of the first particle with the bits below level lev cleared */
    int sh = 3 * (ORC_MAXLEVEL - lev);
    uint64_t pre = (sh >= 64) ? 0 : ((t->key[first] >> sh) << sh);
    deinterleave(pre, &t->ox[c], &t->oy[c], &t->oz[c]);
}

static int cell_is_leaf(const orc_tree *t, int64_t c) { return t->nchild[c] == 0; }

/* Topology (reading of the silent points): the root holds all particles; a
 * cell is split iff it has more than n_leaf particles and level < 21; its
 * children are the non-empty octants, i.e. maximal runs of equal 3-bit key
 * digits at the next level, ordered by octant. Built level by level, which
 * gives the breadth-first order directly. */
static void build_topology(orc_tree *t) {
    if (t->n == 0) return;
    tree_push_cell(t, 0, 0, t->n, -1);
    int64_t lev_begin = 0, lev_end = 1;
    for (int32_t lev = 0; lev < ORC_MAXLEVEL; lev++) {
        for (int64_t c = lev_begin; c < lev_end; c++) {
            if (t->count[c] <= t->n_leaf) continue;
            int sh = 3 * (ORC_MAXLEVEL - (lev + 1));
            int64_t s = t->first[c], e = s + t->count[c];
            int64_t run = s;
            t->child[c] = t->ncell;
            for (int64_t i = s + 1; i <= e; i++) {
                if (i == e || ((t->key[i] >> sh) & 7u) != ((t->key[run] >> sh) & 7u)) {
                    tree_push_cell(t, lev + 1, run, i - run, c);
                    t->nchild[c]++;
                    run = i;
                }
            }
        }
        lev_begin = lev_end;
        lev_end = t->ncell;
        if (lev_begin == lev_end) break;
    }
}

/* Cell multipoles from the cell's own particles (Sect. 1: expansion about the
 * group's centre of mass): M = sum m, COM = sum m x / M, traceless
 * Q_ab = sum m (3 d_a d_b - |d|^2 delta_ab), d = x - COM. A massless cell
 * takes its geometric centre and Q = 0. */
static void build_moments(orc_tree *t) {
    t->cm = (double *)malloc(sizeof(double) * (size_t)(t->ncell + 1));
    t->cx = (double *)malloc(sizeof(double) * (size_t)(t->ncell + 1));
    t->cy = (double *)malloc(sizeof(double) * (size_t)(t->ncell + 1));
    t->cz = (double *)malloc(sizeof(double) * (size_t)(t->ncell + 1));
    t->cq = (double *)malloc(sizeof(double) * 6 * (size_t)(t->ncell + 1));
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t c = 0; c < t->ncell; c++) {
        int64_t s = t->first[c], e = s + t->count[c];
        double M = 0, sx = 0, sy = 0, sz = 0;
        for (int64_t i = s; i < e; i++) {
            M += t->m[i]; sx += t->m[i] * t->x[i]; sy += t->m[i] * t->y[i]; sz += t->m[i] * t->z[i];
        }
        double gx, gy, gz;
        if (M > 0) { gx = sx / M; gy = sy / M; gz = sz / M; }
        else {
            double side = ldexp(1.0, ORC_MAXLEVEL - t->level[c]);
            double u = (t->L > 0) ? t->L / ORC_GRID : 0.0;
            gx = t->lo[0] + ((double)t->ox[c] + 0.5 * side) * u;
            gy = t->lo[1] + ((double)t->oy[c] + 0.5 * side) * u;
            gz = t->lo[2] + ((double)t->oz[c] + 0.5 * side) * u;
        }
        double q[6] = {0, 0, 0, 0, 0, 0};
        if (M > 0) {
            for (int64_t i = s; i < e; i++) {
                double dx = t->x[i] - gx, dy = t->y[i] - gy, dz = t->z[i] - gz;
                double d2 = dx * dx + dy * dy + dz * dz, mi = t->m[i];
                q[0] += mi * (3 * dx * dx - d2); q[1] += mi * (3 * dy * dy - d2);
                q[2] += mi * (3 * dz * dz - d2); q[3] += mi * 3 * dx * dy;
                q[4] += mi * 3 * dx * dz; q[5] += mi * 3 * dy * dz;
            }
        }
        t->cm[c] = M; t->cx[c] = gx; t->cy[c] = gy; t->cz[c] = gz;
        for (int k = 0; k < 6; k++) t->cq[6 * c + k] = q[k];
    }
}

static void push_group(orc_tree *t, int64_t first, int64_t count, const int64_t lo[3], const int64_t hi[3]) {
    if (t->ngroup == t->gcap) {
        t->gcap = t->gcap ? 2 * t->gcap : 64;
        t->gfirst = (int64_t *)realloc(t->gfirst, sizeof(int64_t) * (size_t)t->gcap);
        t->gcount = (int64_t *)realloc(t->gcount, sizeof(int64_t) * (size_t)t->gcap);
        t->glo = (int64_t *)realloc(t->glo, sizeof(int64_t) * 3 * (size_t)t->gcap);
        t->ghi = (int64_t *)realloc(t->ghi, sizeof(int64_t) * 3 * (size_t)t->gcap);
    }
    int64_t g = t->ngroup++;
    t->gfirst[g] = first; t->gcount[g] = count;
    for (int a = 0; a < 3; a++) { t->glo[3 * g + a] = lo[a]; t->ghi[3 * g + a] = hi[a]; }
}

/* Walk groups (reading; the paper does not group targets). A unit is a
 * maximal cell with at most U = 16 G stars (a cell with <= U stars whose
 * parent has more, or the root), or a leaf with more than U stars. Each unit
 * is cut into runs of G consecutive stars in key order, the last run possibly
 * shorter; each run is a group. A group's box is the smallest box on the
 * integer grid that holds its stars' grid cells: per axis lo = min q,
 * hi = max q + 1, with q the star's grid coordinate (its key de-interleaved).
 * Every star of a group lies in the group's box, so a cell the box-box test
 * accepts for the group satisfies the opening-angle test for each of its
 * stars. */
static void push_runs(orc_tree *t, int64_t first, int64_t count) {
    for (int64_t f = first; f < first + count; f += t->group_max) {
        int64_t cnt = first + count - f < t->group_max ? first + count - f : t->group_max;
        int64_t lo[3], hi[3];
        for (int64_t i = f; i < f + cnt; i++) {
            int64_t q[3];
            deinterleave(t->key[i], &q[0], &q[1], &q[2]);
            for (int a = 0; a < 3; a++) {
                if (i == f || q[a] < lo[a]) lo[a] = q[a];
                if (i == f || q[a] + 1 > hi[a]) hi[a] = q[a] + 1;
            }
        }
        push_group(t, f, cnt, lo, hi);
    }
}

static void visit_units(orc_tree *t, int64_t c, int64_t U) {
    if (t->count[c] <= U || cell_is_leaf(t, c)) {
        push_runs(t, t->first[c], t->count[c]);
        return;
    }
    for (int64_t k = 0; k < t->nchild[c]; k++) visit_units(t, t->child[c] + k, U);
}

static void build_groups(orc_tree *t) {
    if (t->ncell == 0) return;
    visit_units(t, 0, 16 * (int64_t)t->group_max);
}

orc_tree *orc_tree_build(int64_t n, const float *x, const float *y, const float *z, const float *m,
                         int32_t n_leaf, int32_t group_max) {
    orc_tree *t = (orc_tree *)calloc(1, sizeof(orc_tree));
    t->n = n; t->n_leaf = n_leaf; t->group_max = group_max;
    orc_bounds(n, x, y, z, t->lo, &t->L, &t->scale);
    size_t nn = (size_t)(n > 0 ? n : 1);
    uint64_t *raw = (uint64_t *)malloc(sizeof(uint64_t) * nn);
    orc_keys(n, x, y, z, t->lo, t->scale, raw);
    t->key = (uint64_t *)malloc(sizeof(uint64_t) * nn);
    t->perm = (int64_t *)malloc(sizeof(int64_t) * nn);
    orc_sort(n, raw, t->key, t->perm);
    free(raw);
    t->x = (double *)malloc(sizeof(double) * nn); t->y = (double *)malloc(sizeof(double) * nn);
    t->z = (double *)malloc(sizeof(double) * nn); t->m = (double *)malloc(sizeof(double) * nn);
    for (int64_t i = 0; i < n; i++) {
        int64_t j = t->perm[i];
        t->x[i] = x[j]; t->y[i] = y[j]; t->z[i] = z[j]; t->m[i] = m[j];
    }
    build_topology(t);
    build_moments(t);
    build_groups(t);
    return t;
}

void orc_tree_free(orc_tree *t) {
    if (!t) return;
    free(t->key); free(t->perm); free(t->x); free(t->y); free(t->z); free(t->m);
    free(t->level); free(t->first); free(t->count); free(t->child); free(t->nchild); free(t->parent);
    free(t->ox); free(t->oy); free(t->oz); free(t->cm); free(t->cx); free(t->cy); free(t->cz); free(t->cq);
    free(t->gfirst); free(t->gcount); free(t->glo); free(t->ghi);
    free(t);
}

void orc_tree_sizes(const orc_tree *t, int64_t out[3]) { out[0] = t->n; out[1] = t->ncell; out[2] = t->ngroup; }
void orc_tree_bounds(const orc_tree *t, double out[5]) {
    out[0] = t->lo[0]; out[1] = t->lo[1]; out[2] = t->lo[2]; out[3] = t->L; out[4] = t->scale;
}
void orc_tree_keys(const orc_tree *t, uint64_t *key, int64_t *perm) {
    memcpy(key, t->key, sizeof(uint64_t) * (size_t)t->n);
    memcpy(perm, t->perm, sizeof(int64_t) * (size_t)t->n);
}
/* cells: [ncell][9] = level, first, count, child, nchild, parent, ox, oy, oz */
void orc_tree_cells(const orc_tree *t, int64_t *out) {
    for (int64_t c = 0; c < t->ncell; c++) {
        int64_t *o = out + 9 * c;
        o[0] = t->level[c]; o[1] = t->first[c]; o[2] = t->count[c]; o[3] = t->child[c];
        o[4] = t->nchild[c]; o[5] = t->parent[c]; o[6] = t->ox[c]; o[7] = t->oy[c]; o[8] = t->oz[c];
    }
}
/* moments: [ncell][10] = M, cx, cy, cz, Qxx, Qyy, Qzz, Qxy, Qxz, Qyz */
void orc_tree_moments(const orc_tree *t, double *out) {
    for (int64_t c = 0; c < t->ncell; c++) {
        double *o = out + 10 * c;
        o[0] = t->cm[c]; o[1] = t->cx[c]; o[2] = t->cy[c]; o[3] = t->cz[c];
        for (int k = 0; k < 6; k++) o[4 + k] = t->cq[6 * c + k];
    }
}
/* groups: [ngroup][8] = first, count, box lo x, y, z, box hi x, y, z */
void orc_tree_groups(const orc_tree *t, int64_t *out) {
    for (int64_t g = 0; g < t->ngroup; g++) {
        int64_t *o = out + 8 * g;
        o[0] = t->gfirst[g]; o[1] = t->gcount[g];
        for (int a = 0; a < 3; a++) { o[2 + a] = t->glo[3 * g + a]; o[5 + a] = t->ghi[3 * g + a]; }
    }
}

/* ------------------------------------------------------------------ */
/* 5. Tree walk                                                         */
/* ------------------------------------------------------------------ */
/* Opening test (reading of the opening-angle criterion): cell C of side
 * s = 2^(21 - level) grid units is accepted for a group whose box is B iff
 * s^2 < theta^2 d^2, with d the minimum Euclidean distance between the boxes
 * of B and C in grid units and theta^2 = theta * theta, all in FP64 (integers
 * below 2^53 are exact). A box that touches or contains the group has d = 0
 * and is opened. */
static int64_t gap1(int64_t blo, int64_t bhi, int64_t clo, int64_t chi) {
    if (clo >= bhi) return clo - bhi;
    if (blo >= chi) return blo - chi;
    return 0;
}
static int mac_accept(const orc_tree *t, const int64_t blo[3], const int64_t bhi[3], int64_t c, double theta2) {
    int64_t s = (int64_t)1 << (ORC_MAXLEVEL - t->level[c]);
    int64_t gx = gap1(blo[0], bhi[0], t->ox[c], t->ox[c] + s);
    int64_t gy = gap1(blo[1], bhi[1], t->oy[c], t->oy[c] + s);
    int64_t gz = gap1(blo[2], bhi[2], t->oz[c], t->oz[c] + s);
    double d2 = (double)(gx * gx + gy * gy + gz * gz);
    double s2 = (double)s * (double)s;
    return s2 < theta2 * d2;
}

/* Softened monopole + quadrupole field of cell c at (px,py,pz) (reading):
 * r = x - COM, rho^2 = r.r + e^2, phi = -M/rho - (r.Q.r)/(2 rho^5),
 * a = -M r/rho^3 + Q r/rho^5 - 5 (r.Q.r) r/(2 rho^7); for e = 0 this is the
 * exact two-term multipole expansion about the centre of mass. */
static void m2p(const orc_tree *t, int64_t c, double px, double py, double pz, double e, int quad,
                nsum *ax, nsum *ay, nsum *az, nsum *ph, int kind) {
    double M = t->cm[c];
    if (M == 0.0) return;
    double rx = px - t->cx[c], ry = py - t->cy[c], rz = pz - t->cz[c];
    if (kind == 1 && e > 0.0) {
        /* spline softening (reading): beyond h = 2.8 e the field is Newton's, so
         * the unsoftened expansion; inside, the cell acts as a softened monopole */
        const double h = ORC_SPLINE_H * e;
        const double r = sqrt(rx * rx + ry * ry + rz * rz);
        if (r < h) {
            double f, p;
            spline_fp(r / h, &f, &p);
            const double s = -M * f / (h * h * h);
            nadd(ax, s * rx); nadd(ay, s * ry); nadd(az, s * rz); nadd(ph, M * p / h);
            return;
        }
        e = 0.0;
    }
    double r2 = rx * rx + ry * ry + rz * rz + e * e;
    if (r2 <= 0.0) return;
    double rinv = 1.0 / sqrt(r2), rinv2 = rinv * rinv, rinv3 = rinv * rinv2;
    double fx = -M * rx * rinv3, fy = -M * ry * rinv3, fz = -M * rz * rinv3, p = -M * rinv;
    if (quad) {
        const double *q = t->cq + 6 * c;
        double qx = q[0] * rx + q[3] * ry + q[4] * rz;
        double qy = q[3] * rx + q[1] * ry + q[5] * rz;
        double qz = q[4] * rx + q[5] * ry + q[2] * rz;
        double rqr = rx * qx + ry * qy + rz * qz;
        double rinv5 = rinv3 * rinv2, rinv7 = rinv5 * rinv2;
        fx += qx * rinv5 - 2.5 * rqr * rx * rinv7;
        fy += qy * rinv5 - 2.5 * rqr * ry * rinv7;
        fz += qz * rinv5 - 2.5 * rqr * rz * rinv7;
        p += -0.5 * rqr * rinv5;
    }
    nadd(ax, fx); nadd(ay, fy); nadd(az, fz); nadd(ph, p);
}

typedef struct {
    const orc_tree *t;
    int64_t blo[3], bhi[3];
    double theta2;
    int quad;
    double px, py, pz, e;
    int64_t self; /* sorted slot of the target, or -1 */
    nsum ax, ay, az, ph;
    int64_t n_p2p, n_m2p;
    int rel;      /* 1: relative criterion with constant K below */
    float K;
    int kind;     /* softening: 0 Plummer, 1 spline */
} walk_state;

/* Relative opening criterion (Sect. 3: the runs use a "Gadget" criterion with
 * an error tolerance; reading: the relative criterion of the Gadget-2 code).
 * A cell of mass M and side s at distance d is used as a multipole for a
 * target whose reference acceleration has magnitude |a| when
 *     M s^2 <= alpha |a| d^4        (G = 1),
 * and only when the target lies outside the cell's box grown by a tenth of its
 * side on every side (a safeguard against a massive cell close to the target).
 * For a group: |a| is the smallest reference magnitude among its stars, d the
 * box-box distance, and the safeguard asks the group's box to lie outside the
 * grown box. The decision is taken in FP32, one rounding per operation, as the
 * CUDA walk takes it: with u the grid unit rounded to FP32,
 * K = (alpha * amin) * (u * u) per group and d2 = d^2 in grid units rounded
 * once to FP32, accept iff M32 * s^2 <= (K * d2) * d2 (M32 = M rounded to
 * FP32). */
static int mac_accept_rel(const orc_tree *t, const int64_t blo[3], const int64_t bhi[3], int64_t c, float K) {
    int64_t s = (int64_t)1 << (ORC_MAXLEVEL - t->level[c]);
    const int64_t o[3] = {t->ox[c], t->oy[c], t->oz[c]};
    int outside = 0;
    for (int a = 0; a < 3; a++)
        if (10 * bhi[a] <= 10 * o[a] - s || 10 * blo[a] >= 10 * (o[a] + s) + s) outside = 1;
    if (!outside) return 0;
    int64_t d2 = 0;
    for (int a = 0; a < 3; a++) {
        int64_t g = gap1(blo[a], bhi[a], o[a], o[a] + s);
        d2 += g * g;
    }
    float d2f = (float)d2;
    float m32 = (float)t->cm[c];
    float s2 = (float)((double)s * (double)s);
    float lhs = m32 * s2;
    float rhs = (K * d2f) * d2f;
    return lhs <= rhs;
}

/* Reference magnitude |a| of a reference acceleration (FP32 components), in
 * FP32 with one rounding per operation: sqrt((x x + y y) + z z). */
static float ref_mag(float x, float y, float z) {
    float s = x * x;
    s = s + y * y;
    s = s + z * z;
    return sqrtf(s);
}

static void walk_cell(walk_state *w, int64_t c) {
    const orc_tree *t = w->t;
    if (w->rel ? mac_accept_rel(t, w->blo, w->bhi, c, w->K) : mac_accept(t, w->blo, w->bhi, c, w->theta2)) {
        m2p(t, c, w->px, w->py, w->pz, w->e, w->quad, &w->ax, &w->ay, &w->az, &w->ph, w->kind);
        w->n_m2p++;
        return;
    }
    if (cell_is_leaf(t, c)) {
        for (int64_t j = t->first[c]; j < t->first[c] + t->count[c]; j++) {
            if (j == w->self) continue;
            p2p_k(w->kind, w->px, w->py, w->pz, t->x[j], t->y[j], t->z[j], t->m[j], w->e, &w->ax, &w->ay, &w->az,
                  &w->ph);
            w->n_p2p++;
        }
        return;
    }
    for (int64_t k = 0; k < t->nchild[c]; k++) walk_cell(w, t->child[c] + k);
}

/* Tree forces on every tree particle, written in caller order.
 * eps_star softens every tree pair (all tree particles are stars).
 * Extra particles (chain centres of mass, unsoftened when xeps = 0) are not in
 * the tree: they act on every tree particle and on each other by the direct
 * pair rule, and each feels the tree through its own walk whose group box is
 * the grid cell [q, q+1)^3 of its position (q unclamped, limited to
 * +-2^23). counts (optional, [n][2]) receives the P2P and M2P interaction
 * counts per tree particle. With nsub >= 0 only the stars whose caller
 * indices are listed in sub[0..nsub) are computed (others untouched).
 * With rx != NULL the stars' groups use the relative criterion above with
 * tolerance alpha and reference accelerations (rx, ry, rz)[i] (caller order,
 * FP32); the extra particles always use the opening angle. kind selects the
 * stars' softening: 0 Plummer, 1 spline (see p2p_k; the extra particles'
 * pairs use Plummer's rule with their own lengths). xq (optional, 6 per
 * extra particle) gives each extra particle a traceless quadrupole about its
 * position, whose field (quad_term) is added wherever that particle acts
 * (reading: a chain seen from outside is its centre of mass plus its
 * quadrupole, the same two-term expansion as a tree cell), except on the
 * stars flagged in xq_skip (caller order, optional): the chain's perturbers,
 * which feel the resolved members instead (Sect. 2) and so keep the
 * centre-of-mass point mass that their correction replaces. */
void orc_tree_forces(const orc_tree *t, double theta, double eps_star, int32_t quad,
                     int32_t nx, const float *xx, const float *xy, const float *xz, const double *xm,
                     const double *xeps,
                     double *ax, double *ay, double *az, double *pot,
                     double *xax, double *xay, double *xaz, double *xpot, int64_t *counts,
                     int64_t nsub, const int64_t *sub,
                     float alpha, const float *rx, const float *ry, const float *rz, int32_t kind,
                     const double *xq, const int8_t *xq_skip) {
    double theta2 = theta * theta;
    const float u = (float)(t->L / ORC_GRID);
    /* optional subset: only sorted slots whose caller index is flagged */
    char *want = NULL;
    if (nsub >= 0) {
        want = (char *)calloc((size_t)(t->n > 0 ? t->n : 1), 1);
        for (int64_t s = 0; s < nsub; s++) want[sub[s]] = 1;
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t g = 0; g < t->ngroup; g++) {
        int64_t blo[3], bhi[3];
        for (int a = 0; a < 3; a++) { blo[a] = t->glo[3 * g + a]; bhi[a] = t->ghi[3 * g + a]; }
        /* relative criterion: K of the group; a group without a reference
         * (smallest |a| = 0, e.g. before any force pass) uses the opening angle */
        int rel = 0;
        float K = 0.0f;
        if (rx) {
            float amin = 0.0f;
            for (int64_t i = t->gfirst[g]; i < t->gfirst[g] + t->gcount[g]; i++) {
                const int64_t j = t->perm[i];
                float v = ref_mag(rx[j], ry[j], rz[j]);
                if (i == t->gfirst[g] || v < amin) amin = v;
            }
            if (amin > 0.0f) { rel = 1; K = (alpha * amin) * (u * u); }
        }
        for (int64_t i = t->gfirst[g]; i < t->gfirst[g] + t->gcount[g]; i++) {
            if (want && !want[t->perm[i]]) continue;
            walk_state w;
            memset(&w, 0, sizeof w);
            w.t = t; w.theta2 = theta2; w.quad = quad; w.e = eps_star; w.self = i; w.rel = rel; w.K = K;
            w.kind = kind;
            memcpy(w.blo, blo, sizeof blo); memcpy(w.bhi, bhi, sizeof bhi);
            w.px = t->x[i]; w.py = t->y[i]; w.pz = t->z[i];
            if (t->ncell > 0) walk_cell(&w, 0);
            for (int32_t k = 0; k < nx; k++) {
                p2p(w.px, w.py, w.pz, xx[k], xy[k], xz[k], xm[k], pair_eps(eps_star, xeps[k]), &w.ax, &w.ay, &w.az, &w.ph);
                if (xq && !(xq_skip && xq_skip[t->perm[i]]))
                    quad_term(w.px - xx[k], w.py - xy[k], w.pz - xz[k], pair_eps(eps_star, xeps[k]), xq + 6 * k,
                              &w.ax, &w.ay, &w.az, &w.ph);
            }
            int64_t o = t->perm[i];
            ax[o] = nval(&w.ax); ay[o] = nval(&w.ay); az[o] = nval(&w.az); pot[o] = nval(&w.ph);
            if (counts) { counts[2 * o] = w.n_p2p; counts[2 * o + 1] = w.n_m2p; }
        }
    }
    free(want);
    for (int32_t k = 0; k < nx; k++) {
        walk_state w;
        memset(&w, 0, sizeof w);
        w.t = t; w.theta2 = theta2; w.quad = quad; w.self = -1;
        w.e = pair_eps(xeps[k], eps_star);
        w.px = xx[k]; w.py = xy[k]; w.pz = xz[k];
        const float pv[3] = {xx[k], xy[k], xz[k]};
        for (int a = 0; a < 3; a++) {
            double q = floor(((double)pv[a] - t->lo[a]) * t->scale);
            if (q < -8388608.0) q = -8388608.0;
            if (q > 8388608.0) q = 8388608.0;
            w.blo[a] = (int64_t)q; w.bhi[a] = (int64_t)q + 1;
        }
        if (t->ncell > 0) walk_cell(&w, 0);
        for (int32_t j = 0; j < nx; j++) {
            if (j == k) continue;
            p2p(w.px, w.py, w.pz, xx[j], xy[j], xz[j], xm[j], pair_eps(xeps[k], xeps[j]), &w.ax, &w.ay, &w.az, &w.ph);
            if (xq)
                quad_term(w.px - xx[j], w.py - xy[j], w.pz - xz[j], pair_eps(xeps[k], xeps[j]), xq + 6 * j, &w.ax,
                          &w.ay, &w.az, &w.ph);
        }
        xax[k] = nval(&w.ax); xay[k] = nval(&w.ay); xaz[k] = nval(&w.az); xpot[k] = nval(&w.ph);
    }
}

/* ------------------------------------------------------------------ */
/* 6. Chain / perturber coupling, unsoftened FP64 (Sect. 2, Eq. 3)      */
/* ------------------------------------------------------------------ */
/* f(r) = r / |r|^3 and the potential -m / |r| (unsoftened). */
static void kepler_pot(double rx, double ry, double rz, double m, double out[4]) {
    double r2 = rx * rx + ry * ry + rz * rz;
    if (r2 <= 0.0) { out[0] = out[1] = out[2] = out[3] = 0.0; return; }
    double rinv = 1.0 / sqrt(r2);
    double s = m * rinv * rinv * rinv;
    out[0] = s * rx; out[1] = s * ry; out[2] = s * rz; out[3] = -m * rinv;
}

/* Chain members k (mass cm[k], position cx[3k..]) and perturbers p (mass pm[p],
 * position px[3p..]) with the chain centre of mass com and total mass
 * M = sum cm (Sect. 2: perturbers feel the resolved members; members feel
 * the perturbers; the centre-of-mass particle's force is corrected, Eq. 3):
 *   a_pert[p], pot_pert[p]   = sum_k cm_k f(x_k - x_p) - M f(com - x_p)
 *                              (resolved chain replaces the centre-of-mass particle);
 *   a_chain[k], pot_chain[k] = sum_p pm_p f(x_p - x_k)   (perturbers on each member);
 *   out[0..3) corr = (1/M) sum_k cm_k a_chain[k]  (Eq. 3);
 *   out[3..6) sub  = sum_p pm_p f(x_p - com), the direct unsoftened terms of the
 *                perturbers on the centre-of-mass particle, to subtract;
 *   out[6] = (1/M) sum_k cm_k pot_chain[k], out[7] = potential of sub;
 *   out[8..11) com, out[11] M. */
void orc_perturber(int32_t nch, const double *cm, const double *cx, int32_t np, const double *pm,
                   const double *px, double *a_pert, double *pot_pert, double *a_chain, double *pot_chain,
                   double out[12]) {
    double M = 0, com[3] = {0, 0, 0};
    for (int32_t k = 0; k < nch; k++) {
        M += cm[k];
        for (int a = 0; a < 3; a++) com[a] += cm[k] * cx[3 * k + a];
    }
    for (int a = 0; a < 3; a++) com[a] = (M > 0) ? com[a] / M : 0.0;
#pragma omp parallel for schedule(static)
    for (int32_t p = 0; p < np; p++) {
        nsum s[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
        double f[4];
        for (int32_t k = 0; k < nch; k++) {
            kepler_pot(cx[3 * k] - px[3 * p], cx[3 * k + 1] - px[3 * p + 1], cx[3 * k + 2] - px[3 * p + 2], cm[k], f);
            for (int a = 0; a < 4; a++) nadd(&s[a], f[a]);
        }
        kepler_pot(com[0] - px[3 * p], com[1] - px[3 * p + 1], com[2] - px[3 * p + 2], M, f);
        for (int a = 0; a < 4; a++) nadd(&s[a], -f[a]);
        for (int a = 0; a < 3; a++) a_pert[3 * p + a] = nval(&s[a]);
        pot_pert[p] = nval(&s[3]);
    }
    nsum cs[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (int32_t k = 0; k < nch; k++) {
        nsum s[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
        double f[4];
        for (int32_t p = 0; p < np; p++) {
            kepler_pot(px[3 * p] - cx[3 * k], px[3 * p + 1] - cx[3 * k + 1], px[3 * p + 2] - cx[3 * k + 2], pm[p], f);
            for (int a = 0; a < 4; a++) nadd(&s[a], f[a]);
        }
        for (int a = 0; a < 3; a++) a_chain[3 * k + a] = nval(&s[a]);
        pot_chain[k] = nval(&s[3]);
        for (int a = 0; a < 3; a++) nadd(&cs[a], cm[k] * a_chain[3 * k + a]);
        nadd(&cs[3], cm[k] * pot_chain[k]);
    }
    nsum ss[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (int32_t p = 0; p < np; p++) {
        double f[4];
        kepler_pot(px[3 * p] - com[0], px[3 * p + 1] - com[1], px[3 * p + 2] - com[2], pm[p], f);
        for (int a = 0; a < 4; a++) nadd(&ss[a], f[a]);
    }
    for (int a = 0; a < 3; a++) { out[a] = (M > 0) ? nval(&cs[a]) / M : 0.0; out[3 + a] = nval(&ss[a]); }
    out[6] = (M > 0) ? nval(&cs[3]) / M : 0.0;
    out[7] = nval(&ss[3]);
    out[8] = com[0]; out[9] = com[1]; out[10] = com[2]; out[11] = M;
}

/* ------------------------------------------------------------------ */
/* 7. Perturber selection                                               */
/* ------------------------------------------------------------------ */
/* Squared distance in FP32, each operation rounded once in this order:
 * d = x - c per axis, d2 = (dx*dx + dy*dy) + dz*dz. */
static float dist2_f32(float x, float y, float z, float cx, float cy, float cz) {
    float dx = x - cx, dy = y - cy, dz = z - cz;
    float a = dx * dx, b = dy * dy, c = dz * dz;
    float s = a + b;
    return s + c;
}

typedef struct { float d2; int64_t idx; } fd;
static int fd_cmp(const void *a, const void *b) {
    const fd *p = (const fd *)a, *q = (const fd *)b;
    if (p->d2 != q->d2) return p->d2 < q->d2 ? -1 : 1;
    return (p->idx > q->idx) - (p->idx < q->idx);
}

/* The k particles nearest to c (ties by lower index), ascending (d2, index). */
int64_t orc_knn(int64_t n, const float *x, const float *y, const float *z, const float c[3], int64_t k, int64_t *out) {
    fd *t = (fd *)malloc(sizeof(fd) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; i++) { t[i].d2 = dist2_f32(x[i], y[i], z[i], c[0], c[1], c[2]); t[i].idx = i; }
    qsort(t, (size_t)n, sizeof(fd), fd_cmp);
    if (k > n) k = n;
    for (int64_t i = 0; i < k; i++) out[i] = t[i].idx;
    free(t);
    return k;
}

/* Ingredients of the chain's start radius (Eq. 1) around a centre c (FP32):
 * stars in ascending FP32 squared distance (ties by index, as orc_knn);
 * out[0] = r(<2 M_bh): the distance (sqrt of the FP64 value of the FP32 d2)
 *          of the star at which the running FP64 sum of masses, taken in that
 *          order, first reaches 2 m_bh (infinity if it never does);
 * out[1] = sigma: the 1D velocity dispersion of the n_sigma nearest stars,
 *          sqrt(sum |v - <v>|^2 / (3 k)), k = min(n_sigma, n), all sums in
 *          FP64 in distance order (<v> their mean velocity);
 * out[2] = G m_bh / sigma^2 (G = 1). */
void orc_influence(int64_t n, const float *x, const float *y, const float *z, const float *vx, const float *vy,
                   const float *vz, const float *m, const float c[3], double m_bh, int64_t n_sigma, double out[3]) {
    fd *t = (fd *)malloc(sizeof(fd) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; i++) { t[i].d2 = dist2_f32(x[i], y[i], z[i], c[0], c[1], c[2]); t[i].idx = i; }
    qsort(t, (size_t)n, sizeof(fd), fd_cmp);
    double cum = 0.0;
    out[0] = INFINITY;
    for (int64_t i = 0; i < n; i++) {
        cum += (double)m[t[i].idx];
        if (cum >= 2.0 * m_bh) { out[0] = sqrt((double)t[i].d2); break; }
    }
    int64_t k = n_sigma < n ? n_sigma : n;
    double mx = 0.0, my = 0.0, mz = 0.0;
    for (int64_t i = 0; i < k; i++) {
        int64_t j = t[i].idx;
        mx += (double)vx[j]; my += (double)vy[j]; mz += (double)vz[j];
    }
    mx /= (double)k; my /= (double)k; mz /= (double)k;
    double s = 0.0;
    for (int64_t i = 0; i < k; i++) {
        int64_t j = t[i].idx;
        double dx = (double)vx[j] - mx, dy = (double)vy[j] - my, dz = (double)vz[j] - mz;
        s += dx * dx;
        s += dy * dy;
        s += dz * dz;
    }
    double s2 = s / (3.0 * (double)k);
    out[1] = sqrt(s2);
    out[2] = m_bh / s2;
    free(t);
}

/* Tidal perturber criterion (Eq. 2): particle j perturbs a chain of total
 * mass M when r_j < (2 m_j / (gamma M))^(1/3) r_crit, r_j its distance to the
 * chain's centre. Taken without a cube root, in FP64 with one rounding per
 * operation on the FP32 squared distance d2 (computed as for the radius
 * search): (d2 d2) d2 < (q q) rc6 with q = (2 m_j) / (gamma M) and
 * rc6 = (rc2 rc2) rc2, rc2 = r_crit r_crit. Ascending index; returns the
 * count (at most cap are written). */
int64_t orc_tidal(int64_t n, const float *x, const float *y, const float *z, const float *m, const float c[3],
                  float mchain, float gamma, float rcrit, int64_t cap, int64_t *out) {
    const double rc2 = (double)rcrit * (double)rcrit;
    const double rc6 = (rc2 * rc2) * rc2;
    const double den = (double)gamma * (double)mchain;
    int64_t k = 0;
    for (int64_t i = 0; i < n; i++) {
        const double d2 = (double)dist2_f32(x[i], y[i], z[i], c[0], c[1], c[2]);
        const double q = (2.0 * (double)m[i]) / den;
        if ((d2 * d2) * d2 < (q * q) * rc6) { if (k < cap) out[k] = i; k++; }
    }
    return k;
}

/* All particles with d2 < r2 (FP32), ascending index; returns the count
 * (at most cap are written). */
int64_t orc_radius(int64_t n, const float *x, const float *y, const float *z, const float c[3], float r2,
                   int64_t cap, int64_t *out) {
    int64_t k = 0;
    for (int64_t i = 0; i < n; i++)
        if (dist2_f32(x[i], y[i], z[i], c[0], c[1], c[2]) < r2) { if (k < cap) out[k] = i; k++; }
    return k;
}

/* ------------------------------------------------------------------ */
/* 8. Chain membership: absorption (Eq. 4)                              */
/* ------------------------------------------------------------------ */
/* The chain's centre of mass c = sum_k m_k x_k / M (FP64, members in index
 * order) and its radius, the largest member distance from c (Sect. 2: the
 * chain radius of the last chain step). Star j (FP32 position) is absorbed
 * when r_j,CoM < r_chain (Eq. 4), decided without a square root in FP64 with
 * one rounding per operation: d_a = (double)x_a - c_a, d2 = (d_x d_x + d_y d_y)
 * + d_z d_z, absorbed iff d2 < rc2 with rc2 the largest member d2 (same
 * formula). Writes the first cap ascending indices to out, returns the count;
 * out2 = (sqrt(rc2), rc2). */
int64_t orc_absorb(int64_t n, const float *x, const float *y, const float *z, int32_t nch, const double *cm,
                   const double *cx, int64_t cap, int64_t *out, double out2[2]) {
    double M = 0.0, c[3] = {0.0, 0.0, 0.0};
    for (int32_t k = 0; k < nch; k++) {
        M += cm[k];
        for (int a = 0; a < 3; a++) c[a] += cm[k] * cx[3 * k + a];
    }
    for (int a = 0; a < 3; a++) c[a] = (M > 0.0) ? c[a] / M : 0.0;
    double rc2 = 0.0;
    for (int32_t k = 0; k < nch; k++) {
        double dx = cx[3 * k] - c[0], dy = cx[3 * k + 1] - c[1], dz = cx[3 * k + 2] - c[2];
        double d2 = (dx * dx + dy * dy) + dz * dz;
        if (d2 > rc2) rc2 = d2;
    }
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; i++) {
        double dx = (double)x[i] - c[0], dy = (double)y[i] - c[1], dz = (double)z[i] - c[2];
        double d2 = (dx * dx + dy * dy) + dz * dz;
        if (d2 < rc2) { if (cnt < cap) out[cnt] = i; cnt++; }
    }
    out2[0] = sqrt(rc2);
    out2[1] = rc2;
    return cnt;
}
