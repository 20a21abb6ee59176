/*
 * hybrid_oracle.c -- plain, slow FP64 CPU oracle of the hybrid tree force path.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library. The CUDA library never
 * calls it, and the two share no source, header, table or helper.
 *
 * It follows Watanabe & Nakasato, "GPU accelerated Hybrid Tree Algorithm for
 * Collision-less N-body Simulations", section by section:
 *   Eq. (1)-(2)  softened gravity                      -> pair_acc, orc_direct
 *   Eq. (3)-(4)  leap-frog kick / drift                -> orc_hybrid_steps
 *   Sec. II-B    tree build, centre of mass, MAC, walk -> orc_tree_*, walk_visit
 *   Eq. (5)-(6)  absolute MAC and B2                   -> moments()
 *   Eq. (7)-(10) hard/soft split with the DLL kernel    -> orc_cutoff_K
 *   Eq. (11)     minimum distance over a sink group     -> dist_point_box
 *   Eq. (15)     R2 + b_max neighbour criterion         -> walk_visit
 *   Sec. III-A1  root cell, Morton keys, sort, split    -> orc_root_box, keys, build
 * Readings taken where the paper is silent are stated beside the code.
 *
 * Build with -ffp-contract=off: every + - * / below rounds once, in the order
 * written. OpenMP is used only to run independent sinks/groups on several
 * threads; it never changes the order of any sum.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_LEVELS 21                       /* 3 x 21 = 63 key bits */
#define ORC_QMAX ((1u << ORC_LEVELS) - 1u)

typedef struct {
    double G, eps, theta, R1, R2, dt_soft, a_err;
    int32_t n_hard, n_leaf, n_crit, mac;   /* mac: 0 = opening angle, 1 = absolute MAC */
} orc_params;

/* ------------------------------------------------------------------------ */
/* Eq. (10): DLL cutoff kernel. Y = (R2 - r)/(R2 - R1); K = 1 for Y >= 1,     */
/* 10Y^6 - 15Y^8 + 6Y^10 for 0 < Y < 1, 0 for Y <= 0. Reading: R1 = R2 = 0    */
/* switches the hard part off (K = 0 everywhere).                            */
/* ------------------------------------------------------------------------ */
double orc_cutoff_K(double r, double R1, double R2)
{
    if (R2 <= 0.0) return 0.0;
    double Y = (R2 - r) / (R2 - R1);
    if (Y >= 1.0) return 1.0;
    if (Y <= 0.0) return 0.0;
    double Y2 = Y * Y;
    double Y6 = Y2 * Y2 * Y2;
    double Y8 = Y6 * Y2;
    double Y10 = Y8 * Y2;
    return 10.0 * Y6 - 15.0 * Y8 + 6.0 * Y10;
}

/* Eq. (2): acceleration on the sink at xi from a source of mass mj at xj,
 * G m_j (r_j - r_i) / (|r_i - r_j|^2 + eps^2)^{3/2}, times the weight w
 * (1, K or 1 - K, Eq. 8-9). scale accumulates |term| for error budgets. */
static void pair_acc(const double xi[3], double xj0, double xj1, double xj2, double mj,
                     double G, double eps, double w, double acc[3], double *scale)
{
    double d0 = xj0 - xi[0], d1 = xj1 - xi[1], d2 = xj2 - xi[2];
    double r2 = d0 * d0 + d1 * d1 + d2 * d2;
    double s2 = r2 + eps * eps;
    double f = G * mj * w / pow(s2, 1.5);
    acc[0] += f * d0;
    acc[1] += f * d1;
    acc[2] += f * d2;
    if (scale) *scale += fabs(f) * sqrt(r2);
}

/* ------------------------------------------------------------------------ */
/* Direct summation, Eq. (1)-(2), split by Eq. (7)-(9).                      */
/* which: 0 = full force, 1 = hard part F*K, 2 = soft part F*(1-K).          */
/* Sinks sink[0..ns) (indices into the arrays); sources are all particles,  */
/* j = i skipped.                                                            */
/* ------------------------------------------------------------------------ */
void orc_direct(int64_t n, const double *x, const double *y, const double *z, const double *m,
                double G, double eps, double R1, double R2, int32_t which,
                int64_t ns, const int64_t *sink, double *ax, double *ay, double *az, double *scale)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t s = 0; s < ns; ++s) {
        int64_t i = sink[s];
        double xi[3] = {x[i], y[i], z[i]};
        double acc[3] = {0.0, 0.0, 0.0};
        double sc = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double w = 1.0;
            if (which != 0) {
                double d0 = x[j] - xi[0], d1 = y[j] - xi[1], d2 = z[j] - xi[2];
                double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
                double K = orc_cutoff_K(r, R1, R2);
                w = (which == 1) ? K : 1.0 - K;
            }
            pair_acc(xi, x[j], y[j], z[j], m[j], G, eps, w, acc, &sc);
        }
        ax[s] = acc[0];
        ay[s] = acc[1];
        az[s] = acc[2];
        if (scale) scale[s] = sc;
    }
}

/* Softened potential energy W = -1/2 sum_i sum_{j != i} G m_i m_j / sqrt(r^2 + eps^2)
 * and kinetic energy T = 1/2 sum_i m_i |v_i|^2 (the "total energy" of Sec. IV-A). */
void orc_energy(int64_t n, const double *x, const double *y, const double *z,
                const double *vx, const double *vy, const double *vz, const double *m,
                double G, double eps, double *kin, double *pot)
{
    double T = 0.0, W = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        T += 0.5 * m[i] * (vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i]);
        double wi = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d0 = x[j] - x[i], d1 = y[j] - y[i], d2 = z[j] - z[i];
            wi += G * m[i] * m[j] / sqrt(d0 * d0 + d1 * d1 + d2 * d2 + eps * eps);
        }
        W += wi;
    }
    *kin = T;
    *pot = -0.5 * W;
}

/* ------------------------------------------------------------------------ */
/* Sec. III-A1: root cell. Reading: the root is the cube anchored at the     */
/* per-axis minimum lo, with side L = the smallest power of two that is      */
/* >= the largest per-axis extent (L = 1 when every particle coincides).     */
/* ------------------------------------------------------------------------ */
void orc_root_box(int64_t n, const double *x, const double *y, const double *z, double lo[3], double *L)
{
    if (n <= 0) {
        lo[0] = lo[1] = lo[2] = 0.0;
        *L = 1.0;
        return;
    }
    double mn[3] = {x[0], y[0], z[0]}, mx[3] = {x[0], y[0], z[0]};
    for (int64_t i = 1; i < n; ++i) {
        double p[3] = {x[i], y[i], z[i]};
        for (int d = 0; d < 3; ++d) {
            if (p[d] < mn[d]) mn[d] = p[d];
            if (p[d] > mx[d]) mx[d] = p[d];
        }
    }
    double ext = 0.0;
    for (int d = 0; d < 3; ++d) {
        double e = mx[d] - mn[d];
        if (e > ext) ext = e;
    }
    double side = 1.0;
    if (ext > 0.0) {
        int e2;
        double f = frexp(ext, &e2);          /* ext = f * 2^e2, f in [0.5, 1) */
        side = (f == 0.5) ? ext : ldexp(1.0, e2);
    }
    lo[0] = mn[0];
    lo[1] = mn[1];
    lo[2] = mn[2];
    *L = side;
}

/* Sec. III-A1: Morton key. Integer cell coordinate per axis,
 * q = clamp(floor((x - lo) * 2^21 / L), 0, 2^21 - 1); the scale 2^21/L is a
 * power of two, so only the subtraction rounds. The 63-bit key interleaves
 * the bits of (qx, qy, qz) from the most significant one down, x first. */
static uint32_t cell_coord(double x, double lo, double scale)
{
    double t = floor((x - lo) * scale);
    if (t < 0.0) t = 0.0;
    if (t > (double)ORC_QMAX) t = (double)ORC_QMAX;
    return (uint32_t)t;
}

void orc_morton_keys(int64_t n, const double *x, const double *y, const double *z,
                     const double lo[3], double L, uint64_t *key)
{
    double scale = ldexp(1.0, ORC_LEVELS) / L;
    for (int64_t i = 0; i < n; ++i) {
        uint32_t q[3] = {cell_coord(x[i], lo[0], scale), cell_coord(y[i], lo[1], scale),
                         cell_coord(z[i], lo[2], scale)};
        uint64_t k = 0;
        for (int b = ORC_LEVELS - 1; b >= 0; --b) {
            k = (k << 3) | ((uint64_t)((q[0] >> b) & 1u) << 2) | ((uint64_t)((q[1] >> b) & 1u) << 1) |
                (uint64_t)((q[2] >> b) & 1u);
        }
        key[i] = k;
    }
}

/* Sec. III-A1: sort by key. Stable: equal keys keep their input order.
 * Plain top-down merge sort of the index array; perm[k] = input index of the
 * k-th smallest key. */
static void merge_sort_rec(const uint64_t *key, int64_t *a, int64_t *tmp, int64_t lo, int64_t hi)
{
    if (hi - lo < 2) return;
    int64_t mid = lo + (hi - lo) / 2;
    merge_sort_rec(key, a, tmp, lo, mid);
    merge_sort_rec(key, a, tmp, mid, hi);
    int64_t i = lo, j = mid, k = lo;
    while (i < mid && j < hi) {
        if (key[a[j]] < key[a[i]]) tmp[k++] = a[j++]; /* left wins ties: stable */
        else tmp[k++] = a[i++];
    }
    while (i < mid) tmp[k++] = a[i++];
    while (j < hi) tmp[k++] = a[j++];
    memcpy(a + lo, tmp + lo, (size_t)(hi - lo) * sizeof(int64_t));
}

void orc_sort(int64_t n, const uint64_t *key, int64_t *perm)
{
    for (int64_t i = 0; i < n; ++i) perm[i] = i;
    if (n < 2) return;
    int64_t *tmp = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    merge_sort_rec(key, perm, tmp, 0, n);
    free(tmp);
}

/* ------------------------------------------------------------------------ */
/* Tree: build, moments, groups (Sec. II-B, Sec. III-A1).                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n;
    orc_params p;
    double lo[3], L;
    /* particles in key order */
    uint64_t *key;
    int64_t *perm;               /* sorted position -> input index */
    double *x, *y, *z, *m;
    /* nodes in canonical breadth-first order */
    int64_t nn, ncap;
    int32_t *level, *nchild;
    int64_t *first, *count, *child, *parent;
    double *M, *cx, *cy, *cz, *bmax, *B2, *delta, *side, *ox, *oy, *oz, *rb;
    /* sink groups in particle order */
    int64_t ng;
    int64_t *gnode;
    double *glo, *ghi;           /* 3 per group: box of the member particles */
} orc_tree;

static void *xmalloc(size_t n) { return malloc(n ? n : 1); }

static void tree_grow(orc_tree *t)
{
    int64_t c = t->ncap ? 2 * t->ncap : 1024;
    t->level = realloc(t->level, (size_t)c * sizeof(int32_t));
    t->nchild = realloc(t->nchild, (size_t)c * sizeof(int32_t));
    t->first = realloc(t->first, (size_t)c * sizeof(int64_t));
    t->count = realloc(t->count, (size_t)c * sizeof(int64_t));
    t->child = realloc(t->child, (size_t)c * sizeof(int64_t));
    t->parent = realloc(t->parent, (size_t)c * sizeof(int64_t));
    t->ncap = c;
}

static void tree_append(orc_tree *t, int32_t level, int64_t first, int64_t count, int64_t parent)
{
    if (t->nn == t->ncap) tree_grow(t);
    int64_t q = t->nn++;
    t->level[q] = level;
    t->first[q] = first;
    t->count[q] = count;
    t->parent[q] = parent;
    t->child[q] = -1;
    t->nchild[q] = 0;
}

/* Sec. III-A1 split rule. Reading: a cell splits while it holds more than
 * n_leaf particles and is above the deepest key level; its children are its
 * non-empty octants in key order. Processing a FIFO queue appends nodes level
 * by level and, inside a level, in key-prefix order: the canonical order. */
static void build(orc_tree *t)
{
    t->nn = 0;
    if (t->n == 0) return;
    tree_append(t, 0, 0, t->n, -1);
    for (int64_t q = 0; q < t->nn; ++q) {
        if (t->count[q] <= t->p.n_leaf || t->level[q] >= ORC_LEVELS) continue;
        int shift = 3 * (ORC_LEVELS - (t->level[q] + 1));
        int64_t i = t->first[q], end = t->first[q] + t->count[q];
        t->child[q] = t->nn;
        while (i < end) {
            uint64_t digit = (t->key[i] >> shift) & 7u;
            int64_t j = i;
            while (j < end && ((t->key[j] >> shift) & 7u) == digit) ++j;
            tree_append(t, t->level[q] + 1, i, j - i, q);
            t->nchild[q] += 1;
            i = j;
        }
    }
}

/* Integer cell coordinate of a key prefix along one axis (axis 0 = x). */
static uint32_t prefix_coord(uint64_t key, int level, int axis)
{
    uint32_t c = 0;
    for (int l = 1; l <= level; ++l) {
        uint64_t digit = (key >> (3 * (ORC_LEVELS - l))) & 7u;
        c = (c << 1) | (uint32_t)((digit >> (2 - axis)) & 1u);
    }
    return c;
}

/* Sec. II-B and Eq. (5)-(6): per cell, by explicit sums over its members:
 * mass M, centre of mass, b_max = max |r_CM - r_i|, B2 = sum m_i |r_CM - r_i|^2;
 * cell geometry (side l = L / 2^level, origin, offset delta = |r_CM - centre|)
 * and the opening radius r_b. Reading for the opening-angle MAC:
 * r_b = l / theta + delta (theta = 0 opens every cell); absolute MAC: Eq. (5). */
static void moments(orc_tree *t)
{
    int64_t nn = t->nn;
    t->M = xmalloc((size_t)nn * sizeof(double));
    t->cx = xmalloc((size_t)nn * sizeof(double));
    t->cy = xmalloc((size_t)nn * sizeof(double));
    t->cz = xmalloc((size_t)nn * sizeof(double));
    t->bmax = xmalloc((size_t)nn * sizeof(double));
    t->B2 = xmalloc((size_t)nn * sizeof(double));
    t->delta = xmalloc((size_t)nn * sizeof(double));
    t->side = xmalloc((size_t)nn * sizeof(double));
    t->ox = xmalloc((size_t)nn * sizeof(double));
    t->oy = xmalloc((size_t)nn * sizeof(double));
    t->oz = xmalloc((size_t)nn * sizeof(double));
    t->rb = xmalloc((size_t)nn * sizeof(double));
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t c = 0; c < nn; ++c) {
        int64_t a = t->first[c], b = a + t->count[c];
        int lev = t->level[c];
        double side = ldexp(t->L, -lev);
        double o[3];
        for (int d = 0; d < 3; ++d) o[d] = t->lo[d] + (double)prefix_coord(t->key[a], lev, d) * side;
        double ctr[3] = {o[0] + 0.5 * side, o[1] + 0.5 * side, o[2] + 0.5 * side};
        /* sum m x / M taken as offsets from the cell's first particle: the same centre of mass, and exactly
         * that particle for a cell of one particle (or of coincident ones), whose B2 and b_max are then 0 */
        double M = 0.0, s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int64_t i = a; i < b; ++i) {
            M += t->m[i];
            s0 += t->m[i] * (t->x[i] - t->x[a]);
            s1 += t->m[i] * (t->y[i] - t->y[a]);
            s2 += t->m[i] * (t->z[i] - t->z[a]);
        }
        double com[3];
        if (M > 0.0) {
            com[0] = t->x[a] + s0 / M;
            com[1] = t->y[a] + s1 / M;
            com[2] = t->z[a] + s2 / M;
        } else { /* reading: a massless cell sits at its geometric centre */
            com[0] = ctr[0];
            com[1] = ctr[1];
            com[2] = ctr[2];
        }
        double bmax = 0.0, B2 = 0.0;
        for (int64_t i = a; i < b; ++i) {
            double d0 = t->x[i] - com[0], d1 = t->y[i] - com[1], d2 = t->z[i] - com[2];
            double r2 = d0 * d0 + d1 * d1 + d2 * d2;
            double r = sqrt(r2);
            if (r > bmax) bmax = r;
            B2 += t->m[i] * r2;
        }
        double e0 = com[0] - ctr[0], e1 = com[1] - ctr[1], e2 = com[2] - ctr[2];
        double delta = sqrt(e0 * e0 + e1 * e1 + e2 * e2);
        double rb;
        if (t->p.mac == 1) {
            rb = 0.5 * bmax + sqrt(0.25 * bmax * bmax + sqrt(3.0 * B2 / t->p.a_err));
        } else {
            rb = (t->p.theta > 0.0) ? side / t->p.theta + delta : INFINITY;
        }
        t->M[c] = M;
        t->cx[c] = com[0];
        t->cy[c] = com[1];
        t->cz[c] = com[2];
        t->bmax[c] = bmax;
        t->B2[c] = B2;
        t->delta[c] = delta;
        t->side[c] = side;
        t->ox[c] = o[0];
        t->oy[c] = o[1];
        t->oz[c] = o[2];
        t->rb[c] = rb;
    }
}

/* Sink groups (the n_vec sinks of Sec. III-A2, Eq. 11, grown to a cell).
 * Reading: descend from the root and stop at the first cell that holds at
 * most n_crit particles or is a leaf; that cell is a group. Depth-first in
 * child order lists the groups in particle order. */
static void groups_rec(orc_tree *t, int64_t c, int64_t *out, int64_t *ng)
{
    if (t->count[c] <= t->p.n_crit || t->nchild[c] == 0) {
        out[(*ng)++] = c;
        return;
    }
    for (int32_t k = 0; k < t->nchild[c]; ++k) groups_rec(t, t->child[c] + k, out, ng);
}

static void groups(orc_tree *t)
{
    t->ng = 0;
    t->gnode = xmalloc((size_t)(t->nn ? t->nn : 1) * sizeof(int64_t));
    if (t->nn) groups_rec(t, 0, t->gnode, &t->ng);
    t->glo = xmalloc((size_t)(3 * t->ng) * sizeof(double));
    t->ghi = xmalloc((size_t)(3 * t->ng) * sizeof(double));
    for (int64_t g = 0; g < t->ng; ++g) {
        int64_t c = t->gnode[g], a = t->first[c], b = a + t->count[c];
        double lo[3] = {t->x[a], t->y[a], t->z[a]}, hi[3] = {t->x[a], t->y[a], t->z[a]};
        for (int64_t i = a + 1; i < b; ++i) {
            double p[3] = {t->x[i], t->y[i], t->z[i]};
            for (int d = 0; d < 3; ++d) {
                if (p[d] < lo[d]) lo[d] = p[d];
                if (p[d] > hi[d]) hi[d] = p[d];
            }
        }
        for (int d = 0; d < 3; ++d) {
            t->glo[3 * g + d] = lo[d];
            t->ghi[3 * g + d] = hi[d];
        }
    }
}

/* The whole tree for one system (Sec. III-A1): root box, keys, stable sort,
 * the particles gathered into key order, split, moments, groups. */
orc_tree *orc_tree_new(int64_t n, const double *x, const double *y, const double *z, const double *m,
                       const orc_params *p)
{
    orc_tree *t = (orc_tree *)calloc(1, sizeof(orc_tree));
    t->n = n;
    t->p = *p;
    orc_root_box(n, x, y, z, t->lo, &t->L);
    uint64_t *key = xmalloc((size_t)n * sizeof(uint64_t));
    orc_morton_keys(n, x, y, z, t->lo, t->L, key);
    t->perm = xmalloc((size_t)n * sizeof(int64_t));
    orc_sort(n, key, t->perm);
    t->key = xmalloc((size_t)n * sizeof(uint64_t));
    t->x = xmalloc((size_t)n * sizeof(double));
    t->y = xmalloc((size_t)n * sizeof(double));
    t->z = xmalloc((size_t)n * sizeof(double));
    t->m = xmalloc((size_t)n * sizeof(double));
    for (int64_t k = 0; k < n; ++k) {
        int64_t i = t->perm[k];
        t->key[k] = key[i];
        t->x[k] = x[i];
        t->y[k] = y[i];
        t->z[k] = z[i];
        t->m[k] = m[i];
    }
    free(key);
    build(t);
    moments(t);
    groups(t);
    return t;
}

void orc_tree_free(orc_tree *t)
{
    if (!t) return;
    void *ptrs[] = {t->key, t->perm, t->x, t->y, t->z, t->m, t->level, t->nchild, t->first, t->count,
                    t->child, t->parent, t->M, t->cx, t->cy, t->cz, t->bmax, t->B2, t->delta, t->side,
                    t->ox, t->oy, t->oz, t->rb, t->gnode, t->glo, t->ghi};
    for (size_t k = 0; k < sizeof(ptrs) / sizeof(ptrs[0]); ++k) free(ptrs[k]);
    free(t);
}

/* Accessors for the Python side. */
int64_t orc_tree_n(const orc_tree *t) { return t->n; }
int64_t orc_tree_nn(const orc_tree *t) { return t->nn; }
int64_t orc_tree_ng(const orc_tree *t) { return t->ng; }
void orc_tree_box(const orc_tree *t, double out[4])
{
    out[0] = t->lo[0];
    out[1] = t->lo[1];
    out[2] = t->lo[2];
    out[3] = t->L;
}
void orc_tree_particles(const orc_tree *t, uint64_t *key, int64_t *perm, double *x, double *y, double *z,
                        double *m)
{
    size_t n = (size_t)t->n;
    memcpy(key, t->key, n * sizeof(uint64_t));
    memcpy(perm, t->perm, n * sizeof(int64_t));
    memcpy(x, t->x, n * sizeof(double));
    memcpy(y, t->y, n * sizeof(double));
    memcpy(z, t->z, n * sizeof(double));
    memcpy(m, t->m, n * sizeof(double));
}
void orc_tree_nodes(const orc_tree *t, int32_t *level, int64_t *first, int64_t *count, int64_t *child,
                    int32_t *nchild, int64_t *parent)
{
    size_t nn = (size_t)t->nn;
    memcpy(level, t->level, nn * sizeof(int32_t));
    memcpy(first, t->first, nn * sizeof(int64_t));
    memcpy(count, t->count, nn * sizeof(int64_t));
    memcpy(child, t->child, nn * sizeof(int64_t));
    memcpy(nchild, t->nchild, nn * sizeof(int32_t));
    memcpy(parent, t->parent, nn * sizeof(int64_t));
}
/* out: nn x 13 doubles: M, cx, cy, cz, bmax, B2, delta, side, ox, oy, oz, rb, (reserved 0) */
void orc_tree_moments(const orc_tree *t, double *out)
{
    for (int64_t c = 0; c < t->nn; ++c) {
        double *o = out + 13 * c;
        o[0] = t->M[c];
        o[1] = t->cx[c];
        o[2] = t->cy[c];
        o[3] = t->cz[c];
        o[4] = t->bmax[c];
        o[5] = t->B2[c];
        o[6] = t->delta[c];
        o[7] = t->side[c];
        o[8] = t->ox[c];
        o[9] = t->oy[c];
        o[10] = t->oz[c];
        o[11] = t->rb[c];
        o[12] = 0.0;
    }
}
void orc_tree_groups(const orc_tree *t, int64_t *gnode, double *glo, double *ghi)
{
    memcpy(gnode, t->gnode, (size_t)t->ng * sizeof(int64_t));
    memcpy(glo, t->glo, (size_t)(3 * t->ng) * sizeof(double));
    memcpy(ghi, t->ghi, (size_t)(3 * t->ng) * sizeof(double));
}

/* ------------------------------------------------------------------------ */
/* Grouped walk (Sec. II-B traversal rule, Eq. 11, Eq. 15).                  */
/* ------------------------------------------------------------------------ */

/* Eq. (11) with a box: the smallest distance from a point to the box of the
 * group's sinks, 0 inside. Per axis the gap is max(lo - p, 0, p - hi). */
static double dist_point_box(double p0, double p1, double p2, const double lo[3], const double hi[3])
{
    double p[3] = {p0, p1, p2}, s = 0.0;
    for (int d = 0; d < 3; ++d) {
        double g = 0.0;
        double a = lo[d] - p[d];
        double b = p[d] - hi[d];
        if (a > g) g = a;
        if (b > g) g = b;
        s += g * g;
    }
    return sqrt(s);
}

typedef struct {
    int64_t *v;
    int64_t n, cap;
} ivec;

static void ivec_push(ivec *a, int64_t x)
{
    if (a->v == NULL && a->cap < 0) { /* counting only */
        a->n++;
        return;
    }
    if (a->n == a->cap) {
        a->cap = a->cap ? 2 * a->cap : 256;
        a->v = realloc(a->v, (size_t)a->cap * sizeof(int64_t));
    }
    a->v[a->n++] = x;
}

/* Visit cell c for group g. Traversal rule of Sec. II-B: open the cell when
 * r_b > r (strict), else take its centre of mass. Reading for the cutoff: a
 * cell is taken whole only when also r >= R2 + b_max (the test of Eq. 15), so
 * every member is at least R2 from every sink and K = 0 for all of its pairs.
 * The hard walk keeps the cells with r < R2 + b_max; its leaves give the
 * neighbour particles. r is measured from the centre of mass to the group box. */
static void walk_visit(const orc_tree *t, int64_t c, const double *glo, const double *ghi, int want_soft,
                       int want_hard, ivec *cells, ivec *parts, ivec *hparts)
{
    double d = dist_point_box(t->cx[c], t->cy[c], t->cz[c], glo, ghi);
    double hard_r = t->p.R2 + t->bmax[c];
    int hard_near = (t->p.R2 > 0.0) && (d < hard_r);
    int accept = (d >= t->rb[c]) && (d >= hard_r);
    int leaf = (t->nchild[c] == 0);
    if (want_soft) {
        if (accept) ivec_push(cells, c);
        else if (leaf)
            for (int64_t i = t->first[c]; i < t->first[c] + t->count[c]; ++i) ivec_push(parts, i);
    }
    if (want_hard && hard_near && leaf)
        for (int64_t i = t->first[c]; i < t->first[c] + t->count[c]; ++i) ivec_push(hparts, i);
    if (!leaf) {
        int ws = want_soft && !accept;
        int wh = want_hard && hard_near;
        if (ws || wh)
            for (int32_t k = 0; k < t->nchild[c]; ++k)
                walk_visit(t, t->child[c] + k, glo, ghi, ws, wh, cells, parts, hparts);
    }
}

static void walk_group(const orc_tree *t, int64_t g, int want_soft, int want_hard, ivec *cells, ivec *parts,
                       ivec *hparts)
{
    if (t->nn == 0) return;
    walk_visit(t, 0, t->glo + 3 * g, t->ghi + 3 * g, want_soft, want_hard, cells, parts, hparts);
}

/* Lists for the selected groups: counts[3*k + {0,1,2}] = soft cells, soft
 * particles, hard particles of group sel[k]. If out is non-NULL the lists are
 * written back to back per group (cells, particles, hard particles), using
 * the offsets given by the counts. mode bit 0 = soft lists, bit 1 = hard. */
void orc_walk(const orc_tree *t, int64_t nsel, const int64_t *sel, int32_t mode, int64_t *counts,
              const int64_t *offsets, int64_t *out)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t k = 0; k < nsel; ++k) {
        ivec cells = {0}, parts = {0}, hparts = {0};
        walk_group(t, sel[k], mode & 1, (mode >> 1) & 1, &cells, &parts, &hparts);
        counts[3 * k + 0] = cells.n;
        counts[3 * k + 1] = parts.n;
        counts[3 * k + 2] = hparts.n;
        if (out) {
            int64_t *o = out + offsets[k];
            memcpy(o, cells.v, (size_t)cells.n * sizeof(int64_t));
            memcpy(o + cells.n, parts.v, (size_t)parts.n * sizeof(int64_t));
            memcpy(o + cells.n + parts.n, hparts.v, (size_t)hparts.n * sizeof(int64_t));
        }
        free(cells.v);
        free(parts.v);
        free(hparts.v);
    }
}

/* Same-tree forces for the sinks of the selected groups (sorted order):
 * soft  = sum over taken cells of F(cell) + sum over listed particles F*(1-K),
 * hard  = sum over hard-listed particles F*K         (Eq. 7-10),
 * each summed in list order. Outputs are indexed by sorted particle position;
 * scale_* gets the sum of term magnitudes. mode bit 0 soft, bit 1 hard. */
void orc_tree_forces(const orc_tree *t, int64_t nsel, const int64_t *sel, int32_t mode, double *as,
                     double *ah, double *scale_s, double *scale_h)
{
    const orc_params *p = &t->p;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < nsel; ++k) {
        int64_t g = sel[k], c0 = t->gnode[g];
        ivec cells = {0}, parts = {0}, hparts = {0};
        walk_group(t, g, mode & 1, (mode >> 1) & 1, &cells, &parts, &hparts);
        for (int64_t i = t->first[c0]; i < t->first[c0] + t->count[c0]; ++i) {
            double xi[3] = {t->x[i], t->y[i], t->z[i]};
            if (mode & 1) {
                double acc[3] = {0, 0, 0}, sc = 0.0;
                for (int64_t e = 0; e < cells.n; ++e) {
                    int64_t c = cells.v[e];
                    pair_acc(xi, t->cx[c], t->cy[c], t->cz[c], t->M[c], p->G, p->eps, 1.0, acc, &sc);
                }
                for (int64_t e = 0; e < parts.n; ++e) {
                    int64_t j = parts.v[e];
                    if (j == i) continue;
                    double d0 = t->x[j] - xi[0], d1 = t->y[j] - xi[1], d2 = t->z[j] - xi[2];
                    double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
                    double w = 1.0 - orc_cutoff_K(r, p->R1, p->R2);
                    pair_acc(xi, t->x[j], t->y[j], t->z[j], t->m[j], p->G, p->eps, w, acc, &sc);
                }
                as[3 * i + 0] = acc[0];
                as[3 * i + 1] = acc[1];
                as[3 * i + 2] = acc[2];
                if (scale_s) scale_s[i] = sc;
            }
            if (mode & 2) {
                double acc[3] = {0, 0, 0}, sc = 0.0;
                for (int64_t e = 0; e < hparts.n; ++e) {
                    int64_t j = hparts.v[e];
                    if (j == i) continue;
                    double d0 = t->x[j] - xi[0], d1 = t->y[j] - xi[1], d2 = t->z[j] - xi[2];
                    double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
                    double w = orc_cutoff_K(r, p->R1, p->R2);
                    pair_acc(xi, t->x[j], t->y[j], t->z[j], t->m[j], p->G, p->eps, w, acc, &sc);
                }
                ah[3 * i + 0] = acc[0];
                ah[3 * i + 1] = acc[1];
                ah[3 * i + 2] = acc[2];
                if (scale_h) scale_h[i] = sc;
            }
        }
        free(cells.v);
        free(parts.v);
        free(hparts.v);
    }
}

/* Interactions the same-tree force evaluates, as sink-source pairs of the
 * lists: soft = |group| * (cells + particles), hard = |group| * hard, summed
 * over groups. A sink's pair with itself is counted (it adds 0 to the force). */
void orc_interactions(const orc_tree *t, int32_t mode, int64_t *soft, int64_t *hard)
{
    int64_t s = 0, h = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : s, h)
    for (int64_t g = 0; g < t->ng; ++g) {
        ivec cells = {0, 0, -1}, parts = {0, 0, -1}, hparts = {0, 0, -1};
        walk_group(t, g, mode & 1, (mode >> 1) & 1, &cells, &parts, &hparts);
        int64_t cnt = t->count[t->gnode[g]];
        s += cnt * (cells.n + parts.n);
        h += cnt * hparts.n;
    }
    *soft = s;
    *hard = h;
}

/* ------------------------------------------------------------------------ */
/* Hybrid integration (Sec. II-C, Eq. 3-4).                                   */
/* ------------------------------------------------------------------------ */

/* Forces at the current positions. The particle arrays are first re-ordered
 * into key order (the tree build of Sec. III-A1 sorts the particle data), so
 * the state stays sorted from one evaluation to the next; perm (optional,
 * length n) is composed with the sort so that it keeps the original ids.
 * mode bit 0 soft, bit 1 hard; as/ah are 3n arrays in the new order. */
static void forces_resort(int64_t n, double *st[7], int64_t *ids, const orc_params *p, int32_t mode, double *as,
                          double *ah)
{
    orc_tree *t = orc_tree_new(n, st[0], st[1], st[2], st[6], p);
    double *tmp = xmalloc((size_t)n * sizeof(double));
    for (int f = 0; f < 7; ++f) {
        for (int64_t k = 0; k < n; ++k) tmp[k] = st[f][t->perm[k]];
        memcpy(st[f], tmp, (size_t)n * sizeof(double));
    }
    free(tmp);
    if (ids) {
        int64_t *itmp = xmalloc((size_t)n * sizeof(int64_t));
        for (int64_t k = 0; k < n; ++k) itmp[k] = ids[t->perm[k]];
        memcpy(ids, itmp, (size_t)n * sizeof(int64_t));
        free(itmp);
    }
    int64_t *sel = xmalloc((size_t)(t->ng ? t->ng : 1) * sizeof(int64_t));
    for (int64_t g = 0; g < t->ng; ++g) sel[g] = g;
    orc_tree_forces(t, t->ng, sel, mode, as, ah, NULL, NULL);
    free(sel);
    orc_tree_free(t);
}

/* Public form of the force evaluation: re-sorts the state in place. */
void orc_forces(int64_t n, double *x, double *y, double *z, double *vx, double *vy, double *vz, double *m,
                int64_t *ids, const orc_params *p, int32_t mode, double *as, double *ah)
{
    double *st[7] = {x, y, z, vx, vy, vz, m};
    forces_resort(n, st, ids, p, mode, as, ah);
}

/* v <- v + h a, one rounding for the product and one for the sum. */
static void kick(int64_t n, double *vx, double *vy, double *vz, const double *a, double h)
{
    for (int64_t i = 0; i < n; ++i) {
        vx[i] = vx[i] + h * a[3 * i + 0];
        vy[i] = vy[i] + h * a[3 * i + 1];
        vz[i] = vz[i] + h * a[3 * i + 2];
    }
}

/* Eq. (4): x <- x + dt v. */
static void drift(int64_t n, double *x, double *y, double *z, const double *vx, const double *vy,
                  const double *vz, double dt)
{
    for (int64_t i = 0; i < n; ++i) {
        x[i] = x[i] + dt * vx[i];
        y[i] = y[i] + dt * vy[i];
        z[i] = z[i] + dt * vz[i];
    }
}

/* Sec. II-C two time-step levels, dt_s = n dt_h. Reading of the (missing)
 * Fig. 1: split-operator kick-drift-kick,
 *   K_s(dt_s/2); n x [K_h(dt_h/2); D(dt_h); rebuild, hard force (and at the
 *   last sub-step also the soft force); K_h(dt_h/2)]; K_s(dt_s/2),
 * i.e. one soft-step and n - 1 hard-steps per dt_s. as/ah (3n) must hold the
 * forces at the current positions unless valid == 0, in which case they are
 * computed first. nsteps soft steps are taken. */
void orc_hybrid_steps(int64_t n, double *x, double *y, double *z, double *vx, double *vy, double *vz, double *m,
                      int64_t *ids, double *as, double *ah, const orc_params *p, int32_t nsteps, int32_t valid)
{
    double *st[7] = {x, y, z, vx, vy, vz, m};
    int nh = p->n_hard;
    double dts = p->dt_soft, dth = p->dt_soft / (double)nh;
    if (!valid) forces_resort(n, st, ids, p, 3, as, ah);
    for (int32_t s = 0; s < nsteps; ++s) {
        kick(n, vx, vy, vz, as, 0.5 * dts);
        for (int k = 1; k <= nh; ++k) {
            kick(n, vx, vy, vz, ah, 0.5 * dth);
            drift(n, x, y, z, vx, vy, vz, dth);
            forces_resort(n, st, ids, p, (k == nh) ? 3 : 2, as, ah);
            kick(n, vx, vy, vz, ah, 0.5 * dth);
        }
        kick(n, vx, vy, vz, as, 0.5 * dts);
    }
}
