/*
 * kitc_oracle.c -- plain, slow, FP64 CPU oracle for the kernel-independent
 * treecode (KITC) of Wang, Krasny & Tlupova, "A kernel-independent treecode
 * based on barycentric Lagrange interpolation" (arXiv 1902.02250).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table
 * or constant generator with the CUDA library under paper_1902_02250_gb300/;
 * neither side includes or links the other.
 *
 * Every function follows the passage of the paper it names.  Nothing is
 * blocked, fused or reordered beyond what the definition states.  Compile
 * with -O2 -ffp-contract=off so that no multiply-add is contracted: the
 * tree-split and MAC predicates below must take the same IEEE decisions as
 * any other implementation that writes the same expressions.
 *
 * Readings of points the paper leaves open:
 *   - leaf rule: a cluster is a leaf iff it holds <= N0 particles (Sec. 6,
 *     "maximum leaf size N0" of Algorithm 2);
 *   - l_max is the longest side of the cluster being split (Sec. 6 says
 *     "of the root"; the rule is applied to every child "in the same way");
 *   - child boxes are the geometric halves of the parent box; the root box
 *     is the smallest box enclosing the particles (Sec. 6);
 *   - a particle on the midpoint goes to the upper half (x >= mid);
 *   - children are ordered by octant code (bit 0 = x upper, bit 1 = y upper,
 *     bit 2 = z upper); the partition is stable; clusters are numbered in
 *     breadth-first order, the children of a cluster being contiguous;
 *   - cluster centre = box midpoint, cluster radius r = half the diagonal;
 *   - MAC (Eq. MAC): the interaction is well separated iff r <= theta * R;
 *   - target batches (not in the paper) take one decision per batch, either
 *     by the box rule r <= theta * dist(box_B, y_c) or by the all-targets
 *     rule (every target of the batch passes Eq. MAC); both are additions;
 *   - the coincident-point tolerance is DBL_MIN, as Sec. 3 states;
 *   - the modified weights are the definition of Eq. modified_weights with
 *     each L_k in barycentric form (Eq. Barycentric-1D), i.e. Algorithm 1
 *     with the division by denom = sum1*sum2*sum3 done per axis;
 *   - the MRS kernels are regular at r = 0, so the self term i = j is kept
 *     (Sec. 1: only a singular kernel omits it);
 *   - the angular-velocity term printed as 1/4 [n.(x-y)] D2 is read as
 *     1/4 [n.(x-y)](x-y) D2 (Eq. AngularVelocity; the printed term is a
 *     scalar added to vectors).
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* kernel identifiers (Sec. 7) */
enum {
    OR_STOKESLET = 0,          /* Eq. Velocity_1: weight f (3) -> u (3)            */
    OR_ROTLET = 1,             /* rotlet part of Eq. MRS_2: torque n (3) -> (u,w)   */
    OR_STOKESLET_ROTLET = 2,   /* Eq. MRS_2: (f,n) (6) -> (u,w) (6)                */
    OR_TEST_POLY = 99          /* test kernel, degree 3 in each y_l: f (3) -> u (3) */
};

int or_kernel_win(int kernel)
{
    return kernel == OR_STOKESLET_ROTLET ? 6 : 3;
}

int or_kernel_wout(int kernel)
{
    return (kernel == OR_ROTLET || kernel == OR_STOKESLET_ROTLET) ? 6 : 3;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Sec. 3: Chebyshev points of the 2nd kind and the simple barycentric       */
/* weights.                                                                  */
/* ------------------------------------------------------------------------ */

/* Eq. Chebyshev_points, s_k = cos(k pi / n), mapped to [a,b] by
 * t -> (a + b + t (b - a)) / 2 (Sec. 3, interval map). */
void or_cheb_points(int n, double a, double b, double *s)
{
    for (int k = 0; k <= n; ++k) {
        double t = cos((double)k * OR_PI / (double)n);
        s[k] = 0.5 * ((a + b) + t * (b - a));
    }
}

/* Eq. barycentric_weights: w_k = (-1)^k delta_k, delta_0 = delta_n = 1/2. */
void or_bary_weights(int n, double *w)
{
    for (int k = 0; k <= n; ++k) {
        double delta = (k == 0 || k == n) ? 0.5 : 1.0;
        w[k] = (k % 2 == 0) ? delta : -delta;
    }
}

/* Eq. Barycentric-1D: L_k(t) = (w_k/(t-s_k)) / sum_m w_m/(t-s_m), with the
 * removable singularity resolved as Sec. 3/Sec. 5 state: if |t - s_j| <=
 * DBL_MIN for some j, L_k(t) = delta_jk (the last such j wins, as in
 * Algorithm 1 where a later k overwrites the flag). */
void or_bary_basis(int n, const double *s, const double *w, double t, double *L)
{
    int flag = -1;
    double sum = 0.0;
    for (int k = 0; k <= n; ++k) {
        double diff = t - s[k];
        if (fabs(diff) <= DBL_MIN) {
            flag = k;
            L[k] = 0.0;
        } else {
            L[k] = w[k] / diff;
            sum += L[k];
        }
    }
    if (flag > -1) {
        for (int k = 0; k <= n; ++k) L[k] = 0.0;
        L[flag] = 1.0;
        return;
    }
    for (int k = 0; k <= n; ++k) L[k] = L[k] / sum;
}

/* ------------------------------------------------------------------------ */
/* Sec. 7: regularized Stokes kernels.                                       */
/* ------------------------------------------------------------------------ */

/* Eq. MRS_kernels: H1, H2, Q, D1, D2 as functions of r^2 and eps. */
void or_mrs_functions(double r2, double eps, double *H)
{
    double e2 = eps * eps;
    double rho2 = r2 + e2;
    double rho = sqrt(rho2);
    double rho3 = rho2 * rho;
    double rho5 = rho3 * rho2;
    double rho7 = rho5 * rho2;
    double c = 8.0 * OR_PI;
    H[0] = (2.0 * e2 + r2) / (c * rho3);                         /* H1 */
    H[1] = 1.0 / (c * rho3);                                     /* H2 */
    H[2] = (5.0 * e2 + 2.0 * r2) / (c * rho5);                   /* Q  */
    H[3] = (10.0 * e2 * e2 - 7.0 * e2 * r2 - 2.0 * r2 * r2) / (c * rho7); /* D1 */
    H[4] = (21.0 * e2 + 6.0 * r2) / (c * rho7);                  /* D2 */
}

static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* u += k(x, y) f for one target x and one source y (the summand of
 * Eq. N-body).  f has or_kernel_win(kernel) components, u has
 * or_kernel_wout(kernel).  d = x - y as in Eqs. Velocity_1 and MRS_2. */
void or_kernel_apply(int kernel, double eps, const double *x, const double *y,
                     const double *f, double *u)
{
    double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
    if (kernel == OR_TEST_POLY) {
        /* k(x,y) = prod_l (1 + x_l y_l / 2)^3: a polynomial of degree 3 in
         * each y_l, reproduced exactly by interpolation of degree n >= 3. */
        double p = 1.0;
        for (int l = 0; l < 3; ++l) {
            double q = 1.0 + 0.5 * x[l] * y[l];
            p = p * (q * q * q);
        }
        for (int c = 0; c < 3; ++c) u[c] += p * f[c];
        return;
    }
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 + eps * eps == 0.0) return; /* eps = 0, x = y: singular, omitted (Sec. 1) */
    double H[5];
    or_mrs_functions(r2, eps, H);
    if (kernel == OR_STOKESLET || kernel == OR_STOKESLET_ROTLET) {
        /* Eq. Velocity_1: f H1 + (f.d) d H2 */
        double fd = f[0] * d[0] + f[1] * d[1] + f[2] * d[2];
        for (int c = 0; c < 3; ++c) u[c] += f[c] * H[0] + fd * d[c] * H[1];
    }
    if (kernel == OR_STOKESLET_ROTLET) {
        /* Eq. AngularVelocity, Stokeslet part: 1/2 (f x d) Q */
        double fxd[3];
        cross3(f, d, fxd);
        for (int c = 0; c < 3; ++c) u[3 + c] += 0.5 * fxd[c] * H[2];
    }
    if (kernel == OR_ROTLET || kernel == OR_STOKESLET_ROTLET) {
        const double *n = (kernel == OR_ROTLET) ? f : f + 3;
        double nxd[3];
        cross3(n, d, nxd);
        double nd = n[0] * d[0] + n[1] * d[1] + n[2] * d[2];
        for (int c = 0; c < 3; ++c) {
            u[c] += 0.5 * nxd[c] * H[2];                         /* Eq. Velocity_2 */
            u[3 + c] += 0.25 * n[c] * H[3] + 0.25 * nd * d[c] * H[4]; /* Eq. AngularVelocity */
        }
    }
}

/* Eq. N-body by direct summation, all j including j = i (the MRS kernels
 * are regular).  tgt: nt x 3, src: ns x 3, w: ns x win, out: nt x wout,
 * all row-major, user order.  out is overwritten. */
void or_direct(int kernel, double eps, const double *tgt, int64_t nt,
               const double *src, const double *w, int64_t ns, double *out)
{
    int win = or_kernel_win(kernel), wout = or_kernel_wout(kernel);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nt; ++i) {
        double u[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t j = 0; j < ns; ++j)
            or_kernel_apply(kernel, eps, tgt + 3 * i, src + 3 * j, w + win * j, u);
        for (int c = 0; c < wout; ++c) out[wout * i + c] = u[c];
    }
}

/* Eq. error: E = (sum_i |ud_i - ut_i|^2 / sum_i |ud_i|^2)^(1/2); rows of m
 * components are concatenated vectors (Sec. 8: u and w together). */
double or_rel_l2(const double *ud, const double *ut, int64_t rows, int m)
{
    double num = 0.0, den = 0.0;
    for (int64_t i = 0; i < rows * (int64_t)m; ++i) {
        double e = ud[i] - ut[i];
        num += e * e;
        den += ud[i] * ud[i];
    }
    return den > 0.0 ? sqrt(num / den) : sqrt(num);
}

/* ------------------------------------------------------------------------ */
/* Sec. 6: tree of particle clusters.                                        */
/* ------------------------------------------------------------------------ */

/* Depth at which splitting stops even above N0; only degenerate inputs
 * (e.g. more than N0 copies of one point) reach it. */
#define OR_MAX_LEVEL 40

typedef struct {
    int64_t n;            /* particles                                        */
    int leaf_size;        /* N0                                               */
    int64_t nclus, cap;   /* clusters in use / allocated                      */
    int64_t *perm;        /* perm[p] = user index of the particle at slot p   */
    double *lo, *hi;      /* box corners, [cluster][3]                        */
    int64_t *begin, *end; /* particle slots [begin, end) of each cluster      */
    int32_t *first_child, *n_child, *level, *parent;
} or_tree;

static void tree_grow(or_tree *t)
{
    if (t->nclus < t->cap) return;
    t->cap = t->cap ? 2 * t->cap : 64;
    t->lo = realloc(t->lo, sizeof(double) * 3 * t->cap);
    t->hi = realloc(t->hi, sizeof(double) * 3 * t->cap);
    t->begin = realloc(t->begin, sizeof(int64_t) * t->cap);
    t->end = realloc(t->end, sizeof(int64_t) * t->cap);
    t->first_child = realloc(t->first_child, sizeof(int32_t) * t->cap);
    t->n_child = realloc(t->n_child, sizeof(int32_t) * t->cap);
    t->level = realloc(t->level, sizeof(int32_t) * t->cap);
    t->parent = realloc(t->parent, sizeof(int32_t) * t->cap);
}

static int64_t tree_push(or_tree *t, const double *lo, const double *hi,
                         int64_t b, int64_t e, int level, int parent)
{
    tree_grow(t);
    int64_t c = t->nclus++;
    for (int l = 0; l < 3; ++l) {
        t->lo[3 * c + l] = lo[l];
        t->hi[3 * c + l] = hi[l];
    }
    t->begin[c] = b;
    t->end[c] = e;
    t->first_child[c] = -1;
    t->n_child[c] = 0;
    t->level[c] = level;
    t->parent[c] = parent;
    return c;
}

/* Sec. 6 tree build.  The root is the smallest box enclosing the particles.
 * A cluster with more than N0 particles is bisected at the midpoint of every
 * side longer than l_max / sqrt(2), giving 8, 4 or 2 sub-boxes; the non-empty
 * ones become its children.  x: n x 3 row-major. */
or_tree *or_tree_build(const double *x, int64_t n, int leaf_size)
{
    or_tree *t = calloc(1, sizeof(or_tree));
    t->n = n;
    t->leaf_size = leaf_size;
    t->perm = malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) t->perm[i] = i;
    if (n <= 0) return t;
    double lo[3], hi[3];
    for (int l = 0; l < 3; ++l) lo[l] = hi[l] = x[l];
    for (int64_t i = 1; i < n; ++i)
        for (int l = 0; l < 3; ++l) {
            if (x[3 * i + l] < lo[l]) lo[l] = x[3 * i + l];
            if (x[3 * i + l] > hi[l]) hi[l] = x[3 * i + l];
        }
    tree_push(t, lo, hi, 0, n, 0, -1);
    int64_t *tmp = malloc(sizeof(int64_t) * n);
    int *code = malloc(sizeof(int) * n);
    for (int64_t c = 0; c < t->nclus; ++c) {  /* breadth-first: nclus grows */
        int64_t b = t->begin[c], e = t->end[c];
        if (e - b <= leaf_size || t->level[c] >= OR_MAX_LEVEL) continue;
        double side[3], lmax = 0.0;
        for (int l = 0; l < 3; ++l) {
            side[l] = t->hi[3 * c + l] - t->lo[3 * c + l];
            if (side[l] > lmax) lmax = side[l];
        }
        if (!(lmax > 0.0)) continue;
        double thr = lmax / sqrt(2.0);
        int split[3];
        double mid[3];
        for (int l = 0; l < 3; ++l) {
            split[l] = side[l] > thr;
            mid[l] = 0.5 * (t->lo[3 * c + l] + t->hi[3 * c + l]);
        }
        int64_t count[8] = {0};
        for (int64_t p = b; p < e; ++p) {
            const double *xp = x + 3 * t->perm[p];
            int k = 0;
            for (int l = 0; l < 3; ++l)
                if (split[l] && xp[l] >= mid[l]) k |= 1 << l;
            code[p] = k;
            count[k]++;
        }
        int64_t start[8], s = b;
        for (int k = 0; k < 8; ++k) {
            start[k] = s;
            s += count[k];
        }
        int64_t pos[8];
        memcpy(pos, start, sizeof(pos));
        for (int64_t p = b; p < e; ++p) tmp[pos[code[p]]++] = t->perm[p];
        memcpy(t->perm + b, tmp + b, sizeof(int64_t) * (e - b));
        int first = -1, nch = 0;
        for (int k = 0; k < 8; ++k) {
            if (count[k] == 0) continue;
            double clo[3], chi[3];
            for (int l = 0; l < 3; ++l) {
                clo[l] = t->lo[3 * c + l];
                chi[l] = t->hi[3 * c + l];
                if (split[l]) {
                    if ((k >> l) & 1) clo[l] = mid[l];
                    else chi[l] = mid[l];
                }
            }
            int64_t ch = tree_push(t, clo, chi, start[k], start[k] + count[k],
                                   t->level[c] + 1, (int)c);
            if (first < 0) first = (int)ch;
            nch++;
        }
        t->first_child[c] = first;
        t->n_child[c] = nch;
    }
    free(tmp);
    free(code);
    return t;
}

void or_tree_free(or_tree *t)
{
    if (!t) return;
    free(t->perm);
    free(t->lo);
    free(t->hi);
    free(t->begin);
    free(t->end);
    free(t->first_child);
    free(t->n_child);
    free(t->level);
    free(t->parent);
    free(t);
}

int64_t or_tree_nclusters(const or_tree *t) { return t->nclus; }

/* Copies the tree out; any pointer may be NULL. */
void or_tree_get(const or_tree *t, int64_t *perm, double *lo, double *hi,
                 int64_t *begin, int64_t *end, int32_t *first_child,
                 int32_t *n_child, int32_t *level, int32_t *parent)
{
    int64_t m = t->nclus;
    if (perm) memcpy(perm, t->perm, sizeof(int64_t) * t->n);
    if (lo) memcpy(lo, t->lo, sizeof(double) * 3 * m);
    if (hi) memcpy(hi, t->hi, sizeof(double) * 3 * m);
    if (begin) memcpy(begin, t->begin, sizeof(int64_t) * m);
    if (end) memcpy(end, t->end, sizeof(int64_t) * m);
    if (first_child) memcpy(first_child, t->first_child, sizeof(int32_t) * m);
    if (n_child) memcpy(n_child, t->n_child, sizeof(int32_t) * m);
    if (level) memcpy(level, t->level, sizeof(int32_t) * m);
    if (parent) memcpy(parent, t->parent, sizeof(int32_t) * m);
}

/* Fig. 1: cluster centre y_c (box midpoint) and radius r (half diagonal). */
static void cluster_geometry(const or_tree *t, int64_t c, double *yc, double *r)
{
    double d[3];
    for (int l = 0; l < 3; ++l) {
        yc[l] = 0.5 * (t->lo[3 * c + l] + t->hi[3 * c + l]);
        d[l] = t->hi[3 * c + l] - t->lo[3 * c + l];
    }
    *r = 0.5 * sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
}

/* ------------------------------------------------------------------------ */
/* Sec. 4-5: Chebyshev grid of a cluster and its modified weights.           */
/* ------------------------------------------------------------------------ */

/* The (n+1) mapped Chebyshev points of each axis of cluster c:
 * s[l*(n+1)+k] = s_k on [lo_l, hi_l] (Sec. 3 interval map, Fig. 1b). */
void or_cluster_points(const or_tree *t, int64_t c, int n, double *s)
{
    for (int l = 0; l < 3; ++l)
        or_cheb_points(n, t->lo[3 * c + l], t->hi[3 * c + l], s + l * (n + 1));
}

/* Eq. modified_weights for every cluster: fhat[c][k1][k2][k3][comp] =
 * sum_{y_j in c} L_k1(y_j1) L_k2(y_j2) L_k3(y_j3) f_j[comp], each L in the
 * barycentric form of Eq. Barycentric-1D with the coincident-point rule.
 * x: n x 3 and w: n x win in user order. */
void or_modified_weights(const or_tree *t, const double *x, const double *w,
                         int win, int n, double *fhat)
{
    int np = n + 1;
    int64_t P = (int64_t)np * np * np;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < t->nclus; ++c) {
        double s[3 * 17], wk[17], L[3][17];
        or_cluster_points(t, c, n, s);
        or_bary_weights(n, wk);
        double *fh = fhat + c * P * win;
        for (int64_t q = 0; q < P * win; ++q) fh[q] = 0.0;
        for (int64_t p = t->begin[c]; p < t->end[c]; ++p) {
            int64_t j = t->perm[p];
            for (int l = 0; l < 3; ++l) or_bary_basis(n, s + l * np, wk, x[3 * j + l], L[l]);
            for (int k1 = 0; k1 < np; ++k1)
                for (int k2 = 0; k2 < np; ++k2)
                    for (int k3 = 0; k3 < np; ++k3) {
                        double prod = L[0][k1] * L[1][k2] * L[2][k3];
                        double *o = fh + ((int64_t)(k1 * np + k2) * np + k3) * win;
                        for (int q = 0; q < win; ++q) o[q] += prod * w[win * j + q];
                    }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 6, Algorithm 2: the treecode.                                        */
/* ------------------------------------------------------------------------ */

#define OR_SMAX (3 * 17)  /* grid coordinates stored per cluster (n <= 16) */

typedef struct {
    const or_tree *t;
    const double *x, *w;   /* sources and weights, user order                    */
    const double *fhat;    /* modified weights, [cluster][P][win]                */
    const double *s;       /* mapped Chebyshev points, [cluster][3][n_c+1]       */
    int n, kernel, win, wout;
    double eps, theta;
    const int32_t *deg;    /* per-cluster degree n_c, or NULL for n everywhere   */
    const int64_t *foff;   /* with deg: offset (doubles) of each cluster's fhat */
    int64_t bad;           /* accepted clusters without weights (deg 0)          */
} tc_ctx;

static int cluster_degree(const tc_ctx *q, int64_t c)
{
    return q->deg ? q->deg[c] : q->n;
}

static void tc_points(tc_ctx *q, double **s_out)
{
    double *s = malloc(sizeof(double) * OR_SMAX * (q->t->nclus > 0 ? q->t->nclus : 1));
    for (int64_t c = 0; c < q->t->nclus; ++c) {
        int n = cluster_degree(q, c);
        if (n > 0) or_cluster_points(q->t, c, n, s + OR_SMAX * c);
    }
    *s_out = s;
}

/* Eq. pc_approximation_3D: u += sum_k k(x, s_k) fhat_k over the (n_c+1)^3
 * grid points of cluster c. */
static void far_field(const tc_ctx *q, int64_t c, const double *x, double *u)
{
    int np = cluster_degree(q, c) + 1;
    int64_t P = (int64_t)np * np * np;
    const double *s = q->s + OR_SMAX * c;
    const double *fh = q->fhat + (q->foff ? q->foff[c] : c * P * q->win);
    for (int k1 = 0; k1 < np; ++k1)
        for (int k2 = 0; k2 < np; ++k2)
            for (int k3 = 0; k3 < np; ++k3) {
                double sk[3] = {s[k1], s[np + k2], s[2 * np + k3]};
                or_kernel_apply(q->kernel, q->eps, x, sk,
                                fh + ((int64_t)(k1 * np + k2) * np + k3) * q->win, u);
            }
}

/* Eq. pc_interaction_3D: u += sum_{y_j in c} k(x, y_j) f_j. */
static void near_field(const tc_ctx *q, int64_t c, const double *x, double *u)
{
    for (int64_t p = q->t->begin[c]; p < q->t->end[c]; ++p) {
        int64_t j = q->t->perm[p];
        or_kernel_apply(q->kernel, q->eps, x, q->x + 3 * j, q->w + q->win * j, u);
    }
}

/* Algorithm 2, subroutine compute_velocity(x, C).  cnt[0] += near pairs,
 * cnt[1] += far grid points, cnt[2] += accepted clusters, cnt[3] += leaves
 * summed directly, cnt[4] += sources inside accepted clusters (so that
 * cnt[0] + cnt[4] counts every source once per target). */
static void compute_velocity(tc_ctx *q, const double *x, int64_t c, double *u,
                             int64_t *cnt)
{
    double yc[3], r;
    cluster_geometry(q->t, c, yc, &r);
    double d0 = x[0] - yc[0], d1 = x[1] - yc[1], d2 = x[2] - yc[2];
    double R = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    if (r <= q->theta * R) {                         /* Eq. MAC */
        int np = cluster_degree(q, c) + 1;
        if (np < 2) {  /* caller error: no modified weights for an accepted cluster */
#pragma omp atomic
            q->bad++;
            return;
        }
        far_field(q, c, x, u);
        cnt[1] += (int64_t)np * np * np;
        cnt[2] += 1;
        cnt[4] += q->t->end[c] - q->t->begin[c];
    } else if (q->t->n_child[c] == 0) {
        near_field(q, c, x, u);
        cnt[0] += q->t->end[c] - q->t->begin[c];
        cnt[3] += 1;
    } else {
        for (int k = 0; k < q->t->n_child[c]; ++k)
            compute_velocity(q, x, q->t->first_child[c] + k, u, cnt);
    }
}

/* Algorithm 2, program main after the tree and the modified weights exist:
 * for each target x_i, compute_velocity(x_i, root).  tgt: nt x 3, out:
 * nt x wout (user order, overwritten).  counts (may be NULL): five totals as
 * in compute_velocity. */
static int64_t treecode_impl(const or_tree *t, const double *x, const double *w,
                             const double *fhat, int n, const int32_t *deg, const int64_t *foff,
                             int kernel, double eps, double theta, const double *tgt, int64_t nt,
                             double *out, int64_t *counts)
{
    tc_ctx q = {t, x, w, fhat, NULL, n, kernel, or_kernel_win(kernel),
                or_kernel_wout(kernel), eps, theta, deg, foff, 0};
    double *s;
    tc_points(&q, &s);
    q.s = s;
    int64_t tot[5] = {0, 0, 0, 0, 0};
#pragma omp parallel
    {
        int64_t loc[5] = {0, 0, 0, 0, 0};
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < nt; ++i) {
            double u[6] = {0, 0, 0, 0, 0, 0};
            if (t->nclus > 0) compute_velocity(&q, tgt + 3 * i, 0, u, loc);
            for (int c = 0; c < q.wout; ++c) out[q.wout * i + c] = u[c];
        }
#pragma omp critical
        for (int k = 0; k < 5; ++k) tot[k] += loc[k];
    }
    if (counts)
        for (int k = 0; k < 5; ++k) counts[k] = tot[k];
    free(s);
    return q.bad;
}

void or_treecode(const or_tree *t, const double *x, const double *w, const double *fhat,
                 int n, int kernel, double eps, double theta,
                 const double *tgt, int64_t nt, double *out, int64_t *counts)
{
    treecode_impl(t, x, w, fhat, n, NULL, NULL, kernel, eps, theta, tgt, nt, out, counts);
}

/* Algorithm 2 with a degree n_c per cluster (deg[c]; the weights of cluster c
 * start at fhat + foff[c]).  Returns the number of (target, cluster) far
 * interactions that met a cluster with deg 0, which must be 0. */
int64_t or_treecode_var(const or_tree *t, const double *x, const double *w, const double *fhat,
                        const int32_t *deg, const int64_t *foff, int kernel, double eps,
                        double theta, const double *tgt, int64_t nt, double *out, int64_t *counts)
{
    return treecode_impl(t, x, w, fhat, 0, deg, foff, kernel, eps, theta, tgt, nt, out, counts);
}

/* ------------------------------------------------------------------------ */
/* Target-batch variant (not in the paper; kept here so that the batch form  */
/* of the traversal has a plain counterpart).  Targets are ordered by the    */
/* Sec. 6 tree built on the targets with leaf size tgt_leaf; batch b holds   */
/* the targets at slots [b*B, (b+1)*B) of that order.  Cluster c is accepted */
/* for the whole batch iff r_c <= theta * dist(box_b, y_c), where box_b is   */
/* the smallest box enclosing the batch's targets and dist is the distance   */
/* from y_c to that box.  Since dist <= |x - y_c| for every target x of the  */
/* batch, a batch-accepted cluster also passes Eq. MAC for every target.     */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t *far, *near;
    int64_t nfar, nnear, capfar, capnear;
} blist;

static void blist_push(int64_t **a, int64_t *m, int64_t *cap, int64_t v)
{
    if (*m == *cap) {
        *cap = *cap ? 2 * *cap : 64;
        *a = realloc(*a, sizeof(int64_t) * *cap);
    }
    (*a)[(*m)++] = v;
}

/* bt == NULL: the box rule, C accepted iff r <= theta * dist(box_B, y_c).
 * bt != NULL (bn targets, 3 coordinates each): the all-targets rule, C accepted
 * iff every target of the batch accepts it by Eq. MAC (the test of
 * compute_velocity); otherwise every target descends. */
static void batch_lists(const tc_ctx *q, const double *blo, const double *bhi, const double *bt,
                        int64_t bn, int64_t c, blist *L)
{
    double yc[3], r, e[3];
    cluster_geometry(q->t, c, yc, &r);
    int accept;
    if (bt) {
        accept = 1;
        for (int64_t i = 0; i < bn && accept; ++i) {
            double d0 = bt[3 * i] - yc[0], d1 = bt[3 * i + 1] - yc[1], d2 = bt[3 * i + 2] - yc[2];
            double R = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
            accept = r <= q->theta * R;
        }
    } else {
        for (int l = 0; l < 3; ++l) {
            if (yc[l] < blo[l]) e[l] = blo[l] - yc[l];
            else if (yc[l] > bhi[l]) e[l] = yc[l] - bhi[l];
            else e[l] = 0.0;
        }
        double dist = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
        accept = r <= q->theta * dist;
    }
    if (accept) {
        blist_push(&L->far, &L->nfar, &L->capfar, c);
    } else if (q->t->n_child[c] == 0) {
        blist_push(&L->near, &L->nnear, &L->capnear, c);
    } else {
        for (int k = 0; k < q->t->n_child[c]; ++k)
            batch_lists(q, blo, bhi, bt, bn, q->t->first_child[c] + k, L);
    }
}

int64_t or_num_batches(int64_t nt, int batch)
{
    return (nt + batch - 1) / batch;
}

/* Batch-MAC treecode.  Outputs (each may be NULL):
 *   out        nt x wout, user order (skipped when lists_only != 0); when sel
 *              is not NULL only the targets i with sel[i] != 0 are summed
 *              and the other rows are set to zero;
 *   counts[5]  as in or_treecode;
 *   tperm      nt, the target order (tperm[slot] = user index);
 *   nfar, nnear  per batch list lengths;
 *   far_list, near_list  concatenated per-batch lists in traversal order,
 *              written only when their capacity (far_cap, near_cap) holds
 *              the totals. */
static void treecode_batch_impl(const or_tree *t, const double *x, const double *w,
                                const double *fhat, int n, const int32_t *deg,
                                const int64_t *foff, int kernel, double eps, double theta,
                                const double *tgt, int64_t nt, int batch, int tgt_leaf,
                                int lists_only, const unsigned char *sel, double *out,
                                int64_t *counts, int64_t *tperm, int64_t *nfar, int64_t *nnear,
                                int64_t *far_list, int64_t far_cap, int64_t *near_list,
                                int64_t near_cap, int all_targets)
{
    tc_ctx q = {t, x, w, fhat, NULL, n, kernel, or_kernel_win(kernel),
                or_kernel_wout(kernel), eps, theta, deg, foff, 0};
    double *s;
    tc_points(&q, &s);
    q.s = s;
    or_tree *tt = or_tree_build(tgt, nt, tgt_leaf);
    if (tperm) memcpy(tperm, tt->perm, sizeof(int64_t) * nt);
    int64_t nb = or_num_batches(nt, batch);
    blist *lists = calloc(nb > 0 ? nb : 1, sizeof(blist));
    int64_t tot[5] = {0, 0, 0, 0, 0};
#pragma omp parallel
    {
        int64_t loc[5] = {0, 0, 0, 0, 0};
#pragma omp for schedule(dynamic, 4)
        for (int64_t b = 0; b < nb; ++b) {
            int64_t s0 = b * batch, s1 = s0 + batch < nt ? s0 + batch : nt;
            double blo[3], bhi[3];
            for (int l = 0; l < 3; ++l) blo[l] = bhi[l] = tgt[3 * tt->perm[s0] + l];
            for (int64_t p = s0; p < s1; ++p)
                for (int l = 0; l < 3; ++l) {
                    double v = tgt[3 * tt->perm[p] + l];
                    if (v < blo[l]) blo[l] = v;
                    if (v > bhi[l]) bhi[l] = v;
                }
            blist *L = &lists[b];
            double *bt = NULL;
            if (all_targets) {
                bt = malloc(sizeof(double) * 3 * (size_t)(s1 - s0));
                for (int64_t p = s0; p < s1; ++p)
                    for (int l = 0; l < 3; ++l) bt[3 * (p - s0) + l] = tgt[3 * tt->perm[p] + l];
            }
            if (t->nclus > 0) batch_lists(&q, blo, bhi, bt, s1 - s0, 0, L);
            free(bt);
            int64_t npair = 0;
            for (int64_t m = 0; m < L->nnear; ++m)
                npair += t->end[L->near[m]] - t->begin[L->near[m]];
            loc[0] += npair * (s1 - s0);
            int64_t pts = 0;
            for (int64_t m = 0; m < L->nfar; ++m) {
                int npc = cluster_degree(&q, L->far[m]) + 1;
                pts += (int64_t)npc * npc * npc;
            }
            loc[1] += pts * (s1 - s0);
            int64_t nsrc = 0;
            for (int64_t m = 0; m < L->nfar; ++m)
                nsrc += t->end[L->far[m]] - t->begin[L->far[m]];
            loc[2] += L->nfar * (s1 - s0);
            loc[3] += L->nnear * (s1 - s0);
            loc[4] += nsrc * (s1 - s0);
            if (lists_only || !out) continue;
            for (int64_t p = s0; p < s1; ++p) {
                int64_t i = tt->perm[p];
                double u[6] = {0, 0, 0, 0, 0, 0};
                if (sel && !sel[i]) {
                    for (int c = 0; c < q.wout; ++c) out[q.wout * i + c] = 0.0;
                    continue;
                }
                for (int64_t m = 0; m < L->nfar; ++m) far_field(&q, L->far[m], tgt + 3 * i, u);
                for (int64_t m = 0; m < L->nnear; ++m) near_field(&q, L->near[m], tgt + 3 * i, u);
                for (int c = 0; c < q.wout; ++c) out[q.wout * i + c] = u[c];
            }
        }
#pragma omp critical
        for (int k = 0; k < 5; ++k) tot[k] += loc[k];
    }
    if (counts)
        for (int k = 0; k < 5; ++k) counts[k] = tot[k];
    int64_t sf = 0, sn = 0;
    for (int64_t b = 0; b < nb; ++b) {
        if (nfar) nfar[b] = lists[b].nfar;
        if (nnear) nnear[b] = lists[b].nnear;
        sf += lists[b].nfar;
        sn += lists[b].nnear;
    }
    if (far_list && far_cap >= sf && near_list && near_cap >= sn) {
        int64_t of = 0, on = 0;
        for (int64_t b = 0; b < nb; ++b) {
            memcpy(far_list + of, lists[b].far, sizeof(int64_t) * lists[b].nfar);
            memcpy(near_list + on, lists[b].near, sizeof(int64_t) * lists[b].nnear);
            of += lists[b].nfar;
            on += lists[b].nnear;
        }
    }
    for (int64_t b = 0; b < nb; ++b) {
        free(lists[b].far);
        free(lists[b].near);
    }
    free(lists);
    or_tree_free(tt);
    free(s);
}

void or_treecode_batch(const or_tree *t, const double *x, const double *w,
                       const double *fhat, int n, int kernel, double eps, double theta,
                       const double *tgt, int64_t nt, int batch, int tgt_leaf,
                       int lists_only, const unsigned char *sel, double *out,
                       int64_t *counts, int64_t *tperm,
                       int64_t *nfar, int64_t *nnear, int64_t *far_list, int64_t far_cap,
                       int64_t *near_list, int64_t near_cap)
{
    treecode_batch_impl(t, x, w, fhat, n, NULL, NULL, kernel, eps, theta, tgt, nt, batch,
                        tgt_leaf, lists_only, sel, out, counts, tperm, nfar, nnear, far_list,
                        far_cap, near_list, near_cap, 0);
}

/* The same with the all-targets rule: a cluster is accepted for a batch iff
 * every target of the batch accepts it by Eq. MAC (so each accepted
 * interaction is one Algorithm 2 also takes), otherwise all targets descend. */
void or_treecode_batch_all(const or_tree *t, const double *x, const double *w,
                           const double *fhat, int n, int kernel, double eps, double theta,
                           const double *tgt, int64_t nt, int batch, int tgt_leaf,
                           int lists_only, const unsigned char *sel, double *out,
                           int64_t *counts, int64_t *tperm,
                           int64_t *nfar, int64_t *nnear, int64_t *far_list, int64_t far_cap,
                           int64_t *near_list, int64_t near_cap)
{
    treecode_batch_impl(t, x, w, fhat, n, NULL, NULL, kernel, eps, theta, tgt, nt, batch,
                        tgt_leaf, lists_only, sel, out, counts, tperm, nfar, nnear, far_list,
                        far_cap, near_list, near_cap, 1);
}

/* Batch-MAC variant with a degree per cluster (see or_treecode_var). */
void or_treecode_batch_var(const or_tree *t, const double *x, const double *w,
                           const double *fhat, const int32_t *deg, const int64_t *foff, int kernel,
                           double eps, double theta, const double *tgt, int64_t nt, int batch,
                           int tgt_leaf, const unsigned char *sel, double *out, int64_t *counts)
{
    treecode_batch_impl(t, x, w, fhat, 0, deg, foff, kernel, eps, theta, tgt, nt, batch, tgt_leaf,
                        0, sel, out, counts, NULL, NULL, NULL, NULL, 0, NULL, 0, 0);
}

/* Eq. modified_weights with a degree n_c per cluster: cluster c (deg[c] > 0)
 * writes (n_c+1)^3 x win values at fhat + foff[c]; clusters with deg 0 get none. */
void or_modified_weights_var(const or_tree *t, const double *x, const double *w, int win,
                             const int32_t *deg, const int64_t *foff, double *fhat)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < t->nclus; ++c) {
        int n = deg[c];
        if (n <= 0) continue;
        int np = n + 1;
        int64_t P = (int64_t)np * np * np;
        double s[3 * 17], wk[17], L[3][17];
        or_cluster_points(t, c, n, s);
        or_bary_weights(n, wk);
        double *fh = fhat + foff[c];
        for (int64_t q = 0; q < P * win; ++q) fh[q] = 0.0;
        for (int64_t p = t->begin[c]; p < t->end[c]; ++p) {
            int64_t j = t->perm[p];
            for (int l = 0; l < 3; ++l) or_bary_basis(n, s + l * np, wk, x[3 * j + l], L[l]);
            for (int k1 = 0; k1 < np; ++k1)
                for (int k2 = 0; k2 < np; ++k2)
                    for (int k3 = 0; k3 < np; ++k3) {
                        double prod = L[0][k1] * L[1][k2] * L[2][k3];
                        double *o = fh + ((int64_t)(k1 * np + k2) * np + k3) * win;
                        for (int q = 0; q < win; ++q) o[q] += prod * w[win * j + q];
                    }
        }
    }
}
