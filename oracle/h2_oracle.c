/*
 * h2_oracle.c -- plain, slow FP64 CPU oracle for the H^2 matrix-vector product.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the CPU-baseline
 * leg of bench.py may load this library. It shares no code with the CUDA library and
 * the CUDA library never calls it.
 *
 * What it follows (Zampini, Boukaram, Turkiyyah, Knio, Keyes, "H2Opus: a distributed-
 * memory multi-GPU software package for non-local operators", arXiv 2109.05451):
 *   Sec. 2.1        A = A_de + <U, S, V^T>: dense m x m leaves at the finest level plus
 *                   coupling blocks S^l_ts on every level, leaf bases U (m x k) and
 *                   k x k interlevel transfers E; U^{l-1}_i = diag(U^l_c) [E^l_c].
 *   Sec. 3.1, Alg 1 upsweep: xhat^q = V^T x at the leaves, then
 *                   xhat^{l-1}_s = sum over children c of F_c^T xhat^l_c.
 *   Sec. 3.2, Alg 4 tree multiply: yhat^l_t = sum_{s in b_t} S^l_ts xhat^l_s on every level.
 *   Sec. 3.3, Alg 6 downsweep: yhat^l_c += E_c yhat^{l-1}_t, then y = U yhat^q.
 *   Sec. 3         the dense product A_de x is added to the low-rank product.
 *   Sec. 6.1       geometric admissibility eta*|C_t - C_s| >= (D_t + D_s)/2 with C the
 *                   centre and D the diagonal of the cluster bounding box; leaf size m.
 *   Sec. 6.3, 6.4  k-d tree clustering, Chebyshev interpolation on the bounding boxes
 *                   (a p x p grid in 2D gives rank p^2, tri-cubic in 3D gives rank 64),
 *                   dense blocks by evaluating the kernel directly.
 *
 * Readings of the paper where it is silent (the same readings the CUDA library takes,
 * written here independently):
 *   - depth q = smallest q >= 0 with n <= m * 2^q; every node above level q is split,
 *     so all leaves are on level q (the level formulas of Alg 1 and Alg 6 assume this).
 *   - k-d split: tight bounding box of the node's points; split dimension = largest
 *     extent (ties -> lowest dimension); order the points by (coordinate, original
 *     index); left child = first floor(n/2) points. Children of heap node i: 2i, 2i+1.
 *   - admissibility compares same-level clusters only, starting at (root, root), and is
 *     evaluated exactly as eta * sqrt(sum_d (c_t,d - c_s,d)^2) >= 0.5 * (D_t + D_s) with
 *     c = (lo + hi) / 2 and D = sqrt(sum_d (hi_d - lo_d)^2); equality is admissible.
 *     Inadmissible pairs recurse into the children pairs (2t,2s), (2t,2s+1), (2t+1,2s),
 *     (2t+1,2s+1) until the leaf level, where they become dense blocks.
 *   - Chebyshev points of the first kind, xi_j = c + (h/2) cos((2j+1) pi / (2p)); the box
 *     extent h is clamped below at 1e-12 * (root diagonal) for these points only.
 *   - multi-index nu = j_0 + p j_1 + p^2 j_2 (dimension 0 fastest); k = p^dim.
 *   - U = V and E = F (one point set, symmetric kernel).
 *   - S_ts[nu][mu] = kappa(xi^t_nu, xi^s_mu); D_ts[i][j] = kappa(x_i, x_j), r = 0 included.
 *   - sums run in ascending index order.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no fused multiply-add contraction, so
 * that the admissibility test is evaluated exactly as written).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

enum { ORC_EXP = 0, ORC_GAUSS = 1, ORC_IMQ = 2, ORC_POLY = 3 };

typedef struct {
    int kind;
    double a, b;
    int deg;
} orc_kernel;

typedef struct {
    int64_t n;
    int dim, m, p, k, q;
    double eta;
    orc_kernel ker;
    double *pts;          /* n * dim, user order */
    int64_t *perm;        /* tree position -> user index */
    int64_t nnodes;       /* heap nodes 1 .. nnodes = 2^(q+1) - 1 */
    int64_t *lo, *hi;     /* [nnodes + 1]: tree-order index range of each node */
    double *bmin, *bmax;  /* [(nnodes + 1) * dim]: tight bounding box */
    double *xi;           /* [(nnodes + 1) * dim * p]: Chebyshev points per node and dim */
    /* admissible (coupling) blocks in traversal order */
    int64_t ncpl, cap_cpl;
    int *cpl_lvl;
    int64_t *cpl_t, *cpl_s;
    /* inadmissible leaf pairs (dense blocks) in traversal order */
    int64_t ndns, cap_dns;
    int64_t *dns_t, *dns_s;
    /* optional stored entries */
    double *S;            /* ncpl * k * k, or NULL: then computed on the fly */
    double *D;            /* dense entries, block b at D + dns_off[b], or NULL */
    int64_t *dns_off;
} orc_h2;

/* ------------------------------------------------------------------ kernel function */

static double kernel_eval(const orc_kernel *kr, const double *x, const double *y, int dim)
{
    if (kr->kind == ORC_POLY) {
        double v = 1.0;
        for (int d = 0; d < dim; d++) {
            double f = 1.0 + x[d] * y[d];
            for (int e = 0; e < kr->deg; e++) v *= f;
        }
        return v;
    }
    double r2 = 0.0;
    for (int d = 0; d < dim; d++) {
        double dx = x[d] - y[d];
        r2 += dx * dx;
    }
    if (kr->kind == ORC_EXP) return exp(-sqrt(r2) / kr->a);
    if (kr->kind == ORC_GAUSS) return exp(-r2 / kr->a);
    return pow(r2 + kr->a, -kr->b); /* ORC_IMQ */
}

/* ------------------------------------------------------------- cluster tree (k-d) */

static const double *g_sort_pts;
static int g_sort_dim, g_sort_d;

static int cmp_coord_then_index(const void *pa, const void *pb)
{
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    double ca = g_sort_pts[a * g_sort_dim + g_sort_d];
    double cb = g_sort_pts[b * g_sort_dim + g_sort_d];
    if (ca < cb) return -1;
    if (ca > cb) return 1;
    return (a > b) - (a < b);
}

static void build_node(orc_h2 *h, int64_t node, int level, int64_t lo, int64_t hi)
{
    int dim = h->dim;
    h->lo[node] = lo;
    h->hi[node] = hi;
    double *bmin = h->bmin + node * dim, *bmax = h->bmax + node * dim;
    for (int d = 0; d < dim; d++) {
        bmin[d] = h->pts[h->perm[lo] * dim + d];
        bmax[d] = bmin[d];
    }
    for (int64_t i = lo; i < hi; i++)
        for (int d = 0; d < dim; d++) {
            double c = h->pts[h->perm[i] * dim + d];
            if (c < bmin[d]) bmin[d] = c;
            if (c > bmax[d]) bmax[d] = c;
        }
    if (level == h->q) return;
    int split = 0;
    for (int d = 1; d < dim; d++)
        if (bmax[d] - bmin[d] > bmax[split] - bmin[split]) split = d;
    g_sort_pts = h->pts;
    g_sort_dim = dim;
    g_sort_d = split;
    qsort(h->perm + lo, (size_t)(hi - lo), sizeof(int64_t), cmp_coord_then_index);
    int64_t mid = lo + (hi - lo) / 2;
    build_node(h, 2 * node, level + 1, lo, mid);
    build_node(h, 2 * node + 1, level + 1, mid, hi);
}

/* -------------------------------------------------------------- admissibility */

static double box_diag(const double *bmin, const double *bmax, int dim)
{
    double s = 0.0;
    for (int d = 0; d < dim; d++) {
        double e = bmax[d] - bmin[d];
        s += e * e;
    }
    return sqrt(s);
}

/* Sec. 6.1: eta * |C_t - C_s| >= (D_t + D_s) / 2 on the tight bounding boxes. */
int orc_admissible_boxes(const double *tmin, const double *tmax, const double *smin,
                         const double *smax, int dim, double eta)
{
    double s = 0.0;
    for (int d = 0; d < dim; d++) {
        double ct = (tmin[d] + tmax[d]) / 2;
        double cs = (smin[d] + smax[d]) / 2;
        double dc = ct - cs;
        s += dc * dc;
    }
    double lhs = eta * sqrt(s);
    double rhs = 0.5 * (box_diag(tmin, tmax, dim) + box_diag(smin, smax, dim));
    return lhs >= rhs;
}

static void push_cpl(orc_h2 *h, int l, int64_t t, int64_t s)
{
    if (h->ncpl == h->cap_cpl) {
        h->cap_cpl = h->cap_cpl ? 2 * h->cap_cpl : 1024;
        h->cpl_lvl = realloc(h->cpl_lvl, h->cap_cpl * sizeof(int));
        h->cpl_t = realloc(h->cpl_t, h->cap_cpl * sizeof(int64_t));
        h->cpl_s = realloc(h->cpl_s, h->cap_cpl * sizeof(int64_t));
    }
    h->cpl_lvl[h->ncpl] = l;
    h->cpl_t[h->ncpl] = t;
    h->cpl_s[h->ncpl] = s;
    h->ncpl++;
}

static void push_dns(orc_h2 *h, int64_t t, int64_t s)
{
    if (h->ndns == h->cap_dns) {
        h->cap_dns = h->cap_dns ? 2 * h->cap_dns : 1024;
        h->dns_t = realloc(h->dns_t, h->cap_dns * sizeof(int64_t));
        h->dns_s = realloc(h->dns_s, h->cap_dns * sizeof(int64_t));
    }
    h->dns_t[h->ndns] = t;
    h->dns_s[h->ndns] = s;
    h->ndns++;
}

static void traverse(orc_h2 *h, int64_t t, int64_t s, int l)
{
    int dim = h->dim;
    if (orc_admissible_boxes(h->bmin + t * dim, h->bmax + t * dim, h->bmin + s * dim,
                             h->bmax + s * dim, dim, h->eta)) {
        push_cpl(h, l, t, s);
    } else if (l == h->q) {
        push_dns(h, t, s);
    } else {
        traverse(h, 2 * t, 2 * s, l + 1);
        traverse(h, 2 * t, 2 * s + 1, l + 1);
        traverse(h, 2 * t + 1, 2 * s, l + 1);
        traverse(h, 2 * t + 1, 2 * s + 1, l + 1);
    }
}

/* ------------------------------------------------------- Chebyshev interpolation */

/* First-kind Chebyshev points of [lo, hi]: xi_j = c + (h/2) cos((2j+1) pi / (2p)). */
void orc_cheb_points(double lo, double hi, int p, double *xi)
{
    double c = (lo + hi) / 2, hh = (hi - lo) / 2;
    for (int j = 0; j < p; j++) xi[j] = c + hh * cos((2.0 * j + 1.0) * M_PI / (2.0 * p));
}

/* Lagrange polynomial L_j(x) = prod_{i != j} (x - xi_i) / (xi_j - xi_i). */
double orc_lagrange(const double *xi, int p, int j, double x)
{
    double v = 1.0;
    for (int i = 0; i < p; i++)
        if (i != j) v *= (x - xi[i]) / (xi[j] - xi[i]);
    return v;
}

static const double *node_xi(const orc_h2 *h, int64_t node, int d)
{
    return h->xi + (node * h->dim + d) * h->p;
}

/* Tensor Chebyshev point nu of node t: (xi^{t,0}_{j0}, xi^{t,1}_{j1}, ...). */
static void node_point(const orc_h2 *h, int64_t t, int nu, double *out)
{
    for (int d = 0; d < h->dim; d++) {
        out[d] = node_xi(h, t, d)[nu % h->p];
        nu /= h->p;
    }
}

/* Tensor Lagrange basis function nu of node t at point x: prod_d L^{t,d}_{nu_d}(x_d). */
static double node_lagrange(const orc_h2 *h, int64_t t, int nu, const double *x)
{
    double v = 1.0;
    for (int d = 0; d < h->dim; d++) {
        v *= orc_lagrange(node_xi(h, t, d), h->p, nu % h->p, x[d]);
        nu /= h->p;
    }
    return v;
}

/* Leaf basis U_t (rows = points of t in tree order, k columns), row-major. */
void orc_leaf_basis(const orc_h2 *h, int64_t t, double *U)
{
    int64_t rows = h->hi[t] - h->lo[t];
    for (int64_t i = 0; i < rows; i++) {
        const double *x = h->pts + h->perm[h->lo[t] + i] * h->dim;
        for (int nu = 0; nu < h->k; nu++) U[i * h->k + nu] = node_lagrange(h, t, nu, x);
    }
}

/* Transfer E_c (k x k, row-major): E_c[mu][nu] = L^{parent}_nu(xi^c_mu). Maps parent
 * coefficients to child coefficients, so U^{l-1}_parent = [U_c1 E_c1; U_c2 E_c2]. */
void orc_transfer(const orc_h2 *h, int64_t c, double *E)
{
    double x[3];
    for (int mu = 0; mu < h->k; mu++) {
        node_point(h, c, mu, x);
        for (int nu = 0; nu < h->k; nu++) E[mu * h->k + nu] = node_lagrange(h, c / 2, nu, x);
    }
}

/* Coupling block S_ts (k x k, row-major): S[nu][mu] = kappa(xi^t_nu, xi^s_mu). */
void orc_coupling(const orc_h2 *h, int64_t t, int64_t s, double *S)
{
    double xt[3], xs[3];
    for (int nu = 0; nu < h->k; nu++) {
        node_point(h, t, nu, xt);
        for (int mu = 0; mu < h->k; mu++) {
            node_point(h, s, mu, xs);
            S[nu * h->k + mu] = kernel_eval(&h->ker, xt, xs, h->dim);
        }
    }
}

/* Dense block D_ts (|t| x |s|, row-major): kappa(x_i, x_j) evaluated directly. */
void orc_dense_block(const orc_h2 *h, int64_t t, int64_t s, double *D)
{
    int64_t rt = h->hi[t] - h->lo[t], rs = h->hi[s] - h->lo[s];
    for (int64_t i = 0; i < rt; i++) {
        const double *xi = h->pts + h->perm[h->lo[t] + i] * h->dim;
        for (int64_t j = 0; j < rs; j++) {
            const double *xj = h->pts + h->perm[h->lo[s] + j] * h->dim;
            D[i * rs + j] = kernel_eval(&h->ker, xi, xj, h->dim);
        }
    }
}

/* ------------------------------------------------------------------- build / free */

void orc_free(orc_h2 *h)
{
    if (!h) return;
    free(h->pts); free(h->perm); free(h->lo); free(h->hi); free(h->bmin); free(h->bmax);
    free(h->xi); free(h->cpl_lvl); free(h->cpl_t); free(h->cpl_s); free(h->dns_t);
    free(h->dns_s); free(h->S); free(h->D); free(h->dns_off);
    free(h);
}

orc_h2 *orc_build(const double *pts, int64_t n, int dim, int kind, double ka, double kb,
                  int kdeg, int m, int p, double eta)
{
    if (n < 1 || dim < 1 || dim > 3 || m < 2 || p < 1 || eta < 0) return NULL;
    orc_h2 *h = calloc(1, sizeof(orc_h2));
    h->n = n; h->dim = dim; h->m = m; h->p = p; h->eta = eta;
    h->ker.kind = kind; h->ker.a = ka; h->ker.b = kb; h->ker.deg = kdeg;
    h->k = 1;
    for (int d = 0; d < dim; d++) h->k *= p;
    h->q = 0;
    while ((int64_t)m << h->q < n) h->q++;
    h->nnodes = ((int64_t)2 << h->q) - 1;
    h->pts = malloc(n * dim * sizeof(double));
    memcpy(h->pts, pts, n * dim * sizeof(double));
    h->perm = malloc(n * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) h->perm[i] = i;
    h->lo = calloc(h->nnodes + 1, sizeof(int64_t));
    h->hi = calloc(h->nnodes + 1, sizeof(int64_t));
    h->bmin = calloc((h->nnodes + 1) * dim, sizeof(double));
    h->bmax = calloc((h->nnodes + 1) * dim, sizeof(double));
    build_node(h, 1, 0, 0, n);

    /* Chebyshev points on the (clamped) bounding boxes */
    double root_diag = box_diag(h->bmin + dim, h->bmax + dim, dim);
    double min_ext = 1e-12 * (root_diag > 0 ? root_diag : 1.0);
    h->xi = calloc((h->nnodes + 1) * dim * p, sizeof(double));
    for (int64_t t = 1; t <= h->nnodes; t++)
        for (int d = 0; d < dim; d++) {
            double lo = h->bmin[t * dim + d], hi = h->bmax[t * dim + d];
            if (hi - lo < min_ext) {
                double c = (lo + hi) / 2;
                lo = c - min_ext / 2;
                hi = c + min_ext / 2;
            }
            orc_cheb_points(lo, hi, p, h->xi + (t * dim + d) * p);
        }

    traverse(h, 1, 1, 0);
    return h;
}

/* Store every coupling and dense block (else they are evaluated on the fly). */
int orc_assemble(orc_h2 *h)
{
    int64_t kk = (int64_t)h->k * h->k;
    h->S = malloc((h->ncpl ? h->ncpl : 1) * kk * sizeof(double));
    if (!h->S) return -1;
    for (int64_t b = 0; b < h->ncpl; b++) orc_coupling(h, h->cpl_t[b], h->cpl_s[b], h->S + b * kk);
    h->dns_off = malloc((h->ndns + 1) * sizeof(int64_t));
    h->dns_off[0] = 0;
    for (int64_t b = 0; b < h->ndns; b++) {
        int64_t t = h->dns_t[b], s = h->dns_s[b];
        h->dns_off[b + 1] = h->dns_off[b] + (h->hi[t] - h->lo[t]) * (h->hi[s] - h->lo[s]);
    }
    h->D = malloc((h->dns_off[h->ndns] ? h->dns_off[h->ndns] : 1) * sizeof(double));
    if (!h->D) return -1;
    for (int64_t b = 0; b < h->ndns; b++) orc_dense_block(h, h->dns_t[b], h->dns_s[b], h->D + h->dns_off[b]);
    return 0;
}

/* --------------------------------------------------------------------- queries */

int64_t orc_n(const orc_h2 *h) { return h->n; }
int orc_depth(const orc_h2 *h) { return h->q; }
int orc_rank(const orc_h2 *h) { return h->k; }
int64_t orc_nnodes(const orc_h2 *h) { return h->nnodes; }
int64_t orc_ncoupling(const orc_h2 *h) { return h->ncpl; }
int64_t orc_ndense(const orc_h2 *h) { return h->ndns; }

void orc_get_perm(const orc_h2 *h, int64_t *out) { memcpy(out, h->perm, h->n * sizeof(int64_t)); }

void orc_get_ranges(const orc_h2 *h, int64_t *lo, int64_t *hi)
{
    memcpy(lo, h->lo, (h->nnodes + 1) * sizeof(int64_t));
    memcpy(hi, h->hi, (h->nnodes + 1) * sizeof(int64_t));
}

void orc_get_boxes(const orc_h2 *h, double *bmin, double *bmax)
{
    memcpy(bmin, h->bmin, (h->nnodes + 1) * h->dim * sizeof(double));
    memcpy(bmax, h->bmax, (h->nnodes + 1) * h->dim * sizeof(double));
}

void orc_get_blocks(const orc_h2 *h, int *lvl, int64_t *t, int64_t *s, int64_t *dt, int64_t *ds)
{
    memcpy(lvl, h->cpl_lvl, h->ncpl * sizeof(int));
    memcpy(t, h->cpl_t, h->ncpl * sizeof(int64_t));
    memcpy(s, h->cpl_s, h->ncpl * sizeof(int64_t));
    memcpy(dt, h->dns_t, h->ndns * sizeof(int64_t));
    memcpy(ds, h->dns_s, h->ndns * sizeof(int64_t));
}

/* ----------------------------------------------------------------------- matvec */

static int node_level(int64_t node)
{
    int l = 0;
    while (node > 1) { node >>= 1; l++; }
    return l;
}

/* S_ts stored or evaluated */
static const double *coupling_of(const orc_h2 *h, int64_t b, double *scratch)
{
    if (h->S) return h->S + b * (int64_t)h->k * h->k;
    orc_coupling(h, h->cpl_t[b], h->cpl_s[b], scratch);
    return scratch;
}

static const double *dense_of(const orc_h2 *h, int64_t b, double *scratch)
{
    if (h->D) return h->D + h->dns_off[b];
    orc_dense_block(h, h->dns_t[b], h->dns_s[b], scratch);
    return scratch;
}

/* Upsweep (Sec. 3.1, Alg 1): xh[node][v][nu], all nodes. xt = x in tree order. */
static void upsweep(const orc_h2 *h, const double *xt, int nv, double *xh)
{
    int k = h->k;
    int64_t first_leaf = (int64_t)1 << h->q;
    double *U = malloc((size_t)h->m * k * sizeof(double));
    double *E = malloc((size_t)k * k * sizeof(double));
    memset(xh, 0, (h->nnodes + 1) * (size_t)k * nv * sizeof(double));
    /* leaf projections xhat^q_t = U_t^T x_t */
    for (int64_t t = first_leaf; t <= h->nnodes; t++) {
        int64_t rows = h->hi[t] - h->lo[t];
        orc_leaf_basis(h, t, U);
        for (int v = 0; v < nv; v++)
            for (int nu = 0; nu < k; nu++) {
                double acc = 0.0;
                for (int64_t i = 0; i < rows; i++) acc += U[i * k + nu] * xt[v * h->n + h->lo[t] + i];
                xh[(t * nv + v) * k + nu] = acc;
            }
    }
    /* transfers xhat^{l-1}_parent = sum_c E_c^T xhat^l_c, for l = q .. 1 */
    for (int l = h->q; l >= 1; l--)
        for (int64_t c = (int64_t)1 << l; c < ((int64_t)2 << l); c++) {
            int64_t par = c / 2;
            orc_transfer(h, c, E);
            for (int v = 0; v < nv; v++)
                for (int nu = 0; nu < k; nu++) {
                    double acc = 0.0;
                    for (int mu = 0; mu < k; mu++) acc += E[mu * k + nu] * xh[(c * nv + v) * k + mu];
                    xh[(par * nv + v) * k + nu] += acc;
                }
        }
    free(U);
    free(E);
}

static void scatter_epilogue(const orc_h2 *h, const double *y, int nv, double alpha,
                             double beta, double *Y)
{
    for (int v = 0; v < nv; v++)
        for (int64_t i = 0; i < h->n; i++) {
            int64_t u = h->perm[i];
            double r = alpha * y[v * h->n + i];
            Y[v * h->n + u] = (beta == 0.0) ? r : r + beta * Y[v * h->n + u];
        }
}

/* Y = alpha * A_H2 * X + beta * Y. X, Y: n x nv column-major in user order. When
 * beta == 0, Y is not read. Steps in the order of Sec. 3 (Alg 1, Alg 4, Alg 6). */
int orc_matvec(const orc_h2 *h, const double *X, double *Y, int nv, double alpha, double beta)
{
    int k = h->k;
    int64_t n = h->n;
    double *xt = malloc(n * (size_t)nv * sizeof(double));
    double *y = calloc(n * (size_t)nv, sizeof(double));
    double *xh = malloc((h->nnodes + 1) * (size_t)k * nv * sizeof(double));
    double *yh = calloc((h->nnodes + 1) * (size_t)k * nv, sizeof(double));
    double *U = malloc((size_t)h->m * k * sizeof(double));
    double *E = malloc((size_t)k * k * sizeof(double));
    double *blk = malloc((size_t)(k * k > h->m * h->m ? k * k : h->m * h->m) * sizeof(double));
    if (!xt || !y || !xh || !yh || !U || !E || !blk) return -1;

    /* 1. x in tree order */
    for (int v = 0; v < nv; v++)
        for (int64_t i = 0; i < n; i++) xt[v * n + i] = X[v * n + h->perm[i]];
    /* 2-3. upsweep */
    upsweep(h, xt, nv, xh);
    /* 4. tree multiply: yhat^l_t += S^l_ts xhat^l_s, blocks in traversal order */
    for (int64_t b = 0; b < h->ncpl; b++) {
        int64_t t = h->cpl_t[b], s = h->cpl_s[b];
        const double *S = coupling_of(h, b, blk);
        for (int v = 0; v < nv; v++)
            for (int nu = 0; nu < k; nu++) {
                double acc = 0.0;
                for (int mu = 0; mu < k; mu++) acc += S[nu * k + mu] * xh[(s * nv + v) * k + mu];
                yh[(t * nv + v) * k + nu] += acc;
            }
    }
    /* 5. downsweep: yhat^l_c += E_c yhat^{l-1}_parent, for l = 1 .. q */
    for (int l = 1; l <= h->q; l++)
        for (int64_t c = (int64_t)1 << l; c < ((int64_t)2 << l); c++) {
            orc_transfer(h, c, E);
            for (int v = 0; v < nv; v++)
                for (int mu = 0; mu < k; mu++) {
                    double acc = 0.0;
                    for (int nu = 0; nu < k; nu++) acc += E[mu * k + nu] * yh[((c / 2) * nv + v) * k + nu];
                    yh[(c * nv + v) * k + mu] += acc;
                }
        }
    /* 6a. leaf expansion y_t = U_t yhat^q_t */
    for (int64_t t = (int64_t)1 << h->q; t <= h->nnodes; t++) {
        int64_t rows = h->hi[t] - h->lo[t];
        orc_leaf_basis(h, t, U);
        for (int v = 0; v < nv; v++)
            for (int64_t i = 0; i < rows; i++) {
                double acc = 0.0;
                for (int nu = 0; nu < k; nu++) acc += U[i * k + nu] * yh[(t * nv + v) * k + nu];
                y[v * n + h->lo[t] + i] = acc;
            }
    }
    /* 6b. dense near field y_t += D_ts x_s */
    for (int64_t b = 0; b < h->ndns; b++) {
        int64_t t = h->dns_t[b], s = h->dns_s[b];
        int64_t rt = h->hi[t] - h->lo[t], rs = h->hi[s] - h->lo[s];
        const double *D = dense_of(h, b, blk);
        for (int v = 0; v < nv; v++)
            for (int64_t i = 0; i < rt; i++) {
                double acc = 0.0;
                for (int64_t j = 0; j < rs; j++) acc += D[i * rs + j] * xt[v * n + h->lo[s] + j];
                y[v * n + h->lo[t] + i] += acc;
            }
    }
    /* 7. Y[perm] = alpha y + beta Y */
    scatter_epilogue(h, y, nv, alpha, beta, Y);
    free(xt); free(y); free(xh); free(yh); free(U); free(E); free(blk);
    return 0;
}

/* The output rows of a few leaves only, for checks at sizes where the full product is
 * too slow. The upsweep is complete (every xhat is needed); the tree multiply and the
 * downsweep are restricted to the ancestors of each sampled leaf, which is all that
 * leaf's rows depend on. out: for each sampled leaf (in the given order) its rows in
 * tree order, nv values per row (row-major, out[(r) * nv + v]); the caller maps rows to
 * user indices with the permutation. Yin (user order, n x nv column-major) supplies the
 * beta term; it is not read when beta == 0. */
int orc_matvec_leaves(const orc_h2 *h, const double *X, int nv, double alpha, double beta,
                      const double *Yin, const int64_t *leaves, int64_t nleaves, double *out)
{
    int k = h->k;
    int64_t n = h->n;
    double *xt = malloc(n * (size_t)nv * sizeof(double));
    double *xh = malloc((h->nnodes + 1) * (size_t)k * nv * sizeof(double));
    double *acc_path = malloc((size_t)k * nv * sizeof(double));
    double *row = malloc((size_t)k * nv * sizeof(double));
    double *tmp = malloc((size_t)k * nv * sizeof(double));
    double *U = malloc((size_t)h->m * k * sizeof(double));
    double *E = malloc((size_t)k * k * sizeof(double));
    double *blk = malloc((size_t)(k * k > h->m * h->m ? k * k : h->m * h->m) * sizeof(double));
    /* block-row index: first block of each node (blocks are grouped by traversal, not by
     * row, so build a per-node list) */
    int64_t *cnt = calloc(h->nnodes + 2, sizeof(int64_t));
    int64_t *idx = malloc((h->ncpl ? h->ncpl : 1) * sizeof(int64_t));
    int64_t *dcnt = calloc(h->nnodes + 2, sizeof(int64_t));
    int64_t *didx = malloc((h->ndns ? h->ndns : 1) * sizeof(int64_t));
    if (!xt || !xh || !acc_path || !row || !tmp || !U || !E || !blk || !cnt || !idx || !dcnt || !didx) return -1;
    for (int64_t b = 0; b < h->ncpl; b++) cnt[h->cpl_t[b] + 1]++;
    for (int64_t t = 1; t <= h->nnodes + 1; t++) cnt[t] += cnt[t - 1];
    {
        int64_t *fill = calloc(h->nnodes + 2, sizeof(int64_t));
        for (int64_t b = 0; b < h->ncpl; b++) {
            int64_t t = h->cpl_t[b];
            idx[cnt[t] + fill[t]++] = b;
        }
        free(fill);
    }
    for (int64_t b = 0; b < h->ndns; b++) dcnt[h->dns_t[b] + 1]++;
    for (int64_t t = 1; t <= h->nnodes + 1; t++) dcnt[t] += dcnt[t - 1];
    {
        int64_t *fill = calloc(h->nnodes + 2, sizeof(int64_t));
        for (int64_t b = 0; b < h->ndns; b++) {
            int64_t t = h->dns_t[b];
            didx[dcnt[t] + fill[t]++] = b;
        }
        free(fill);
    }

    for (int v = 0; v < nv; v++)
        for (int64_t i = 0; i < n; i++) xt[v * n + i] = X[v * n + h->perm[i]];
    upsweep(h, xt, nv, xh);

    int64_t orow = 0;
    for (int64_t li = 0; li < nleaves; li++) {
        int64_t leaf = leaves[li];
        memset(acc_path, 0, (size_t)k * nv * sizeof(double));
        /* walk root -> leaf: acc^l = E_c acc^{l-1} + (S^l xhat^l)_c */
        for (int l = 0; l <= h->q; l++) {
            int64_t c = leaf >> (h->q - l);
            if (l >= 1) {
                orc_transfer(h, c, E);
                for (int v = 0; v < nv; v++)
                    for (int mu = 0; mu < k; mu++) {
                        double a = 0.0;
                        for (int nu = 0; nu < k; nu++) a += E[mu * k + nu] * acc_path[v * k + nu];
                        tmp[v * k + mu] = a;
                    }
                memcpy(acc_path, tmp, (size_t)k * nv * sizeof(double));
            }
            memset(row, 0, (size_t)k * nv * sizeof(double));
            for (int64_t e = cnt[c]; e < cnt[c + 1]; e++) {
                int64_t b = idx[e], s = h->cpl_s[b];
                const double *S = coupling_of(h, b, blk);
                for (int v = 0; v < nv; v++)
                    for (int nu = 0; nu < k; nu++) {
                        double a = 0.0;
                        for (int mu = 0; mu < k; mu++) a += S[nu * k + mu] * xh[(s * nv + v) * k + mu];
                        row[v * k + nu] += a;
                    }
            }
            for (int64_t e = 0; e < (int64_t)k * nv; e++) acc_path[e] += row[e];
        }
        int64_t rows = h->hi[leaf] - h->lo[leaf];
        orc_leaf_basis(h, leaf, U);
        for (int64_t i = 0; i < rows; i++)
            for (int v = 0; v < nv; v++) {
                double a = 0.0;
                for (int nu = 0; nu < k; nu++) a += U[i * k + nu] * acc_path[v * k + nu];
                out[(orow + i) * nv + v] = a;
            }
        for (int64_t e = dcnt[leaf]; e < dcnt[leaf + 1]; e++) {
            int64_t b = didx[e], s = h->dns_s[b];
            int64_t rs = h->hi[s] - h->lo[s];
            const double *D = dense_of(h, b, blk);
            for (int64_t i = 0; i < rows; i++)
                for (int v = 0; v < nv; v++) {
                    double a = 0.0;
                    for (int64_t j = 0; j < rs; j++) a += D[i * rs + j] * xt[v * n + h->lo[s] + j];
                    out[(orow + i) * nv + v] += a;
                }
        }
        for (int64_t i = 0; i < rows; i++)
            for (int v = 0; v < nv; v++) {
                int64_t u = h->perm[h->lo[leaf] + i];
                double r = alpha * out[(orow + i) * nv + v];
                out[(orow + i) * nv + v] = (beta == 0.0) ? r : r + beta * Yin[v * n + u];
            }
        orow += rows;
    }
    free(xt); free(xh); free(acc_path); free(row); free(tmp); free(U); free(E); free(blk);
    free(cnt); free(idx); free(dcnt); free(didx);
    return 0;
}

/* ------------------------------------------------- explicit forms for small n */

/* Explicit nested basis U^l_t (|t| x k, row-major) built from the leaf bases and the
 * transfers, U^{l-1}_i = [U^l_c1 E_c1; U^l_c2 E_c2] (Sec. 2.1). */
void orc_nested_basis(const orc_h2 *h, int64_t t, double *out)
{
    int k = h->k;
    if (node_level(t) == h->q) {
        orc_leaf_basis(h, t, out);
        return;
    }
    double *E = malloc((size_t)k * k * sizeof(double));
    for (int64_t c = 2 * t; c <= 2 * t + 1; c++) {
        int64_t rc = h->hi[c] - h->lo[c];
        double *Uc = malloc((size_t)rc * k * sizeof(double));
        orc_nested_basis(h, c, Uc);
        orc_transfer(h, c, E);
        double *dst = out + (h->lo[c] - h->lo[t]) * k;
        for (int64_t i = 0; i < rc; i++)
            for (int nu = 0; nu < k; nu++) {
                double a = 0.0;
                for (int mu = 0; mu < k; mu++) a += Uc[i * k + mu] * E[mu * k + nu];
                dst[i * k + nu] = a;
            }
        free(Uc);
    }
    free(E);
}

/* Direct interpolation basis of node t at its own points: prod_d L^{t,d}_{nu_d}(x_{i,d}). */
void orc_direct_basis(const orc_h2 *h, int64_t t, double *out)
{
    int64_t rows = h->hi[t] - h->lo[t];
    for (int64_t i = 0; i < rows; i++) {
        const double *x = h->pts + h->perm[h->lo[t] + i] * h->dim;
        for (int nu = 0; nu < h->k; nu++) out[i * h->k + nu] = node_lagrange(h, t, nu, x);
    }
}

/* Dense n x n A_H2 (row-major, user order): A_de + sum over coupling blocks of
 * U^l_t S_ts U^l_s^T with the explicit nested bases. */
int orc_assemble_h2_dense(const orc_h2 *h, double *A)
{
    int k = h->k;
    int64_t n = h->n;
    memset(A, 0, n * n * sizeof(double));
    double *blk = malloc((size_t)(k * k > h->m * h->m ? k * k : h->m * h->m) * sizeof(double));
    for (int64_t b = 0; b < h->ndns; b++) {
        int64_t t = h->dns_t[b], s = h->dns_s[b];
        int64_t rt = h->hi[t] - h->lo[t], rs = h->hi[s] - h->lo[s];
        const double *D = dense_of(h, b, blk);
        for (int64_t i = 0; i < rt; i++)
            for (int64_t j = 0; j < rs; j++)
                A[h->perm[h->lo[t] + i] * n + h->perm[h->lo[s] + j]] += D[i * rs + j];
    }
    for (int64_t b = 0; b < h->ncpl; b++) {
        int64_t t = h->cpl_t[b], s = h->cpl_s[b];
        int64_t rt = h->hi[t] - h->lo[t], rs = h->hi[s] - h->lo[s];
        double *Ut = malloc((size_t)rt * k * sizeof(double));
        double *Us = malloc((size_t)rs * k * sizeof(double));
        double *US = malloc((size_t)rt * k * sizeof(double));
        orc_nested_basis(h, t, Ut);
        orc_nested_basis(h, s, Us);
        const double *S = coupling_of(h, b, blk);
        for (int64_t i = 0; i < rt; i++)
            for (int mu = 0; mu < k; mu++) {
                double a = 0.0;
                for (int nu = 0; nu < k; nu++) a += Ut[i * k + nu] * S[nu * k + mu];
                US[i * k + mu] = a;
            }
        for (int64_t i = 0; i < rt; i++)
            for (int64_t j = 0; j < rs; j++) {
                double a = 0.0;
                for (int mu = 0; mu < k; mu++) a += US[i * k + mu] * Us[j * k + mu];
                A[h->perm[h->lo[t] + i] * n + h->perm[h->lo[s] + j]] += a;
            }
        free(Ut); free(Us); free(US);
    }
    free(blk);
    return 0;
}

/* Brute-force dense product Y = K X with K_ij = kappa(x_i, x_j) (no H^2 structure). */
void orc_dense_kx(const double *pts, int64_t n, int dim, int kind, double ka, double kb,
                  int kdeg, const double *X, int nv, double *Y)
{
    orc_kernel kr = {kind, ka, kb, kdeg};
    for (int v = 0; v < nv; v++)
        for (int64_t i = 0; i < n; i++) {
            double a = 0.0;
            for (int64_t j = 0; j < n; j++) a += kernel_eval(&kr, pts + i * dim, pts + j * dim, dim) * X[v * n + j];
            Y[v * n + i] = a;
        }
}

/* Rows `rows[0..nr)` of K X (brute force), out[r * nv + v]. */
void orc_dense_kx_rows(const double *pts, int64_t n, int dim, int kind, double ka, double kb,
                       int kdeg, const double *X, int nv, const int64_t *rows, int64_t nr,
                       double *out)
{
    orc_kernel kr = {kind, ka, kb, kdeg};
    for (int64_t r = 0; r < nr; r++)
        for (int v = 0; v < nv; v++) {
            double a = 0.0;
            for (int64_t j = 0; j < n; j++)
                a += kernel_eval(&kr, pts + rows[r] * dim, pts + j * dim, dim) * X[v * n + j];
            out[r * nv + v] = a;
        }
}

/* Kernel value at one pair of points (for tests of the kernel definitions). */
double orc_kernel_value(int kind, double ka, double kb, int kdeg, const double *x,
                        const double *y, int dim)
{
    orc_kernel kr = {kind, ka, kb, kdeg};
    return kernel_eval(&kr, x, y, dim);
}
