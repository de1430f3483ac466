// h2_host.cpp -- host construction of the H^2 operator (FP64).
//
// Follows the construction the paper describes for its test matrices: a k-d tree over
// the points (Sec. 6.4), the geometric admissibility condition of Sec. 6.1 applied by a
// same-level dual traversal starting at the root pair (Sec. 2.2), and tensor Chebyshev
// interpolation on the cluster bounding boxes for leaf bases and interlevel transfers
// (Sec. 6.3: a p x p grid gives rank p^2, tri-cubic gives rank 64). The nested-basis
// relation U^{l-1}_i = diag(U^l_c)[E^l_c] of Sec. 2.1 holds exactly for these transfers
// because the children's Lagrange bases reproduce polynomials of degree < p.
//
// The tree is built one level at a time; the admissible partition is found one level at
// a time from the pairs the previous level had to refine; both end as level-ordered
// block-row CSR arrays that the device kernels stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <utility>

#include "h2_internal.h"

namespace {

constexpr double kPi = 3.14159265358979323846;

// Tight bounding box of the points of one cluster.
void cluster_box(const h2_op &op, int64_t lo, int64_t hi, double *bmin, double *bmax)
{
    const int dim = op.dim;
    for (int d = 0; d < dim; ++d) bmin[d] = bmax[d] = op.pts[op.perm[lo] * dim + d];
    for (int64_t i = lo + 1; i < hi; ++i) {
        const double *x = &op.pts[op.perm[i] * dim];
        for (int d = 0; d < dim; ++d) {
            bmin[d] = std::min(bmin[d], x[d]);
            bmax[d] = std::max(bmax[d], x[d]);
        }
    }
}

double diagonal(const double *bmin, const double *bmax, int dim)
{
    double s = 0.0;
    for (int d = 0; d < dim; ++d) {
        const double e = bmax[d] - bmin[d];
        s += e * e;
    }
    return std::sqrt(s);
}

// Sec. 6.1 geometric admissibility, evaluated in this exact operation order (the file is
// compiled without floating-point contraction).
bool admissible(const h2_op &op, int64_t t, int64_t s)
{
    const int dim = op.dim;
    const double *tmin = &op.bmin[t * dim], *tmax = &op.bmax[t * dim];
    const double *smin = &op.bmin[s * dim], *smax = &op.bmax[s * dim];
    double dist2 = 0.0;
    for (int d = 0; d < dim; ++d) {
        const double ct = (tmin[d] + tmax[d]) / 2;
        const double cs = (smin[d] + smax[d]) / 2;
        const double dc = ct - cs;
        dist2 += dc * dc;
    }
    return op.eta * std::sqrt(dist2) >= 0.5 * (diagonal(tmin, tmax, dim) + diagonal(smin, smax, dim));
}

// Values of the p Lagrange polynomials of the points xi at x.
void lagrange_values(const double *xi, int p, double x, double *out)
{
    for (int j = 0; j < p; ++j) {
        double v = 1.0;
        for (int i = 0; i < p; ++i)
            if (i != j) v *= (x - xi[i]) / (xi[j] - xi[i]);
        out[j] = v;
    }
}

void build_tree(h2_op &op)
{
    const int dim = op.dim;
    op.perm.resize(op.n);
    for (int64_t i = 0; i < op.n; ++i) op.perm[i] = i;
    op.lo.assign(op.nnodes + 1, 0);
    op.hi.assign(op.nnodes + 1, 0);
    op.bmin.assign((op.nnodes + 1) * dim, 0.0);
    op.bmax.assign((op.nnodes + 1) * dim, 0.0);
    op.lo[1] = 0;
    op.hi[1] = op.n;
    for (int l = 0; l <= op.q; ++l) {
        const int64_t first = int64_t(1) << l, last = int64_t(2) << l;
#pragma omp parallel for schedule(dynamic, 1) if (last - first >= 8)
        for (int64_t t = first; t < last; ++t) {
            const int64_t lo = op.lo[t], hi = op.hi[t];
            double *bmin = &op.bmin[t * dim], *bmax = &op.bmax[t * dim];
            cluster_box(op, lo, hi, bmin, bmax);
            if (l == op.q) continue;
            int split = 0;
            for (int d = 1; d < dim; ++d)
                if (bmax[d] - bmin[d] > bmax[split] - bmin[split]) split = d;
            const double *pts = op.pts.data();
            std::sort(op.perm.begin() + lo, op.perm.begin() + hi, [&](int64_t a, int64_t b) {
                const double ca = pts[a * dim + split], cb = pts[b * dim + split];
                return ca < cb || (ca == cb && a < b);
            });
            const int64_t mid = lo + (hi - lo) / 2;
            op.lo[2 * t] = lo;
            op.hi[2 * t] = mid;
            op.lo[2 * t + 1] = mid;
            op.hi[2 * t + 1] = hi;
        }
    }
}

void chebyshev_points(h2_op &op)
{
    const int dim = op.dim, p = op.p;
    const double root_diag = diagonal(&op.bmin[dim], &op.bmax[dim], dim);
    const double min_extent = 1e-12 * (root_diag > 0 ? root_diag : 1.0);
    op.cheb.assign((op.nnodes + 1) * dim * p, 0.0);
    for (int64_t t = 1; t <= op.nnodes; ++t)
        for (int d = 0; d < dim; ++d) {
            double lo = op.bmin[t * dim + d], hi = op.bmax[t * dim + d];
            if (hi - lo < min_extent) {
                const double c = (lo + hi) / 2;
                lo = c - min_extent / 2;
                hi = c + min_extent / 2;
            }
            const double c = (lo + hi) / 2, half = (hi - lo) / 2;
            for (int j = 0; j < p; ++j)
                op.cheb[(t * dim + d) * p + j] = c + half * std::cos((2.0 * j + 1.0) * kPi / (2.0 * p));
        }
}

// Leaf bases U_t[i][nu] = prod_d L^{t,d}_{nu_d}(x_{i,d}), rows in tree order.
void leaf_bases(h2_op &op)
{
    const int dim = op.dim, p = op.p, k = op.k;
    op.U.assign(op.n * k, 0.0);
    const int64_t first = op.first_leaf();
#pragma omp parallel for schedule(static)
    for (int64_t t = first; t <= op.nnodes; ++t) {
        double lv[3][16];
        for (int64_t i = op.lo[t]; i < op.hi[t]; ++i) {
            const double *x = &op.pts[op.perm[i] * dim];
            for (int d = 0; d < dim; ++d) lagrange_values(&op.cheb[(t * dim + d) * p], p, x[d], lv[d]);
            for (int nu = 0; nu < k; ++nu) {
                double v = 1.0;
                int r = nu;
                for (int d = 0; d < dim; ++d) {
                    v *= lv[d][r % p];
                    r /= p;
                }
                op.U[i * k + nu] = v;
            }
        }
    }
}

// Transfers E_c[mu][nu] = prod_d L^{parent,d}_{nu_d}(xi^{c,d}_{mu_d}): a Kronecker product
// of the per-dimension p x p matrices that map parent coefficients to child coefficients.
void transfers(h2_op &op)
{
    const int dim = op.dim, p = op.p, k = op.k;
    op.E.assign((op.nnodes + 1) * k * k, 0.0);
#pragma omp parallel for schedule(static)
    for (int64_t c = 2; c <= op.nnodes; ++c) {
        double T[3][16][16];
        for (int d = 0; d < dim; ++d)
            for (int a = 0; a < p; ++a)
                lagrange_values(&op.cheb[((c / 2) * dim + d) * p], p, op.cheb[(c * dim + d) * p + a], T[d][a]);
        double *Ec = &op.E[c * k * k];
        for (int mu = 0; mu < k; ++mu)
            for (int nu = 0; nu < k; ++nu) {
                double v = 1.0;
                int rm = mu, rn = nu;
                for (int d = 0; d < dim; ++d) {
                    v *= T[d][rm % p][rn % p];
                    rm /= p;
                    rn /= p;
                }
                Ec[mu * k + nu] = v;
            }
    }
}

// Same-level dual traversal, one level at a time: admissible pairs become coupling
// leaves, inadmissible leaf pairs become dense leaves, other inadmissible pairs are
// refined into their four children pairs.
void partition(h2_op &op)
{
    std::vector<std::pair<int32_t, int32_t>> cand{{1, 1}}, next, cpl, dns;
    for (int l = 0; l <= op.q && !cand.empty(); ++l) {
        next.clear();
        for (const auto &ts : cand) {
            const int64_t t = ts.first, s = ts.second;
            if (admissible(op, t, s)) {
                cpl.push_back(ts);
            } else if (l == op.q) {
                dns.push_back(ts);
            } else {
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b)
                        next.emplace_back(int32_t(2 * t + a), int32_t(2 * s + b));
            }
        }
        cand.swap(next);
    }
    std::sort(cpl.begin(), cpl.end());
    std::sort(dns.begin(), dns.end());
    op.cpl_rowptr.assign(op.nnodes + 2, 0);
    op.cpl_col.resize(cpl.size());
    for (size_t b = 0; b < cpl.size(); ++b) {
        op.cpl_rowptr[cpl[b].first + 1]++;
        op.cpl_col[b] = cpl[b].second;
    }
    for (int64_t t = 1; t <= op.nnodes + 1; ++t) op.cpl_rowptr[t] += op.cpl_rowptr[t - 1];
    const int64_t first = op.first_leaf();
    op.dns_rowptr.assign(op.nleaves() + 1, 0);
    op.dns_col.resize(dns.size());
    for (size_t b = 0; b < dns.size(); ++b) {
        op.dns_rowptr[dns[b].first - first + 1]++;
        op.dns_col[b] = int32_t(dns[b].second - first);
    }
    for (int64_t t = 1; t <= op.nleaves(); ++t) op.dns_rowptr[t] += op.dns_rowptr[t - 1];
}

}  // namespace

int h2_host_build(h2_op *op, const double *points, int64_t n, int dim, h2_kernel kernel,
                  int leaf_size, int cheb_order, double eta)
{
    if (!op || !points || n < 1 || n >= (int64_t(1) << 31) || dim < 1 || dim > 3 || leaf_size < 2 ||
        cheb_order < 1 || !(eta >= 0))
        return H2_EINVAL;
    int k = 1;
    for (int d = 0; d < dim; ++d) k *= cheb_order;
    if (k > 64 || cheb_order > 16) return H2_EINVAL;
    if (kernel.kind < H2_K_EXP || kernel.kind > H2_K_POLY) return H2_EINVAL;
    if ((kernel.kind == H2_K_EXP || kernel.kind == H2_K_GAUSS) && !(kernel.a > 0)) return H2_EINVAL;
    if (kernel.kind == H2_K_POLY && kernel.deg < 0) return H2_EINVAL;
    for (int64_t i = 0; i < n * dim; ++i)
        if (!std::isfinite(points[i])) return H2_EINVAL;
    try {
        op->n = n;
        op->dim = dim;
        op->m = leaf_size;
        op->p = cheb_order;
        op->k = k;
        op->eta = eta;
        op->ker = kernel;
        op->q = 0;
        while ((int64_t(leaf_size) << op->q) < n) ++op->q;
        if (op->q >= H2_MAX_LEVELS - 1) return H2_EINVAL;
        op->nnodes = (int64_t(2) << op->q) - 1;
        op->pts.assign(points, points + n * dim);
        build_tree(*op);
        chebyshev_points(*op);
        leaf_bases(*op);
        transfers(*op);
        partition(*op);
    } catch (const std::bad_alloc &) {
        return H2_ENOMEM;
    }
    return H2_OK;
}

// ---------------------------------------------------------------- save / load

namespace {

constexpr char kMagic[8] = {'H', '2', 'G', 'B', '3', '0', '0', 'o'};
constexpr uint32_t kFormat = 1;

template <typename V>
bool put_vec(FILE *f, const std::vector<V> &v)
{
    const uint64_t n = v.size();
    return std::fwrite(&n, sizeof(n), 1, f) == 1 && (n == 0 || std::fwrite(v.data(), sizeof(V), n, f) == n);
}

template <typename V>
bool get_vec(FILE *f, std::vector<V> &v, uint64_t expect)
{
    uint64_t n = 0;
    if (std::fread(&n, sizeof(n), 1, f) != 1 || n != expect) return false;
    v.resize(n);
    return n == 0 || std::fread(v.data(), sizeof(V), n, f) == n;
}

// Every index a loaded operator hands to the device (permutation, ranges, block columns)
// stays inside its array, so a damaged file is refused on the host.
bool consistent(const h2_op &o)
{
    const int64_t n = o.n, nn = o.nnodes, first = o.first_leaf(), leaves = o.nleaves();
    int64_t k = 1;
    for (int d = 0; d < o.dim; ++d) k *= o.p;
    if (o.m < 1 || o.k < 1) return false;
    if (o.p == 0) {  // compressed: explicit blocks, level ranks within the stored rank
        for (int r : o.level_rank)
            if (r < 0 || r > o.k) return false;
    } else if (o.p < 0 || o.k != k) {
        return false;
    }
    std::vector<char> seen(size_t(n), 0);
    for (int64_t v : o.perm) {
        if (v < 0 || v >= n || seen[size_t(v)]) return false;
        seen[size_t(v)] = 1;
    }
    if (o.lo[1] != 0 || o.hi[1] != n) return false;
    for (int64_t c = 1; c <= nn; ++c) {
        if (o.lo[c] < 0 || o.lo[c] > o.hi[c] || o.hi[c] > n) return false;
        if (c < first && (o.lo[2 * c] != o.lo[c] || o.hi[2 * c] != o.lo[2 * c + 1] || o.hi[2 * c + 1] != o.hi[c]))
            return false;
        if (c >= first && o.hi[c] - o.lo[c] > o.m) return false;
    }
    auto csr_ok = [](const std::vector<int64_t> &rp, const auto &col, int64_t lo, int64_t hi) {
        if (rp.front() != 0) return false;
        for (size_t i = 1; i < rp.size(); ++i)
            if (rp[i] < rp[i - 1]) return false;
        for (auto c : col)
            if (int64_t(c) < lo || int64_t(c) > hi) return false;
        return true;
    };
    return csr_ok(o.cpl_rowptr, o.cpl_col, 1, nn) && csr_ok(o.dns_rowptr, o.dns_col, 0, leaves - 1);
}

}  // namespace

extern "C" int h2_save(h2_handle h, const char *path)
{
    if (!h || !path) return H2_EINVAL;
    FILE *f = std::fopen(path, "wb");
    if (!f) return H2_EINVAL;
    const h2_op &o = *h;
    const int64_t ints[7] = {o.n, o.dim, o.m, o.p, o.k, o.q, o.nnodes};
    bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(&kFormat, sizeof(kFormat), 1, f) == 1 &&
              std::fwrite(ints, sizeof(ints), 1, f) == 1 && std::fwrite(&o.eta, sizeof(o.eta), 1, f) == 1 &&
              std::fwrite(&o.ker, sizeof(o.ker), 1, f) == 1;
    ok = ok && put_vec(f, o.pts) && put_vec(f, o.perm) && put_vec(f, o.lo) && put_vec(f, o.hi) &&
         put_vec(f, o.bmin) && put_vec(f, o.bmax) && put_vec(f, o.cheb) && put_vec(f, o.U) && put_vec(f, o.E) &&
         put_vec(f, o.cpl_rowptr) && put_vec(f, o.cpl_col) && put_vec(f, o.dns_rowptr) && put_vec(f, o.dns_col) &&
         put_vec(f, o.S) && put_vec(f, o.level_rank);
    ok = (std::fclose(f) == 0) && ok;
    return ok ? H2_OK : H2_EINVAL;
}

extern "C" int h2_load(const char *path, h2_handle *out)
{
    if (!out) return H2_EINVAL;
    *out = nullptr;
    if (!path) return H2_EINVAL;
    FILE *f = std::fopen(path, "rb");
    if (!f) return H2_EINVAL;
    h2_op *o = new (std::nothrow) h2_op;
    if (!o) {
        std::fclose(f);
        return H2_ENOMEM;
    }
    char magic[8];
    uint32_t format = 0;
    int64_t ints[7];
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
              std::fread(&format, sizeof(format), 1, f) == 1 && format == kFormat &&
              std::fread(ints, sizeof(ints), 1, f) == 1 && std::fread(&o->eta, sizeof(o->eta), 1, f) == 1 &&
              std::fread(&o->ker, sizeof(o->ker), 1, f) == 1;
    if (ok) {
        o->n = ints[0];
        o->dim = int(ints[1]);
        o->m = int(ints[2]);
        o->p = int(ints[3]);
        o->k = int(ints[4]);
        o->q = int(ints[5]);
        o->nnodes = ints[6];
        ok = o->n >= 1 && o->dim >= 1 && o->dim <= 3 && o->q >= 0 && o->q < 40 && o->nnodes == (int64_t(2) << o->q) - 1 &&
             o->k >= 1 && o->k <= 4096 && o->p >= 0;
    }
    if (ok) {
        const uint64_t n = uint64_t(o->n), nodes = uint64_t(o->nnodes + 1), k = uint64_t(o->k);
        const uint64_t leaves = uint64_t(1) << o->q;
        ok = get_vec(f, o->pts, n * o->dim) && get_vec(f, o->perm, n) && get_vec(f, o->lo, nodes) &&
             get_vec(f, o->hi, nodes) && get_vec(f, o->bmin, nodes * o->dim) && get_vec(f, o->bmax, nodes * o->dim) &&
             get_vec(f, o->cheb, nodes * o->dim * o->p) && get_vec(f, o->U, n * k) && get_vec(f, o->E, nodes * k * k) &&
             get_vec(f, o->cpl_rowptr, nodes + 1);
        if (ok) ok = get_vec(f, o->cpl_col, uint64_t(o->cpl_rowptr.back()));
        if (ok) ok = get_vec(f, o->dns_rowptr, leaves + 1);
        if (ok) ok = get_vec(f, o->dns_col, uint64_t(o->dns_rowptr.back()));
        // a compressed operator carries its coupling blocks and level ranks (p = 0)
        const bool compressed = o->p == 0;
        if (ok) ok = get_vec(f, o->S, compressed ? uint64_t(o->cpl_col.size()) * k * k : 0);
        if (ok) ok = get_vec(f, o->level_rank, compressed ? uint64_t(o->q + 1) : 0);
    }
    std::fclose(f);
    if (ok) ok = consistent(*o);
    if (!ok) {
        delete o;
        return H2_EINVAL;
    }
    *out = o;
    return H2_OK;
}
