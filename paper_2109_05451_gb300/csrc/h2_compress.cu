// h2_compress.cu -- algebraic recompression of an H^2 operator on the GPU (Sec. 5), FP64.
//
// The four steps run level by level on one stream, every node or block of a level in its own
// CTA (h2_cmpk.cuh): orthogonalization (leaf QR, the sibling-pair QR upsweep, S <- R S R^T),
// the new-basis downsweep (Eq. for B_i^q, one QR update per stacked block), the truncation
// upsweep (Jacobi SVDs; a node keeps the singular values above tau times its largest, and
// each level's rank is the largest such count over its nodes, decided on the device), and the
// projection S' = T_t S T_s^T. The result is compacted to the largest level rank and copied
// into a new host operator.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "h2_cmpk.cuh"
#include "h2_internal.h"
#include "h2_nvtx.h"

namespace {

int cstat(cudaError_t e)
{
    if (e == cudaSuccess) return H2_OK;
    if (e == cudaErrorMemoryAllocation) return H2_ENOMEM;
    return H2_ECUDA;
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

template <typename K>
int allow_smem(K kernel, size_t bytes)
{
    return cstat(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)));
}

unsigned grid_for(int64_t items, int64_t cap = 8192) { return unsigned(std::max<int64_t>(1, std::min(items, cap))); }

// Householder QR of rows x k plus its explicit Q (Golub & Van Loan flop counts).
double qr_flops(double rows, double k)
{
    const double p = std::min(rows, k), c = std::max(rows, k);
    return 2.0 * (2.0 * c * p * p - 2.0 / 3.0 * p * p * p);
}

}  // namespace

extern "C" int h2_compress(h2_handle h, double tau, void *cuda_stream, h2_handle *out, h2_compress_info *info)
{
    h2n::Range range("h2_compress");
    if (!out) return H2_EINVAL;
    *out = nullptr;
    if (!h || !(tau >= 0.0) || !std::isfinite(tau)) return H2_EINVAL;
    const h2_op &op = *h;
    const int k = op.k, q = op.q;
    const int64_t nn = op.nnodes, first = op.first_leaf(), nleaves = op.nleaves(), ncpl = int64_t(op.cpl_col.size());
    int M = 0;
    for (int64_t t = 0; t < nleaves; ++t) M = std::max<int>(M, int(op.hi[first + t] - op.lo[first + t]));
    if (k > h2c::kMaxK || M > h2c::kMaxRows || M < 1) return H2_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const size_t kk = size_t(k) * k;

    // ---- device arena
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += up256(std::max<size_t>(bytes, 1));
        return o;
    };
    const int64_t max_parents = std::max<int64_t>(1, nleaves / 2);
    const size_t o_U = take(size_t(op.n) * k * 8), o_E0 = take((nn + 1) * kk * 8), o_S = take(ncpl * kk * 8);
    const size_t o_Q = take(size_t(nleaves) * M * k * 8), o_R = take((nn + 1) * kk * 8), o_E1 = take((nn + 1) * kk * 8);
    const bool gram_route = tau >= h2c::kGramMinTau;
    const size_t o_Rh = take((nn + 1) * kk * 8), o_G = take(gram_route ? (nn + 1) * kk * 8 : 0), o_W = take(size_t(nleaves) * M * k * 8);
    const size_t o_sig = take((nn + 1) * k * 8), o_T = take((nn + 1) * kk * 8), o_E2 = take((nn + 1) * kk * 8);
    const size_t o_Zb = take(max_parents * 2 * kk * 8), o_Wb = take(max_parents * 2 * kk * 8);
    const size_t o_leaf = take((nleaves + 1) * 4), o_rp = take((nn + 2) * 8), o_brow = take(ncpl * 4),
                 o_bcol = take(ncpl * 4);
    const size_t o_norm = take(16), o_rank = take(size_t(q + 1) * 4), o_sweeps = take(size_t(q + 1) * 8);
    char *arena = nullptr;
    if (cudaMalloc(&arena, off) != cudaSuccess) {
        cudaGetLastError();
        return H2_ENOMEM;
    }
    auto D = [&](size_t o) { return reinterpret_cast<double *>(arena + o); };
    double *dU = D(o_U), *dE0 = D(o_E0), *dS = D(o_S), *dQ = D(o_Q), *dR = D(o_R), *dE1 = D(o_E1), *dRh = D(o_Rh), *dG = D(o_G),
           *dW = D(o_W), *dsig = D(o_sig), *dT = D(o_T), *dE2 = D(o_E2), *dZb = D(o_Zb), *dWb = D(o_Wb),
           *dnorm = D(o_norm);
    int32_t *dleaf = reinterpret_cast<int32_t *>(arena + o_leaf), *dbrow = reinterpret_cast<int32_t *>(arena + o_brow),
            *dbcol = reinterpret_cast<int32_t *>(arena + o_bcol);
    int64_t *drp = reinterpret_cast<int64_t *>(arena + o_rp);
    int *drank = reinterpret_cast<int *>(arena + o_rank);
    unsigned long long *dsweeps = reinterpret_cast<unsigned long long *>(arena + o_sweeps);

    std::vector<int32_t> leaf_lo(nleaves + 1), brow(ncpl);
    for (int64_t t = 0; t < nleaves; ++t) leaf_lo[t] = int32_t(op.lo[first + t]);
    leaf_lo[nleaves] = int32_t(op.n);
    for (int64_t t = 1; t <= nn; ++t)
        for (int64_t b = op.cpl_rowptr[t]; b < op.cpl_rowptr[t + 1]; ++b) brow[b] = int32_t(t);

    int rc = H2_OK;
    auto cp = [&](void *dst, const void *src, size_t bytes) {
        if (rc == H2_OK && bytes) rc = cstat(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
    };
    cp(dU, op.U.data(), op.U.size() * 8);
    cp(dE0, op.E.data(), op.E.size() * 8);
    cp(dleaf, leaf_lo.data(), leaf_lo.size() * 4);
    cp(drp, op.cpl_rowptr.data(), op.cpl_rowptr.size() * 8);
    cp(dbrow, brow.data(), brow.size() * 4);
    cp(dbcol, op.cpl_col.data(), op.cpl_col.size() * 4);
    auto zero = [&](void *p, size_t bytes) {
        if (rc == H2_OK) rc = cstat(cudaMemsetAsync(p, 0, bytes, st));
    };
    zero(dR, (nn + 1) * kk * 8);
    zero(dE1, (nn + 1) * kk * 8);
    zero(dRh, (nn + 1) * kk * 8);
    zero(dT, (nn + 1) * kk * 8);
    zero(dE2, (nn + 1) * kk * 8);
    zero(drank, size_t(q + 1) * 4);
    zero(dsweeps, size_t(q + 1) * 8);
    zero(dnorm, 16);
    if (rc == H2_OK) rc = h2_coupling_fp64(op, dS, st);

    using namespace h2c;
    const size_t sm_lqr = smem_leaf_qr(M, k), sm_tqr = smem_transfer_qr(k), sm_sw = smem_sandwich(k),
                 sm_dn = smem_down_gram(k), sm_dq = smem_down(k), sm_lsvd = smem_leaf_svd(M, k), sm_nsvd = smem_node_svd(k);
    if (rc == H2_OK) rc = allow_smem(k_leaf_qr, sm_lqr);
    if (rc == H2_OK) rc = allow_smem(k_transfer_qr, sm_tqr);
    if (rc == H2_OK) rc = allow_smem(k_orth_blocks, sm_sw);
    if (rc == H2_OK) rc = allow_smem(k_down_gram, sm_dn);
    if (rc == H2_OK) rc = allow_smem(k_down_qr, sm_dq);
    const bool gram = tau >= kGramMinTau;
    if (rc == H2_OK) rc = allow_smem(k_leaf_svd, sm_lsvd);
    if (rc == H2_OK) rc = allow_smem(k_node_svd, sm_nsvd);
    if (rc == H2_OK) rc = allow_smem(k_project, sm_sw);

    cudaEvent_t ev[5] = {};
    for (auto &e : ev)
        if (rc == H2_OK) rc = cstat(cudaEventCreate(&e));
    if (rc == H2_OK) {
        cudaEventRecord(ev[0], st);
        // 1. orthogonalization
        k_leaf_qr<<<grid_for(nleaves), kThreads, sm_lqr, st>>>(dU, dleaf, nleaves, k, M, dQ, dR, first);
        for (int lp = q - 1; lp >= 0; --lp)
            k_transfer_qr<<<grid_for(int64_t(1) << lp), kThreads, sm_tqr, st>>>(lp, k, dE0, dE1, dR);
        if (ncpl > 0) k_orth_blocks<<<grid_for(ncpl, 65535), kThreads, sm_sw, st>>>(dS, dbrow, dbcol, ncpl, dR, k);
        cudaEventRecord(ev[1], st);
        // 2. new-basis downsweep
        // Gram route for tolerances it resolves (singular values down to ~1e-8 of a node's
        // largest), else the QR updates of the stacked block rows as the paper writes them
        for (int l = 0; l <= q; ++l) {
            if (gram)
                k_down_gram<<<grid_for(int64_t(1) << l), kThreads, sm_dn, st>>>(l, k, drp, dS, dE1, dG, dRh);
            else
                k_down_qr<<<grid_for(int64_t(1) << l), kThreads, sm_dq, st>>>(l, k, drp, dS, dE1, dRh);
        }
        k_norm<<<1, kThreads, 0, st>>>(gram ? dG : dRh, first, nleaves, k, gram, dnorm);
        cudaEventRecord(ev[2], st);
        // 3. truncation upsweep
        k_leaf_svd<<<grid_for(nleaves), kThreads, sm_lsvd, st>>>(dQ, dleaf, nleaves, k, M, dRh, first, tau, dW,
                                                                 dsig + first * k, drank, q, dsweeps + q);
        k_leaf_t<<<grid_for(nleaves), kThreads, 0, st>>>(dQ, dW, dleaf, nleaves, k, M, drank, q, first, dT, dsig,
                                                         dnorm + 1);
        for (int lp = q - 1; lp >= 0; --lp) {
            k_node_svd<<<grid_for(int64_t(1) << lp), kThreads, sm_nsvd, st>>>(lp, k, dT, dE1, dRh, tau, dZb, dWb, dsig,
                                                                               drank, dsweeps + lp);
            k_node_t<<<grid_for(int64_t(1) << lp), kThreads, 0, st>>>(lp, k, dZb, dWb, drank, dE2, dT, dsig, dnorm + 1);
        }
        cudaEventRecord(ev[3], st);
        // 4. projection
        if (ncpl > 0) k_project<<<grid_for(ncpl, 65535), kThreads, sm_sw, st>>>(dS, dbrow, dbcol, ncpl, dT, drank, k);
        cudaEventRecord(ev[4], st);
        rc = cstat(cudaGetLastError());
    }
    std::vector<int> ranks(q + 1, 0);
    std::vector<unsigned long long> sweeps(q + 1, 0);
    double norms[2] = {0, 0};  // ||A_lr||_F, dropped energy
    if (rc == H2_OK) rc = cstat(cudaMemcpyAsync(ranks.data(), drank, size_t(q + 1) * 4, cudaMemcpyDeviceToHost, st));
    if (rc == H2_OK) rc = cstat(cudaMemcpyAsync(sweeps.data(), dsweeps, size_t(q + 1) * 8, cudaMemcpyDeviceToHost, st));
    if (rc == H2_OK) rc = cstat(cudaMemcpyAsync(norms, dnorm, 16, cudaMemcpyDeviceToHost, st));
    if (rc == H2_OK) rc = cstat(cudaStreamSynchronize(st));
    float ms[4] = {0, 0, 0, 0};
    if (rc == H2_OK)
        for (int i = 0; i < 4; ++i) cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
    for (auto &e : ev)
        if (e) cudaEventDestroy(e);

    // ---- compaction to the stored rank kc and the new host operator
    const int kc = std::max(1, *std::max_element(ranks.begin(), ranks.end()));
    h2_op *o = nullptr;
    if (rc == H2_OK) {
        o = new (std::nothrow) h2_op;
        if (!o) rc = H2_ENOMEM;
    }
    if (rc == H2_OK) {
        o->n = op.n;
        o->dim = op.dim;
        o->m = op.m;
        o->p = 0;
        o->k = kc;
        o->q = q;
        o->eta = op.eta;
        o->ker = op.ker;
        o->pts = op.pts;
        o->perm = op.perm;
        o->nnodes = nn;
        o->lo = op.lo;
        o->hi = op.hi;
        o->bmin = op.bmin;
        o->bmax = op.bmax;
        o->cpl_rowptr = op.cpl_rowptr;
        o->cpl_col = op.cpl_col;
        o->dns_rowptr = op.dns_rowptr;
        o->dns_col = op.dns_col;
        o->level_rank = ranks;
        try {
            o->U.assign(size_t(op.n) * kc, 0.0);
            o->E.assign(size_t(nn + 1) * kc * kc, 0.0);
            o->S.assign(size_t(ncpl) * kc * kc, 0.0);
        } catch (...) {
            rc = H2_ENOMEM;
        }
    }
    double *dUc = dQ, *dEc = dR, *dSc = nullptr;  // the compacted copies reuse dead buffers
    if (rc == H2_OK && ncpl > 0 && cudaMalloc(&dSc, size_t(ncpl) * kc * kc * 8) != cudaSuccess) {
        cudaGetLastError();
        rc = H2_ENOMEM;
    }
    if (rc == H2_OK) {
        k_compact_u<<<grid_for(nleaves), 128, 0, st>>>(dW, dleaf, nleaves, k, M, drank, q, kc, dUc);
        k_compact_slabs<<<grid_for((nn + 1) * kc * kc / 256 + 1, 65535), 256, 0, st>>>(dE2, nn + 1, k, kc, dEc);
        if (ncpl > 0) k_compact_slabs<<<grid_for(ncpl * kc * kc / 256 + 1, 65535), 256, 0, st>>>(dS, ncpl, k, kc, dSc);
        rc = cstat(cudaGetLastError());
    }
    if (rc == H2_OK) rc = cstat(cudaMemcpyAsync(o->U.data(), dUc, o->U.size() * 8, cudaMemcpyDeviceToHost, st));
    if (rc == H2_OK) rc = cstat(cudaMemcpyAsync(o->E.data(), dEc, o->E.size() * 8, cudaMemcpyDeviceToHost, st));
    if (rc == H2_OK && ncpl > 0)
        rc = cstat(cudaMemcpyAsync(o->S.data(), dSc, o->S.size() * 8, cudaMemcpyDeviceToHost, st));
    if (rc == H2_OK) rc = cstat(cudaStreamSynchronize(st));
    if (dSc) cudaFree(dSc);
    cudaFree(arena);
    if (rc != H2_OK) {
        delete o;
        return rc;
    }

    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->tau = tau;
        info->norm_lowrank = norms[0];
        info->dropped_energy = norms[1];
        info->depth = q;
        info->rank_in = k;
        info->rank_out = kc;
        for (int l = 0; l <= q && l < H2_MAX_LEVELS; ++l) info->level_rank[l] = ranks[l];
        for (int i = 0; i < 4; ++i) info->ms[i] = ms[i];
        // operation counts of the kernels as written (triangular factors exploited)
        const double K = k, dk3 = K * K * K;
        double f1 = 0, f2 = 0, f3 = 0, f4 = 0;
        for (int64_t t = 0; t < nleaves; ++t) f1 += qr_flops(double(leaf_lo[t + 1] - leaf_lo[t]), K);
        f1 += double(nn - nleaves) * (2 * dk3 + qr_flops(2 * K, K)) + double(ncpl) * 2 * dk3;
        f2 = double(nn - 1) * (dk3 + 2 * dk3) + double(ncpl) * 2 * dk3;
        // one-sided Jacobi: 12 flops per row per pair and sweep (three dot products and the
        // rotation), 8 per pair row more where the rotations are accumulated; FP32 sweeps are
        // not counted
        auto jac = [&](double sweeps_l, double rows, double cols, bool acc) {
            return sweeps_l * (cols * (cols - 1) / 2) * (12.0 * rows + (acc ? 8.0 * cols : 0.0));
        };
        double leaf_p = 0;
        for (int64_t t = 0; t < nleaves; ++t) {
            const double rows = leaf_lo[t + 1] - leaf_lo[t], p = std::min(rows, K);
            leaf_p += p / double(nleaves);
            // V re-orthogonalization, A Vq, W = Q W', T = W^T Q
            f3 += qr_flops(K, K) + 2.0 * p * K * K + 2.0 * rows * p * K + 2.0 * ranks[q] * rows * K;
        }
        f3 += jac(double(sweeps[q]), leaf_p, K, false);
        for (int lp = q - 1; lp >= 0; --lp) {
            const double parents = double(int64_t(1) << lp), r = ranks[lp + 1], rp = ranks[lp], n = 2 * r;
            const bool wide = n < K;
            const double cols = wide ? n : K, rows = wide ? K : n;
            f3 += parents * (2 * 2 * r * K * K + n * K * K + qr_flops(cols, cols) + 2.0 * rows * cols * cols +
                             2 * rp * n * K) +
                  jac(double(sweeps[lp]), rows, cols, wide);
        }
        for (int64_t b = 0; b < ncpl; ++b) {
            int l = 0;
            for (int64_t x = brow[b]; x > 1; x >>= 1) ++l;
            const double r = ranks[l];
            f4 += 2.0 * (K * K * r + r * r * K);
        }
        info->flops[0] = f1;
        info->flops[1] = f2;
        info->flops[2] = f3;
        info->flops[3] = f4;
        for (auto s : sweeps) info->jacobi_sweeps += int64_t(s);
        info->lowrank_bytes_in = size_t(op.n * k + (nn - 1) * k * k + ncpl * k * k) * 8;
        size_t after = size_t(op.n) * ranks[q];
        for (int64_t c = 2; c <= nn; ++c) {
            int l = 0;
            for (int64_t x = c; x > 1; x >>= 1) ++l;
            after += size_t(ranks[l]) * ranks[l - 1];
        }
        for (int64_t b = 0; b < ncpl; ++b) {
            int l = 0;
            for (int64_t x = brow[b]; x > 1; x >>= 1) ++l;
            after += size_t(ranks[l]) * ranks[l];
        }
        info->lowrank_bytes_out = after * 8;
    }
    *out = o;
    return H2_OK;
}
