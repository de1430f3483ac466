// h2_internal.h -- host-side operator state shared by the host build (h2_host.cpp) and
// the device upload / matvec (h2_device.cu). Not part of the public ABI.
#pragma once

#include <cstdint>
#include <vector>

#include "../../include/h2.h"

struct h2_device;  // device copy, defined in h2_device.cu

struct h2_op {
    // parameters
    int64_t n = 0;
    int dim = 0, m = 0, p = 0, k = 0, q = 0;
    double eta = 0;
    h2_kernel ker{};

    // geometry (FP64, host)
    std::vector<double> pts;         // n * dim, caller order
    std::vector<int64_t> perm;       // tree position -> caller index
    int64_t nnodes = 0;              // heap nodes 1 .. nnodes
    std::vector<int64_t> lo, hi;     // [nnodes + 1] tree-order ranges
    std::vector<double> bmin, bmax;  // [(nnodes + 1) * dim] tight boxes
    std::vector<double> cheb;        // [(nnodes + 1) * dim * p] 1-D Chebyshev points

    // bases (FP64, host)
    std::vector<double> U;           // n * k, rows in tree order
    std::vector<double> E;           // (nnodes + 1) * k * k, E_c[mu][nu]

    // partition
    std::vector<int64_t> cpl_rowptr; // nnodes + 2, rows = heap indices (level-ordered)
    std::vector<int32_t> cpl_col;    // heap index of the column cluster
    std::vector<int64_t> dns_rowptr; // nleaves + 1
    std::vector<int32_t> dns_col;    // leaf index of the column cluster

    // explicit coupling blocks of a compressed operator (n_coupling x k x k, CSR order,
    // S_ts[nu][mu] row-major);
    // empty when the blocks are the kernel at the clusters' Chebyshev points (then p > 0)
    std::vector<double> S;
    std::vector<int> level_rank;     // per level, compressed operators only

    int64_t nleaves() const { return int64_t(1) << q; }
    int64_t first_leaf() const { return int64_t(1) << q; }

    h2_device *dev = nullptr;
};

// Fork/join context of one product: the high-priority side stream that runs the upper tree
// levels next to the main stream, and the events that order them (cudaStream_t /
// cudaEvent_t, kept opaque here). Each handle keeps a pool of them for h2_matvec /
// h2_matvec_ws (a product borrows one while its launches are enqueued); the serving loop
// gives each of its slots its own.
struct h2_exec {
    void *side = nullptr;
    void *ev_up = nullptr;
    void *ev_top = nullptr;
    void *ev_topup = nullptr;  // the side stream's upsweep is done (matrix-free schedule)
};

// h2_device.cu
// H2_OK if the current CUDA device holds h's device copy; H2_ESTATE without a device copy,
// H2_EINVAL if another device is current.
int h2_device_check(h2_handle h);
int h2_exec_create(h2_exec *ex);
void h2_exec_destroy(h2_exec *ex);
// h2_matvec_ws with an explicit fork/join context (nullptr: the handle's own).
int h2_matvec_exec(h2_handle h, const void *X, void *Y, int nv, double alpha, double beta, void *workspace,
                   size_t ws_bytes, void *cuda_stream, const h2_exec *ex);

// FP64 coupling blocks (n_coupling x k x k, CSR order, each S_ts[nu][mu] row-major) on the
// device: generated from the kernel, or copied when explicit. Synchronises the stream.
int h2_coupling_fp64(const h2_op &op, double *dS, void *cuda_stream);

// h2_host.cpp
int h2_host_build(h2_op *op, const double *points, int64_t n, int dim, h2_kernel kernel,
                  int leaf_size, int cheb_order, double eta);
// h2_device.cu
void h2_device_free(h2_op *op);
