// h2_cg.cu -- conjugate gradients for (A_H2 + sigma2 I) x = b on the device.
//
// The paper solves its integral equation with a Krylov method whose products are the H^2
// matvec (Sec. 6.4, preconditioned CG). This is unpreconditioned CG: the products run in the
// uploaded precision through h2_matvec; the Krylov vectors, inner products and updates are
// FP64 on the device. Inner products use a fixed two-stage reduction (a fixed number of
// blocks, fixed summation order), so a solve is bitwise repeatable. The step lengths are
// computed on the device from the inner products; the host reads one residual norm per
// iteration for the stopping test.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "h2_cgk.cuh"
#include "h2_internal.h"
#include "h2_nvtx.h"

namespace {

using namespace h2cg;

struct CgState {
    int64_t n;
    cudaStream_t st;
    double *r, *p, *Ap, *partial, *scal;  // scal: [0] rr, [1] pAp, [2] rr_new, [3] bb
    float *pf, *Apf;
    void *mem;
};

void dot(const CgState &c, const double *a, const double *b, double *out) { h2cg::dot(a, b, c.n, c.partial, out, c.st); }

// out = (A + sigma2 I) v
int apply(h2_handle h, const CgState &c, const double *v, double *out, double sigma2, bool fp64)
{
    int rc;
    if (fp64) {
        rc = h2_matvec(h, v, out, 1, 1.0, 0.0, c.st);
        if (rc != H2_OK) return rc;
        k_shift<double><<<grid_for(c.n), kThreads, 0, c.st>>>(out, v, sigma2, out, c.n);
    } else {
        k_to_float<<<grid_for(c.n), kThreads, 0, c.st>>>(v, c.pf, c.n);
        rc = h2_matvec(h, c.pf, c.Apf, 1, 1.0, 0.0, c.st);
        if (rc != H2_OK) return rc;
        k_shift<float><<<grid_for(c.n), kThreads, 0, c.st>>>(c.Apf, v, sigma2, out, c.n);
    }
    return cuda_status(cudaGetLastError());
}

double read_scalar(const CgState &c, int idx, int *rc)
{
    double v = 0.0;
    const cudaError_t e = cudaMemcpyAsync(&v, c.scal + idx, sizeof(double), cudaMemcpyDeviceToHost, c.st);
    const cudaError_t e2 = cudaStreamSynchronize(c.st);
    if (e != cudaSuccess || e2 != cudaSuccess) *rc = H2_ECUDA;
    return v;
}

}  // namespace

extern "C" int h2_cg_solve(h2_handle h, double sigma2, const double *b, double *x, double tol, int maxit,
                           int *iters, double *true_relres, void *cuda_stream)
{
    h2n::Range range("h2_cg_solve");
    if (iters) *iters = 0;
    if (true_relres) *true_relres = 0.0;
    if (!h || !b || !x || maxit < 0 || !(tol >= 0) || !(sigma2 >= 0)) return H2_EINVAL;
    h2_info info;
    h2_get_info(h, &info);
    if (info.uploaded_prec < 0) return H2_ESTATE;
    const bool fp64 = info.uploaded_prec == H2_FP64;
    CgState c{};
    c.n = info.n;
    c.st = static_cast<cudaStream_t>(cuda_stream);
    const size_t nd = size_t(c.n) * sizeof(double), nf = size_t(c.n) * sizeof(float);
    const size_t bytes = 3 * nd + (fp64 ? 0 : 2 * nf) + kDotBlocks * sizeof(double) + 8 * sizeof(double) + 1024;
    if (cudaMalloc(&c.mem, bytes) != cudaSuccess) {
        cudaGetLastError();
        return H2_ENOMEM;
    }
    char *m = static_cast<char *>(c.mem);
    c.r = reinterpret_cast<double *>(m);
    c.p = reinterpret_cast<double *>(m + nd);
    c.Ap = reinterpret_cast<double *>(m + 2 * nd);
    c.partial = reinterpret_cast<double *>(m + 3 * nd);
    c.scal = c.partial + kDotBlocks;
    c.pf = fp64 ? nullptr : reinterpret_cast<float *>(m + 3 * nd + (kDotBlocks + 8) * sizeof(double) + 256);
    c.Apf = fp64 ? nullptr : c.pf + c.n + 64;
    int rc = H2_OK;

    // r = b - (A + sigma2 I) x0; p = r; rr = r.r; bb = b.b
    rc = apply(h, c, x, c.Ap, sigma2, fp64);
    if (rc == H2_OK) {
        k_residual<<<grid_for(c.n), kThreads, 0, c.st>>>(b, c.Ap, c.r, c.p, c.n);
        dot(c, c.r, c.r, c.scal + 0);
        dot(c, b, b, c.scal + 3);
    }
    const double bb = rc == H2_OK ? read_scalar(c, 3, &rc) : 0.0;
    double rr = rc == H2_OK ? read_scalar(c, 0, &rc) : 0.0;
    int it = 0;
    bool converged = false;
    if (rc == H2_OK) {
        if (bb == 0.0) {
            // b = 0: the solution is x = 0
            cudaMemsetAsync(x, 0, nd, c.st);
            converged = true;
            rr = 0.0;
        } else if (std::sqrt(rr / bb) < tol) {
            converged = true;
        }
    }
    while (rc == H2_OK && !converged && it < maxit) {
        rc = apply(h, c, c.p, c.Ap, sigma2, fp64);
        if (rc != H2_OK) break;
        dot(c, c.p, c.Ap, c.scal + 1);
        k_update_xr<<<grid_for(c.n), kThreads, 0, c.st>>>(x, c.r, c.p, c.Ap, c.scal, c.n);
        dot(c, c.r, c.r, c.scal + 2);
        ++it;
        const double rr_new = read_scalar(c, 2, &rc);
        if (rc != H2_OK) break;
        if (!std::isfinite(rr_new)) {
            rc = H2_ENOTCONV;  // breakdown (the operator is not positive definite in this precision)
            break;
        }
        if (std::sqrt(rr_new / bb) < tol) {
            converged = true;
            break;
        }
        k_update_p<<<grid_for(c.n), kThreads, 0, c.st>>>(c.p, c.r, c.scal, c.n);
        k_copy_scalar<<<1, 1, 0, c.st>>>(c.scal, 0, 2);
        rr = rr_new;
    }
    // true residual |b - (A + sigma2 I) x| / |b|, recomputed with one more product
    if ((rc == H2_OK || rc == H2_ENOTCONV) && bb > 0.0) {
        int rc2 = apply(h, c, x, c.Ap, sigma2, fp64);
        if (rc2 == H2_OK) {
            k_residual<<<grid_for(c.n), kThreads, 0, c.st>>>(b, c.Ap, c.r, nullptr, c.n);
            dot(c, c.r, c.r, c.scal + 2);
            const double res = read_scalar(c, 2, &rc2);
            if (true_relres) *true_relres = std::sqrt(res / bb);
        }
        if (rc2 != H2_OK) rc = rc2;
    }
    if (rc == H2_OK && !converged) rc = H2_ENOTCONV;
    if (iters) *iters = it;
    cudaStreamSynchronize(c.st);
    cudaFree(c.mem);
    return rc;
}
