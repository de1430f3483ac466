// h2_noalloc.cu -- H^2 product for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need a product: code that
// runs inside a memory-pool budget it may not grow, code that is itself called from an
// allocator or a memory-pressure handler (an allocation there can recurse or deadlock),
// and real-time loops where an allocation's device-wide synchronisation is not allowed.
// For them h2_matvec_noalloc runs the same product as h2_matvec_ws, with its workspace
// taken from one fixed scratch area that every GPU reserves when it loads this library
// and keeps until the process exits.
//
// The scratch area is a file-scope __device__ array. In host code its name is only a
// host-side stand-in, not a device address, so the address the kernels get is looked up
// once per device (with that device current) through cudaGetSymbolAddress.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/h2.h"
#include "h2_internal.h"

static __device__ __align__(256) unsigned char h2_noalloc_scratch[H2_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of this device's scratch area; looked up on the first call per device.
int scratch_address(int device, void **out)
{
    if (device < 0 || device >= kMaxDevices) return H2_EINVAL;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        // with lazy module loading this first lookup is what loads the module on this device
        // and reserves the scratch area, so it can fail for lack of device memory
        const cudaError_t e = cudaGetSymbolAddress(&p, h2_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? H2_ENOMEM : H2_ECUDA;
        }
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return H2_OK;
}

}  // namespace

extern "C" int h2_matvec_noalloc(h2_handle h, const void *X, void *Y, int nv, double alpha, double beta,
                                 void *cuda_stream)
{
    if (!h || !X || !Y || nv < 1) return H2_EINVAL;
    // the current device must hold the operator: its scratch area is the one the kernels get
    const int dc = h2_device_check(h);
    if (dc != H2_OK) return dc;
    const size_t need = h2_workspace_bytes(h, nv);
    if (need == 0) return H2_ESTATE;
    if (need > size_t(H2_NOALLOC_SCRATCH_BYTES)) return H2_EINVAL;  // operator too large for the scratch area
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return H2_ECUDA;
    }
    void *scratch = nullptr;
    const int rc = scratch_address(device, &scratch);
    if (rc != H2_OK) return rc;
    // the product's scheduling counters live in this workspace and are reset by the product
    // itself before use; everything else in it is fully overwritten by each product
    return h2_matvec_ws(h, X, Y, nv, alpha, beta, scratch, size_t(H2_NOALLOC_SCRATCH_BYTES), cuda_stream);
}
