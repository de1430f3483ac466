// h2_nvtx.h -- NVTX ranges (domain "h2") around the library's entry points and the phases of
// one product, so that timelines taken with NVIDIA's tools show which kernels belong to which
// call and phase. Without a tool attached a range costs one test of a function pointer.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace h2n {

inline nvtxDomainHandle_t domain()
{
    static const nvtxDomainHandle_t d = nvtxDomainCreateA("h2");
    return d;
}

// Scoped range on the calling thread (push on construction, pop on destruction).
struct Range {
    explicit Range(const char *name)
    {
        nvtxEventAttributes_t a{};
        a.version = NVTX_VERSION;
        a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
        a.messageType = NVTX_MESSAGE_TYPE_ASCII;
        a.message.ascii = name;
        nvtxDomainRangePushEx(domain(), &a);
    }
    ~Range() { nvtxDomainRangePop(domain()); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

}  // namespace h2n
