// Read-only sample of the current device's SM clock, for the timing table
// (a time means little without the clock it was measured at).  NVML is
// loaded at run time; without it (or without a device) the sample is 0.
// Nothing here changes any setting of the GPU.
#include "ct_internal.hpp"

#include <dlfcn.h>
#include <nvml.h>

namespace ct {

namespace {

struct Nvml {
    bool ok = false;
    nvmlReturn_t (*init)() = nullptr;
    nvmlReturn_t (*by_bus)(const char*, nvmlDevice_t*) = nullptr;
    nvmlReturn_t (*clock)(nvmlDevice_t, nvmlClockType_t, unsigned int*) = nullptr;
    Nvml()
    {
        void* h = dlopen("libnvidia-ml.so.1", RTLD_NOW | RTLD_LOCAL);
        if (!h) return;
        init = reinterpret_cast<decltype(init)>(dlsym(h, "nvmlInit_v2"));
        by_bus = reinterpret_cast<decltype(by_bus)>(dlsym(h, "nvmlDeviceGetHandleByPciBusId_v2"));
        clock = reinterpret_cast<decltype(clock)>(dlsym(h, "nvmlDeviceGetClockInfo"));
        ok = init && by_bus && clock && init() == NVML_SUCCESS;
    }
};

}  // namespace

int sample_sm_mhz()
{
    static Nvml nv;
    static std::mutex mu;
    static nvmlDevice_t handles[64] = {};
    static bool looked[64] = {};
    if (!nv.ok) return 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 0;
    }
    nvmlDevice_t d = nullptr;
    {
        std::lock_guard<std::mutex> g(mu);
        if (!looked[dev]) {
            looked[dev] = true;
            char bus[64] = {};
            if (cudaDeviceGetPCIBusId(bus, (int)sizeof bus, dev) != cudaSuccess || nv.by_bus(bus, &handles[dev]) !=
                                                                                        NVML_SUCCESS) {
                cudaGetLastError();
                handles[dev] = nullptr;
            }
        }
        d = handles[dev];
    }
    unsigned int mhz = 0;
    if (!d || nv.clock(d, NVML_CLOCK_SM, &mhz) != NVML_SUCCESS) return 0;
    return (int)mhz;
}

}  // namespace ct
