// Per-device launch configuration shared by the kernel launchers.
#include "ufvc_internal.h"

#include <map>
#include <mutex>
#include <utility>

namespace ufvc {

namespace {
std::mutex g_mu;
std::map<std::pair<const void*, int>, int> g_optin;  // (kernel, device) -> largest opt-in set there
std::map<int, int> g_sms;                            // device -> SM count
std::map<std::pair<const void*, int>, int> g_pairs;  // (kernel, device) -> co-resident CTA pairs
}  // namespace

cudaError_t smem_optin(const void* func, int bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_optin.find({func, dev});
    if (it != g_optin.end() && it->second >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) g_optin[{func, dev}] = bytes;
    return e;
}

int sm_count() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_sms.find(dev);
    if (it != g_sms.end()) return it->second;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return 148;
    g_sms[dev] = sms;
    return sms;
}

int max_pairs(const void* func, int smem, int threads) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_pairs.find({func, dev});
        if (it != g_pairs.end()) return it->second;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * sm_count());
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, func, &cfg) != cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    g_pairs[{func, dev}] = n;
    return n;
}

}  // namespace ufvc
