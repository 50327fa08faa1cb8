// Host side of the kernel timeline tracer (trace.cuh): included at the end of
// solver.cu, whose module holds the traced kernels and the tracer state.
#pragma once

#include <mutex>

namespace fa {

struct TraceHost {
    std::mutex mu;
    bool on = false;
    int device = -1;
    TraceRec* rec = nullptr;
    unsigned* pos = nullptr;      // [nsm + 1]: per-SM counts, then the dropped count
    size_t cap = 0;               // records allocated
    unsigned per_sm = 0, nsm = 0;
};
static TraceHost g_trace_host;

static int trace_install(const TraceState& ts) {
    const cudaError_t e = cudaMemcpyToSymbol(g_trace, &ts, sizeof(ts));
    return e == cudaSuccess ? FA_OK : cuda_fail(e, "trace: set tracer state");
}

}  // namespace fa

extern "C" int fa_trace_start(long long capacity) {
    using namespace fa;
    if (capacity < 1) return FA_EINVAL;
    TraceHost& H = g_trace_host;
    std::lock_guard<std::mutex> lock(H.mu);
    int dev = -1, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "fa_trace_start: device");
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || nsm < 1) return cuda_fail(e, "fa_trace_start: SM count");
    const unsigned per = (unsigned)std::min<long long>((capacity + nsm - 1) / nsm, 1ll << 24);
    const size_t need = (size_t)per * (size_t)nsm;
    if (H.device != dev || H.cap < need || H.nsm != (unsigned)nsm) {
        if (H.rec) {
            int cur = dev;
            if (H.device >= 0 && H.device != dev) cudaSetDevice(H.device);
            cudaFree(H.rec);
            cudaFree(H.pos);
            if (H.device >= 0 && H.device != dev) cudaSetDevice(cur);
            H.rec = nullptr;
            H.pos = nullptr;
            H.cap = 0;
        }
        if (cudaMalloc(&H.rec, need * sizeof(TraceRec)) != cudaSuccess ||
            cudaMalloc(&H.pos, (size_t)(nsm + 1) * sizeof(unsigned)) != cudaSuccess) {
            cudaGetLastError();
            if (H.rec) cudaFree(H.rec);
            H.rec = nullptr;
            H.pos = nullptr;
            set_error("fa_trace_start: no room for %zu trace records", need);
            return FA_ENOMEM;
        }
        H.cap = need;
        H.device = dev;
        H.nsm = (unsigned)nsm;
    }
    H.per_sm = per;
    e = cudaDeviceSynchronize();   // no traced kernel of a previous session still running
    if (e == cudaSuccess) e = cudaMemset(H.pos, 0, (size_t)(nsm + 1) * sizeof(unsigned));
    if (e != cudaSuccess) return cuda_fail(e, "fa_trace_start: clear");
    const int rc = trace_install(TraceState{H.rec, H.pos, H.pos + nsm, per, (unsigned)nsm});
    if (rc != FA_OK) return rc;
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "fa_trace_start: sync");
    H.on = true;
    return FA_OK;
}

extern "C" int fa_trace_stop(fa_trace_record* records, long long capacity, long long* n, long long* dropped) {
    using namespace fa;
    if (!records || !n || !dropped || capacity < 0) return FA_EINVAL;
    TraceHost& H = g_trace_host;
    std::lock_guard<std::mutex> lock(H.mu);
    if (!H.on) return FA_ESTATE;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "fa_trace_stop: device");
    if (dev != H.device) {
        set_error("fa_trace_stop: tracing runs on device %d, the current device is %d", H.device, dev);
        return FA_EINVAL;
    }
    e = cudaDeviceSynchronize();   // every traced block has written its record
    if (e != cudaSuccess) return cuda_fail(e, "fa_trace_stop: sync");
    int rc = trace_install(TraceState{nullptr, nullptr, nullptr, 0u, 1u});
    H.on = false;
    if (rc != FA_OK) return rc;
    std::vector<unsigned> pos(H.nsm + 1);
    e = cudaMemcpy(pos.data(), H.pos, pos.size() * sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "fa_trace_stop: read counts");
    long long copied = 0, lost = pos[H.nsm];
    for (unsigned sm = 0; sm < H.nsm; ++sm) {
        const long long have = std::min<long long>(pos[sm], H.per_sm);
        const long long take = std::min<long long>(have, capacity - copied);
        if (take > 0) {
            e = cudaMemcpy(records + copied, H.rec + (size_t)sm * H.per_sm, (size_t)take * sizeof(TraceRec),
                           cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(e, "fa_trace_stop: read records");
        }
        copied += std::max(0ll, take);
        lost += have - std::max(0ll, take);
    }
    *n = copied;
    *dropped = lost;
    return FA_OK;
}
