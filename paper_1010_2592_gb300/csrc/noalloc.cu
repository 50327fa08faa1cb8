// fa_apply_A_noalloc: out = A in (FP64) without any device allocation.
//
// Who needs this: callers that must not have the library allocate device
// memory on their behalf.  A caller recording a CUDA graph under global
// stream-capture mode cannot call cudaMalloc (the runtime rejects it while
// the capture is open), and a caller whose device memory is owned by a
// framework's caching allocator or a fixed budget wants no hidden
// cudaMalloc/cudaFree that could fail or fragment that budget.  fa_apply_A
// grows per-context scratch buffers on first use; this variant instead keeps
// its two working spinors in one file-scope device array whose size is fixed
// when the library is loaded.
//
// Limits: lattices up to kNoAllocMaxSites = 8192 sites (8^3 x 16); larger
// ones are rejected with FA_EINVAL before any device work.  The array
// (2 x 12 x 8192 complex doubles = 3 MiB) is resident on every GPU that loads
// the library until the process exits.  All calls share it: calls that
// overlap on a GPU (other streams, other contexts on the same device) race
// on it and must be serialised by the caller.  Nothing in it needs clearing
// between calls: each call writes every element it later reads.
#include <cmath>
#include <mutex>

#include "fa_context.h"

namespace fa {

constexpr int kNoAllocMaxSites = 8192;
constexpr int kNoAllocMaxDevices = 64;

// two internal-layout FP64 spinors: [2][12][kNoAllocMaxSites] double2
static __device__ __align__(256) double2 g_noalloc_scratch[2 * 12 * kNoAllocMaxSites];

// Device address of g_noalloc_scratch per device, resolved once per device
// with that device current.  In host code the symbol itself is only a
// stand-in for the device array, never a usable device pointer.
static void* g_scratch_addr[kNoAllocMaxDevices] = {};
static std::mutex g_scratch_mu;

static int scratch_address(int device, double2** out) {
    if (device < 0 || device >= kNoAllocMaxDevices) {
        set_error("fa_apply_A_noalloc: device %d beyond the supported %d", device, kNoAllocMaxDevices);
        return FA_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (g_scratch_addr[device] == nullptr) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            return cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                             "fa_apply_A_noalloc: cudaGetSymbolAddress");
        g_scratch_addr[device] = p;
    }
    *out = static_cast<double2*>(g_scratch_addr[device]);
    return FA_OK;
}

}  // namespace fa

using namespace fa;

extern "C" int fa_apply_A_noalloc(fa_ctx* c, const double* in, double* out, int dagger) {
    if (!c || !in || !out || in == out) return FA_EINVAL;
    if (c->g.V > kNoAllocMaxSites) {
        set_error("fa_apply_A_noalloc: lattice of %d sites exceeds the static scratch limit of %d sites",
                  c->g.V, kNoAllocMaxSites);
        return FA_EINVAL;
    }
    if (!c->have_gauge || !c->have_params) return FA_ESTATE;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "fa_apply_A_noalloc: cudaGetDevice");
    if (dev != c->device) {
        set_error("fa_apply_A_noalloc: current device %d is not the context's device %d", dev, c->device);
        return FA_EINVAL;
    }
    double2* scratch = nullptr;
    int rc = scratch_address(dev, &scratch);
    if (rc != FA_OK) return rc;
    double2* a = scratch;                                   // packed input, later the packed result
    double2* t = scratch + (size_t)12 * kNoAllocMaxSites;   // g5 D in
    // A = c g5 D g5 D; A^H = A(-mu).  The hop kernels are launched directly,
    // so the call leaves the context's solver state and timing untouched.
    const double mu = dagger != 0 ? -c->mu : c->mu;
    const double ef = std::exp(mu), eb = std::exp(-mu), diag = 4.0 + c->mass;
    rc = launch_pack_spinor_f64(c->g, in, a, c->stream);
    if (rc == FA_OK)
        rc = launch_hop_f64(c->g, links64_of(c), a, t, diag, ef, eb, c->t_bc, 1.0, false, true, nullptr, nullptr,
                            nullptr, c->stream);
    if (rc == FA_OK)
        rc = launch_hop_f64(c->g, links64_of(c), t, a, diag, ef, eb, c->t_bc, c->scale_c, false, true, nullptr,
                            nullptr, nullptr, c->stream);
    if (rc == FA_OK) rc = launch_unpack_spinor_f64(c->g, a, out, c->stream);
    if (rc != FA_OK) return rc;   // the launch error is recorded for fa_last_error
    c->launches += 4;
    return FA_OK;
}
