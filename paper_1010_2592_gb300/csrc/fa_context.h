// Host-side context of libfapath (the opaque fa_ctx of the C-ABI).
#pragma once

#include <cuda_runtime.h>
#include <vector>
#include <string>

#include "fa_internal.cuh"

struct fa_ctx;

namespace fa {

// Device allocation that frees itself.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    // (re)allocate to at least n bytes; contents undefined
    cudaError_t ensure(size_t n) {
        if (bytes >= n && p) return cudaSuccess;
        release();
        cudaError_t e = cudaMalloc(&p, n);
        if (e != cudaSuccess) { p = nullptr; return e; }
        bytes = n;
        return cudaSuccess;
    }
    template <typename T> T* as() const { return static_cast<T*>(p); }
};

// An instantiated outer iteration.  (key, L, dev, n, V) select the entry;
// `sig` holds every value that the captured launches took as a kernel
// argument and that can change between solves on the same context (buffer
// addresses, operator scalars, link pointer, launch shape, launch attributes).
// An entry whose signature differs from the current one is re-captured.
struct GraphEntry {
    int key, L;
    void* dev;
    int n, V;
    cudaGraphExec_t exec;
    long long kernels;
    std::vector<unsigned long long> sig;
};

void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

}  // namespace fa

struct fa_ctx {
    fa::Geom g{};
    cudaStream_t stream = nullptr;
    int device = 0;

    // gauge field (own packed copy, or the packed copy of another context)
    fa::DevBuf links64, links32, linksdf;
    const fa_ctx* links_owner = nullptr;
    bool have_gauge = false;
    // operator parameters
    double mass = 0.0, mu = 0.0, t_bc = -1.0, scale_c = 1.0;
    bool have_params = false;
    // poles
    int ns = 0;
    double omega[fa::kMaxShifts] = {}, sigma[fa::kMaxShifts] = {};
    bool have_poles = false;

    // scratch of the operator entry points and the solver
    fa::DevBuf io64a, io64b, io32a, io32b, tmp64, tmp32;
    fa::DevBuf partials;                 // reduction partials
    fa::DevBuf state;                    // DevState
    fa::DevBuf shiftbuf;                 // sigma, omega, zeta, zeta_p, active, iters
    fa::DevBuf rec;                      // alpha, beta, gamma records
    fa::DevBuf prec, coef, cs;           // per-shift record, pass-2 weights, sweep output
    fa::DevBuf coef4;                    // pass-2 weights as FP32 pairs (gathers of FP32 / double-float stores)
    fa::DevBuf r64, u64, rt64, r32, u32, rt32;   // seed vectors (l+1 each, contiguous)
    fa::DevBuf y64;                      // accumulated result (FP64 internal)
    fa::DevBuf xs64, us64;               // single-pass shift vectors
    fa::DevBuf bhost_dev, yhost_dev;     // canonical staging for fa_apply_f_host
    fa::DevBuf gx, gpart;                // gradient: saved x_s, force partials
    fa::DevBuf store64, store32;         // pseudo-double-pass occurrence stores
    fa::DevBuf snap64, snap32;           // seed state at the first unstored outer iteration
    fa::DevBuf descbuf, flagbuf;         // batch descriptors and done flags (first context of a batch)
    fa::DevBuf tabbuf;                   // batch work tables and lattice groups (first context of a batch)
    int mrhs_rpb = 0, mrhs_mb = 0;       // multi-RHS FP32 sweep shape of batches led by this context (0: default)
    fa::DevBuf xrel, brel, snapx;        // reliable updates: seed solution, packed source, snapshot
    fa::DevBuf defl;                     // deflated sign: partial sums, coefficients, projected source
    fa::DevBuf eig;                      // eigensolver: Krylov basis, work spinors, partials
    std::vector<fa::GraphEntry> graphs;  // captured outer iterations
    void* pinned = nullptr;              // host copy of DevState
    size_t pinned_bytes = 0;

    long long launches = 0;
    // hop-kernel timing: index FP64 0, FP32 1, double-float 2; + 3 for the
    // sweeps that also form <dot_with, out> (and run a scalar step in a solve);
    // 6: the FP32 sweep with the Gram-matrix epilogue (the last of an outer iteration)
    double hop_ms[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    long long hop_count[7] = {0, 0, 0, 0, 0, 0, 0};
    bool hop_timing = false;
    int hop_shape = 0;                   // FP32 sweep launch shape (fa_hop_shape; 0: automatic)
    std::vector<cudaEvent_t> hop_ev;     // start/stop pairs, reused across solves
    std::vector<int> hop_ev_kind;        // timing index of each recorded pair
    size_t hop_ev_used = 0;              // pairs recorded since the last collection
    std::vector<int> hop_ev_outer;       // pass-1 outer iteration of each pair (-1: other)
    int hop_outer = -1;                  // outer iteration being enqueued in pass 1
};

namespace fa {
inline const double2* links64_of(const fa_ctx* c) {
    return c->links_owner ? c->links_owner->links64.as<double2>() : c->links64.as<double2>();
}
inline const float4* links32_of(const fa_ctx* c) {
    return c->links_owner ? c->links_owner->links32.as<float4>() : c->links32.as<float4>();
}
inline const float4* linksdf_of(const fa_ctx* c) {
    return c->links_owner ? c->links_owner->linksdf.as<float4>() : c->linksdf.as<float4>();
}
// operator application on internal layouts (used by the C-ABI and the solver)
int hop_f64(fa_ctx* c, const double2* in, double2* out, double scale, bool g5in, bool g5out, bool dagger_mu,
            const double2* dot_with, double2* partials, const int* done);
int hop_f32(fa_ctx* c, const float4* in, float4* out, double scale, bool g5in, bool g5out, bool dagger_mu,
            const float4* dot_with, double2* partials, const int* done);
int hop_df(fa_ctx* c, const float4* in, float4* out, double scale, bool g5in, bool g5out, bool dagger_mu,
           const float4* dot_with, double2* partials, const int* done);
int solve(fa_ctx* c, const double* b_canon, double* y_canon, double* const* xs_canon,
          const fa_solver_params* p, fa_solver_stats* stats);
int solve_batch(fa_ctx* const* ctxs, int n, const double* const* b, double* const* y_canon,
                double* const* xs_canon, const fa_solver_params* p, fa_solver_stats* stats);
int estimate_scale(fa_ctx* c, const double* v0, int iters, double* scale_out);
int eigs_smallest(fa_ctx* c, int k, int m, double tol, int max_restarts, const fa_solver_params* p,
                  unsigned long long seed, double* lambda, double* R, double* Lv, int* nconv, int* nsolve);
int autotune_batch(fa_ctx* const* ctxs, int n, int reps, int* rhs_per_block, int* min_blocks, double* times_ms,
                   int ntimes);
int apply_sign(fa_ctx* c, const double* b, double* out, const fa_solver_params* p, fa_solver_stats* stats,
               bool overlap);
int apply_sign_deflated(fa_ctx* c, const double* b, double* out, int k, const double* lambda, const double* R,
                        const double* Lv, bool overlap, const fa_solver_params* p, fa_solver_stats* stats);
int grad(fa_ctx* c, const double* b, const double* eta, double* dLdU, double* dLdmu, double* L, double* dLdb,
         const fa_solver_params* p, fa_solver_stats* stats);
}  // namespace fa
