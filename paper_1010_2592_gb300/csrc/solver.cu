// Host driver of multi-shift BiCGstab(l): single-pass (shift vectors updated
// alongside the seed) and the double-pass form of Sec. 2 (pass 1: seed
// recurrence + scalars only; backward sweep over the recorded per-shift
// operations gives the weight of every seed-vector occurrence in
// sum_s omega_s x_s, the resolved recursion of Eq. 3; pass 2: the seed
// recurrence is rerun with the recorded scalars and the weighted
// occurrences are summed into y).  Everything between "pack b" and "unpack y"
// runs in the kernels of solver_kernels.cuh and dslash.cu; the host only
// enqueues them and polls a done flag.
#include <cmath>
#include <cstring>
#include <algorithm>
#include <vector>

#include "fa_context.h"
#include "solver_kernels.cuh"

namespace fa {

static inline int ok(cudaError_t e, const char* what) { return e == cudaSuccess ? FA_OK : cuda_fail(e, what); }
#define FA_TRY(x)                      \
    do {                               \
        int _rc = (x);                 \
        if (_rc != FA_OK) return _rc;  \
    } while (0)
#define FA_CUDA(x, what) FA_TRY(ok((x), what))
#define FA_LAUNCHED(c, what)                                   \
    do {                                                       \
        (c)->launches++;                                       \
        cudaError_t _e = cudaGetLastError();                   \
        if (_e != cudaSuccess) return cuda_fail(_e, what);     \
    } while (0)

// ------------------------------------------------------------------ operator helpers
static void hop_timing_begin(fa_ctx* c, int kind) {
    if (!c->hop_timing) return;
    const size_t need = 2 * (c->hop_ev_used + 1);
    while (c->hop_ev.size() < need) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) { c->hop_timing = false; return; }
        c->hop_ev.push_back(e);
    }
    if (c->hop_ev_kind.size() < c->hop_ev_used + 1) c->hop_ev_kind.resize(c->hop_ev_used + 1);
    c->hop_ev_kind[c->hop_ev_used] = kind;
    cudaEventRecord(c->hop_ev[2 * c->hop_ev_used], c->stream);
}
static void hop_timing_end(fa_ctx* c) {
    if (!c->hop_timing) return;
    cudaEventRecord(c->hop_ev[2 * c->hop_ev_used + 1], c->stream);
    c->hop_ev_used++;
}
// after a stream synchronisation: fold the recorded pairs into the means
static void hop_timing_collect(fa_ctx* c) {
    for (size_t k = 0; k < c->hop_ev_used; ++k) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->hop_ev[2 * k], c->hop_ev[2 * k + 1]) == cudaSuccess) {
            c->hop_ms[c->hop_ev_kind[k]] += ms;
            c->hop_count[c->hop_ev_kind[k]] += 1;
        }
    }
    c->hop_ev_used = 0;
}

int hop_f64(fa_ctx* c, const double2* in, double2* out, double scale, bool g5in, bool g5out, bool dagger_mu,
            const double2* dot_with, double2* partials, const int* done) {
    const double mu = dagger_mu ? -c->mu : c->mu;
    hop_timing_begin(c, 0);
    int rc = launch_hop_f64(c->g, c->links64.as<double2>(), in, out, 4.0 + c->mass, std::exp(mu), std::exp(-mu),
                            c->t_bc, scale, g5in, g5out, dot_with, partials, done, c->stream);
    hop_timing_end(c);
    c->launches++;
    if (rc == FA_ECUDA) return cuda_fail(cudaGetLastError(), "hop_f64");
    return rc;
}

int hop_f32(fa_ctx* c, const float4* in, float4* out, double scale, bool g5in, bool g5out, bool dagger_mu,
            const float4* dot_with, double2* partials, const int* done) {
    const double mu = dagger_mu ? -c->mu : c->mu;
    hop_timing_begin(c, 1);
    int rc = launch_hop_f32(c->g, c->links32.as<float4>(), in, out, 4.0 + c->mass, std::exp(mu), std::exp(-mu),
                            c->t_bc, scale, g5in, g5out, dot_with, partials, done, c->stream);
    hop_timing_end(c);
    c->launches++;
    if (rc == FA_ECUDA) return cuda_fail(cudaGetLastError(), "hop_f32");
    return rc;
}

// A v = c g5 D g5 D v through the scratch spinor tmp; optional <dot_with, A v> partials.
static int apply_A_64(fa_ctx* c, const double2* in, double2* out, double2* tmp, const double2* dot_with,
                      double2* partials, const int* done, double scale) {
    FA_TRY(hop_f64(c, in, tmp, 1.0, false, true, false, nullptr, nullptr, done));
    return hop_f64(c, tmp, out, scale, false, true, false, dot_with, partials, done);
}
static int apply_A_32(fa_ctx* c, const float4* in, float4* out, float4* tmp, const float4* dot_with,
                      double2* partials, const int* done, double scale) {
    FA_TRY(hop_f32(c, in, tmp, 1.0, false, true, false, nullptr, nullptr, done));
    return hop_f32(c, tmp, out, scale, false, true, false, dot_with, partials, done);
}

// ------------------------------------------------------------------ small FP64 kernels
__global__ void k_sc_invnorm(const double2* part, int nblk, double* out) {
    const dcx v = reduce_partials(part, 1, nblk);
    if (threadIdx.x == 0) {
        out[0] = 1.0 / sqrt(v.r);
        out[1] = sqrt(v.r);
    }
}
__global__ void k_scale_f64(int n, double2* v, const double* s) {
    const int idx = blockIdx.x * kThreads + threadIdx.x;
    if (idx >= n) return;
    const double a = s[0];
    double2 t = v[idx];
    v[idx] = make_double2(t.x * a, t.y * a);
}

// ------------------------------------------------------------------ workspace
struct Layout {
    int L, ns, max_outer, V;
    bool need64, need32, single;
    size_t vs64, vs32;         // one spinor in elements of double2 / float4
    int nblk, red_grid, part_slots;
};

static int red_grid_for(int V) { return std::min(nblocks(V), 8 * 152); }

static int ensure_workspace(fa_ctx* c, const Layout& Lo) {
    const int V = Lo.V, L = Lo.L, ns = Lo.ns, MO = Lo.max_outer;
    const size_t s64 = (size_t)12 * V * sizeof(double2), s32 = (size_t)6 * V * sizeof(float4);
    FA_CUDA(c->partials.ensure((size_t)std::max(Lo.nblk, Lo.red_grid) * Lo.part_slots * sizeof(double2)),
            "alloc partials");
    FA_CUDA(c->state.ensure(sizeof(DevState)), "alloc state");
    FA_CUDA(c->shiftbuf.ensure((size_t)kMaxShifts * (2 * sizeof(double) + 2 * sizeof(double2) + 2 * sizeof(int))),
            "alloc shifts");
    FA_CUDA(c->rec.ensure((size_t)MO * (3 * L + 1) * sizeof(double2)), "alloc record");
    FA_CUDA(c->prec.ensure((size_t)ns * MO * ps_stride(L) * sizeof(double2)), "alloc shift record");
    FA_CUDA(c->coef.ensure((size_t)MO * nc_slots(L) * sizeof(double2)), "alloc weights");
    if (!Lo.single) FA_CUDA(c->cs.ensure((size_t)ns * MO * nc_slots(L) * sizeof(double2)), "alloc sweep");
    FA_CUDA(c->y64.ensure(s64), "alloc y");
    if (Lo.need64) {
        FA_CUDA(c->r64.ensure((L + 1) * s64), "alloc r64");
        FA_CUDA(c->u64.ensure((L + 1) * s64), "alloc u64");
        FA_CUDA(c->rt64.ensure(s64), "alloc rt64");
        FA_CUDA(c->tmp64.ensure(s64), "alloc tmp64");
    }
    if (Lo.need32) {
        FA_CUDA(c->r32.ensure((L + 1) * s32), "alloc r32");
        FA_CUDA(c->u32.ensure((L + 1) * s32), "alloc u32");
        FA_CUDA(c->rt32.ensure(s32), "alloc rt32");
        FA_CUDA(c->tmp32.ensure(s32), "alloc tmp32");
    }
    if (Lo.single) {
        FA_CUDA(c->xs64.ensure((size_t)ns * s64), "alloc shift solutions");
        FA_CUDA(c->us64.ensure((size_t)ns * (L + 1) * s64), "alloc shift directions");
    }
    if (!c->pinned) {
        FA_CUDA(cudaMallocHost(&c->pinned, 2 * sizeof(DevState)), "alloc pinned");
        c->pinned_bytes = 2 * sizeof(DevState);
    }
    return FA_OK;
}

static SolverDev make_dev(fa_ctx* c, const Layout& Lo) {
    SolverDev d{};
    d.st = c->state.as<DevState>();
    d.ns = Lo.ns;
    d.L = Lo.L;
    d.max_outer = Lo.max_outer;
    d.V = Lo.V;
    char* sb = c->shiftbuf.as<char>();
    d.sigma = reinterpret_cast<const double*>(sb);
    d.omega = reinterpret_cast<const double*>(sb + kMaxShifts * sizeof(double));
    d.zeta = reinterpret_cast<double2*>(sb + 2 * kMaxShifts * sizeof(double));
    d.zeta_p = d.zeta + kMaxShifts;
    d.active = reinterpret_cast<int*>(d.zeta_p + kMaxShifts);
    d.iters = d.active + kMaxShifts;
    double2* rb = c->rec.as<double2>();
    d.rec_alpha = rb;
    d.rec_beta = rb + (size_t)Lo.max_outer * Lo.L;
    d.rec_gamma = rb + (size_t)2 * Lo.max_outer * Lo.L;
    d.prec = c->prec.as<double2>();
    d.coef = c->coef.as<double2>();
    d.cs = Lo.single ? nullptr : c->cs.as<double2>();
    return d;
}

// ------------------------------------------------------------------ one outer iteration
// Pass 1 (pass2 = false): seed recurrence with inner products and the scalar
// kernels.  Pass 2 (pass2 = true): the same vector kernels with the recorded
// scalars, no inner products, and y accumulation.  single: shift vectors too.
template <typename R, int L>
static int enqueue_outer(fa_ctx* c, const Layout& Lo, const SolverDev& d, bool pass2, bool single, bool head,
                         void* store_v) {
    using T = typename Ch<R>::T;
    constexpr bool F64 = sizeof(R) == 8;
    T* r = F64 ? (T*)c->r64.p : (T*)c->r32.p;
    T* u = F64 ? (T*)c->u64.p : (T*)c->u32.p;
    T* rt = F64 ? (T*)c->rt64.p : (T*)c->rt32.p;
    T* tmp = F64 ? (T*)c->tmp64.p : (T*)c->tmp32.p;
    const size_t vs = F64 ? Lo.vs64 : Lo.vs32;
    T* store = static_cast<T*>(store_v);
    const int* done = pass2 ? nullptr : &d.st->done;
    double2* part = c->partials.as<double2>();
    double2* y = c->y64.as<double2>();
    double2* xs = single ? c->xs64.as<double2>() : nullptr;
    double2* us = single ? c->us64.as<double2>() : nullptr;
    const size_t svs = Lo.vs64;
    const int nb = Lo.nblk;
    cudaStream_t st = c->stream;

    auto A = [&](const T* in, T* out, const T* dotw) -> int {
        if constexpr (F64)
            return apply_A_64(c, (const double2*)in, (double2*)out, (double2*)tmp, (const double2*)dotw, part, done,
                              c->scale_c);
        else
            return apply_A_32(c, (const float4*)in, (float4*)out, (float4*)tmp, (const float4*)dotw, part, done,
                              c->scale_c);
    };

    for (int j = 0; j < L; ++j) {
        if (!pass2 && j > 0) {
            k_sc_beta<<<1, kScalarThreads, 0, st>>>(d, j, part, nb);
            FA_LAUNCHED(c, "k_sc_beta");
        }
        k_update_u<R><<<nb, kThreads, 0, st>>>(d, j, r, u, vs, done);
        FA_LAUNCHED(c, "k_update_u");
        FA_TRY(A(u + j * vs, u + (j + 1) * vs, pass2 ? nullptr : rt));
        if (!pass2) {
            k_sc_alpha<<<1, kScalarThreads, 0, st>>>(d, j, part, nb);
            FA_LAUNCHED(c, "k_sc_alpha");
        }
        if (pass2) {
            k_update_r<R, true, false><<<nb, kThreads, 0, st>>>(d, j, r, u, vs, y, nullptr, nullptr, svs, nullptr,
                                                                done);
        } else if (single) {
            if constexpr (F64)
                k_update_r<R, false, true><<<nb, kThreads, 0, st>>>(d, j, r, u, vs, nullptr, xs, us, svs, nullptr,
                                                                    done);
        } else {
            k_update_r<R, false, false><<<nb, kThreads, 0, st>>>(d, j, r, u, vs, nullptr, nullptr, nullptr, svs,
                                                                 store, done);
        }
        FA_LAUNCHED(c, "k_update_r");
        FA_TRY(A(r + j * vs, r + (j + 1) * vs, (!pass2 && j < L - 1) ? rt : nullptr));
    }
    const int rg = Lo.red_grid;
    if (!pass2) {
        k_gram<R, L><<<rg, kThreads, 0, st>>>(d, r, vs, part, done);
        FA_LAUNCHED(c, "k_gram");
        k_sc_mr<L><<<1, kScalarThreads, 0, st>>>(d, part, rg);
        FA_LAUNCHED(c, "k_sc_mr");
    }
    if (pass2) {
        k_mr<R, L, true, false, false><<<rg, kThreads, 0, st>>>(d, r, u, rt, vs, y, nullptr, nullptr, svs, nullptr,
                                                                 part, done);
    } else if (single) {
        if constexpr (F64)
            k_mr<R, L, false, true, true><<<rg, kThreads, 0, st>>>(d, r, u, rt, vs, nullptr, xs, us, svs, nullptr,
                                                                   part, done);
    } else {
        k_mr<R, L, false, false, true><<<rg, kThreads, 0, st>>>(d, r, u, rt, vs, nullptr, nullptr, nullptr, svs,
                                                                 store, part, done);
    }
    FA_LAUNCHED(c, "k_mr");
    if (!pass2) {
        k_sc_conv<<<1, kScalarThreads, 0, st>>>(d, part, rg, head ? 1 : 0);
        FA_LAUNCHED(c, "k_sc_conv");
    } else {
        k_advance<<<1, 1, 0, st>>>(d);
        FA_LAUNCHED(c, "k_advance");
    }
    return FA_OK;
}

template <int L>
static int enqueue_outer_p(fa_ctx* c, const Layout& Lo, const SolverDev& d, bool f64, bool pass2, bool single,
                           bool head, void* store) {
    return f64 ? enqueue_outer<double, L>(c, Lo, d, pass2, single, head, store)
               : enqueue_outer<float, L>(c, Lo, d, pass2, single, head, store);
}

static int enqueue_outer_any(fa_ctx* c, const Layout& Lo, const SolverDev& d, bool f64, bool pass2, bool single,
                             bool head, void* store = nullptr) {
    switch (Lo.L) {
        case 1: return enqueue_outer_p<1>(c, Lo, d, f64, pass2, single, head, store);
        case 2: return enqueue_outer_p<2>(c, Lo, d, f64, pass2, single, head, store);
        case 3: return enqueue_outer_p<3>(c, Lo, d, f64, pass2, single, head, store);
        case 4: return enqueue_outer_p<4>(c, Lo, d, f64, pass2, single, head, store);
        case 8: return enqueue_outer_p<8>(c, Lo, d, f64, pass2, single, head, store);
        default: return FA_EINVAL;
    }
}

static int launch_sweep(fa_ctx* c, const Layout& Lo, const SolverDev& d) {
    const int th = 32;
    const int bl = (Lo.ns + th - 1) / th;
    switch (Lo.L) {
        case 1: k_sweep<1><<<bl, th, 0, c->stream>>>(d); break;
        case 2: k_sweep<2><<<bl, th, 0, c->stream>>>(d); break;
        case 3: k_sweep<3><<<bl, th, 0, c->stream>>>(d); break;
        case 4: k_sweep<4><<<bl, th, 0, c->stream>>>(d); break;
        case 8: k_sweep<8><<<bl, th, 0, c->stream>>>(d); break;
        default: return FA_EINVAL;
    }
    FA_LAUNCHED(c, "k_sweep");
    return FA_OK;
}

// b (canonical) -> r_0 and rt of the requested precision, u_0 = 0
static int load_source(fa_ctx* c, const Layout& Lo, const double* b, bool f64) {
    if (f64) {
        FA_TRY(launch_pack_spinor_f64(c->g, b, c->r64.as<double2>(), c->stream));
        FA_CUDA(cudaMemcpyAsync(c->rt64.p, c->r64.p, (size_t)12 * Lo.V * sizeof(double2), cudaMemcpyDeviceToDevice,
                                c->stream), "copy rt");
        FA_CUDA(cudaMemsetAsync(c->u64.p, 0, (size_t)12 * Lo.V * sizeof(double2), c->stream), "zero u");
    } else {
        FA_TRY(launch_pack_spinor_f32(c->g, b, c->r32.as<float4>(), c->stream));
        FA_CUDA(cudaMemcpyAsync(c->rt32.p, c->r32.p, (size_t)6 * Lo.V * sizeof(float4), cudaMemcpyDeviceToDevice,
                                c->stream), "copy rt");
        FA_CUDA(cudaMemsetAsync(c->u32.p, 0, (size_t)6 * Lo.V * sizeof(float4), c->stream), "zero u");
    }
    c->launches += 3;
    return FA_OK;
}

// FP64 -> FP32 hand-over of the live seed vectors (r_0, u_0, rt) at an outer-iteration boundary
static int switch_to_f32(fa_ctx* c, const Layout& Lo) {
    FA_TRY(launch_convert_f64_to_f32(c->g, c->r64.as<double2>(), c->r32.as<float4>(), c->stream));
    FA_TRY(launch_convert_f64_to_f32(c->g, c->u64.as<double2>(), c->u32.as<float4>(), c->stream));
    FA_TRY(launch_convert_f64_to_f32(c->g, c->rt64.as<double2>(), c->rt32.as<float4>(), c->stream));
    c->launches += 3;
    return FA_OK;
}

static int read_state(fa_ctx* c, DevState* out) {
    FA_CUDA(cudaMemcpyAsync(out, c->state.p, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream), "read state");
    FA_CUDA(cudaStreamSynchronize(c->stream), "sync state");
    return FA_OK;
}

// ------------------------------------------------------------------ the solve
int solve(fa_ctx* c, const double* b, double* y_canon, double* const* xs_canon, const fa_solver_params* p,
          fa_solver_stats* stats) {
    if (!c->have_gauge || !c->have_params || !c->have_poles) return FA_ESTATE;
    const int L = p->ell;
    if (!(L == 1 || L == 2 || L == 3 || L == 4 || L == 8)) return FA_EINVAL;
    if (!(p->tol > 0.0) || p->max_outer < 1 || p->max_outer > 1000000) return FA_EINVAL;
    const bool single = p->mode == FA_SINGLE;
    const bool pseudo = p->mode == FA_PSEUDO;
    if (!single && !pseudo && p->mode != FA_DOUBLE) return FA_EINVAL;
    const int prec = p->precision;
    if (prec != FA_F64 && prec != FA_F32 && prec != FA_MIXED) return FA_EINVAL;
    if (single && prec != FA_F64) return FA_EINVAL;
    // FA_MIXED: switch_resid <= 0 selects the default 0.04 / l^2 (the FP32
    // error of the power-basis recurrence grows with l)
    const double switch_resid = (p->switch_resid > 0.0) ? p->switch_resid : 0.04 / ((double)L * L);
    if (prec == FA_MIXED && !(switch_resid < 1.0)) return FA_EINVAL;

    Layout Lo{};
    Lo.L = L;
    Lo.ns = c->ns;
    Lo.max_outer = p->max_outer;
    Lo.V = c->g.V;
    Lo.single = single;
    Lo.need64 = prec != FA_F32;
    Lo.need32 = prec != FA_F64;
    Lo.vs64 = (size_t)12 * Lo.V;
    Lo.vs32 = (size_t)6 * Lo.V;
    Lo.nblk = nblocks(Lo.V);
    Lo.red_grid = red_grid_for(Lo.V);
    Lo.part_slots = std::max(n_gram(L), 2);
    FA_TRY(ensure_workspace(c, Lo));
    SolverDev d = make_dev(c, Lo);
    cudaStream_t st = c->stream;
    const bool timing = (p->flags & 1) != 0;
    c->hop_timing = (p->flags & 2) != 0;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    if (timing)
        for (auto& e : ev) FA_CUDA(cudaEventCreate(&e), "event");

    // poles
    FA_CUDA(cudaMemcpyAsync((void*)d.sigma, c->sigma, Lo.ns * sizeof(double), cudaMemcpyHostToDevice, st), "poles");
    FA_CUDA(cudaMemcpyAsync((void*)d.omega, c->omega, Lo.ns * sizeof(double), cudaMemcpyHostToDevice, st), "poles");
    FA_CUDA(cudaMemsetAsync(c->y64.p, 0, (size_t)12 * Lo.V * sizeof(double2), st), "zero y");
    if (single) {
        FA_CUDA(cudaMemsetAsync(c->xs64.p, 0, (size_t)Lo.ns * 12 * Lo.V * sizeof(double2), st), "zero xs");
        FA_CUDA(cudaMemsetAsync(c->us64.p, 0, (size_t)Lo.ns * (L + 1) * 12 * Lo.V * sizeof(double2), st), "zero us");
    }
    // ---- pseudo-double-pass store (Sec. 2, option 2): pass 1 keeps the seed-vector
    // occurrences of a contiguous prefix [0, K) of outer iterations, as many as
    // the budget holds (FP64 slots while in FP64, FP32 slots after the switch)
    const int NC = nc_slots(L);
    const size_t s64 = Lo.vs64 * sizeof(double2), s32 = Lo.vs32 * sizeof(float4);
    const size_t per64 = (size_t)NC * s64, per32 = (size_t)NC * s32;
    long long cap64 = 0, cap32 = 0;
    if (pseudo) {
        size_t fb = 0, tb = 0;
        FA_CUDA(cudaMemGetInfo(&fb, &tb), "memory info");
        const double held = (double)c->store64.bytes + (double)c->store32.bytes;
        double budget = p->store_gb > 0.0 ? p->store_gb * 1e9 : std::min(0.25 * ((double)fb + held), 16e9);
        budget = std::min(budget, 0.9 * ((double)fb + held));
        if (prec == FA_F64) {
            cap64 = (long long)std::min<double>(Lo.max_outer, budget / per64);
        } else if (prec == FA_F32) {
            cap32 = (long long)std::min<double>(Lo.max_outer, budget / per32);
        } else {
            cap64 = (long long)std::min<double>(std::min(Lo.max_outer, 64), 0.4 * budget / per64);
            cap32 = (long long)std::min<double>(Lo.max_outer, (budget - (double)cap64 * per64) / per32);
        }
        cap64 = std::max(0LL, cap64);
        cap32 = std::max(0LL, cap32);
        if (cap64 > 0) FA_CUDA(c->store64.ensure((size_t)cap64 * per64), "alloc occurrence store");
        if (cap32 > 0) FA_CUDA(c->store32.ensure((size_t)cap32 * per32), "alloc occurrence store");
        if (Lo.need64) FA_CUDA(c->snap64.ensure(3 * s64), "alloc snapshot");
        if (Lo.need32) FA_CUDA(c->snap32.ensure(3 * s32), "alloc snapshot");
    }
    int K = pseudo ? -1 : 0;            // first outer iteration not stored (-1: still storing)
    int m0_32 = prec == FA_F32 ? 0 : -1;  // first FP32 outer iteration
    bool snap_f64 = true;
    int snap_rc = FA_OK;
    // r_0, u_0, rt of the current precision -> snapshot (pass 2 restarts from it)
    auto snapshot = [&](bool f64now) {
        snap_f64 = f64now;
        const size_t sb = f64now ? s64 : s32;
        char* dst = f64now ? c->snap64.as<char>() : c->snap32.as<char>();
        void* src[3] = {f64now ? c->r64.p : c->r32.p, f64now ? c->u64.p : c->u32.p, f64now ? c->rt64.p : c->rt32.p};
        for (int k = 0; k < 3; ++k)
            if (cudaMemcpyAsync(dst + k * sb, src[k], sb, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                snap_rc = cuda_fail(cudaGetLastError(), "snapshot");
    };
    auto store_for = [&](int m, bool f64now) -> void* {
        if (K >= 0) return nullptr;
        void* ptr = nullptr;
        if (f64now && m < cap64) ptr = c->store64.as<char>() + (size_t)m * per64;
        if (!f64now && m0_32 >= 0 && m - m0_32 < cap32) ptr = c->store32.as<char>() + (size_t)(m - m0_32) * per32;
        if (!ptr) {
            K = m;
            snapshot(f64now);
        }
        return ptr;
    };
    if (timing) cudaEventRecord(ev[0], st);

    // ---- pass 1
    bool f64 = prec != FA_F32;
    bool head = prec == FA_MIXED;
    FA_TRY(load_source(c, Lo, b, f64));
    if (f64)
        k_dot2<double><<<Lo.red_grid, kThreads, 0, st>>>(Lo.V, c->rt64.as<double2>(), c->r64.as<double2>(),
                                                          c->partials.as<double2>());
    else
        k_dot2<float><<<Lo.red_grid, kThreads, 0, st>>>(Lo.V, c->rt32.as<float4>(), c->r32.as<float4>(),
                                                         c->partials.as<double2>());
    FA_LAUNCHED(c, "k_dot2");
    k_sc_init<<<1, kScalarThreads, 0, st>>>(d, c->partials.as<double2>(), Lo.red_grid, p->tol,
                                            prec == FA_MIXED ? switch_resid : 0.0);
    FA_LAUNCHED(c, "k_sc_init");

    DevState hs{};
    int switch_outer = -1;
    int enq = 0;
    // FP64 head of FA_MIXED: one outer iteration at a time until the switch
    while (head && enq < Lo.max_outer) {
        FA_TRY(enqueue_outer_any(c, Lo, d, true, false, single, true, store_for(enq, true)));
        ++enq;
        FA_TRY(read_state(c, &hs));
        if (hs.done) break;
        if (hs.switch_req) {
            FA_TRY(switch_to_f32(c, Lo));
            switch_outer = hs.m;
            m0_32 = switch_outer;
            head = false;
            f64 = false;
        }
    }
    if (!hs.done) {
        // main loop: chunks of outer iterations, polling the previous chunk's flag
        const int chunk = Lo.V >= (1 << 17) ? 2 : 8;
        DevState* pin = static_cast<DevState*>(c->pinned);
        cudaEvent_t pe[2];
        FA_CUDA(cudaEventCreateWithFlags(&pe[0], cudaEventDisableTiming), "event");
        FA_CUDA(cudaEventCreateWithFlags(&pe[1], cudaEventDisableTiming), "event");
        int k = 0;
        bool stop = false;
        int rc = FA_OK;
        while (!stop && enq < Lo.max_outer) {
            for (int i = 0; i < chunk && enq < Lo.max_outer; ++i, ++enq) {
                rc = enqueue_outer_any(c, Lo, d, f64, false, single, false, store_for(enq, f64));
                if (rc != FA_OK) break;
            }
            if (rc != FA_OK) break;
            cudaMemcpyAsync(&pin[k & 1], c->state.p, sizeof(DevState), cudaMemcpyDeviceToHost, st);
            cudaEventRecord(pe[k & 1], st);
            if (k > 0) {
                cudaEventSynchronize(pe[(k - 1) & 1]);
                if (pin[(k - 1) & 1].done) stop = true;
            }
            ++k;
        }
        cudaEventDestroy(pe[0]);
        cudaEventDestroy(pe[1]);
        FA_TRY(rc);
        FA_TRY(read_state(c, &hs));
    }
    if (timing) cudaEventRecord(ev[1], st);
    const int M = hs.n_outer;
    int status = hs.status;
    if (status == FA_OK && !hs.done) status = FA_ENOCONV;

    FA_TRY(snap_rc);
    const int Kst = pseudo ? (K < 0 ? M : std::min(K, M)) : 0;   // stored prefix

    // ---- backward sweep, gather of the stored prefix, pass 2 for the rest
    if (status == FA_OK && !single) {
        FA_CUDA(cudaMemsetAsync(c->cs.p, 0, (size_t)Lo.ns * Lo.max_outer * nc_slots(L) * sizeof(double2), st),
                "zero sweep");
        FA_TRY(launch_sweep(c, Lo, d));
        const int n = M * nc_slots(L);
        k_coef_reduce<<<(n + 255) / 256, 256, 0, st>>>(d, M);
        FA_LAUNCHED(c, "k_coef_reduce");
        if (timing) cudaEventRecord(ev[2], st);
        if (Kst > 0) {
            // FP64 slots cover [0, end64), FP32 slots [m0_32, Kst)
            const int end64 = prec == FA_F64 ? Kst : (prec == FA_MIXED ? (m0_32 >= 0 ? std::min(Kst, m0_32) : Kst) : 0);
            if (end64 > 0) {
                k_gather<double><<<Lo.nblk, kThreads, 0, st>>>(d, c->store64.as<double2>(), Lo.vs64, 0, end64, 0,
                                                                c->y64.as<double2>());
                FA_LAUNCHED(c, "k_gather<double>");
            }
            if (m0_32 >= 0 && Kst > m0_32) {
                k_gather<float><<<Lo.nblk, kThreads, 0, st>>>(d, c->store32.as<float4>(), Lo.vs32, m0_32, Kst, m0_32,
                                                               c->y64.as<double2>());
                FA_LAUNCHED(c, "k_gather<float>");
            }
        }
        const int mstart = Kst;
        if (mstart < M) {
            bool p2f64 = prec == FA_F64 || (prec == FA_MIXED && (switch_outer < 0 || mstart < switch_outer));
            if (mstart == 0) {
                FA_TRY(load_source(c, Lo, b, p2f64));
            } else {
                // restart from the snapshot taken before outer iteration K
                if (snap_f64 != p2f64) return FA_ESTATE;
                const size_t sb = p2f64 ? s64 : s32;
                const char* src = p2f64 ? c->snap64.as<char>() : c->snap32.as<char>();
                void* dst[3] = {p2f64 ? c->r64.p : c->r32.p, p2f64 ? c->u64.p : c->u32.p, p2f64 ? c->rt64.p : c->rt32.p};
                for (int k = 0; k < 3; ++k)
                    FA_CUDA(cudaMemcpyAsync(dst[k], src + k * sb, sb, cudaMemcpyDeviceToDevice, st), "restore");
            }
            k_set_m<<<1, 1, 0, st>>>(d, mstart);
            FA_LAUNCHED(c, "k_set_m");
            for (int m = mstart; m < M; ++m) {
                if (p2f64 && prec == FA_MIXED && m == switch_outer) {
                    FA_TRY(switch_to_f32(c, Lo));
                    p2f64 = false;
                }
                FA_TRY(enqueue_outer_any(c, Lo, d, p2f64, true, false, false));
            }
        }
        if (timing) cudaEventRecord(ev[3], st);
        FA_TRY(launch_unpack_spinor_f64(c->g, c->y64.as<double2>(), y_canon, st));
        c->launches++;
    } else if (status == FA_OK && single) {
        if (timing) { cudaEventRecord(ev[2], st); cudaEventRecord(ev[3], st); }
        if (y_canon) {
            k_combine<<<(12 * Lo.V + kThreads - 1) / kThreads, kThreads, 0, st>>>(
                Lo.V, Lo.ns, d.omega, c->xs64.as<double2>(), Lo.vs64, c->y64.as<double2>());
            FA_LAUNCHED(c, "k_combine");
            FA_TRY(launch_unpack_spinor_f64(c->g, c->y64.as<double2>(), y_canon, st));
            c->launches++;
        }
        if (xs_canon) {
            for (int s = 0; s < Lo.ns; ++s) {
                FA_TRY(launch_unpack_spinor_f64(c->g, c->xs64.as<double2>() + (size_t)s * Lo.vs64, xs_canon[s], st));
                c->launches++;
            }
        }
    }
    FA_CUDA(cudaStreamSynchronize(st), "sync solve");
    if (c->hop_timing) hop_timing_collect(c);
    c->hop_timing = false;

    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->status = status;
        stats->outer_iters = M;
        stats->switch_outer = switch_outer;
        stats->ns = Lo.ns;
        int iters[kMaxShifts];
        FA_CUDA(cudaMemcpy(iters, d.iters, Lo.ns * sizeof(int), cudaMemcpyDeviceToHost), "read iters");
        for (int s = 0; s < Lo.ns; ++s) stats->iters_per_shift[s] = iters[s];
        stats->resid_recurrence = std::sqrt(hs.rnorm2 / hs.bnorm2);
        const long long per = 2LL * L * M;
        stats->n_mv = single ? per : per + 2LL * L * (M - Kst);
        stats->stored_outer = Kst;
        stats->n_dot = (long long)M * (L * (L + 7) / 2 + 1);
        stats->n_launch = c->launches;
        if (timing) {
            float a = 0.f, b2 = 0.f, c2 = 0.f;
            cudaEventElapsedTime(&a, ev[0], ev[1]);
            cudaEventElapsedTime(&b2, ev[1], ev[2]);
            cudaEventElapsedTime(&c2, ev[2], ev[3]);
            stats->t_pass1_ms = a;
            stats->t_sweep_ms = b2;
            stats->t_pass2_ms = c2;
        }
    }
    if (timing)
        for (auto& e : ev) cudaEventDestroy(e);
    return status;
}

// ------------------------------------------------------------------ adjoint gradient
// L = Re <eta, y>, y = sum_s omega_s x_s, x_s = (A + sigma_s)^{-1} b.
// dL = -Re sum_s omega_s <lambda_s, dA x_s>, lambda_s = (A^H + sigma_s)^{-1} eta with
// A^H = A(-mu); <lambda, dA x> = c [<g5 lambda, dD (g5 D x)> + <D(-mu) lambda, dD x>]
// (c held fixed).  x_s and lambda_s come from two single-pass FP64 solves (the
// forward solution is recomputed here rather than stored by the forward call).
int grad(fa_ctx* c, const double* b, const double* eta, double* dLdU, double* dLdmu, double* L, double* dLdb,
         const fa_solver_params* p, fa_solver_stats* stats) {
    if (!c->have_gauge || !c->have_params || !c->have_poles) return FA_ESTATE;
    if (!b || !eta || !dLdU || !dLdmu || !L || !p) return FA_EINVAL;
    fa_solver_params ps = *p;
    ps.mode = FA_SINGLE;
    ps.precision = FA_F64;
    fa_solver_stats st1{}, st2{};
    FA_TRY(solve(c, b, nullptr, nullptr, &ps, &st1));
    const int V = c->g.V, ns = c->ns;
    const size_t vs = (size_t)12 * V;
    const size_t sb = vs * sizeof(double2);
    cudaStream_t st = c->stream;
    FA_CUDA(c->gx.ensure(ns * sb), "alloc gradient");
    FA_CUDA(cudaMemcpyAsync(c->gx.p, c->xs64.p, ns * sb, cudaMemcpyDeviceToDevice, st), "save x_s");
    const double mu0 = c->mu;
    c->mu = -mu0;
    const int rc2 = solve(c, eta, nullptr, nullptr, &ps, &st2);
    c->mu = mu0;
    FA_TRY(rc2);
    const int nb = nblocks(V), rg = red_grid_for(V);
    FA_CUDA(c->io64a.ensure(sb), "alloc");
    FA_CUDA(c->io64b.ensure(sb), "alloc");
    FA_CUDA(c->gpart.ensure(((size_t)ns * nb + 2 * (size_t)rg) * sizeof(double2)), "alloc");
    FA_CUDA(cudaMemsetAsync(dLdU, 0, (size_t)V * 72 * sizeof(double), st), "zero dL/dU");
    double2* gxs = c->gx.as<double2>();
    double2* lam = c->xs64.as<double2>();
    double2* t1 = c->io64a.as<double2>();
    double2* t2 = c->io64b.as<double2>();
    double2* part = c->gpart.as<double2>();
    for (int s = 0; s < ns; ++s) {
        const double2* xs = gxs + s * vs;
        const double2* ls = lam + s * vs;
        FA_TRY(hop_f64(c, xs, t1, 1.0, false, true, false, nullptr, nullptr, nullptr));   // g5 D x
        FA_TRY(hop_f64(c, ls, t2, 1.0, false, false, true, nullptr, nullptr, nullptr));   // D(-mu) lambda
        FA_TRY(launch_force(c->g, c->links64.as<double2>(), ls, t1, t2, xs, dLdU, -c->scale_c * c->omega[s],
                            std::exp(c->mu), std::exp(-c->mu), c->t_bc, part + (size_t)s * nb, st));
        c->launches++;
    }
    // y = sum omega x, L = Re <eta, y>; dL/db = sum omega lambda
    // the pole weights omega were uploaded by the solves (shift buffer, after sigma)
    const double* om_dev = reinterpret_cast<const double*>(c->shiftbuf.as<char>() + kMaxShifts * sizeof(double));
    k_combine<<<(12 * V + kThreads - 1) / kThreads, kThreads, 0, st>>>(V, ns, om_dev, gxs, vs, c->y64.as<double2>());
    FA_LAUNCHED(c, "k_combine");
    FA_TRY(launch_pack_spinor_f64(c->g, eta, t1, st));
    k_dot2<double><<<rg, kThreads, 0, st>>>(V, t1, c->y64.as<double2>(), part + (size_t)ns * nb);
    FA_LAUNCHED(c, "k_dot2");
    if (dLdb) {
        k_combine<<<(12 * V + kThreads - 1) / kThreads, kThreads, 0, st>>>(V, ns, om_dev, lam, vs, t2);
        FA_LAUNCHED(c, "k_combine");
        FA_TRY(launch_unpack_spinor_f64(c->g, t2, dLdb, st));
    }
    std::vector<double2> h((size_t)ns * nb + 2 * (size_t)rg);
    FA_CUDA(cudaMemcpyAsync(h.data(), part, h.size() * sizeof(double2), cudaMemcpyDeviceToHost, st), "read partials");
    FA_CUDA(cudaStreamSynchronize(st), "sync gradient");
    double dmu = 0.0, lre = 0.0;
    for (size_t k = 0; k < (size_t)ns * nb; ++k) dmu += h[k].x;
    for (int k = 0; k < rg; ++k) lre += h[(size_t)ns * nb + k].x;
    *dLdmu = dmu;
    *L = lre;
    if (stats) {
        *stats = st1;
        stats->n_mv += st2.n_mv;
        stats->n_dot += st2.n_dot;
        stats->outer_iters = st1.outer_iters + st2.outer_iters;
        stats->n_launch = c->launches;
    }
    return FA_OK;
}

// ------------------------------------------------------------------ power iteration for the scale c
int estimate_scale(fa_ctx* c, const double* v0, int iters, double* scale_out) {
    if (!c->have_gauge || !c->have_params) return FA_ESTATE;
    if (iters < 1 || !v0 || !scale_out) return FA_EINVAL;
    const int V = c->g.V;
    const size_t s64 = (size_t)12 * V * sizeof(double2);
    const int rg = red_grid_for(V);
    FA_CUDA(c->io64a.ensure(s64), "alloc");
    FA_CUDA(c->io64b.ensure(s64), "alloc");
    FA_CUDA(c->tmp64.ensure(s64), "alloc");
    FA_CUDA(c->partials.ensure((size_t)std::max(nblocks(V), rg) * 2 * sizeof(double2)), "alloc");
    FA_CUDA(c->state.ensure(sizeof(DevState)), "alloc");
    double2* v = c->io64a.as<double2>();
    double2* w = c->io64b.as<double2>();
    double* sc = reinterpret_cast<double*>(c->state.p);
    cudaStream_t st = c->stream;
    const int n = 12 * V, g = (n + kThreads - 1) / kThreads;
    FA_TRY(launch_pack_spinor_f64(c->g, v0, v, st));
    auto normalise = [&](double2* x) -> int {
        k_dot2<double><<<rg, kThreads, 0, st>>>(V, x, x, c->partials.as<double2>());
        FA_LAUNCHED(c, "k_dot2");
        k_sc_invnorm<<<1, kScalarThreads, 0, st>>>(c->partials.as<double2>(), rg, sc);
        FA_LAUNCHED(c, "k_sc_invnorm");
        k_scale_f64<<<g, kThreads, 0, st>>>(n, x, sc);
        FA_LAUNCHED(c, "k_scale_f64");
        return FA_OK;
    };
    FA_TRY(normalise(v));
    for (int it = 0; it < iters; ++it) {
        FA_TRY(apply_A_64(c, v, w, c->tmp64.as<double2>(), nullptr, nullptr, nullptr, 1.0));
        FA_TRY(normalise(w));
        std::swap(v, w);
    }
    FA_TRY(apply_A_64(c, v, w, c->tmp64.as<double2>(), nullptr, nullptr, nullptr, 1.0));
    k_dot2<double><<<rg, kThreads, 0, st>>>(V, w, w, c->partials.as<double2>());
    FA_LAUNCHED(c, "k_dot2");
    k_sc_invnorm<<<1, kScalarThreads, 0, st>>>(c->partials.as<double2>(), rg, sc);
    FA_LAUNCHED(c, "k_sc_invnorm");
    double h[2];
    FA_CUDA(cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, st), "read norm");
    FA_CUDA(cudaStreamSynchronize(st), "sync");
    if (!(h[1] > 0.0) || !std::isfinite(h[1])) return FA_ENONFINITE;
    *scale_out = 1.0 / h[1];
    return FA_OK;
}

}  // namespace fa
