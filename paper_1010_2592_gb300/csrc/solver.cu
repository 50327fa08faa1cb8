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
#include <cstdint>
#include <cstring>
#include <algorithm>
#include <vector>
#include <type_traits>

#include "fa_context.h"
#include "fused_sweep.cuh"

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
    if (c->hop_ev_outer.size() < c->hop_ev_used + 1) c->hop_ev_outer.resize(c->hop_ev_used + 1);
    c->hop_ev_kind[c->hop_ev_used] = kind;
    c->hop_ev_outer[c->hop_ev_used] = c->hop_outer;
    cudaEventRecord(c->hop_ev[2 * c->hop_ev_used], c->stream);
}
static void hop_timing_end(fa_ctx* c) {
    if (!c->hop_timing) return;
    cudaEventRecord(c->hop_ev[2 * c->hop_ev_used + 1], c->stream);
    c->hop_ev_used++;
}
// after a stream synchronisation: fold the recorded pairs into the means.
// Pass-1 outer iterations from `m_run` on were enqueued ahead of the host's
// convergence poll and returned at once (the done flag): not counted.
static void hop_timing_collect(fa_ctx* c, int m_run = 1 << 30) {
    for (size_t k = 0; k < c->hop_ev_used; ++k) {
        if (c->hop_ev_outer[k] >= m_run) continue;
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
    hop_timing_begin(c, 0 + (dot_with ? 3 : 0));
    int rc = launch_hop_f64(c->g, links64_of(c), in, out, 4.0 + c->mass, std::exp(mu), std::exp(-mu),
                            c->t_bc, scale, g5in, g5out, dot_with, partials, done, c->stream);
    hop_timing_end(c);
    c->launches++;
    return rc;
}

int hop_f32(fa_ctx* c, const float4* in, float4* out, double scale, bool g5in, bool g5out, bool dagger_mu,
            const float4* dot_with, double2* partials, const int* done) {
    const double mu = dagger_mu ? -c->mu : c->mu;
    hop_timing_begin(c, 1 + (dot_with ? 3 : 0));
    int rc = launch_hop_f32(c->g, links32_of(c), in, out, 4.0 + c->mass, std::exp(mu), std::exp(-mu),
                            c->t_bc, scale, g5in, g5out, dot_with, partials, done, c->stream, c->hop_shape);
    hop_timing_end(c);
    c->launches++;
    return rc;
}

int hop_df(fa_ctx* c, const float4* in, float4* out, double scale, bool g5in, bool g5out, bool dagger_mu,
           const float4* dot_with, double2* partials, const int* done) {
    const double mu = dagger_mu ? -c->mu : c->mu;
    hop_timing_begin(c, 2 + (dot_with ? 3 : 0));
    int rc = launch_hop_df(c->g, linksdf_of(c), in, out, 4.0 + c->mass, std::exp(mu), std::exp(-mu), c->t_bc, scale,
                           g5in, g5out, dot_with, partials, done, c->stream);
    hop_timing_end(c);
    c->launches++;
    return rc;
}

// A v = c g5 D g5 D v through the scratch spinor tmp; optional <dot_with, A v> partials.
static int apply_A_64(fa_ctx* c, const double2* in, double2* out, double2* tmp, const double2* dot_with,
                      double2* partials, const int* done, double scale) {
    FA_TRY(hop_f64(c, in, tmp, 1.0, false, true, false, nullptr, nullptr, done));
    return hop_f64(c, tmp, out, scale, false, true, false, dot_with, partials, done);
}
// ------------------------------------------------------------------ small FP64 kernels
__global__ void k_sc_invnorm(const double2* part, int nblk, double* out) {
    __shared__ dcx red[2];
    reduce_slots<2, false>(part, nblk, 2, red);
    const dcx v = red[1];
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

// y += x over n double2 elements
__global__ void k_add_f64(int n, const double2* __restrict__ x, double2* __restrict__ y) {
    const int idx = blockIdx.x * kThreads + threadIdx.x;
    if (idx >= n) return;
    const double2 a = x[idx], t = y[idx];
    y[idx] = make_double2(t.x + a.x, t.y + a.y);
}

// Deflation on canonical spinors (n = 12 V complex elements each).
// part[i * gridDim.x + block] = partial sum of conj(V_i) b over the block's elements
__global__ void __launch_bounds__(kThreads) k_dots_canon(int n, const double2* __restrict__ V,
                                                         const double2* __restrict__ b, double2* __restrict__ part) {
    const double2* v = V + (size_t)blockIdx.y * n;
    double re = 0.0, im = 0.0;
    for (int e = blockIdx.x * kThreads + threadIdx.x; e < n; e += gridDim.x * kThreads) {
        const double2 x = v[e], y = b[e];
        re = fma(x.x, y.x, fma(x.y, y.y, re));
        im = fma(x.x, y.y, fma(-x.y, y.x, im));
    }
    __shared__ double sre[kThreads], sim[kThreads];
    const int t = threadIdx.x;
    sre[t] = re;
    sim[t] = im;
    __syncthreads();
    for (int h = kThreads / 2; h > 0; h >>= 1) {
        if (t < h) {
            sre[t] += sre[t + h];
            sim[t] += sim[t + h];
        }
        __syncthreads();
    }
    if (t == 0) part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = make_double2(sre[0], sim[0]);
}
// out[e] = base[e] + g(e) sum_i coef[i] V_i[e]; g(e) = -1 on spins 2, 3 (the
// canonical site holds 4 spins x 3 colours) when g5, else 1.  base may be out,
// or null (then out = the combination alone).
__global__ void __launch_bounds__(kThreads) k_lincomb_canon(int n, int k, const double2* __restrict__ coef,
                                                            const double2* __restrict__ V, const double2* base,
                                                            double2* out, int g5) {
    for (int e = blockIdx.x * kThreads + threadIdx.x; e < n; e += gridDim.x * kThreads) {
        double re = 0.0, im = 0.0;
        for (int i = 0; i < k; ++i) {
            const double2 a = coef[i], x = V[(size_t)i * n + e];
            re = fma(a.x, x.x, fma(-a.y, x.y, re));
            im = fma(a.x, x.y, fma(a.y, x.x, im));
        }
        if (g5 && (e % 12) >= 6) {
            re = -re;
            im = -im;
        }
        const double2 c = base != nullptr ? base[e] : make_double2(0.0, 0.0);
        out[e] = make_double2(c.x + re, c.y + im);
    }
}

// ------------------------------------------------------------------ workspace
struct Layout {
    int L, ns, max_outer, V;
    bool need64, need32, single;
    bool gram_hop;             // FP32 pass 1: the Gram matrix in the last sweep's epilogue (one system, l <= 4)
    size_t vs64, vs32;         // one spinor in elements of double2 / float4
    int nblk, red_grid, part_slots;
    int vgrid;                 // balanced vector kernels: kVecBlocks per SM
};

static int sms() {
    const int n = sm_count();
    return n > 0 ? n : 152;
}
static int red_grid_for(int V) { return std::min(nblocks(V), 8 * sms()); }

static int ensure_workspace(fa_ctx* c, const Layout& Lo) {
    const int V = Lo.V, L = Lo.L, ns = c->ns, MO = Lo.max_outer;
    const size_t s64 = (size_t)12 * V * sizeof(double2), s32 = (size_t)6 * V * sizeof(float4);
    // the Gram epilogue of the FP32 sweep writes n_gram(l) partials per block
    const size_t hop_blk = (size_t)std::max(nblocks(V), (V + kHopNarrowThreads - 1) / kHopNarrowThreads) + 1;
    FA_CUDA(c->partials.ensure(std::max({(size_t)std::max({Lo.nblk, Lo.red_grid, Lo.vgrid + 1}) * Lo.part_slots,
                                         (size_t)row_blocks(V), hop_blk * (size_t)Lo.part_slots}) *
                               sizeof(double2)),
            "alloc partials");
    FA_CUDA(c->state.ensure(sizeof(DevState)), "alloc state");
    FA_CUDA(c->shiftbuf.ensure((size_t)kMaxShifts * (2 * sizeof(double) + 2 * sizeof(double2) + 2 * sizeof(int))),
            "alloc shifts");
    FA_CUDA(c->rec.ensure((size_t)MO * (3 * L + 1) * sizeof(double2)), "alloc record");
    FA_CUDA(c->prec.ensure((size_t)ns * MO * ps_stride(L) * sizeof(double2)), "alloc shift record");
    FA_CUDA(c->coef.ensure((size_t)MO * nc_slots(L) * sizeof(double2)), "alloc weights");
    FA_CUDA(c->coef4.ensure((size_t)MO * nc_slots(L) * sizeof(float4)), "alloc weights");
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
        FA_CUDA(cudaMallocHost(&c->pinned, 4096), "alloc pinned");
        c->pinned_bytes = 4096;
    }
    return FA_OK;
}

static SolverDev make_dev(fa_ctx* c, const Layout& Lo) {
    SolverDev d{};
    d.st = c->state.as<DevState>();
    d.ns = c->ns;
    d.L = Lo.L;
    d.max_outer = Lo.max_outer;
    d.V = Lo.V;
    d.g = c->g;
    d.links64 = links64_of(c);
    d.links32 = links32_of(c);
    d.linksdf = linksdf_of(c);
    d.diag = 4.0 + c->mass;
    d.ef = std::exp(c->mu);
    d.eb = std::exp(-c->mu);
    d.bc = c->t_bc;
    d.scale = c->scale_c;
    d.fdiag1 = host_cvt<float>(1.0 * d.diag);
    d.fhop1 = host_cvt<float>(-0.5 * 1.0);
    d.fdiag2 = host_cvt<float>(d.scale * d.diag);
    d.fhop2 = host_cvt<float>(-0.5 * d.scale);
    d.fef = host_cvt<float>(d.ef);
    d.feb = host_cvt<float>(d.eb);
    d.fbc = host_cvt<float>(d.bc);
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
    d.coef4 = c->coef4.as<float4>();
    d.cs = Lo.single ? nullptr : c->cs.as<double2>();
    d.r64 = c->r64.as<double2>();
    d.u64 = c->u64.as<double2>();
    d.rt64 = c->rt64.as<double2>();
    d.tmp64 = c->tmp64.as<double2>();
    d.r32 = c->r32.as<float4>();
    d.u32 = c->u32.as<float4>();
    d.rt32 = c->rt32.as<float4>();
    d.tmp32 = c->tmp32.as<float4>();
    d.y = c->y64.as<double2>();
    d.xs = Lo.single ? c->xs64.as<double2>() : nullptr;
    d.us = Lo.single ? c->us64.as<double2>() : nullptr;
    d.store64 = nullptr;
    d.store32 = nullptr;
    d.cap64 = d.cap32 = 0;
    d.m0_32 = -1;
    d.nblk = Lo.nblk;
    d.red_grid = Lo.red_grid;
    d.part = c->partials.as<double2>();
    d.x64 = nullptr;
    d.b64 = nullptr;
    d.fixed_iters = 0;
    return d;
}

// Work tables of a batch launch (see `where` in solver_kernels.cuh): per kernel
// kind, one entry (system, block, vector blocks, tickets) per block of the launch.
enum TabKind { TB_VEC = 0, TB_VECX, TB_RG, TB_RGX, TB_HOP, TB_ROWS, TB_KINDS };

// A batch: systems whose kernels share each launch.  One system, or systems of
// one lattice shape without work tables (grid.y = systems), or systems of any
// shapes with work tables (grid.x = the table).
struct Batch {
    fa_ctx* c0 = nullptr;                 // owner of the stream and the descriptor array
    std::vector<fa_ctx*> sys;
    std::vector<SolverDev> host;          // host copy of the descriptors
    SolverDev* dev = nullptr;             // device array
    int* flags = nullptr;                 // device done flags
    Layout Lo{};                          // layout of system 0 (all systems without tables)
    std::vector<Layout> lo;               // layout of each system
    bool tables = false;                  // launches follow the work tables
    const int4* tab[TB_KINDS] = {};       // device tables
    int tab_n[TB_KINDS] = {};             // their lengths (blocks of the launch)
    const GroupDev* groups = nullptr;     // systems sharing a gauge field (multi-RHS FP32 sweep)
    const int4* items = nullptr;          // (group, tile, first, end) per block of that sweep
    int n_items = 0;
    int rhs_per_block = 1;
    int mrhs_min_blocks = kHopNarrowBlocks;
    std::vector<char> tab_host;           // staging of the tables (alive until the solve's final sync)
    int n = 0;
    bool use_graph = false;
    bool pdl = true;                      // programmatic dependent launch inside an outer iteration
};


// Kernel launch, with programmatic stream serialization when `pdl` is set: the
// kernel may then be placed on the SMs while its predecessor (a kernel) finishes,
// and it waits in dep_sync() before its first memory access.  Used only for
// kernels that call dep_sync() first and follow another kernel in the stream.
template <typename... KArgs, typename... Args>
static void launch(bool pdl, void (*k)(KArgs...), dim3 grid, int block, cudaStream_t st, Args... args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    (void)cudaLaunchKernelEx(&cfg, k, args...);   // errors surface through cudaGetLastError
}

static int upload(Batch& B) {
    FA_CUDA(cudaMemcpyAsync(B.dev, B.host.data(), B.n * sizeof(SolverDev), cudaMemcpyHostToDevice, B.c0->stream),
            "upload descriptors");
    return FA_OK;
}

static inline ScalarStep none_step() { return ScalarStep{STEP_NONE, 0}; }

// working precision of a stretch of outer iterations
enum Rp { RP64 = 0, RP32 = 1, RPDF = 2 };
template <typename R> constexpr int rp_of() {
    return std::is_same<R, double>::value ? RP64 : (std::is_same<R, float>::value ? RP32 : RPDF);
}

// ------------------------------------------------------------------ one outer iteration
// Pass 1 (pass2 = false): seed recurrence with inner products and the scalar
// kernels.  Pass 2 (pass2 = true): the same vector kernels with the recorded
// scalars, no inner products, and y accumulation.  single: shift vectors too.
// Each launch covers the whole batch (grid.y = systems).
template <typename R, int L>
static int enqueue_outer(Batch& B, bool pass2, bool single, bool head, bool reliable) {
    fa_ctx* c = B.c0;
    const int n = B.n, nb = B.Lo.nblk, rg = B.Lo.red_grid, vg = B.Lo.vgrid;
    const int p2 = pass2 ? 1 : 0;
    // The vector kernels run vg blocks (one site per thread while the lattice
    // fits one wave); their XS variants add the shift block, which finishes
    // early (taking one of the vector blocks for it would give the others 257
    // sites for 256 threads, a second pass for one thread of every block).
    // k_gram / k_mr use vg where their register budget gives kVecBlocks
    // resident blocks per SM, else the reduction grid.
    dim3 gs(nb, n), gv(vg, n), gvx(vg + 1, n);
    const bool gram_vec = gram_min_blocks<R, L>() >= kVecBlocks, mr_vec = mr_min_blocks<R, L>() >= kVecBlocks;
    dim3 gg(gram_vec ? vg : rg, n);
    const int mg = mr_vec ? vg : rg;
    dim3 gm(mg, n), gmx(mg + 1, n);
    // work tables (systems of different lattice shapes in one launch)
    const int4 *tv = nullptr, *tvx = nullptr, *tg = nullptr, *tm = nullptr, *tmx = nullptr;
    if (B.tables) {
        auto T = [&](int k, dim3& g, const int4*& t) {
            g = dim3(B.tab_n[k]);
            t = B.tab[k];
        };
        T(TB_VEC, gv, tv);
        T(TB_VECX, gvx, tvx);
        T(gram_vec ? TB_VEC : TB_RG, gg, tg);
        T(mr_vec ? TB_VEC : TB_RG, gm, tm);
        T(mr_vec ? TB_VECX : TB_RGX, gmx, tmx);
    }
    const SolverDev* ds = B.dev;
    cudaStream_t st = c->stream;
    constexpr int kind = rp_of<R>() == RP64 ? 0 : (rp_of<R>() == RP32 ? 1 : 2);
    const bool timing = c->hop_timing && !B.use_graph;
    const bool pdl = B.pdl && !timing;
    // One system: the stand-alone hop kernel with its pointers as kernel
    // parameters (no descriptor fields held in registers).  A batch: the
    // descriptor-driven hop, one launch for all systems.
    using T = typename Ch<R>::T;
    const SolverDev& h0 = B.host[0];
    auto vsel = [&](int sel, int j) -> T* {
        constexpr bool wide = rp_of<R>() != RP32;   // FP64 and double-float use the wide buffers
        T* base = wide ? (T*)(sel == 0 ? (void*)h0.u64 : sel == 1 ? (void*)h0.r64 : (void*)h0.tmp64)
                       : (T*)(sel == 0 ? (void*)h0.u32 : sel == 1 ? (void*)h0.r32 : (void*)h0.tmp32);
        return base + (size_t)j * (size_t)Ch<R>::N * h0.V;
    };
    const ScalarStep none{STEP_NONE, 0};
    auto hop = [&](int in_sel, int in_j, int out_sel, int out_j, int second, bool dot, ScalarStep step) -> int {
        if (timing) hop_timing_begin(c, kind + (dot ? 3 : 0));
        if (n == 1) {
            const T* rt = rp_of<R>() != RP32 ? (const T*)(const void*)h0.rt64 : (const T*)(const void*)h0.rt32;
            const int* done = pass2 ? nullptr : &h0.st->done;
            const double sc = second ? h0.scale : 1.0;
            const int V = h0.V;
            LinkView<R> U;
            if constexpr (rp_of<R>() == RP64) U = LinkView<R>{h0.links64, V};
            else if constexpr (rp_of<R>() == RPDF) U = LinkView<R>{h0.linksdf, V};
            else U = LinkView<R>{h0.links32, V};
            const SpinorView<R> vin{vsel(in_sel, in_j), V}, vout{vsel(out_sel, out_j), V};
            const SpinorView<R> vdot{const_cast<T*>(rt), V};
            const R cdiag = host_cvt<R>(sc * h0.diag), chop = host_cvt<R>(-0.5 * sc);
            const R ef = host_cvt<R>(h0.ef), eb = host_cvt<R>(h0.eb), bc = host_cvt<R>(h0.bc);
            if constexpr (rp_of<R>() == RPDF) {
                const int nbh = row_blocks(V);
                if (dot)
                    launch(pdl, k_hop1_rows<R, true>, nbh, kRowThreads, st, h0.g, U, vin, vout, cdiag, chop, ef, eb, bc,
                                                                       vdot, h0.part, done, ds, step);
                else
                    launch(pdl, k_hop1_rows<R, false>, nbh, kRowThreads, st, h0.g, U, vin, vout, cdiag, chop, ef, eb, bc,
                                                                        vdot, nullptr, done, ds, none);
            } else {
                bool narrow = false;
                if constexpr (rp_of<R>() == RP32) {
                    if (hop_use_narrow(c->hop_shape, V)) {
                        narrow = true;
                        constexpr int NT = kHopNarrowThreads, MB = kHopNarrowBlocks;
                        const int nbh = (V + NT - 1) / NT;
                        if (dot)
                            launch(pdl, k_hop1<R, true, NT, MB>, nbh, NT, st, h0.g, U, vin, vout, cdiag, chop, ef, eb, bc,
                                                                        vdot, h0.part, done, ds, step);
                        else
                            launch(pdl, k_hop1<R, false, NT, MB>, nbh, NT, st, h0.g, U, vin, vout, cdiag, chop, ef, eb, bc,
                                                                         vdot, nullptr, done, ds, none);
                    }
                }
                if (!narrow) {
                    const int nbh = nblocks(V);
                    if (dot)
                        launch(pdl, k_hop1<R, true>, nbh, kThreads, st, h0.g, U, vin, vout, cdiag, chop, ef, eb, bc, vdot,
                                                                  h0.part, done, ds, step);
                    else
                        launch(pdl, k_hop1<R, false>, nbh, kThreads, st, h0.g, U, vin, vout, cdiag, chop, ef, eb, bc, vdot,
                                                                   nullptr, done, ds, none);
                }
            }
            if (timing) hop_timing_end(c);
            FA_LAUNCHED(c, "k_hop1");
            return FA_OK;
        }
        if constexpr (rp_of<R>() == RP32) {
            if (B.items != nullptr) {
                // the sources of one lattice share each tile's links
                const dim3 gi(B.n_items);
                const ScalarStep e = dot ? step : none;
                if (B.mrhs_min_blocks == 4) {
                    if (dot) launch(pdl, k_hop_mrhs<true, 4>, gi, kHopNarrowThreads, st, ds, B.groups, B.items, in_sel,
                                    in_j, out_sel, out_j, second, p2, e);
                    else launch(pdl, k_hop_mrhs<false, 4>, gi, kHopNarrowThreads, st, ds, B.groups, B.items, in_sel,
                                in_j, out_sel, out_j, second, p2, e);
                } else {
                    if (dot) launch(pdl, k_hop_mrhs<true, kHopNarrowBlocks>, gi, kHopNarrowThreads, st, ds, B.groups,
                                    B.items, in_sel, in_j, out_sel, out_j, second, p2, e);
                    else launch(pdl, k_hop_mrhs<false, kHopNarrowBlocks>, gi, kHopNarrowThreads, st, ds, B.groups,
                                B.items, in_sel, in_j, out_sel, out_j, second, p2, e);
                }
                if (timing) hop_timing_end(c);
                FA_LAUNCHED(c, "k_hop_mrhs");
                return FA_OK;
            }
        }
        if constexpr (rp_of<R>() == RPDF) {
            dim3 gw(row_blocks(h0.V), n);
            const int4* tw = nullptr;
            if (B.tables) {
                gw = dim3(B.tab_n[TB_ROWS]);
                tw = B.tab[TB_ROWS];
            }
            if (dot) launch(pdl, k_hop_sys_rows<R, true>, gw, kRowThreads, st, ds, in_sel, in_j, out_sel, out_j, second, p2,
                            step, tw);
            else launch(pdl, k_hop_sys_rows<R, false>, gw, kRowThreads, st, ds, in_sel, in_j, out_sel, out_j, second, p2,
                        none, tw);
        } else {
            const int4* th = nullptr;
            if (B.tables) {
                gs = dim3(B.tab_n[TB_HOP]);
                th = B.tab[TB_HOP];
            }
            if (dot) launch(pdl, k_hop_sys<R, true>, gs, kThreads, st, ds, in_sel, in_j, out_sel, out_j, second, p2, step,
                            th);
            else launch(pdl, k_hop_sys<R, false>, gs, kThreads, st, ds, in_sel, in_j, out_sel, out_j, second, p2, none,
                        th);
        }
        if (timing) hop_timing_end(c);
        FA_LAUNCHED(c, "k_hop_sys");
        return FA_OK;
    };
    // FP32 pass 1 of a one-system double-pass solve: the last sweep forms the
    // Gram matrix (fused_sweep.cuh) instead of a kernel of its own
    const bool gram_hop = rp_of<R>() == RP32 && L <= 4 && B.Lo.gram_hop && n == 1 && !pass2 && !single;
    auto gram_sweep = [&]() -> int {
        if constexpr (rp_of<R>() == RP32 && L <= 4) {
            GramHop a{};
            a.g = h0.g;
            a.U = LinkView<float>{h0.links32, h0.V};
            a.in = h0.tmp32;
            a.out = h0.r32 + (size_t)L * 6 * h0.V;
            a.part = h0.part;
            for (int i = 0; i < L; ++i) a.r[i] = h0.r32 + (size_t)i * 6 * h0.V;
            a.cdiag = host_cvt<float>(h0.scale * h0.diag);
            a.chop = host_cvt<float>(-0.5 * h0.scale);
            a.ef = host_cvt<float>(h0.ef);
            a.eb = host_cvt<float>(h0.eb);
            a.bc = host_cvt<float>(h0.bc);
            if (timing) hop_timing_begin(c, 6);
            if (hop_use_narrow(c->hop_shape, h0.V)) {
                constexpr int NT = kHopNarrowThreads, MB = kHopNarrowBlocks;
                launch(pdl, k_hop_gram<L, NT, MB>, dim3((h0.V + NT - 1) / NT), NT, st, a, ds);
            } else {
                launch(pdl, k_hop_gram<L, kThreads, FA_HOP_MINB>, dim3(nblocks(h0.V)), kThreads, st, a, ds);
            }
            if (timing) hop_timing_end(c);
            FA_LAUNCHED(c, "k_hop_gram");
        }
        return FA_OK;
    };
    // Pass 1: the seed parts of the scalar steps run in the last block of the
    // reduction that precedes them (alpha after <rt, u_{j+1}>, the next beta
    // after <rt, r_{j+1}>, the MR coefficients after the Gram matrix,
    // convergence after |r_0|^2); the shift parts in block 0 of the next
    // vector kernel (double-pass forms) or with the seed part (single pass).
    for (int j = 0; j < L; ++j) {
        launch(j > 0 && pdl, k_update_u<R>, gv, kThreads, st, ds, j, p2, tv);
        FA_LAUNCHED(c, "k_update_u");
        FA_TRY(hop(0, j, 2, 0, 0, false, none));                                   // tmp = g5 D u_j
        const ScalarStep alpha{single ? STEP_ALPHA_ALL : STEP_ALPHA, j};
        FA_TRY(hop(2, 0, 0, j + 1, 1, !pass2, pass2 ? none : alpha));              // u_{j+1}
        if (pass2) {
            launch(pdl, k_update_r<R, true, false>, gv, kThreads, st, ds, j, p2, tv);
        } else if (single) {
            if constexpr (rp_of<R>() == RP64) launch(pdl, k_update_r<R, false, true>, gv, kThreads, st, ds, j, p2, tv);
        } else {
            // block 0: shift part of sub-step j beside the vector blocks
            launch(pdl, k_update_r<R, false, false, true>, gvx, kThreads, st, ds, j, p2, tvx);
        }
        FA_LAUNCHED(c, "k_update_r");
        FA_TRY(hop(1, j, 2, 0, 0, false, none));                                   // tmp = g5 D r_j
        const bool next_beta = !pass2 && j < L - 1;
        if (gram_hop && j == L - 1) {
            FA_TRY(gram_sweep());   // r_l and, in the epilogue, the Gram matrix and gamma
        } else {
            FA_TRY(hop(2, 0, 1, j + 1, 1, next_beta, next_beta ? ScalarStep{STEP_BETA, j + 1} : none));   // r_{j+1}
        }
    }
    if (!pass2 && !gram_hop) {
        launch(pdl, k_gram<R, L>, gg, kThreads, st, ds, single ? 1 : 0, tg);
        FA_LAUNCHED(c, "k_gram");
    }
    const ScalarStep conv = pass2 ? none : ScalarStep{STEP_CONV, head ? 1 : 0};
    if (pass2) {
        launch(pdl, k_mr<R, L, true, false, false>, gm, kThreads, st, ds, p2, none, tm);
    } else if (single) {
        if constexpr (rp_of<R>() == RP64)
            launch(pdl, k_mr<R, L, false, true, true>, gm, kThreads, st, ds, p2, reliable ? none : conv, tm);
    } else {
        // block 0: shift part of the MR step beside the vector blocks
        launch(pdl, k_mr<R, L, false, false, true, true>, gmx, kThreads, st, ds, p2, reliable ? none : conv, tmx);
    }
    FA_LAUNCHED(c, "k_mr");
    if (reliable) {
        // r_0 <- b - A x in FP64 (one system): A x through two FP64 hops, then the
        // replacement and fresh <rt, r_0>, |r_0|^2 for the convergence step
        double2* t1 = c->io64a.as<double2>();
        double2* t2 = c->io64b.as<double2>();
        const int* done = pass2 ? nullptr : &h0.st->done;
        int rc = launch_hop_f64(h0.g, h0.links64, h0.x64, t1, h0.diag, h0.ef, h0.eb, h0.bc, 1.0, false, true,
                                nullptr, nullptr, done, st);
        if (rc == FA_OK)
            rc = launch_hop_f64(h0.g, h0.links64, t1, t2, h0.diag, h0.ef, h0.eb, h0.bc, h0.scale, false, true,
                                nullptr, nullptr, done, st);
        c->launches += 2;
        if (rc != FA_OK) return rc;
        k_reliable<R><<<gv, kThreads, 0, st>>>(ds, t2, p2, conv);
        FA_LAUNCHED(c, "k_reliable");
    }
    if (pass2) {
        launch(pdl, k_advance, dim3(n), 1, st, ds);
        FA_LAUNCHED(c, "k_advance");
    }
    return FA_OK;
}

template <int L>
static int enqueue_outer_p(Batch& B, int rp, bool pass2, bool single, bool head, bool rel) {
    if (rp == RP64) return enqueue_outer<double, L>(B, pass2, single, head, rel);
    if (rp == RPDF) return enqueue_outer<df, L>(B, pass2, single, head, rel);
    return enqueue_outer<float, L>(B, pass2, single, head, rel);
}

static int enqueue_outer_direct(Batch& B, int rp, bool pass2, bool single, bool head, bool rel) {
    switch (B.Lo.L) {
        case 1: return enqueue_outer_p<1>(B, rp, pass2, single, head, rel);
        case 2: return enqueue_outer_p<2>(B, rp, pass2, single, head, rel);
        case 3: return enqueue_outer_p<3>(B, rp, pass2, single, head, rel);
        case 4: return enqueue_outer_p<4>(B, rp, pass2, single, head, rel);
        case 8: return enqueue_outer_p<8>(B, rp, pass2, single, head, rel);
        default: return FA_EINVAL;
    }
}

// Everything the launches of one outer iteration take as kernel arguments
// that is not part of the cache key: for a batch of one the stand-alone hop
// kernel gets its vectors, links, reduction partials, state and the operator
// scalars (4+m, e^{+-mu}, boundary sign, c) as parameters, and its launch shape;
// the reliable update's FP64 hops read the scratch pair io64a/io64b.  A batch
// reads its systems from the descriptor array, re-uploaded before every solve.
static std::vector<unsigned long long> graph_signature(const Batch& B) {
    std::vector<unsigned long long> s;
    auto p = [&](const void* v) { s.push_back((unsigned long long)(uintptr_t)v); };
    auto d = [&](double v) {
        unsigned long long u;
        std::memcpy(&u, &v, sizeof(u));
        s.push_back(u);
    };
    const fa_ctx* c = B.c0;
    s.push_back((unsigned long long)B.pdl);
    s.push_back((unsigned long long)(long long)c->hop_shape);
    // batches: the tables' addresses and lengths set the launches' grids
    p(c->tabbuf.p);
    for (int k = 0; k < TB_KINDS; ++k) s.push_back((unsigned long long)B.tab_n[k]);
    s.push_back((unsigned long long)B.n_items);
    s.push_back((unsigned long long)B.mrhs_min_blocks);
    p(c->io64a.p);
    p(c->io64b.p);
    if (B.n == 1) {
        const SolverDev& h = B.host[0];
        for (const void* v : {(const void*)h.st, (const void*)h.part, (const void*)h.links64,
                              (const void*)h.links32, (const void*)h.linksdf, (const void*)h.r64,
                              (const void*)h.u64, (const void*)h.rt64, (const void*)h.tmp64, (const void*)h.r32,
                              (const void*)h.u32, (const void*)h.rt32, (const void*)h.tmp32, (const void*)h.x64,
                              (const void*)h.b64})
            p(v);
        d(h.diag);
        d(h.ef);
        d(h.eb);
        d(h.bc);
        d(h.scale);
    }
    return s;
}

// One outer iteration, replayed from a captured CUDA graph when the batch
// uses graphs (every launch argument is iteration-independent: the kernels
// read m and their scalars from the device).  A cached graph whose launch
// arguments no longer match the context (new mu, mass, scale, gauge field,
// launch shape or reallocated buffers) is destroyed and captured again.
static int enqueue_outer_any(Batch& B, int rp, bool pass2, bool single, bool head, bool rel = false) {
    if (!B.use_graph) return enqueue_outer_direct(B, rp, pass2, single, head, rel);
    fa_ctx* c = B.c0;
    const int key = rp | (pass2 ? 4 : 0) | (single ? 8 : 0) | (head ? 16 : 0) | (rel ? 32 : 0) |
                    (B.Lo.gram_hop ? 64 : 0);
    std::vector<unsigned long long> sig = graph_signature(B);
    GraphEntry* ge = nullptr;
    for (auto& e : c->graphs)
        if (e.key == key && e.L == B.Lo.L && e.dev == (void*)B.dev && e.n == B.n && e.V == B.Lo.V) ge = &e;
    if (ge && ge->sig != sig) {
        if (ge->exec) cudaGraphExecDestroy(ge->exec);
        ge->exec = nullptr;
    }
    if (!ge || !ge->exec) {
        const long long n0 = c->launches;
        cudaGraph_t g = nullptr;
        FA_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        const int rc = enqueue_outer_direct(B, rp, pass2, single, head, rel);
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (rc != FA_OK) { if (g) cudaGraphDestroy(g); return rc; }
        FA_CUDA(e, "end capture");
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        FA_CUDA(e, "instantiate graph");
        if (!ge) {
            c->graphs.push_back(GraphEntry{key, B.Lo.L, (void*)B.dev, B.n, B.Lo.V, nullptr, 0, {}});
            ge = &c->graphs.back();
        }
        ge->exec = ex;
        ge->kernels = c->launches - n0;
        ge->sig = std::move(sig);
        c->launches = n0;
    }
    FA_CUDA(cudaGraphLaunch(ge->exec, c->stream), "graph launch");
    c->launches += ge->kernels;
    return FA_OK;
}

static int launch_sweep(Batch& B) {
    const int th = 32;
    int maxns = 0;
    for (auto* c : B.sys) maxns = std::max(maxns, c->ns);
    const dim3 g((maxns + th - 1) / th, B.n);
    cudaStream_t st = B.c0->stream;
    switch (B.Lo.L) {
        case 1: k_sweep<1><<<g, th, 0, st>>>(B.dev); break;
        case 2: k_sweep<2><<<g, th, 0, st>>>(B.dev); break;
        case 3: k_sweep<3><<<g, th, 0, st>>>(B.dev); break;
        case 4: k_sweep<4><<<g, th, 0, st>>>(B.dev); break;
        case 8: k_sweep<8><<<g, th, 0, st>>>(B.dev); break;
        default: return FA_EINVAL;
    }
    FA_LAUNCHED(B.c0, "k_sweep");
    return FA_OK;
}

// b (canonical) -> r_0 and rt of the requested precision, u_0 = 0, for system i
static int load_source(Batch& B, int i, const double* b, int rp) {
    fa_ctx* c = B.sys[i];
    cudaStream_t st = B.c0->stream;
    const int V = B.lo[i].V;
    if (rp != RP32) {
        if (rp == RP64) FA_TRY(launch_pack_spinor_f64(c->g, b, c->r64.as<double2>(), st));
        else FA_TRY(launch_pack_spinor_df(c->g, b, c->r64.as<float4>(), st));
        FA_CUDA(cudaMemcpyAsync(c->rt64.p, c->r64.p, (size_t)12 * V * sizeof(double2), cudaMemcpyDeviceToDevice, st),
                "copy rt");
        FA_CUDA(cudaMemsetAsync(c->u64.p, 0, (size_t)12 * V * sizeof(double2), st), "zero u");
    } else {
        FA_TRY(launch_pack_spinor_f32(c->g, b, c->r32.as<float4>(), st));
        FA_CUDA(cudaMemcpyAsync(c->rt32.p, c->r32.p, (size_t)6 * V * sizeof(float4), cudaMemcpyDeviceToDevice, st),
                "copy rt");
        FA_CUDA(cudaMemsetAsync(c->u32.p, 0, (size_t)6 * V * sizeof(float4), st), "zero u");
    }
    B.c0->launches += 1;
    return FA_OK;
}

// head (FP64 or double-float) -> FP32 hand-over of the live seed vectors
// (r_0, u_0, rt) at an outer-iteration boundary
static int switch_to_f32(Batch& B, int i, int from) {
    fa_ctx* c = B.sys[i];
    cudaStream_t st = B.c0->stream;
    DevBuf* src[3] = {&c->r64, &c->u64, &c->rt64};
    DevBuf* dst[3] = {&c->r32, &c->u32, &c->rt32};
    for (int k = 0; k < 3; ++k) {
        if (from == RPDF) FA_TRY(launch_convert_df_to_f32(c->g, src[k]->as<float4>(), dst[k]->as<float4>(), st));
        else FA_TRY(launch_convert_f64_to_f32(c->g, src[k]->as<double2>(), dst[k]->as<float4>(), st));
    }
    B.c0->launches += 3;
    return FA_OK;
}

// r_0, u_0, rt of system i <-> its snapshot buffer
static int snapshot(Batch& B, int i, bool f64, bool restore) {
    fa_ctx* c = B.sys[i];
    const size_t sb = f64 ? B.lo[i].vs64 * sizeof(double2) : B.lo[i].vs32 * sizeof(float4);
    char* snap = f64 ? c->snap64.as<char>() : c->snap32.as<char>();
    void* v[3] = {f64 ? c->r64.p : c->r32.p, f64 ? c->u64.p : c->u32.p, f64 ? c->rt64.p : c->rt32.p};
    for (int k = 0; k < 3; ++k) {
        void* dst = restore ? v[k] : (void*)(snap + k * sb);
        const void* src = restore ? (const void*)(snap + k * sb) : v[k];
        FA_CUDA(cudaMemcpyAsync(dst, src, sb, cudaMemcpyDeviceToDevice, B.c0->stream), "snapshot");
    }
    if (B.host[i].x64) {   // reliable updates: the seed solution belongs to the state
        const size_t xb = B.lo[i].vs64 * sizeof(double2);
        void* dst = restore ? (void*)B.host[i].x64 : c->snapx.p;
        const void* src = restore ? c->snapx.p : (const void*)B.host[i].x64;
        FA_CUDA(cudaMemcpyAsync(dst, src, xb, cudaMemcpyDeviceToDevice, B.c0->stream), "snapshot x");
    }
    return FA_OK;
}

static int read_states(Batch& B, std::vector<DevState>& hs) {
    hs.resize(B.n);
    for (int i = 0; i < B.n; ++i)
        FA_CUDA(cudaMemcpyAsync(&hs[i], B.sys[i]->state.p, sizeof(DevState), cudaMemcpyDeviceToHost, B.c0->stream),
                "read state");
    FA_CUDA(cudaStreamSynchronize(B.c0->stream), "sync state");
    return FA_OK;
}

// Work tables and lattice groups of a batch of several systems, in one device
// buffer of the first context.  Shift blocks come first in their tables (they
// run the per-shift FP64 recurrences, the longest blocks of a launch).
static int build_tables(Batch& B) {
    fa_ctx* c0 = B.c0;
    const int n = B.n;
    std::vector<int4> t[TB_KINDS];
    auto blocks = [&](std::vector<int4>& v, int i, int nb, bool xs) {
        for (int b = 0; b < nb; ++b) v.push_back(make_int4(i, b, nb, nb + (xs ? 1 : 0)));
    };
    for (int i = 0; i < n; ++i) {
        t[TB_VECX].push_back(make_int4(i, -1, B.lo[i].vgrid, B.lo[i].vgrid + 1));
        t[TB_RGX].push_back(make_int4(i, -1, B.lo[i].red_grid, B.lo[i].red_grid + 1));
    }
    for (int i = 0; i < n; ++i) {
        const Layout& lo = B.lo[i];
        blocks(t[TB_VEC], i, lo.vgrid, false);
        blocks(t[TB_VECX], i, lo.vgrid, true);
        blocks(t[TB_RG], i, lo.red_grid, false);
        blocks(t[TB_RGX], i, lo.red_grid, true);
        blocks(t[TB_HOP], i, lo.nblk, false);
        blocks(t[TB_ROWS], i, row_blocks(lo.V), false);
    }
    // lattice groups for the FP32 multi-RHS sweep: systems sharing the packed
    // links and the lattice shape, at most kMaxRhs per group
    std::vector<GroupDev> groups;
    std::vector<const void*> gkey;
    std::vector<int4> items;
    if (B.Lo.need32) {
        for (int i = 0; i < n; ++i) {
            const void* key = B.host[i].links32;
            int gi = -1;
            for (size_t g = 0; g < groups.size(); ++g)
                if (gkey[g] == key && groups[g].nsys < kMaxRhs && B.host[groups[g].sys[0]].V == B.host[i].V &&
                    B.host[groups[g].sys[0]].g.X == B.host[i].g.X && B.host[groups[g].sys[0]].g.Y == B.host[i].g.Y &&
                    B.host[groups[g].sys[0]].g.Z == B.host[i].g.Z)
                    gi = (int)g;
            if (gi < 0) {
                GroupDev gd{};
                gd.nsys = 0;
                gd.ntile = (B.host[i].V + kHopNarrowThreads - 1) / kHopNarrowThreads;
                groups.push_back(gd);
                gkey.push_back(key);
                gi = (int)groups.size() - 1;
            }
            groups[gi].sys[groups[gi].nsys++] = i;
        }
        const int rpb = c0->mrhs_rpb > 0 ? c0->mrhs_rpb : kMaxRhs;
        for (size_t g = 0; g < groups.size(); ++g)
            for (int tile = 0; tile < groups[g].ntile; ++tile)
                for (int r0 = 0; r0 < groups[g].nsys; r0 += rpb)
                    items.push_back(make_int4((int)g, tile, r0, std::min(r0 + rpb, groups[g].nsys)));
        B.rhs_per_block = rpb;
        B.mrhs_min_blocks = c0->mrhs_mb == 4 ? 4 : kHopNarrowBlocks;
    }
    size_t off[TB_KINDS + 2], bytes = 0;
    for (int k = 0; k < TB_KINDS; ++k) {
        off[k] = bytes;
        bytes += t[k].size() * sizeof(int4);
    }
    off[TB_KINDS] = bytes;
    bytes += items.size() * sizeof(int4);
    off[TB_KINDS + 1] = bytes;
    bytes += groups.size() * sizeof(GroupDev);
    FA_CUDA(c0->tabbuf.ensure(std::max<size_t>(bytes, 16)), "alloc work tables");
    B.tab_host.assign(bytes, 0);
    for (int k = 0; k < TB_KINDS; ++k)
        if (!t[k].empty()) std::memcpy(B.tab_host.data() + off[k], t[k].data(), t[k].size() * sizeof(int4));
    if (!items.empty()) std::memcpy(B.tab_host.data() + off[TB_KINDS], items.data(), items.size() * sizeof(int4));
    if (!groups.empty())
        std::memcpy(B.tab_host.data() + off[TB_KINDS + 1], groups.data(), groups.size() * sizeof(GroupDev));
    char* base = c0->tabbuf.as<char>();
    FA_CUDA(cudaMemcpyAsync(base, B.tab_host.data(), bytes, cudaMemcpyHostToDevice, c0->stream), "upload work tables");
    B.tables = true;
    for (int k = 0; k < TB_KINDS; ++k) {
        B.tab[k] = reinterpret_cast<const int4*>(base + off[k]);
        B.tab_n[k] = (int)t[k].size();
    }
    if (!items.empty()) {
        B.items = reinterpret_cast<const int4*>(base + off[TB_KINDS]);
        B.n_items = (int)items.size();
        B.groups = reinterpret_cast<const GroupDev*>(base + off[TB_KINDS + 1]);
    }
    return FA_OK;
}

// ------------------------------------------------------------------ the solve (a batch of n systems)// ------------------------------------------------------------------ the solve (a batch of n systems)
int solve_batch(fa_ctx* const* ctxs, int n, const double* const* b, double* const* y_canon, double* const* xs_canon,
                const fa_solver_params* p, fa_solver_stats* stats) {
    if (n < 1 || !ctxs || !b || !p) return FA_EINVAL;
    fa_ctx* c0 = ctxs[0];
    for (int i = 0; i < n; ++i) {
        fa_ctx* c = ctxs[i];
        if (!c || !b[i]) return FA_EINVAL;
        if (!c->have_gauge || !c->have_params || !c->have_poles) return FA_ESTATE;
        if (c->device != c0->device) return FA_EINVAL;
    }
    bool same_shape = true;
    for (int i = 0; i < n; ++i) {
        const Geom& g = ctxs[i]->g;
        same_shape = same_shape && g.X == c0->g.X && g.Y == c0->g.Y && g.Z == c0->g.Z && g.T == c0->g.T;
    }
    const int L = p->ell;
    if (!(L == 1 || L == 2 || L == 3 || L == 4 || L == 8)) return FA_EINVAL;
    if (!(p->tol > 0.0) || p->max_outer < 1 || p->max_outer > 1000000) return FA_EINVAL;
    const bool single = p->mode == FA_SINGLE;
    const bool pseudo = p->mode == FA_PSEUDO;
    if (!single && !pseudo && p->mode != FA_DOUBLE) return FA_EINVAL;
    const int prec = p->precision;
    if (prec != FA_F64 && prec != FA_F32 && prec != FA_MIXED && prec != FA_MIXED_DF) return FA_EINVAL;
    if (single && prec != FA_F64) return FA_EINVAL;
    const bool mixed = prec == FA_MIXED || prec == FA_MIXED_DF;
    const int head_rp = prec == FA_MIXED_DF ? RPDF : RP64;   // working precision of the head
    const int rel_every = p->reliable_every;
    if (rel_every < 0 || (rel_every > 0 && n != 1)) return FA_EINVAL;
    // FA_MIXED: switch_resid <= 0 selects the default min(0.04 / l^2, 0.4 / l^6):
    // the FP32 error of the power-basis recurrence grows steeply with l (FP32-only
    // solves on 4^3 x 8: 9.1e-8 at l = 2, 1.7e-6 to 3.8e-6 at l = 4), and at l = 4
    // a threshold of 6.25e-4 left one of nine point sources at 2.4e-8 while 1e-4
    // kept all of them below 4.3e-10
    const double Ld = (double)L, L2 = Ld * Ld;
    const double switch_resid = (p->switch_resid > 0.0) ? p->switch_resid : std::min(0.04 / L2, 0.4 / (L2 * L2 * L2));
    if (mixed && !(switch_resid < 1.0)) return FA_EINVAL;

    Batch B;
    B.c0 = c0;
    B.n = n;
    B.sys.assign(ctxs, ctxs + n);
    // the layout of each system (its lattice size decides its grids)
    auto layout_of = [&](const fa_ctx* c) {
        Layout Lo{};
        Lo.L = L;
        Lo.max_outer = p->max_outer;
        Lo.V = c->g.V;
        Lo.single = single;
        Lo.need64 = prec != FA_F32;
        Lo.need32 = prec != FA_F64;
        Lo.vs64 = (size_t)12 * Lo.V;
        Lo.vs32 = (size_t)6 * Lo.V;
        Lo.nblk = nblocks(Lo.V);
        Lo.red_grid = red_grid_for(Lo.V);
        // at most one wave of kVecBlocks blocks per SM, one site per thread where
        // the lattice is smaller (a wave of exactly kVecBlocks per SM with fewer
        // sites per block measured 3-5% slower on 16^3 x 32: the kernels are bound
        // by HBM, not by the per-SM imbalance)
        Lo.vgrid = std::min(Lo.nblk, kVecBlocks * sms());
        Lo.part_slots = std::max(n_gram(L), 2);
        // FP32 stretches of a one-system double-pass solve form the MR Gram matrix in
        // the epilogue of their last sweep (flags bit 5: the Gram kernel instead)
        Lo.gram_hop = n == 1 && !single && L <= 4 && prec != FA_F64 && (p->flags & 32) == 0;
        return Lo;
    };
    for (auto* c : B.sys) B.lo.push_back(layout_of(c));
    B.Lo = B.lo[0];
    const Layout& Lo = B.Lo;
    for (int i = 0; i < n; ++i) FA_TRY(ensure_workspace(B.sys[i], B.lo[i]));
    FA_CUDA(c0->descbuf.ensure((size_t)n * sizeof(SolverDev)), "alloc descriptors");
    FA_CUDA(c0->flagbuf.ensure((size_t)2 * n * sizeof(int)), "alloc flags");
    if (c0->pinned_bytes < 2 * n * sizeof(int) + 64) {
        if (c0->pinned) cudaFreeHost(c0->pinned);
        c0->pinned = nullptr;
        c0->pinned_bytes = 0;
        FA_CUDA(cudaMallocHost(&c0->pinned, 2 * n * sizeof(int) + 4096), "alloc pinned");
        c0->pinned_bytes = 2 * n * sizeof(int) + 4096;
    }
    B.dev = c0->descbuf.as<SolverDev>();
    B.flags = c0->flagbuf.as<int>();
    // graphs need a capturable stream (not the legacy default stream)
    B.use_graph = (p->flags & 4) != 0 && c0->stream != nullptr && c0->stream != cudaStreamLegacy;
    // programmatic dependent launch for direct launches only: under CUDA-graph
    // replay it measured slower (16^3 x 32 headline: 15.00 against 14.62 ms)
    B.pdl = (p->flags & 16) == 0 && !B.use_graph;
    for (int i = 0; i < n; ++i) B.host.push_back(make_dev(B.sys[i], B.lo[i]));
    for (auto& h : B.host) h.fixed_iters = (p->flags & 8) ? 1 : 0;
    // Several systems: every launch serves all of them through work tables (any
    // mix of lattice shapes); FP32 sweeps go by lattice groups (systems that
    // share one gauge field and shape) so that a block's right-hand sides read
    // its tile's links once.
    if (n > 1) FA_TRY(build_tables(B));
    (void)same_shape;
    cudaStream_t st = c0->stream;
    const bool timing = (p->flags & 1) != 0;
    c0->hop_timing = (p->flags & 2) != 0;
    c0->hop_outer = -1;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    if (timing)
        for (auto& e : ev) FA_CUDA(cudaEventCreate(&e), "event");

    // ---- pseudo-double-pass stores (Sec. 2, option 2): pass 1 keeps the seed-vector
    // occurrences of a contiguous prefix [0, K) of outer iterations, as many as the
    // budget holds (FP64 slots while in FP64, FP32 slots after the switch)
    const int NC = nc_slots(L);
    const size_t s64 = Lo.vs64 * sizeof(double2);   // system 0 (reliable updates: one system)
    // one stored outer iteration of every system (FP64 / FP32 slots): the budget
    // holds the same number of outer iterations for all systems of a batch
    double per64t = 0.0, per32t = 0.0;
    for (int i = 0; i < n; ++i) {
        per64t += (double)NC * (double)(B.lo[i].vs64 * sizeof(double2));
        per32t += (double)NC * (double)(B.lo[i].vs32 * sizeof(float4));
    }
    long long cap64 = 0, cap32 = 0;
    if (pseudo) {
        size_t fb = 0, tb = 0;
        FA_CUDA(cudaMemGetInfo(&fb, &tb), "memory info");
        double held = 0.0;
        for (auto* c : B.sys) held += (double)c->store64.bytes + (double)c->store32.bytes;
        double budget = p->store_gb > 0.0 ? p->store_gb * 1e9 : std::min(0.25 * ((double)fb + held), 16e9);
        budget = std::min(budget, 0.9 * ((double)fb + held));     // all systems together
        if (prec == FA_F64) {
            cap64 = (long long)std::min<double>(Lo.max_outer, budget / per64t);
        } else if (prec == FA_F32) {
            cap32 = (long long)std::min<double>(Lo.max_outer, budget / per32t);
        } else {
            // the head's (wider) slots take up to half of the budget
            cap64 = (long long)std::min<double>(std::min(Lo.max_outer, 64), 0.5 * budget / per64t);
            cap32 = (long long)std::min<double>(Lo.max_outer, (budget - (double)cap64 * per64t) / per32t);
        }
        cap64 = std::max(0LL, cap64);
        cap32 = std::max(0LL, cap32);
        for (int i = 0; i < n; ++i) {
            fa_ctx* c = B.sys[i];
            const size_t s64i = B.lo[i].vs64 * sizeof(double2), s32i = B.lo[i].vs32 * sizeof(float4);
            if (cap64 > 0) FA_CUDA(c->store64.ensure((size_t)cap64 * NC * s64i), "alloc occurrence store");
            if (cap32 > 0) FA_CUDA(c->store32.ensure((size_t)cap32 * NC * s32i), "alloc occurrence store");
            if (Lo.need64) FA_CUDA(c->snap64.ensure(3 * s64i), "alloc snapshot");
            if (Lo.need32) FA_CUDA(c->snap32.ensure(3 * s32i), "alloc snapshot");
            B.host[i].store64 = c->store64.as<char>();
            B.host[i].store32 = c->store32.as<char>();
            B.host[i].cap64 = (int)cap64;
            B.host[i].cap32 = (int)cap32;
            B.host[i].m0_32 = prec == FA_F32 ? 0 : -1;
        }
    }
    if (rel_every > 0) {
        fa_ctx* c = B.sys[0];
        FA_CUDA(c->xrel.ensure(s64), "alloc x");
        FA_CUDA(c->brel.ensure(s64), "alloc b");
        FA_CUDA(c->io64a.ensure(s64), "alloc");
        FA_CUDA(c->io64b.ensure(s64), "alloc");
        if (pseudo) FA_CUDA(c->snapx.ensure(s64), "alloc snapshot x");
        FA_TRY(launch_pack_spinor_f64(c->g, b[0], c->brel.as<double2>(), st));
        FA_CUDA(cudaMemsetAsync(c->xrel.p, 0, s64, st), "zero x");
        B.host[0].x64 = c->xrel.as<double2>();
        B.host[0].b64 = c->brel.as<double2>();
    }
    // outer iteration m ends with a reliable update
    auto reliable_at = [&](int m) { return rel_every > 0 && (m + 1) % rel_every == 0; };
    FA_TRY(upload(B));
    int K = pseudo ? -1 : 0;                // first outer iteration not stored (-1: still storing)
    int m0_32 = prec == FA_F32 ? 0 : -1;    // first FP32 outer iteration (one value for the batch)
    bool snap_wide = true;
    // called before outer iteration m is enqueued: at the first unstored one,
    // snapshot the seed state so that a pass 2 can restart there (FP64 and
    // double-float states use the wide buffers and stores)
    auto before_outer = [&](int m, int rp) -> int {
        if (K >= 0) return FA_OK;
        const bool wide = rp != RP32;
        const bool stored = wide ? (m < cap64) : (m0_32 >= 0 && m - m0_32 < cap32);
        if (stored) return FA_OK;
        K = m;
        snap_wide = wide;
        for (int i = 0; i < n; ++i) FA_TRY(snapshot(B, i, wide, false));
        return FA_OK;
    };

    // poles, y, shift vectors
    for (int i = 0; i < n; ++i) {
        fa_ctx* c = B.sys[i];
        const SolverDev& d = B.host[i];
        FA_CUDA(cudaMemcpyAsync((void*)d.sigma, c->sigma, c->ns * sizeof(double), cudaMemcpyHostToDevice, st), "poles");
        FA_CUDA(cudaMemcpyAsync((void*)d.omega, c->omega, c->ns * sizeof(double), cudaMemcpyHostToDevice, st), "poles");
        FA_CUDA(cudaMemsetAsync(d.y, 0, (size_t)12 * B.lo[i].V * sizeof(double2), st), "zero y");
        if (single) {
            const size_t vb = (size_t)12 * B.lo[i].V * sizeof(double2);
            FA_CUDA(cudaMemsetAsync(d.xs, 0, (size_t)c->ns * vb, st), "zero xs");
            FA_CUDA(cudaMemsetAsync(d.us, 0, (size_t)c->ns * (L + 1) * vb, st), "zero us");
        }
    }
    if (timing) cudaEventRecord(ev[0], st);

    // ---- pass 1
    int rp = prec == FA_F32 ? RP32 : (prec == FA_F64 ? RP64 : head_rp);
    bool head = mixed;
    for (int i = 0; i < n; ++i) FA_TRY(load_source(B, i, b[i], rp));
    dim3 gr(Lo.vgrid, n);
    const int4* tr = nullptr;
    if (B.tables) {
        gr = dim3(B.tab_n[TB_VEC]);
        tr = B.tab[TB_VEC];
    }
    for (int i = 0; i < n; ++i)
        FA_CUDA(cudaMemsetAsync(B.host[i].st, 0, sizeof(DevState), st), "clear state");
    const double theta = mixed ? switch_resid : 0.0;
    if (rp == RP64) k_dot2_sys<double><<<gr, kThreads, 0, st>>>(B.dev, p->tol, theta, tr);
    else if (rp == RPDF) k_dot2_sys<df><<<gr, kThreads, 0, st>>>(B.dev, p->tol, theta, tr);
    else k_dot2_sys<float><<<gr, kThreads, 0, st>>>(B.dev, p->tol, theta, tr);
    FA_LAUNCHED(c0, "k_dot2_sys");

    std::vector<DevState> hs(n);
    int switch_outer = -1;
    int enq = 0;
    bool all_done = false;
    // head of FA_MIXED / FA_MIXED_DF: one outer iteration at a time until every
    // system (that has not finished) asks for the switch; a batch switches at one
    // outer iteration (a system that asked earlier runs its head longer, which
    // only makes its result more accurate)
    while (head && enq < Lo.max_outer) {
        FA_TRY(before_outer(enq, rp));
        c0->hop_outer = enq;
        FA_TRY(enqueue_outer_any(B, rp, false, single, true, reliable_at(enq)));
        ++enq;
        FA_TRY(read_states(B, hs));
        bool every_done = true, every_switch = true;
        for (int i = 0; i < n; ++i) {
            every_done = every_done && hs[i].done;
            every_switch = every_switch && (hs[i].done || hs[i].switch_req);
        }
        if (every_done) { all_done = true; break; }
        if (every_switch) {
            for (int i = 0; i < n; ++i) FA_TRY(switch_to_f32(B, i, rp));
            switch_outer = enq;
            m0_32 = switch_outer;
            // the stored prefix must stay contiguous: no FP32 slots if the head outran its slots
            if (K >= 0) cap32 = 0;
            for (int i = 0; i < n; ++i) {
                B.host[i].m0_32 = m0_32;
                if (K >= 0) B.host[i].cap32 = 0;
            }
            FA_TRY(upload(B));
            head = false;
            rp = RP32;
        }
    }
    if (!all_done) {
        // main loop: chunks of outer iterations; poll the previous chunk's done
        // flags (iterations enqueued past convergence return at once)
        const int chunk = (Lo.V * (long long)n) >= (1 << 17) ? 4 : 8;
        int* pin = static_cast<int*>(c0->pinned);
        cudaEvent_t pe[2];
        FA_CUDA(cudaEventCreateWithFlags(&pe[0], cudaEventDisableTiming), "event");
        FA_CUDA(cudaEventCreateWithFlags(&pe[1], cudaEventDisableTiming), "event");
        int k = 0;
        bool stop = false;
        int rc = FA_OK;
        while (!stop && enq < Lo.max_outer) {
            for (int i = 0; i < chunk && enq < Lo.max_outer; ++i, ++enq) {
                rc = before_outer(enq, rp);
                c0->hop_outer = enq;
                if (rc == FA_OK) rc = enqueue_outer_any(B, rp, false, single, false, reliable_at(enq));
                if (rc != FA_OK) break;
            }
            if (rc != FA_OK) break;
            if (n == 1) {
                // one system: its done flag straight from the device state
                cudaMemcpyAsync(pin + (k & 1), &B.host[0].st->done, sizeof(int), cudaMemcpyDeviceToHost, st);
            } else {
                k_flags<<<(n + 127) / 128, 128, 0, st>>>(B.dev, n, B.flags + (k & 1) * n);
                c0->launches++;
                cudaMemcpyAsync(pin + (k & 1) * n, B.flags + (k & 1) * n, n * sizeof(int), cudaMemcpyDeviceToHost, st);
            }
            cudaEventRecord(pe[k & 1], st);
            if (k > 0) {
                cudaEventSynchronize(pe[(k - 1) & 1]);
                bool all = true;
                for (int i = 0; i < n; ++i) all = all && pin[((k - 1) & 1) * n + i] != 0;
                if (all) stop = true;
            }
            ++k;
        }
        cudaEventDestroy(pe[0]);
        cudaEventDestroy(pe[1]);
        FA_TRY(rc);
        FA_TRY(read_states(B, hs));
    }
    c0->hop_outer = -1;
    if (timing) cudaEventRecord(ev[1], st);
    std::vector<int> status(n);
    int M = 0, rc_all = FA_OK;
    for (int i = 0; i < n; ++i) {
        status[i] = hs[i].status;
        if (status[i] == FA_OK && !hs[i].done) status[i] = FA_ENOCONV;
        if (status[i] != FA_OK && rc_all == FA_OK) rc_all = status[i];
        M = std::max(M, hs[i].n_outer);
    }
    const int Kst = pseudo ? (K < 0 ? M : std::min(K, M)) : 0;   // stored prefix (all systems)

    // ---- backward sweep, gather of the stored prefix, pass 2 for the rest
    if (rc_all == FA_OK && !single) {
        for (int i = 0; i < n; ++i)
            FA_CUDA(cudaMemsetAsync(B.host[i].cs, 0, (size_t)B.sys[i]->ns * Lo.max_outer * NC * sizeof(double2), st),
                    "zero sweep");
        FA_TRY(launch_sweep(B));
        k_coef_reduce<<<dim3((M * NC + 255) / 256, n), 256, 0, st>>>(B.dev);
        FA_LAUNCHED(c0, "k_coef_reduce");
        if (timing) cudaEventRecord(ev[2], st);
        // the largest lattice of the batch sets the grids (blocks beyond a smaller
        // system's sites return at once)
        int max_nblk = 0, max_V = 0;
        for (int i = 0; i < n; ++i) {
            max_nblk = std::max(max_nblk, B.lo[i].nblk);
            max_V = std::max(max_V, B.lo[i].V);
        }
        if (pseudo && Kst > 0) {
            // one thread per site and chunk: 12 chunks per site (FP64, double-float), 6 (FP32)
            if (cap64 > 0) {
                const dim3 gw(max_nblk * 12, n);
                if (prec == FA_MIXED_DF) k_gather<df><<<gw, kThreads, 0, st>>>(B.dev);
                else k_gather<double><<<gw, kThreads, 0, st>>>(B.dev);
                FA_LAUNCHED(c0, "k_gather (head store)");
            }
            if (cap32 > 0 && m0_32 >= 0) {
                k_gather<float><<<dim3(max_nblk * 6, n), kThreads, 0, st>>>(B.dev);
                FA_LAUNCHED(c0, "k_gather<float>");
            }
        }
        const int mstart = Kst;
        if (mstart < M) {
            int p2 = prec == FA_F64 ? RP64
                   : (prec == FA_F32 ? RP32 : ((switch_outer < 0 || mstart < switch_outer) ? head_rp : RP32));
            for (int i = 0; i < n; ++i) {
                if (mstart == 0) {
                    FA_TRY(load_source(B, i, b[i], p2));
                    if (B.host[i].x64)
                        FA_CUDA(cudaMemsetAsync(B.host[i].x64, 0, s64, st), "zero x");
                } else {
                    if (snap_wide != (p2 != RP32)) return FA_ESTATE;
                    FA_TRY(snapshot(B, i, p2 != RP32, true));
                }
            }
            k_set_m<<<n, 1, 0, st>>>(B.dev, mstart);
            FA_LAUNCHED(c0, "k_set_m");
            for (int m = mstart; m < M; ++m) {
                if (p2 != RP32 && mixed && m == switch_outer) {
                    for (int i = 0; i < n; ++i) FA_TRY(switch_to_f32(B, i, p2));
                    p2 = RP32;
                }
                FA_TRY(enqueue_outer_any(B, p2, true, false, false, reliable_at(m)));
            }
        }
        if (timing) cudaEventRecord(ev[3], st);
        if (y_canon)
            for (int i = 0; i < n; ++i) {
                FA_TRY(launch_unpack_spinor_f64(B.sys[i]->g, B.host[i].y, y_canon[i], st));
                c0->launches++;
            }
    } else if (rc_all == FA_OK && single) {
        if (timing) { cudaEventRecord(ev[2], st); cudaEventRecord(ev[3], st); }
        if (y_canon) {
            int max_V = 0;
            for (int i = 0; i < n; ++i) max_V = std::max(max_V, B.lo[i].V);
            k_combine_sys<<<dim3((12 * max_V + kThreads - 1) / kThreads, n), kThreads, 0, st>>>(B.dev);
            FA_LAUNCHED(c0, "k_combine_sys");
            for (int i = 0; i < n; ++i) {
                FA_TRY(launch_unpack_spinor_f64(B.sys[i]->g, B.host[i].y, y_canon[i], st));
                c0->launches++;
            }
        }
        if (xs_canon && n == 1) {
            for (int s = 0; s < c0->ns; ++s) {
                FA_TRY(launch_unpack_spinor_f64(c0->g, B.host[0].xs + (size_t)s * Lo.vs64, xs_canon[s], st));
                c0->launches++;
            }
        }
    }
    FA_CUDA(cudaStreamSynchronize(st), "sync solve");
    if (c0->hop_timing) hop_timing_collect(c0, M);
    c0->hop_timing = false;

    if (stats) {
        for (int i = 0; i < n; ++i) {
            fa_solver_stats& S = stats[i];
            std::memset(&S, 0, sizeof(S));
            const int Mi = hs[i].n_outer;
            S.status = status[i];
            S.outer_iters = Mi;
            S.switch_outer = switch_outer;
            S.ns = B.sys[i]->ns;
            int iters[kMaxShifts];
            FA_CUDA(cudaMemcpy(iters, B.host[i].iters, S.ns * sizeof(int), cudaMemcpyDeviceToHost), "read iters");
            for (int s = 0; s < S.ns; ++s) S.iters_per_shift[s] = iters[s];
            S.resid_recurrence = std::sqrt(hs[i].rnorm2 / hs[i].bnorm2);
            const int Ki = std::min(Kst, Mi);
            const long long per = 2LL * L * Mi;
            S.n_mv = single ? per : per + 2LL * L * (Mi - (pseudo ? Ki : 0));
            S.stored_outer = pseudo ? Ki : 0;
            S.n_dot = (long long)Mi * (L * (L + 7) / 2 + 1);
            S.n_launch = c0->launches;
            if (timing) {
                float a = 0.f, b2 = 0.f, c2 = 0.f;
                cudaEventElapsedTime(&a, ev[0], ev[1]);
                cudaEventElapsedTime(&b2, ev[1], ev[2]);
                cudaEventElapsedTime(&c2, ev[2], ev[3]);
                S.t_pass1_ms = a;
                S.t_sweep_ms = b2;
                S.t_pass2_ms = c2;
            }
        }
    }
    if (timing)
        for (auto& e : ev) cudaEventDestroy(e);
    return rc_all;
}

int solve(fa_ctx* c, const double* b, double* y_canon, double* const* xs_canon, const fa_solver_params* p,
          fa_solver_stats* stats) {
    return solve_batch(&c, 1, &b, y_canon ? &y_canon : nullptr, xs_canon, p, stats);
}

// ------------------------------------------------------------------ batched sweep autotuner
// Times the multi-RHS FP32 sweep of a batch (r_0 -> tmp, the first hop of A)
// for each right-hand-side count per block and residency; keeps the fastest in
// ctxs[0].  The sweep's results do not depend on the choice.
int autotune_batch(fa_ctx* const* ctxs, int n, int reps, int* rpb_out, int* mb_out, double* times, int ntimes) {
    fa_ctx* c0 = ctxs[0];
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]->have_gauge || !ctxs[i]->have_params || !ctxs[i]->have_poles) return FA_ESTATE;
        if (ctxs[i]->device != c0->device) return FA_EINVAL;
    }
    Batch B;
    B.c0 = c0;
    B.n = n;
    B.sys.assign(ctxs, ctxs + n);
    for (int i = 0; i < n; ++i) {
        Layout lo{};
        lo.L = 1;
        lo.max_outer = 1;
        lo.V = ctxs[i]->g.V;
        lo.need32 = true;
        lo.vs64 = (size_t)12 * lo.V;
        lo.vs32 = (size_t)6 * lo.V;
        lo.nblk = nblocks(lo.V);
        lo.red_grid = red_grid_for(lo.V);
        lo.vgrid = std::min(lo.nblk, kVecBlocks * sms());
        lo.part_slots = 2;
        B.lo.push_back(lo);
        FA_TRY(ensure_workspace(ctxs[i], lo));
    }
    B.Lo = B.lo[0];
    cudaStream_t st = c0->stream;
    FA_CUDA(c0->descbuf.ensure((size_t)n * sizeof(SolverDev)), "alloc descriptors");
    B.dev = c0->descbuf.as<SolverDev>();
    for (int i = 0; i < n; ++i) {
        B.host.push_back(make_dev(ctxs[i], B.lo[i]));
        FA_CUDA(cudaMemsetAsync(B.host[i].st, 0, sizeof(DevState), st), "clear state");
        FA_CUDA(cudaMemsetAsync(ctxs[i]->r32.p, 0, B.lo[i].vs32 * sizeof(float4), st), "clear r");
    }
    FA_TRY(upload(B));
    const int rpbs[] = {1, 2, 3, 4, 6, 12, kMaxRhs};
    const int mbs[] = {kHopNarrowBlocks, 4};
    constexpr int NR = sizeof(rpbs) / sizeof(rpbs[0]), NM = sizeof(mbs) / sizeof(mbs[0]);
    double best[NR][NM];
    for (auto& row : best)
        for (auto& v : row) v = 1e30;
    const int saved_rpb = c0->mrhs_rpb, saved_mb = c0->mrhs_mb;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    FA_CUDA(cudaEventCreate(&e0), "event");
    FA_CUDA(cudaEventCreate(&e1), "event");
    int rc = FA_OK;
    const ScalarStep none{STEP_NONE, 0};
    for (int round = 0; round < 3 && rc == FA_OK; ++round)
        for (int a = 0; a < NR && rc == FA_OK; ++a)
            for (int m = 0; m < NM && rc == FA_OK; ++m) {
                c0->mrhs_rpb = rpbs[a];
                c0->mrhs_mb = mbs[m];
                B.items = nullptr;
                rc = build_tables(B);
                if (rc != FA_OK) break;
                auto go = [&](int k) {
                    for (int i = 0; i < k; ++i) {
                        if (B.mrhs_min_blocks == 4)
                            k_hop_mrhs<false, 4><<<B.n_items, kHopNarrowThreads, 0, st>>>(B.dev, B.groups, B.items, 1,
                                                                                          0, 2, 0, 0, 0, none);
                        else
                            k_hop_mrhs<false, kHopNarrowBlocks><<<B.n_items, kHopNarrowThreads, 0, st>>>(
                                B.dev, B.groups, B.items, 1, 0, 2, 0, 0, 0, none);
                    }
                };
                go(3);
                cudaEventRecord(e0, st);
                go(reps);
                cudaEventRecord(e1, st);
                cudaError_t e = cudaEventSynchronize(e1);
                if (e == cudaSuccess) e = cudaGetLastError();
                if (e != cudaSuccess) { rc = cuda_fail(e, "fa_autotune_batched"); break; }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                best[a][m] = std::min(best[a][m], (double)ms / reps);
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != FA_OK) {
        c0->mrhs_rpb = saved_rpb;
        c0->mrhs_mb = saved_mb;
        return rc;
    }
    int ba = NR - 1, bm = 0;
    for (int a = 0; a < NR; ++a)
        for (int m = 0; m < NM; ++m)
            if (best[a][m] < best[ba][bm]) ba = a, bm = m;
    c0->mrhs_rpb = rpbs[ba];
    c0->mrhs_mb = mbs[bm];
    *rpb_out = rpbs[ba];
    *mb_out = mbs[bm];
    if (times)
        for (int a = 0, k = 0; a < NR; ++a)
            for (int m = 0; m < NM; ++m, ++k)
                if (k < ntimes) times[k] = best[a][m];
    FA_CUDA(cudaStreamSynchronize(st), "sync");
    return FA_OK;
}

// ------------------------------------------------------------------ sign function, overlap operator
// Sec. 1: D_ov(mu) = 1 + g5 sign(g5 D_w(mu)), sign z = z / sqrt(z^2).  With
// A = c H^2, H = g5 D_w: sign(H) b = sqrt(c) H f(A) b, f(A) b the solver's y
// (poles approximating z^{-1/2}); D_ov b = b + g5 sign(H) b = b + sqrt(c) D_w y.
// One FP64 sweep on the solver's internal y after the solve.
int apply_sign(fa_ctx* c, const double* b, double* out, const fa_solver_params* p, fa_solver_stats* stats,
               bool overlap) {
    const int rc = solve(c, b, out, nullptr, p, stats);   // out holds y for now
    if (rc != FA_OK) return rc;
    const int V = c->g.V;
    const size_t s64 = (size_t)12 * V * sizeof(double2);
    cudaStream_t st = c->stream;
    FA_CUDA(c->io64b.ensure(s64), "alloc");
    double2* o = c->io64b.as<double2>();
    FA_TRY(hop_f64(c, c->y64.as<double2>(), o, std::sqrt(c->scale_c), false, !overlap, false, nullptr, nullptr,
                   nullptr));
    if (overlap) {
        FA_CUDA(c->io64a.ensure(s64), "alloc");
        double2* bp = c->io64a.as<double2>();
        FA_TRY(launch_pack_spinor_f64(c->g, b, bp, st));
        k_add_f64<<<(12 * V + kThreads - 1) / kThreads, kThreads, 0, st>>>(12 * V, bp, o);
        c->launches++;
        FA_LAUNCHED(c, "k_add_f64");
    }
    FA_TRY(launch_unpack_spinor_f64(c->g, o, out, st));
    c->launches++;
    FA_CUDA(cudaStreamSynchronize(st), "sync sign");
    return FA_OK;
}

// sign(H) b with k eigenpairs of H = g5 D_w treated exactly: a_i = <l_i, b>,
// sign(H) b = sum_i sign(Re lambda_i) a_i r_i + sign-by-poles(b - sum_i a_i r_i);
// D_ov b = b + g5 sign(H) b.  The k inner products are summed on the host in
// a fixed order (deterministic).
int apply_sign_deflated(fa_ctx* c, const double* b, double* out, int k, const double* lambda, const double* R,
                        const double* Lv, bool overlap, const fa_solver_params* p, fa_solver_stats* stats) {
    if (k == 0) return apply_sign(c, b, out, p, stats, overlap);
    if (!c->have_gauge || !c->have_params || !c->have_poles) return FA_ESTATE;
    const int n = 12 * c->g.V;
    const int nb = std::min((n + kThreads - 1) / kThreads, 4 * sms());
    cudaStream_t st = c->stream;
    const size_t part_n = (size_t)k * nb, coef_n = (size_t)3 * k;
    FA_CUDA(c->defl.ensure((part_n + coef_n + (size_t)n) * sizeof(double2)), "alloc deflation");
    double2* part = c->defl.as<double2>();
    double2* coef = part + part_n;     // [-a_i | sign(Re lambda_i) a_i | a_i]
    double2* bp = coef + coef_n;       // b - sum_i a_i r_i
    const double2* Rv = reinterpret_cast<const double2*>(R);
    const double2* Lw = reinterpret_cast<const double2*>(Lv);
    const double2* bv = reinterpret_cast<const double2*>(b);
    k_dots_canon<<<dim3(nb, k), kThreads, 0, st>>>(n, Lw, bv, part);
    FA_LAUNCHED(c, "k_dots_canon");
    std::vector<double2> hp(part_n), hc(coef_n);
    FA_CUDA(cudaMemcpyAsync(hp.data(), part, part_n * sizeof(double2), cudaMemcpyDeviceToHost, st), "copy partials");
    FA_CUDA(cudaStreamSynchronize(st), "sync deflation");
    for (int i = 0; i < k; ++i) {
        double re = 0.0, im = 0.0;
        for (int j = 0; j < nb; ++j) {
            re += hp[(size_t)i * nb + j].x;
            im += hp[(size_t)i * nb + j].y;
        }
        const double lr = lambda[2 * i];
        if (!std::isfinite(re) || !std::isfinite(im) || !std::isfinite(lr) || lr == 0.0) return FA_EINVAL;
        const double sg = lr > 0.0 ? 1.0 : -1.0;
        hc[i] = make_double2(-re, -im);
        hc[k + i] = make_double2(sg * re, sg * im);
        hc[2 * k + i] = make_double2(re, im);
    }
    FA_CUDA(cudaMemcpyAsync(coef, hc.data(), coef_n * sizeof(double2), cudaMemcpyHostToDevice, st), "copy coefficients");
    k_lincomb_canon<<<nb, kThreads, 0, st>>>(n, k, coef, Rv, bv, bp, 0);
    FA_LAUNCHED(c, "k_lincomb_canon");
    const int rc = apply_sign(c, reinterpret_cast<const double*>(bp), out, p, stats, overlap);
    if (rc != FA_OK) return rc;
    double2* o = reinterpret_cast<double2*>(out);
    if (!overlap) {
        k_lincomb_canon<<<nb, kThreads, 0, st>>>(n, k, coef + k, Rv, o, o, 0);
        FA_LAUNCHED(c, "k_lincomb_canon");
    } else {
        // out = b' + g5 sign(H) b'; add back sum_i a_i r_i and g5 sum_i sign_i a_i r_i
        k_lincomb_canon<<<nb, kThreads, 0, st>>>(n, k, coef + 2 * k, Rv, o, o, 0);
        FA_LAUNCHED(c, "k_lincomb_canon");
        k_lincomb_canon<<<nb, kThreads, 0, st>>>(n, k, coef + k, Rv, o, o, 1);
        FA_LAUNCHED(c, "k_lincomb_canon");
    }
    FA_CUDA(cudaStreamSynchronize(st), "sync deflation");
    return FA_OK;
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
    const int V = c->g.V, ns = c->ns;
    const int chunk = (p->shift_chunk > 0 && p->shift_chunk < ns) ? p->shift_chunk : ns;
    const size_t vs = (size_t)12 * V;
    const size_t sb = vs * sizeof(double2);
    cudaStream_t st = c->stream;
    const int nb = nblocks(V), rg = red_grid_for(V);
    FA_CUDA(c->gx.ensure((size_t)chunk * sb), "alloc gradient");
    FA_CUDA(c->io64a.ensure(sb), "alloc");
    FA_CUDA(c->io64b.ensure(sb), "alloc");
    FA_CUDA(c->tmp64.ensure(sb), "alloc");
    // mu-derivative partials of one chunk (summed on the host chunk by chunk, in
    // shift order) and the partials of <eta, y>
    FA_CUDA(c->gpart.ensure(((size_t)chunk * nb + 2 * (size_t)rg) * sizeof(double2)), "alloc");
    FA_CUDA(c->defl.ensure(2 * sb), "alloc");             // y and dL/db accumulators
    double2* yacc = c->defl.as<double2>();
    double2* bacc = yacc + vs;
    FA_CUDA(cudaMemsetAsync(dLdU, 0, (size_t)V * 72 * sizeof(double), st), "zero dL/dU");
    FA_CUDA(cudaMemsetAsync(yacc, 0, 2 * sb, st), "zero accumulators");
    double2* gxs = c->gx.as<double2>();
    double2* t1 = c->io64a.as<double2>();
    double2* t2 = c->io64b.as<double2>();
    double2* part = c->gpart.as<double2>();
    // the poles of the whole expansion; each chunk solves with a slice of them
    std::vector<double> om_all(c->omega, c->omega + ns), sg_all(c->sigma, c->sigma + ns);
    const double mu0 = c->mu;
    fa_solver_stats st1{}, st2{}, acc{};
    int rc = FA_OK;
    double dmu = 0.0;
    std::vector<double2> hmu((size_t)chunk * nb);
    for (int s0 = 0; s0 < ns && rc == FA_OK; s0 += chunk) {
        const int k = std::min(chunk, ns - s0);
        c->ns = k;
        for (int i = 0; i < k; ++i) {
            c->omega[i] = om_all[s0 + i];
            c->sigma[i] = sg_all[s0 + i];
        }
        rc = solve(c, b, nullptr, nullptr, &ps, &st1);
        if (rc != FA_OK) break;
        rc = ok(cudaMemcpyAsync(gxs, c->xs64.p, (size_t)k * sb, cudaMemcpyDeviceToDevice, st), "save x_s");
        if (rc != FA_OK) break;
        c->mu = -mu0;
        rc = solve(c, eta, nullptr, nullptr, &ps, &st2);
        c->mu = mu0;
        if (rc != FA_OK) break;
        const double2* lam = c->xs64.as<double2>();
        for (int i = 0; i < k && rc == FA_OK; ++i) {
            const double2* xs = gxs + i * vs;
            const double2* ls = lam + i * vs;
            rc = hop_f64(c, xs, t1, 1.0, false, true, false, nullptr, nullptr, nullptr);   // g5 D x
            if (rc == FA_OK) rc = hop_f64(c, ls, t2, 1.0, false, false, true, nullptr, nullptr, nullptr);   // D(-mu) lambda
            if (rc == FA_OK)
                rc = launch_force(c->g, links64_of(c), ls, t1, t2, xs, dLdU, -c->scale_c * om_all[s0 + i],
                                  std::exp(c->mu), std::exp(-c->mu), c->t_bc, part + (size_t)i * nb, st);
            c->launches++;
        }
        if (rc != FA_OK) break;
        // y += sum_chunk omega x; dL/db += sum_chunk omega lambda (the pole weights of the
        // chunk were uploaded by its solves: shift buffer, after sigma)
        const double* om_dev = reinterpret_cast<const double*>(c->shiftbuf.as<char>() + kMaxShifts * sizeof(double));
        k_combine<<<(12 * V + kThreads - 1) / kThreads, kThreads, 0, st>>>(V, k, om_dev, gxs, vs, yacc, 1);
        c->launches++;
        if (dLdb) {
            k_combine<<<(12 * V + kThreads - 1) / kThreads, kThreads, 0, st>>>(V, k, om_dev, lam, vs, bacc, 1);
            c->launches++;
        }
        rc = ok(cudaGetLastError(), "k_combine");
        if (rc == FA_OK)
            rc = ok(cudaMemcpyAsync(hmu.data(), part, (size_t)k * nb * sizeof(double2), cudaMemcpyDeviceToHost, st),
                    "read partials");
        if (rc == FA_OK) rc = ok(cudaStreamSynchronize(st), "sync gradient chunk");
        for (size_t q = 0; rc == FA_OK && q < (size_t)k * nb; ++q) dmu += hmu[q].x;
        acc.n_mv += st1.n_mv + st2.n_mv;
        acc.n_dot += st1.n_dot + st2.n_dot;
        acc.outer_iters += st1.outer_iters + st2.outer_iters;
        if (s0 == 0) acc.status = st1.status;
    }
    c->ns = ns;
    for (int i = 0; i < ns; ++i) {
        c->omega[i] = om_all[i];
        c->sigma[i] = sg_all[i];
    }
    c->mu = mu0;
    FA_TRY(rc);
    // L = Re <eta, y>
    FA_TRY(launch_pack_spinor_f64(c->g, eta, t1, st));
    k_dot2<double><<<rg, kThreads, 0, st>>>(V, t1, yacc, part);
    FA_LAUNCHED(c, "k_dot2");
    if (dLdb) FA_TRY(launch_unpack_spinor_f64(c->g, bacc, dLdb, st));
    std::vector<double2> h((size_t)rg);
    FA_CUDA(cudaMemcpyAsync(h.data(), part, h.size() * sizeof(double2), cudaMemcpyDeviceToHost, st), "read partials");
    FA_CUDA(cudaStreamSynchronize(st), "sync gradient");
    double lre = 0.0;
    for (int k = 0; k < rg; ++k) lre += h[k].x;
    *dLdmu = dmu;
    *L = lre;
    if (stats) {
        *stats = st1;
        stats->n_mv = acc.n_mv;
        stats->n_dot = acc.n_dot;
        stats->outer_iters = acc.outer_iters;
        stats->status = acc.status;
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

#include "eigs_impl.cuh"
#include "trace_impl.cuh"
