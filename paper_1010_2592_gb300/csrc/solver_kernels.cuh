// Device kernels of the multi-shift BiCGstab(l) solver (single-pass and
// double-pass forms of Sec. 2), shared by solver.cu.
//
// Seed recurrence (BiCGstab(l), Sleijpen-Fokkema, cited in Sec. 2):
//   outer m: rho0 <- -omega rho0; for j = 0..l-1:
//     rho1 = <rt, r_j>, beta = alpha rho1/rho0, rho0 = rho1
//     u_i <- r_i - beta u_i (i <= j);  u_{j+1} = A u_j;  alpha = rho0/<rt, u_{j+1}>
//     r_i <- r_i - alpha u_{i+1} (i <= j);  r_{j+1} = A r_j
//   MR: gamma minimises |r_0 - sum gamma_j r_j| (normal equations, pivoted elimination),
//     r_0 <- r_0 - sum gamma_j r_j, u_0 <- u_0 - sum gamma_j u_j, omega = gamma_l.
// Shifted systems (shift invariance, Sec. 1) carry zeta_s with r^s = r_0/zeta_s:
//   BiCG: zeta_new = (1 + alpha sigma) zeta + (alpha beta/alpha_prev)(zeta' - zeta),
//         alpha_s = alpha zeta/zeta_new, beta_s = beta (zeta'/zeta)^2,
//         u^s_i <- r_old_i/zeta - beta_s u^s_i, u^s_{j+1} <- (r_old_j/zeta - r_j/zeta_new)/alpha_s
//         - sigma u^s_j, x_s <- x_s + alpha_s u^s_0
//   MR:   p_s = 1 - sum gamma_j (-sigma)^j, c_k = sum_{j>k} gamma_j (-sigma)^{j-1-k},
//         x_s <- x_s + sum_k c_k r_k/(zeta p_s), u^s_0 <- (u^s_0 - sum gamma_j u^s_j)/p_s,
//         zeta <- zeta p_s, zeta' <- zeta' p_s.
// All scalars are FP64 and live on the device; vector kernels read the
// current outer iteration m and their scalars from the device record, so
// pass 1, pass 2 and any replay run the same kernels with the same
// arithmetic (explicit fma intrinsics, no contraction by the compiler).
#pragma once

#include "hop_device.cuh"
#include "trace.cuh"

namespace fa {

// ------------------------------------------------------------------ solver state
struct DevState {
    double2 rho0, alpha, omega, alpha_prev;
    double bnorm2, tol2b, theta2b, rnorm2;
    int m;           // current outer iteration
    int done;        // nonzero: pass-1 kernels return at once
    int status;      // fa_status of the solve
    int n_active;    // shifts not frozen
    int n_outer;     // M, set when pass 1 ends
    int switch_req;  // FA_MIXED: head residuals below the switch threshold
    int max_outer;
    unsigned ticket; // blocks of the current reduction that have stored their partials
};

// Per-shift record of pass 1 at outer iteration m (complex FP64):
//   sub-step j: [5j+0] alpha_s, [5j+1] beta_s, [5j+2] 1/zeta, [5j+3] 1/(alpha_s zeta),
//               [5j+4] 1/(alpha_s zeta_new)
//   MR:         [5l] 1/p_s, [5l+1+k] c_k/(zeta p_s), k < l
__host__ __device__ constexpr int ps_stride(int L) { return 6 * L + 1; }
// Pass-2 weights per outer iteration: slot (j, i) of the BiCG sub-step j for the
// occurrence r_i before its update (i <= j), then l MR slots for r_0..r_{l-1}.
__host__ __device__ constexpr int nc_slots(int L) { return L * (L + 1) / 2 + L; }
__host__ __device__ constexpr int slot_old(int j, int i) { return j * (j + 1) / 2 + i; }
__host__ __device__ constexpr int slot_mr(int L, int k) { return L * (L + 1) / 2 + k; }
__host__ __device__ constexpr int n_gram(int L) { return (L + 1) * (L + 2) / 2; }

// Everything one system needs on the device.  Kernels read their system's
// descriptor from an array (ds[blockIdx.y] for site kernels, ds[blockIdx.x]
// for the kernels with one block per system), so one launch serves a batch of
// systems of the same lattice shape; a single solve is a batch of one.
struct SolverDev {
    DevState* st;
    int ns, L, max_outer, V;
    Geom g;
    const double2* links64;
    const float4* links32;
    const float4* linksdf;            // double-float links [4][9][V]
    double diag, ef, eb, bc, scale;   // 4+m, e^{+mu}, e^{-mu}, time-boundary sign, c
    // the same operator scalars rounded to FP32 (multi-RHS sweep): 4+m and -1/2 for the
    // first hop of A, c (4+m) and -c/2 for the second, e^{+-mu}, the boundary sign
    float fdiag1, fhop1, fdiag2, fhop2, fef, feb, fbc;
    const double* sigma;   // [ns]
    const double* omega;   // [ns]
    double2* zeta;         // [ns]
    double2* zeta_p;       // [ns]
    int* active;           // [ns]
    int* iters;            // [ns]
    double2* rec_alpha;    // [max_outer][L]
    double2* rec_beta;     // [max_outer][L]
    double2* rec_gamma;    // [max_outer][L+1]
    double2* prec;         // [ns][max_outer][ps_stride]
    double2* coef;         // [max_outer][nc_slots]
    float4* coef4;         // the same weights as FP32 pairs (hi, lo) per part
    double2* cs;           // [ns][max_outer][nc_slots]   per-shift sweep output
    // seed vectors: r_0..r_l and u_0..u_l contiguous, the shadow vector, scratch
    double2 *r64, *u64, *rt64, *tmp64;
    float4 *r32, *u32, *rt32, *tmp32;
    double2* y;            // FP64 [12][V] result
    double2* xs;           // single-pass x_s   [ns][12][V]
    double2* us;           // single-pass u^s_i [ns][l+1][12][V]
    // pseudo-double-pass occurrence stores: outer iteration m is stored in the
    // FP64 store if m < cap64, in the FP32 store if 0 <= m - m0_32 < cap32
    char* store64;
    char* store32;
    int cap64, cap32, m0_32;
    int nblk, red_grid;    // hop partials per launch, grid of the reduction kernels
    double2* part;         // this system's reduction partials
    // reliable updates: seed solution x (FP64, [12][V], accumulated alongside the
    // recurrence when not null) and the packed source b (FP64)
    double2* x64;
    const double2* b64;
    // nonzero: max_outer is the planned number of outer iterations, reaching it
    // freezes the remaining shifts instead of failing (fixed-cost runs)
    int fixed_iters;
};

template <typename R> struct Vec;
template <> struct Vec<double> {
    using T = double2;
    __device__ static T* r(const SolverDev& d) { return d.r64; }
    __device__ static T* u(const SolverDev& d) { return d.u64; }
    __device__ static T* rt(const SolverDev& d) { return d.rt64; }
    __device__ static T* tmp(const SolverDev& d) { return d.tmp64; }
    __device__ static LinkView<double> links(const SolverDev& d) { return {d.links64, d.V}; }
};
// double-float vectors live in the FP64 buffers (same bytes: one float4 per complex)
template <> struct Vec<df> {
    using T = float4;
    __device__ static T* r(const SolverDev& d) { return reinterpret_cast<T*>(d.r64); }
    __device__ static T* u(const SolverDev& d) { return reinterpret_cast<T*>(d.u64); }
    __device__ static T* rt(const SolverDev& d) { return reinterpret_cast<T*>(d.rt64); }
    __device__ static T* tmp(const SolverDev& d) { return reinterpret_cast<T*>(d.tmp64); }
    __device__ static LinkView<df> links(const SolverDev& d) { return {d.linksdf, d.V}; }
};
template <> struct Vec<float> {
    using T = float4;
    __device__ static T* r(const SolverDev& d) { return d.r32; }
    __device__ static T* u(const SolverDev& d) { return d.u32; }
    __device__ static T* rt(const SolverDev& d) { return d.rt32; }
    __device__ static T* tmp(const SolverDev& d) { return d.tmp32; }
    __device__ static LinkView<float> links(const SolverDev& d) { return {d.links32, d.V}; }
};

// Position of a block in a launch that serves one or several systems.  Without
// a work table: system blockIdx.y, block blockIdx.x of gridDim.x (every system of
// the launch has the same lattice shape).  With a table (systems of different
// lattice shapes in one launch): tab[blockIdx.x] = (system, block within the
// system, vector blocks of the system, blocks of the system in this launch =
// the tickets of its reductions).  XS kernels: block -1 is the system's shift
// block (block 0 of the launch without a table).
struct Where {
    int sys, bx, nbx, ntk;
};
template <bool XS>
__device__ __forceinline__ Where where(const int4* tab) {
    if (tab != nullptr) {
        const int4 t = tab[blockIdx.x];
        return {t.x, t.y, t.z, t.w};
    }
    return {(int)blockIdx.y, (int)blockIdx.x - (XS ? 1 : 0), (int)gridDim.x - (XS ? 1 : 0), (int)gridDim.x};
}

// pass 1: the system has finished (converged, failed or max_outer);
// pass 2: the system has replayed all its outer iterations.
__device__ __forceinline__ bool sys_idle(const SolverDev& d, int pass2) {
    return pass2 ? (d.st->m >= d.st->n_outer) : (d.st->done != 0);
}

// ------------------------------------------------------------------ chunk IO
// A chunk is the vector unit of one load: FP64 one complex (double2, 12 per
// site), FP32 two complex (float4, 6 per site).
template <typename R> struct Ch;
template <> struct Ch<double> {
    static constexpr int W = 1, N = 12;
    using T = double2;
    cx<double> c[1];
    __device__ __forceinline__ static Ch ld(const T* b, int q, int V, int s) {
        double2 t = b[(size_t)q * V + s];
        Ch r; r.c[0] = {t.x, t.y}; return r;
    }
    __device__ __forceinline__ void stv(T* b, int q, int V, int s) const {
        b[(size_t)q * V + s] = make_double2(c[0].r, c[0].i);
    }
    // evict-first store / load (occurrence store: written once, read once by the gather)
    __device__ __forceinline__ void stv_cs(T* b, int q, int V, int s) const {
        __stcs(b + (size_t)q * V + s, make_double2(c[0].r, c[0].i));
    }
    __device__ __forceinline__ static Ch ld_cs(const T* b, int q, int V, int s) {
        double2 t = __ldcs(b + (size_t)q * V + s);
        Ch r; r.c[0] = {t.x, t.y}; return r;
    }
};
template <> struct Ch<df> {
    static constexpr int W = 1, N = 12;
    using T = float4;
    cx<df> c[1];
    __device__ __forceinline__ static Ch ld(const T* b, int q, int V, int s) {
        float4 t = b[(size_t)q * V + s];
        Ch r; r.c[0] = {df(t.x, t.y), df(t.z, t.w)}; return r;
    }
    __device__ __forceinline__ void stv(T* b, int q, int V, int s) const {
        b[(size_t)q * V + s] = make_float4(c[0].r.hi, c[0].r.lo, c[0].i.hi, c[0].i.lo);
    }
    __device__ __forceinline__ void stv_cs(T* b, int q, int V, int s) const {
        __stcs(b + (size_t)q * V + s, make_float4(c[0].r.hi, c[0].r.lo, c[0].i.hi, c[0].i.lo));
    }
    __device__ __forceinline__ static Ch ld_cs(const T* b, int q, int V, int s) {
        float4 t = __ldcs(b + (size_t)q * V + s);
        Ch r; r.c[0] = {df(t.x, t.y), df(t.z, t.w)}; return r;
    }
};
template <> struct Ch<float> {
    static constexpr int W = 2, N = 6;
    using T = float4;
    cx<float> c[2];
    __device__ __forceinline__ static Ch ld(const T* b, int q, int V, int s) {
        float4 t = b[(size_t)q * V + s];
        Ch r; r.c[0] = {t.x, t.y}; r.c[1] = {t.z, t.w}; return r;
    }
    __device__ __forceinline__ void stv(T* b, int q, int V, int s) const {
        b[(size_t)q * V + s] = make_float4(c[0].r, c[0].i, c[1].r, c[1].i);
    }
    __device__ __forceinline__ void stv_cs(T* b, int q, int V, int s) const {
        __stcs(b + (size_t)q * V + s, make_float4(c[0].r, c[0].i, c[1].r, c[1].i));
    }
    __device__ __forceinline__ static Ch ld_cs(const T* b, int q, int V, int s) {
        float4 t = __ldcs(b + (size_t)q * V + s);
        Ch r; r.c[0] = {t.x, t.y}; r.c[1] = {t.z, t.w}; return r;
    }
};

template <typename R> __device__ __forceinline__ size_t vstride(const SolverDev& d) {
    return (size_t)Ch<R>::N * d.V;
}

// store slots of outer iteration m, or nullptr when m is not stored
template <typename R>
__device__ __forceinline__ typename Ch<R>::T* store_at(const SolverDev& d, int m) {
    const size_t per = (size_t)nc_slots(d.L) * vstride<R>(d) * sizeof(typename Ch<R>::T);
    if (sizeof(R) == 8) {
        if (m < d.cap64) return reinterpret_cast<typename Ch<R>::T*>(d.store64 + (size_t)m * per);
    } else {
        const int k = m - d.m0_32;
        if (d.m0_32 >= 0 && k >= 0 && k < d.cap32) return reinterpret_cast<typename Ch<R>::T*>(d.store32 + (size_t)k * per);
    }
    return nullptr;
}

template <typename R> __device__ __forceinline__ cx<R> tocx(double2 v) { return {fromdbl<R>(v.x), fromdbl<R>(v.y)}; }
template <typename R> __device__ __forceinline__ cx<R> negcx(double2 v) {
    return {fromdbl<R>(-v.x), fromdbl<R>(-v.y)};
}
// pass-2 weight k in R from its FP64 and FP32-pair copies (the same value as
// tocx<R>(cf[k]); the pair form needs no FP64 conversion per thread)
template <typename R> __device__ __forceinline__ cx<R> weight(const double2* cf, const float4* cf4, size_t k) {
    if constexpr (std::is_same<R, double>::value) {
        return tocx<double>(cf[k]);
    } else {
        const float4 t = cf4[k];
        if constexpr (std::is_same<R, float>::value) return {t.x, t.z};
        else return {df(t.x, t.y), df(t.z, t.w)};
    }
}

// y (FP64, [12][V]) += t for the W complex components of chunk q
template <typename R>
__device__ __forceinline__ void acc_y(double2* y, int q, int V, int s, const cx<R> (&t)[Ch<R>::W]) {
#pragma unroll
    for (int w = 0; w < Ch<R>::W; ++w) {
        double2* p = y + (size_t)(q * Ch<R>::W + w) * V + s;
        double2 a = *p;
        a.x = __dadd_rn(a.x, todbl(t[w].r));
        a.y = __dadd_rn(a.y, todbl(t[w].i));
        *p = a;
    }
}

// x (FP64) += a v for the W components of chunk q
template <typename R>
__device__ __forceinline__ void acc_x(double2* x, int q, int V, int s, double2 a, const Ch<R>& v) {
#pragma unroll
    for (int w = 0; w < Ch<R>::W; ++w) {
        double2* p = x + (size_t)(q * Ch<R>::W + w) * V + s;
        double2 t = *p;
        const double vr = todbl(v.c[w].r), vi = todbl(v.c[w].i);
        t.x = __fma_rn(a.x, vr, t.x);
        t.x = __fma_rn(-a.y, vi, t.x);
        t.y = __fma_rn(a.x, vi, t.y);
        t.y = __fma_rn(a.y, vr, t.y);
        *p = t;
    }
}

// ------------------------------------------------------------------ scalar steps
// The scalar steps of the recurrence run inside the vector kernels, in two
// parts.  The seed part (beta, alpha, the MR coefficients gamma, convergence)
// runs in the last block of the reduction kernel whose partials it reads: each
// block stores its partials, fences and takes a ticket, and the block holding
// the last ticket sums all partials in a fixed order (so the result does not
// depend on which block finished last) and runs the step.  The shift part (the
// zeta recurrences and the per-shift scalars of every BiCG sub-step and MR
// step) is not needed by the next seed-vector kernel: in the double-pass forms
// it runs in an extra block 0 of that next kernel, beside its vector blocks.
// Single-pass solves consume the shift scalars at once and run both parts in
// the last block.
//
// FP64 instructions are scarce on this part (one warp instruction occupies a
// sub-partition's FP64 pipe for tens of cycles, a division for hundreds), so
// the steps use fused multiply-adds, one real division per complex inverse,
// and reuse inverses between the per-shift scalars.
//
// The step's code runs once per launch, in whichever block takes the last
// ticket, so its instructions are usually not in that SM's instruction cache:
// on GB300 (16^3 x 32 solve) fetching them from L2 took most of the last
// block's time (a reduction of 2 x 512 partials: 4.6 us with cold code, 1.3 us
// with the same code run once before on other data).  So the blocks that take
// one of the last kWarmTickets tickets, other than the last, run the step as a
// dry run (no partial loads, no stores; `dry` below) before they exit: the
// blocks that share an SM with the last block finish shortly before it, and
// their dry runs bring the code into that SM's instruction cache while the
// last block still works.  Results do not change: a dry run reads state but
// writes nothing outside its own shared memory.  Only in launches of at most
// about one wave (8 blocks per SM): in a longer launch a block that lingers
// for its dry run holds back the blocks still waiting for a slot (the
// 72-system batch, one launch for all systems, measured 3-10 % slower).
constexpr unsigned kWarmTickets = 1024, kWarmSkip = 32;
enum { LB_NONE = 0, LB_WARM = 1, LB_LAST = 2 };
__device__ __forceinline__ unsigned sm_count_dev() {
    unsigned n;
    asm("mov.u32 %0, %%nsmid;" : "=r"(n));
    return n;
}
__device__ __forceinline__ int last_block(DevState* S, int ntickets) {
    __shared__ int is_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        // thread 0 stored the block's partials; the fence is cumulative over
        // what the barrier ordered before it (release), and the one after the
        // last ticket orders the reads that follow (acquire; the other threads
        // read the partials after the barrier, from L2)
        __threadfence();
        const unsigned t = atomicAdd(&S->ticket, 1u);
        // (the last kWarmSkip before the last block run no dry run: they would
        // end after it on an SM whose code is still cold)
        const bool one_wave = gridDim.x * gridDim.y <= 8u * sm_count_dev();
        is_last = t == (unsigned)ntickets - 1u ? LB_LAST
                  : (one_wave && t + kWarmTickets >= (unsigned)ntickets && t + 1u + kWarmSkip < (unsigned)ntickets
                         ? LB_WARM
                         : LB_NONE);
        if (is_last == LB_LAST) {
            S->ticket = 0u;   // every block of this launch has taken its ticket
            __threadfence();
        }
    }
    __syncthreads();
    return is_last;
}

__device__ __forceinline__ dcx zneg(dcx a) { return {-a.r, -a.i}; }   // a sign flip, free on FMA operands
__device__ __forceinline__ dcx zmul(dcx a, dcx b) {
    return {__fma_rn(a.r, b.r, -__dmul_rn(a.i, b.i)), __fma_rn(a.r, b.i, __dmul_rn(a.i, b.r))};
}
__device__ __forceinline__ dcx zfma(dcx a, dcx b, dcx c) {   // a b + c
    return {__fma_rn(a.r, b.r, __fma_rn(-a.i, b.i, c.r)), __fma_rn(a.r, b.i, __fma_rn(a.i, b.r, c.i))};
}
__device__ __forceinline__ dcx zrfma(double a, dcx b, dcx c) { return {__fma_rn(a, b.r, c.r), __fma_rn(a, b.i, c.i)}; }
__device__ __forceinline__ dcx zscale(double a, dcx b) { return {__dmul_rn(a, b.r), __dmul_rn(a, b.i)}; }
__device__ __forceinline__ dcx zsub(dcx a, dcx b) { return {__dsub_rn(a.r, b.r), __dsub_rn(a.i, b.i)}; }
__device__ __forceinline__ double zabs2(dcx a) { return __fma_rn(a.r, a.r, __dmul_rn(a.i, a.i)); }
__device__ __forceinline__ dcx zconj_scale(double a, dcx b) { return {__dmul_rn(a, b.r), -__dmul_rn(a, b.i)}; }
__device__ __forceinline__ dcx zinv(dcx a) { return zconj_scale(1.0 / zabs2(a), a); }
__device__ __forceinline__ bool zfinite(dcx a) { return isfinite(a.r) && isfinite(a.i); }
// 2^-floor(e/2) for x = f 2^e (x > 0, normal): x * result^2 lies in [1, 4).
// Integer work on the exponent bits only.
__device__ __forceinline__ double pow2_rsqrt(double x) {
    const long long bits = __double_as_longlong(x);
    const int e = (int)((bits >> 52) & 0x7ff) - 1023;
    const int h = e >= 0 ? e / 2 : -((1 - e) / 2);     // floor(e / 2)
    return __longlong_as_double((long long)(1023 - h) << 52);
}
// 1/p and 1/q (p, q > 0) from one division while p q stays well inside the
// FP64 range, else from two
__device__ __forceinline__ void recip2(double p, double q, double& ip, double& iq) {
    const double pq = __dmul_rn(p, q);
    if (pq > 1e-280 && pq < 1e280) {
        const double r = 1.0 / pq;
        ip = __dmul_rn(q, r);
        iq = __dmul_rn(p, r);
    } else {
        ip = 1.0 / p;
        iq = 1.0 / q;
    }
}

// Sums of the nblk partials of slots 0..ns-1 into out[0..ns-1], fixed order:
// each slot is split into four quarters, one warp each (consecutive warps sit
// on different sub-partitions), summed by the lanes in strided order and a
// shuffle tree; the quarters are then added in order.  Partials are read from
// L2 (other blocks of the same launch stored them).  DFP: the partials are
// FP32 pairs (float4: re.hi, re.lo, im.hi, im.lo; the FP32 and double-float
// kernels store them so) and are summed in double-float on the FP32 pipe;
// otherwise FP64 values summed in FP64.
template <typename R> constexpr bool dfp_of() { return !std::is_same<R, double>::value; }

// dry: warp 0 runs the code of one quarter once, every load predicated off
// (the sums are 0); the other warps only meet the barriers.
template <int NSMAX, bool DFP>
__device__ __forceinline__ void reduce_slots(const double2* part, int nblk, int ns, dcx* out, bool dry = false) {
    __shared__ double2 qs[4 * NSMAX];
    __shared__ float4 qf[4 * NSMAX];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int per = (nblk + 3) >> 2;
    const int ntask = dry ? 1 : 4 * ns;
    if (dry && (int)threadIdx.x < 4 * ns) {   // the quarters a dry run leaves out
        qs[threadIdx.x] = make_double2(0.0, 0.0);
        qf[threadIdx.x] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    // Several slots (the Gram matrix) and quarters of at most 256 partials: each
    // warp takes two quarters at a time, u and u + nw, with the sixteen loads in
    // flight together (the loads were the time: six rounds of them for 6 x 1024
    // partials in a 128-thread block).  The additions of each quarter are those
    // of the loop below, in the same order.  A dry run takes this path too (its
    // code is the one to bring into the instruction cache).
    int u_first = warp;
    if constexpr (DFP && NSMAX >= 3) {
        if (per <= 256) {
            for (int u = warp; u < ntask; u += 2 * nw) {
                const int u2 = u + nw;
                const bool two = u2 < ntask;
                const int i0 = (u & 3) * per, i1 = dry ? i0 : min(nblk, i0 + per);
                const int j0 = (u2 & 3) * per, j1 = (two && !dry) ? min(nblk, j0 + per) : j0;
                const float4* pf = reinterpret_cast<const float4*>(part) + (size_t)(u >> 2) * nblk;
                const float4* pg = reinterpret_cast<const float4*>(part) + (size_t)(u2 >> 2) * nblk;
                float4 v[8], x[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int i = i0 + lane + 32 * t, j = j0 + lane + 32 * t;
                    v[t] = i < i1 ? __ldcg(pf + i) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    x[t] = j < j1 ? __ldcg(pg + j) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                }
                df a(0.0f), b(0.0f), c(0.0f), e(0.0f);
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    a = addR(a, df(v[t].x, v[t].y));
                    b = addR(b, df(v[t].z, v[t].w));
                    c = addR(c, df(x[t].x, x[t].y));
                    e = addR(e, df(x[t].z, x[t].w));
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    a = addR(a, shfl_down_df(a, o));
                    b = addR(b, shfl_down_df(b, o));
                    c = addR(c, shfl_down_df(c, o));
                    e = addR(e, shfl_down_df(e, o));
                }
                if (lane == 0) {
                    qf[u] = make_float4(a.hi, a.lo, b.hi, b.lo);
                    if (two) qf[u2] = make_float4(c.hi, c.lo, e.hi, e.lo);
                }
            }
            u_first = ntask;   // every quarter done
        }
    }
    for (int u = u_first; u < ntask; u += nw) {
        const int k = u >> 2;
        const int i0 = (u & 3) * per, i1 = dry ? i0 : min(nblk, i0 + per);
        const int iend = dry ? i0 + 32 : i1;
        if constexpr (DFP) {
            const float4* pf = reinterpret_cast<const float4*>(part) + (size_t)k * nblk;
            df a(0.0f), b(0.0f);
            // eight loads in flight per lane before the adds (zero padding
            // leaves the sums unchanged)
            for (int ib = i0 + lane; ib < iend; ib += 32 * 8) {
                float4 v[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int i = ib + 32 * t;
                    v[t] = i < i1 ? __ldcg(pf + i) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                }
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    a = addR(a, df(v[t].x, v[t].y));
                    b = addR(b, df(v[t].z, v[t].w));
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a = addR(a, shfl_down_df(a, o));
                b = addR(b, shfl_down_df(b, o));
            }
            if (lane == 0) qf[u] = make_float4(a.hi, a.lo, b.hi, b.lo);
        } else {
            const double2* pd = part + (size_t)k * nblk;
            double a = 0.0, b = 0.0;
            for (int ib = i0 + lane; ib < iend; ib += 32 * 8) {
                double2 v[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int i = ib + 32 * t;
                    v[t] = i < i1 ? __ldcg(pd + i) : make_double2(0.0, 0.0);
                }
                const int nt = min(8, (max(i1, ib + 1) - ib + 31) >> 5);   // loads that hit (FP64 adds are scarce)
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    if (t < nt) {
                        a = __dadd_rn(a, v[t].x);
                        b = __dadd_rn(b, v[t].y);
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a = __dadd_rn(a, __shfl_down_sync(0xffffffffu, a, o));
                b = __dadd_rn(b, __shfl_down_sync(0xffffffffu, b, o));
            }
            if (lane == 0) qs[u] = make_double2(a, b);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < ns; k += blockDim.x) {
        if constexpr (DFP) {
            df a(0.0f), b(0.0f);
#pragma unroll 1
            for (int q = 0; q < 4; ++q) {
                const float4 t = qf[4 * k + q];
                a = addR(a, df(t.x, t.y));
                b = addR(b, df(t.z, t.w));
            }
            out[k] = {todbl(a), todbl(b)};
        } else {
            const double2 q0 = qs[4 * k], q1 = qs[4 * k + 1], q2 = qs[4 * k + 2], q3 = qs[4 * k + 3];
            out[k] = {__dadd_rn(__dadd_rn(q0.x, q1.x), __dadd_rn(q2.x, q3.x)),
                      __dadd_rn(__dadd_rn(q0.y, q1.y), __dadd_rn(q2.y, q3.y))};
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void fail(DevState* S, int code) {
    if (S->status == FA_OK) S->status = code;
    S->done = 1;
}

// start of pass 1: partials hold <rt, r0> and |r0|^2 with r0 = rt = b
template <bool DFP>
__device__ __noinline__ void sc_init(const SolverDev& d, int nblk, double tol, double theta) {
    DevState* S = d.st;
    __shared__ dcx red[2];
    reduce_slots<2, DFP>(d.part, nblk, 2, red);
    const dcx rtr = red[0];
    const double bb = red[1].r;
    for (int sh = threadIdx.x; sh < d.ns; sh += blockDim.x) {
        d.zeta[sh] = pk(mk(1.0));
        d.zeta_p[sh] = pk(mk(1.0));
        d.active[sh] = 1;
        d.iters[sh] = 0;
    }
    if (threadIdx.x == 0) {
        S->bnorm2 = bb;
        S->tol2b = tol * tol * bb;
        S->theta2b = theta * theta * bb;
        S->rnorm2 = bb;
        S->m = 0;
        S->done = 0;
        S->status = FA_OK;
        S->n_active = d.ns;
        S->n_outer = 0;
        S->switch_req = 0;
        S->max_outer = d.max_outer;
        S->omega = pk(mk(1.0));
        S->alpha = pk(mk(0.0));
        S->alpha_prev = pk(mk(1.0));
        // first BiCG sub-step: rho0 <- -omega rho0 with rho0 = 1; beta = alpha rho1/rho0 = 0
        S->rho0 = pk(rtr);
        d.rec_beta[0] = pk(mk(0.0));
        if (!(bb > 0.0) || !isfinite(bb)) fail(S, FA_EINVAL);
    }
}

// beta of BiCG sub-step j >= 1 from partials of <rt, r_j>
template <bool DFP>
__device__ __noinline__ void sc_beta(const SolverDev& d, int j, int nblk, bool dry) {
    DevState* S = d.st;
    // the state loads are issued with the partial loads and consumed after the
    // reduction (one memory round trip; the done flag only matters then)
    const int done = S->done, m = S->m;
    const dcx rho0 = ld(S->rho0), alpha = ld(S->alpha);
    __shared__ dcx red[1];
    reduce_slots<1, DFP>(d.part, nblk, 1, red, dry);
    if (done) return;
    if (threadIdx.x == 0) {
        const dcx rho1 = red[0];
        if (zabs2(rho0) == 0.0) { if (!dry) fail(S, FA_EBREAKDOWN); return; }
        const dcx beta = zmul(zmul(alpha, rho1), zinv(rho0));
        if (!zfinite(beta)) { if (!dry) fail(S, FA_ENONFINITE); return; }
        if (dry) { red[0] = beta; return; }   // (kept, so that the arithmetic stays on the dry path)
        S->rho0 = pk(rho1);
        d.rec_beta[m * d.L + j] = pk(beta);
    }
}

// alpha of BiCG sub-step j from partials of <rt, u_{j+1}> (seed part)
template <bool DFP>
__device__ __noinline__ void sc_alpha_seed(const SolverDev& d, int j, int nblk, bool dry) {
    DevState* S = d.st;
    const int done = S->done, m = S->m;
    const dcx rho0 = ld(S->rho0);
    __shared__ dcx red[1];
    reduce_slots<1, DFP>(d.part, nblk, 1, red, dry);
    if (done) return;
    if (threadIdx.x == 0) {
        const dcx den = dry ? mk(1.0) : red[0];
        if (zabs2(den) == 0.0) { fail(S, FA_EBREAKDOWN); return; }
        const dcx alpha = zmul(rho0, zinv(den));
        if (!zfinite(alpha)) { if (!dry) fail(S, FA_ENONFINITE); return; }
        if (dry) { red[0] = alpha; return; }
        d.rec_alpha[m * d.L + j] = pk(alpha);
        S->alpha = pk(alpha);
        S->alpha_prev = pk(alpha);
    }
}

// Shift part of BiCG sub-step j of the current outer iteration, from the
// recorded alpha, beta and the previous sub-step's alpha:
//   zeta_new = (1 + sigma alpha) zeta + (alpha beta / alpha_prev)(zeta' - zeta)
//   alpha_s = alpha zeta / zeta_new,  beta_s = beta (zeta' / zeta)^2
// and the weights 1/zeta, 1/(alpha_s zeta) = zeta_new / (alpha zeta^2),
// 1/(alpha_s zeta_new) = 1/(alpha zeta) that the sweep and the single-pass
// shift updates use.  One division per shift (recip2).
__device__ __noinline__ void sc_alpha_shifts(const SolverDev& d, int j) {
    DevState* S = d.st;
    if (S->done) return;
    const int m = S->m;
    const int t = m * d.L + j;
    const dcx alpha = ld(d.rec_alpha[t]);
    const dcx beta = ld(d.rec_beta[t]);
    const dcx aprev = t > 0 ? ld(d.rec_alpha[t - 1]) : mk(1.0);
    // 1/alpha and 1/alpha_prev from one division
    double ina, inp;
    recip2(zabs2(alpha), zabs2(aprev), ina, inp);
    const dcx inv_a = zconj_scale(ina, alpha);
    const dcx inv_p = zconj_scale(inp, aprev);
    const dcx c1 = zmul(zmul(alpha, beta), inv_p);
    for (int sh = threadIdx.x; sh < d.ns; sh += blockDim.x) {
        if (!d.active[sh]) continue;
        const double sg = d.sigma[sh];
        const dcx z = ld(d.zeta[sh]), zp = ld(d.zeta_p[sh]);
        const dcx zs = zrfma(sg, zmul(alpha, z), z);            // (1 + sigma alpha) zeta
        const dcx zn = zfma(c1, zsub(zp, z), zs);
        const double nzn = zabs2(zn);
        double izn, iz;
        recip2(nzn, zabs2(z), izn, iz);
        const dcx inv_zn = zconj_scale(izn, zn);
        const dcx inv_z = zconj_scale(iz, z);
        const dcx as = zmul(zmul(alpha, z), inv_zn);
        const dcx r = zmul(zp, inv_z);
        const dcx bs = zmul(beta, zmul(r, r));
        const dcx iaz = zmul(inv_a, inv_z);                       // 1/(alpha zeta)
        double2* P = d.prec + ((size_t)sh * d.max_outer + m) * ps_stride(d.L) + 5 * j;
        P[0] = pk(as);
        P[1] = pk(bs);
        P[2] = pk(inv_z);
        P[3] = pk(zmul(zn, zmul(iaz, inv_z)));
        P[4] = pk(iaz);
        if (!(nzn > 0.0) || !isfinite(izn) || !zfinite(as) || !zfinite(zn)) fail(S, FA_ENONFINITE);
        d.zeta_p[sh] = pk(z);
        d.zeta[sh] = pk(zn);
    }
}

// MR coefficients gamma (seed part) from the Gram partials: diagonally scaled
// normal equations, Gaussian elimination with partial pivoting.
template <int L, bool DFP>
__device__ __noinline__ void sc_mr_seed(const SolverDev& d, int nblk, bool dry) {
    DevState* S = d.st;
    const int done = S->done, m = S->m;
    constexpr int NG = n_gram(L);
    __shared__ dcx G[NG];
    reduce_slots<NG, DFP>(d.part, nblk, NG, G, dry);
    if (done || threadIdx.x != 0) return;
    int bad = 0;
    // slot of (i, k), i <= k, in the row-major upper triangle
    auto slot = [](int i, int k) { return i * (L + 1) - i * (i - 1) / 2 + (k - i); };
    if (dry)   // a regular Gram matrix, so that the dry run takes the solving path
        for (int i = 0; i <= L; ++i) G[slot(i, i)] = mk(1.0);
    dcx gam[L + 1];
    gam[0] = mk(-1.0);
    for (int i = 1; i <= L; ++i) {
        const double gii = G[slot(i, i)].r;
        if (!(gii > 0.0) || !isfinite(gii)) bad = FA_EBREAKDOWN;
    }
    if constexpr (L == 1) {
        // gamma_1 = <r_1, r_0> / <r_1, r_1>
        if (!bad) gam[1] = zscale(1.0 / G[slot(1, 1)].r, conjd(G[slot(0, 1)]));
    } else if constexpr (L == 2) {
        // Cramer's rule on the Hermitian 2 x 2 normal equations (no scaling:
        // the rule is covariant under it)
        const double g11 = G[slot(1, 1)].r, g22 = G[slot(2, 2)].r;
        const dcx g12 = G[slot(1, 2)];
        const dcx b1 = conjd(G[slot(0, 1)]), b2 = conjd(G[slot(0, 2)]);   // <r_i, r_0>
        const double det = __fma_rn(g11, g22, -zabs2(g12));
        if (bad || !(det != 0.0) || !isfinite(det)) {
            bad = bad ? bad : FA_EBREAKDOWN;
        } else {
            const double idet = 1.0 / det;
            gam[1] = zscale(idet, zsub(zscale(g22, b1), zmul(g12, b2)));
            gam[2] = zscale(idet, zsub(zscale(g11, b2), zmul(conjd(g12), b1)));
        }
    } else {
        // Diagonal scaling by powers of two (exact; integer work only), so that
        // the scaled diagonal lies in [1, 4).
        double dsc[L];
        for (int i = 1; i <= L; ++i) dsc[i - 1] = pow2_rsqrt(G[slot(i, i)].r);
        dcx Ab[L][L + 1];
        for (int i = 1; i <= L; ++i) {
            for (int k = 1; k <= L; ++k) {
                const dcx gik = (i <= k) ? G[slot(i, k)] : conjd(G[slot(k, i)]);
                Ab[i - 1][k - 1] = zscale(__dmul_rn(dsc[i - 1], dsc[k - 1]), gik);
            }
            Ab[i - 1][L] = zscale(dsc[i - 1], conjd(G[slot(0, i)]));   // <r_i, r_0>
        }
        dcx z[L];
        {
            // elimination with partial pivoting (the power basis r_1..r_l can
            // make the normal equations numerically indefinite for large l; any
            // solution is a valid MR polynomial); one inverse per pivot
            dcx ipiv[L];
            for (int k = 0; k < L && !bad; ++k) {
                int pr = k;
                double best = zabs2(Ab[k][k]);
                for (int i = k + 1; i < L; ++i)
                    if (zabs2(Ab[i][k]) > best) { best = zabs2(Ab[i][k]); pr = i; }
                if (!(best > 0.0)) { bad = FA_EBREAKDOWN; break; }
                if (pr != k)
                    for (int q = k; q <= L; ++q) { dcx tq = Ab[k][q]; Ab[k][q] = Ab[pr][q]; Ab[pr][q] = tq; }
                ipiv[k] = zinv(Ab[k][k]);
                for (int i = k + 1; i < L; ++i) {
                    const dcx f = zmul(Ab[i][k], ipiv[k]);
                    for (int q = k + 1; q <= L; ++q) Ab[i][q] = zsub(Ab[i][q], zmul(f, Ab[k][q]));
                }
            }
            if (!bad) {
                for (int i = L - 1; i >= 0; --i) {
                    dcx v = Ab[i][L];
                    for (int q = i + 1; q < L; ++q) v = zsub(v, zmul(Ab[i][q], z[q]));
                    z[i] = zmul(v, ipiv[i]);
                }
            }
        }
        if (!bad)
            for (int j = 1; j <= L; ++j) gam[j] = zscale(dsc[j - 1], z[j - 1]);
    }
    if (!bad)
        for (int j = 1; j <= L; ++j)
            if (!zfinite(gam[j])) bad = FA_ENONFINITE;
    if (dry) {
        if (!bad) G[0] = gam[L];
        return;
    }
    if (bad) { fail(S, bad); return; }
    for (int j = 0; j <= L; ++j) d.rec_gamma[m * (L + 1) + j] = pk(gam[j]);
    S->omega = pk(gam[L]);
}

// Shift part of the MR step: p_s = 1 - sum_j gamma_j (-sigma)^j, the weights
// 1/p_s and c_k/(zeta p_s) with c_k = sum_{j>k} gamma_j (-sigma)^{j-1-k}, and
// zeta <- zeta p_s, zeta' <- zeta' p_s.  The powers of -sigma are real.
template <int L>
__device__ __noinline__ void sc_mr_shifts(const SolverDev& d) {
    DevState* S = d.st;
    if (S->done) return;
    const int m = S->m;
    dcx gam[L + 1];
#pragma unroll
    for (int j = 0; j <= L; ++j) gam[j] = ld(d.rec_gamma[m * (L + 1) + j]);
    for (int sh = threadIdx.x; sh < d.ns; sh += blockDim.x) {
        if (!d.active[sh]) continue;
        const double ms = -d.sigma[sh];
        double pw[L + 1];
        pw[0] = 1.0;
#pragma unroll
        for (int j = 1; j <= L; ++j) pw[j] = __dmul_rn(pw[j - 1], ms);
        dcx ps = mk(1.0);
#pragma unroll
        for (int j = 1; j <= L; ++j) ps = zrfma(-pw[j], gam[j], ps);
        const dcx z = ld(d.zeta[sh]);
        const dcx zps = zmul(z, ps);
        const double nps = zabs2(ps);
        double ips, izps;
        recip2(nps, zabs2(zps), ips, izps);
        const dcx inv_ps = zconj_scale(ips, ps);
        const dcx inv_zps = zconj_scale(izps, zps);
        double2* P = d.prec + ((size_t)sh * d.max_outer + m) * ps_stride(L) + 5 * L;
        P[0] = pk(inv_ps);
#pragma unroll
        for (int k = 0; k < L; ++k) {
            dcx c = mk(0.0);
#pragma unroll
            for (int j = k + 1; j <= L; ++j) c = zrfma(pw[j - 1 - k], gam[j], c);
            P[1 + k] = pk(zmul(c, inv_zps));
        }
        if (!(nps > 0.0) || !isfinite(ips) || !isfinite(izps) || !zfinite(ps)) fail(S, FA_ENONFINITE);
        d.zeta[sh] = pk(zps);
        d.zeta_p[sh] = pk(zmul(ld(d.zeta_p[sh]), ps));
    }
}

// end of an outer iteration: convergence and freezing of shifts, next beta
template <bool DFP>
__device__ __noinline__ void sc_conv(const SolverDev& d, int nblk, int head, bool dry) {
    DevState* S = d.st;
    // every load the step needs is issued with the partial loads and consumed
    // after the reduction (one memory round trip)
    const int done = S->done, m = S->m;
    const double tol2b = S->tol2b, theta2b = S->theta2b;
    const dcx omega = ld(S->omega), rho_old = ld(S->rho0), alpha = ld(S->alpha);
    const int sh = threadIdx.x;     // one thread per shift (kMaxShifts <= blockDim.x)
    const int act = sh < d.ns ? d.active[sh] : 0;
    const double2 zv = sh < d.ns ? d.zeta[sh] : make_double2(0.0, 0.0);
    __shared__ dcx red[2];
    reduce_slots<2, DFP>(d.part, nblk, 2, red, dry);
    if (done) return;
    const dcx rtr = dry ? mk(1.0) : red[0];
    const double rn2 = dry ? 1.0 : red[1].r;
    __shared__ int n_act, all_small;
    if (threadIdx.x == 0) { n_act = 0; all_small = 1; }
    __syncthreads();
    const bool last = d.fixed_iters && m + 1 >= d.max_outer;
    if (act) {
        const double z2 = zabs2(ld(zv));
        if (last || rn2 <= tol2b * z2) {
            if (!dry) {
                d.active[sh] = 0;
                d.iters[sh] = m + 1;
            }
        } else {
            atomicAdd(&n_act, 1);
            if (rn2 > theta2b * z2) atomicAnd(&all_small, 0);
        }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    if (!dry) {
        S->rnorm2 = rn2;
        S->m = m + 1;
        S->n_active = n_act;
    }
    if (!isfinite(rn2) || !zfinite(rtr)) {
        if (!dry) { fail(S, FA_ENONFINITE); S->n_outer = m + 1; }
        return;
    }
    if (head && all_small && !dry) S->switch_req = 1;
    if (n_act == 0) {
        if (!dry) { S->done = 1; S->n_outer = m + 1; }
        return;
    }
    if (m + 1 >= d.max_outer) {
        if (!dry) { fail(S, FA_ENOCONV); S->n_outer = m + 1; }
        return;
    }
    const dcx rho0 = zneg(zmul(omega, rho_old));
    if (zabs2(rho0) == 0.0) {
        if (!dry) { fail(S, FA_EBREAKDOWN); S->n_outer = m + 1; }
        return;
    }
    const dcx beta = zmul(zmul(alpha, rtr), zinv(rho0));
    if (dry) { red[0] = beta; return; }
    S->rho0 = pk(rtr);
    d.rec_beta[(m + 1) * d.L] = pk(beta);
}

// Step run by the last block of a reduction over the pass-1 seed vectors.
enum StepKind : int {
    STEP_NONE = 0,
    STEP_BETA = 1,          // beta of sub-step arg
    STEP_ALPHA = 2,         // alpha of sub-step arg (seed part)
    STEP_ALPHA_ALL = 3,     // alpha of sub-step arg, seed and shift parts (single pass)
    STEP_CONV = 4           // convergence; arg = head flag
};
struct ScalarStep {
    int kind;
    int arg;
};

// nblk: partials of the reduction; ntickets: blocks of the system in this launch;
// warm: a late block that is not the last may run the step dry (last_block)
template <bool DFP>
__device__ __forceinline__ void run_step(const SolverDev& d, ScalarStep e, int nblk, int ntickets, bool warm = true) {
    if (e.kind == STEP_NONE) return;
    const int lb = last_block(d.st, ntickets);
    // (FP64 kernels run no dry runs: their sweeps are bound by the FP64 pipe,
    // which the dry step would share)
    if (lb == LB_NONE || (lb == LB_WARM && (!warm || !DFP))) return;
    const bool dry = lb == LB_WARM;
    if (e.kind == STEP_BETA) {
        sc_beta<DFP>(d, e.arg, nblk, dry);
    } else if (e.kind == STEP_ALPHA || e.kind == STEP_ALPHA_ALL) {
        sc_alpha_seed<DFP>(d, e.arg, nblk, dry);
        if (e.kind == STEP_ALPHA_ALL && !dry) {
            __syncthreads();
            sc_alpha_shifts(d, e.arg);
        }
    } else {
        sc_conv<DFP>(d, nblk, e.arg, dry);
    }
}

// Resident blocks per SM of the balanced vector kernels (register budget <= 64).
constexpr int kVecBlocks = 4;

// Contiguous site range [s0, s1) of block bx of nbx (V/nbx sites, +-1).  The
// vector kernels run at most one wave (kVecBlocks per SM, which their register
// budget guarantees); larger lattices loop over their range.
__device__ __forceinline__ void site_range(int V, unsigned bx, unsigned nbx, int& s0, int& s1) {
    s0 = (int)(((long long)V * bx) / nbx);
    s1 = (int)(((long long)V * (bx + 1)) / nbx);
}

// ------------------------------------------------------------------ BiCG sub-step kernels
// u_i <- r_i - beta u_i, i = 0..j (r, u: l+1 spinors each, contiguous, stride vs)
template <typename R>
__global__ void __launch_bounds__(kThreads, kVecBlocks)
k_update_u(const SolverDev* __restrict__ ds, int j, int pass2, const int4* tab) {
    dep_sync();
    const TraceScope trace_(trace_kind<R>(FA_TK_UPDATE_U));
    const Where w = where<false>(tab);
    const SolverDev& d = ds[w.sys];
    if (sys_idle(d, pass2)) return;
    int s0, s1;
    site_range(d.V, w.bx, w.nbx, s0, s1);
    const typename Ch<R>::T* r = Vec<R>::r(d);
    typename Ch<R>::T* u = Vec<R>::u(d);
    const size_t vs = vstride<R>(d);
    const int m = d.st->m;
    const cx<R> nb = negcx<R>(d.rec_beta[m * d.L + j]);
    for (int s = s0 + threadIdx.x; s < s1; s += kThreads) {
    for (int i = 0; i <= j; ++i) {
        const typename Ch<R>::T* ri = r + i * vs;
        typename Ch<R>::T* ui = u + i * vs;
#pragma unroll
        for (int q = 0; q < Ch<R>::N; ++q) {
            Ch<R> a = Ch<R>::ld(ri, q, d.V, s), b = Ch<R>::ld(ui, q, d.V, s);
#pragma unroll
            for (int w = 0; w < Ch<R>::W; ++w) b.c[w] = cfma(nb, b.c[w], a.c[w]);
            b.stv(ui, q, d.V, s);
        }
    }
    }
}

// r_i <- r_i - alpha u_{i+1}, i = 0..j.
// ACC (pass 2): y += sum_i coef[m][slot_old(j,i)] r_i(before the update).
// SHIFTS (single-pass, FP64): the shift-vector updates of the BiCG sub-step,
// reading each seed vector once for all active shifts.
// XS (pass 1 of the double-pass forms): block 0 runs the shift part of sub-step
// j (sc_alpha_shifts) beside the vector blocks 1..nblk.
template <typename R, bool ACC, bool SHIFTS, bool XS = false>
__global__ void __launch_bounds__(kThreads, kVecBlocks)
k_update_r(const SolverDev* __restrict__ ds, int j, int pass2, const int4* tab) {
    dep_sync();
    const TraceScope trace_(trace_kind<R>(FA_TK_UPDATE_R, XS));
    const Where w = where<XS>(tab);
    const SolverDev& d = ds[w.sys];
    if (sys_idle(d, pass2)) return;
    if (XS && w.bx < 0) {
        sc_alpha_shifts(d, j);
        return;
    }
    int s0, s1;
    site_range(d.V, w.bx, w.nbx, s0, s1);
    const int m = d.st->m;
    typename Ch<R>::T* r = Vec<R>::r(d);
    const typename Ch<R>::T* u = Vec<R>::u(d);
    const size_t vs = vstride<R>(d);
    double2* y = d.y;
    double2* xs = d.xs;
    double2* us = d.us;
    const size_t svs = (size_t)12 * d.V;
    typename Ch<R>::T* store = pass2 ? nullptr : store_at<R>(d, m);
    const int L = d.L;
    const cx<R> na = negcx<R>(d.rec_alpha[m * L + j]);
    const size_t cf0 = (size_t)m * nc_slots(L);
    for (int s = s0 + threadIdx.x; s < s1; s += kThreads) {
#pragma unroll
    for (int q = 0; q < Ch<R>::N; ++q) {
        cx<R> t[Ch<R>::W];
#pragma unroll
        for (int w = 0; w < Ch<R>::W; ++w) t[w] = czero<R>();
        for (int i = 0; i <= j; ++i) {
            typename Ch<R>::T* ri = r + i * vs;
            Ch<R> a = Ch<R>::ld(ri, q, d.V, s), b = Ch<R>::ld(u + (i + 1) * vs, q, d.V, s);
            if (store != nullptr) a.stv_cs(store + slot_old(j, i) * vs, q, d.V, s);
            if (ACC) {
                const cx<R> c = weight<R>(d.coef, d.coef4, cf0 + slot_old(j, i));
#pragma unroll
                for (int w = 0; w < Ch<R>::W; ++w) t[w] = cfma(c, a.c[w], t[w]);
            }
            if (SHIFTS) {
                // u^s_i <- r_old_i/zeta - beta_s u^s_i   (FP64 only)
                for (int sh = 0; sh < d.ns; ++sh) {
                    if (!d.active[sh]) continue;
                    const double2* P = d.prec + ((size_t)sh * d.max_outer + m) * ps_stride(L) + 5 * j;
                    const cx<R> bs = negcx<R>(P[1]), iz = tocx<R>(P[2]);
                    double2* usi = us + ((size_t)sh * (L + 1) + i) * svs;
                    Ch<R> v = Ch<R>::ld((const typename Ch<R>::T*)usi, q, d.V, s);
#pragma unroll
                    for (int w = 0; w < Ch<R>::W; ++w) v.c[w] = cfma(bs, v.c[w], cmul(iz, a.c[w]));
                    v.stv((typename Ch<R>::T*)usi, q, d.V, s);
                }
            }
            Ch<R> n;
#pragma unroll
            for (int w = 0; w < Ch<R>::W; ++w) n.c[w] = cfma(na, b.c[w], a.c[w]);
            n.stv(ri, q, d.V, s);
            if (SHIFTS && i == j) {
                // u^s_{j+1} <- r_old_j/(alpha_s zeta) - r_j/(alpha_s zeta_new) - sigma u^s_j;
                // x_s <- x_s + alpha_s u^s_0
                for (int sh = 0; sh < d.ns; ++sh) {
                    if (!d.active[sh]) continue;
                    const double2* P = d.prec + ((size_t)sh * d.max_outer + m) * ps_stride(L) + 5 * j;
                    const cx<R> as = tocx<R>(P[0]), iaz = tocx<R>(P[3]), niazn = negcx<R>(P[4]);
                    const R nsig = (R)(-d.sigma[sh]);
                    double2* usj = us + ((size_t)sh * (L + 1) + j) * svs;
                    double2* usj1 = us + ((size_t)sh * (L + 1) + j + 1) * svs;
                    double2* us0 = us + ((size_t)sh * (L + 1)) * svs;
                    double2* xsh = xs + (size_t)sh * svs;
                    Ch<R> vj = Ch<R>::ld((const typename Ch<R>::T*)usj, q, d.V, s);
                    Ch<R> v0 = Ch<R>::ld((const typename Ch<R>::T*)us0, q, d.V, s);
                    Ch<R> xv = Ch<R>::ld((const typename Ch<R>::T*)xsh, q, d.V, s);
                    Ch<R> nv;
#pragma unroll
                    for (int w = 0; w < Ch<R>::W; ++w) {
                        cx<R> e = cmul(iaz, a.c[w]);
                        e = cfma(niazn, n.c[w], e);
                        nv.c[w] = crfma(nsig, vj.c[w], e);
                        xv.c[w] = cfma(as, v0.c[w], xv.c[w]);
                    }
                    nv.stv((typename Ch<R>::T*)usj1, q, d.V, s);
                    xv.stv((typename Ch<R>::T*)xsh, q, d.V, s);
                }
            }
        }
        if (ACC) acc_y<R>(y, q, d.V, s, t);
        if (d.x64 != nullptr) acc_x<R>(d.x64, q, d.V, s, d.rec_alpha[m * L + j], Ch<R>::ld(u, q, d.V, s));
    }
    }
}

// ------------------------------------------------------------------ MR part
// Gram matrix <r_i, r_k>, 0 <= i <= k <= L, grid-stride, per-block partials.
// Last block: the MR coefficients (sc_mr_seed) and, for single-pass solves
// (shifts != 0), their shift part.
// l <= 2: registers capped for 4 blocks/SM (one wave of 512 blocks)
template <typename R, int L> constexpr int gram_min_blocks() { return L <= 2 ? 4 : 1; }
template <typename R, int L>
__global__ void __launch_bounds__(kThreads, gram_min_blocks<R, L>())
k_gram(const SolverDev* __restrict__ ds, int shifts, const int4* tab) {
    dep_sync();
    const TraceScope trace_(trace_kind<R>(FA_TK_GRAM));
    const Where w = where<false>(tab);
    const SolverDev& d = ds[w.sys];
    if (sys_idle(d, 0)) return;
    const typename Ch<R>::T* r = Vec<R>::r(d);
    const size_t vs = vstride<R>(d);
    double2* partials = d.part;
    constexpr int NG = n_gram(L);
    cx<R> acc[NG];
#pragma unroll
    for (int k = 0; k < NG; ++k) acc[k] = czero<R>();
    int s0, s1;
    site_range(d.V, w.bx, w.nbx, s0, s1);
    for (int s = s0 + threadIdx.x; s < s1; s += kThreads) {
#pragma unroll
        for (int q = 0; q < Ch<R>::N; ++q) {
            Ch<R> v[L + 1];
#pragma unroll
            for (int i = 0; i <= L; ++i) v[i] = Ch<R>::ld(r + i * vs, q, d.V, s);
            int g = 0;
#pragma unroll
            for (int i = 0; i <= L; ++i)
#pragma unroll
                for (int k = i; k <= L; ++k) {
#pragma unroll
                    for (int w = 0; w < Ch<R>::W; ++w) acc[g] = cjfma(v[i].c[w], v[k].c[w], acc[g]);
                    ++g;
                }
        }
    }
    block_reduce_store<NG, R>(acc, partials, w.nbx, w.bx);
    const int lb = last_block(d.st, w.ntk);
    if (lb == LB_LAST || (lb == LB_WARM && dfp_of<R>())) {
        sc_mr_seed<L, dfp_of<R>()>(d, w.nbx, lb == LB_WARM);
        if (shifts && lb == LB_LAST) {
            __syncthreads();
            sc_mr_shifts<L>(d);
        }
    }
}

// MR update: r_0 -= sum gamma_j r_j, u_0 -= sum gamma_j u_j.
// ACC: y += sum_k coef[m][slot_mr(k)] r_k (before the update).
// SHIFTS: x_s += sum_k c_k/(zeta p_s) r_k, u^s_0 <- (u^s_0 - sum gamma_j u^s_j)/p_s.
// DOT: per-block partials of <rt, r_0> (slot 0) and |r_0|^2 (slot 1), grid-stride,
// then `step` (convergence) in the last block.
// XS (pass 1 of the double-pass forms): block 0 runs the shift part of the MR
// step (sc_mr_shifts) and takes a ticket too, so that the convergence step sees
// the new zeta; blocks 1.. are the vector blocks.
// FP32 and double-float, l <= 3: registers capped for 4 blocks/SM (64; some
// bytes spilled), so that a 16^3 x 32 lattice (512 blocks) runs in one wave
// instead of 1.12 (left alone, the compiler takes up to 167 registers here)
template <typename R, int L> constexpr int mr_min_blocks() {
    return (!std::is_same<R, double>::value && L <= 3) ? 4 : 1;
}
template <typename R, int L, bool ACC, bool SHIFTS, bool DOT, bool XS = false>
__global__ void __launch_bounds__(kThreads, mr_min_blocks<R, L>())
k_mr(const SolverDev* __restrict__ ds, int pass2, ScalarStep step, const int4* tab) {
    dep_sync();
    const TraceScope trace_(trace_kind<R>(FA_TK_MR, XS));
    const Where w = where<XS>(tab);
    const SolverDev& d = ds[w.sys];
    if (sys_idle(d, pass2)) return;
    const int bx = w.bx, nbx = w.nbx;
    if (XS && bx < 0) {
        sc_mr_shifts<L>(d);
        __threadfence();   // the new zeta of every thread before the ticket
        run_step<dfp_of<R>()>(d, step, nbx, w.ntk);
        return;
    }
    const int m = d.st->m;
    typename Ch<R>::T* r = Vec<R>::r(d);
    typename Ch<R>::T* u = Vec<R>::u(d);
    const typename Ch<R>::T* rt = Vec<R>::rt(d);
    const size_t vs = vstride<R>(d);
    double2* y = d.y;
    double2* xs = d.xs;
    double2* us = d.us;
    const size_t svs = (size_t)12 * d.V;
    typename Ch<R>::T* store = pass2 ? nullptr : store_at<R>(d, m);
    double2* partials = d.part;
    cx<R> ng[L + 1];
    ng[0] = czero<R>();
#pragma unroll
    for (int j = 1; j <= L; ++j) ng[j] = negcx<R>(d.rec_gamma[m * (L + 1) + j]);
    const size_t cf0 = (size_t)m * nc_slots(L);
    cx<R> dots[2] = {czero<R>(), czero<R>()};
    int s0, s1;
    site_range(d.V, bx, nbx, s0, s1);
    for (int s = s0 + threadIdx.x; s < s1; s += kThreads) {
#pragma unroll
        for (int q = 0; q < Ch<R>::N; ++q) {
            Ch<R> rv[L + 1];
#pragma unroll
            for (int i = 0; i <= L; ++i) rv[i] = Ch<R>::ld(r + i * vs, q, d.V, s);
            if (store != nullptr) {
#pragma unroll
                for (int k = 0; k < L; ++k) rv[k].stv_cs(store + slot_mr(L, k) * vs, q, d.V, s);
            }
            if (ACC) {
                cx<R> t[Ch<R>::W];
#pragma unroll
                for (int w = 0; w < Ch<R>::W; ++w) t[w] = czero<R>();
#pragma unroll
                for (int k = 0; k < L; ++k) {
                    const cx<R> c = weight<R>(d.coef, d.coef4, cf0 + slot_mr(L, k));
#pragma unroll
                    for (int w = 0; w < Ch<R>::W; ++w) t[w] = cfma(c, rv[k].c[w], t[w]);
                }
                acc_y<R>(y, q, d.V, s, t);
            }
            if (SHIFTS) {
                for (int sh = 0; sh < d.ns; ++sh) {
                    if (!d.active[sh]) continue;
                    const double2* P = d.prec + ((size_t)sh * d.max_outer + m) * ps_stride(L) + 5 * L;
                    const cx<R> ips = tocx<R>(P[0]);
                    double2* xsh = xs + (size_t)sh * svs;
                    Ch<R> xv = Ch<R>::ld((const typename Ch<R>::T*)xsh, q, d.V, s);
                    Ch<R> u0 = Ch<R>::ld((const typename Ch<R>::T*)(us + (size_t)sh * (L + 1) * svs), q, d.V, s);
#pragma unroll
                    for (int k = 0; k < L; ++k) {
                        const cx<R> c = tocx<R>(P[1 + k]);
#pragma unroll
                        for (int w = 0; w < Ch<R>::W; ++w) xv.c[w] = cfma(c, rv[k].c[w], xv.c[w]);
                    }
#pragma unroll
                    for (int j = 1; j <= L; ++j) {
                        Ch<R> uj = Ch<R>::ld((const typename Ch<R>::T*)(us + ((size_t)sh * (L + 1) + j) * svs),
                                             q, d.V, s);
#pragma unroll
                        for (int w = 0; w < Ch<R>::W; ++w) u0.c[w] = cfma(ng[j], uj.c[w], u0.c[w]);
                    }
#pragma unroll
                    for (int w = 0; w < Ch<R>::W; ++w) u0.c[w] = cmul(ips, u0.c[w]);
                    xv.stv((typename Ch<R>::T*)xsh, q, d.V, s);
                    u0.stv((typename Ch<R>::T*)(us + (size_t)sh * (L + 1) * svs), q, d.V, s);
                }
            }
            if (d.x64 != nullptr) {
#pragma unroll
                for (int j = 1; j <= L; ++j) acc_x<R>(d.x64, q, d.V, s, d.rec_gamma[m * (L + 1) + j], rv[j - 1]);
            }
            Ch<R> r0 = rv[0];
            Ch<R> u0 = Ch<R>::ld(u, q, d.V, s);
#pragma unroll
            for (int j = 1; j <= L; ++j) {
                Ch<R> uj = Ch<R>::ld(u + j * vs, q, d.V, s);
#pragma unroll
                for (int w = 0; w < Ch<R>::W; ++w) {
                    r0.c[w] = cfma(ng[j], rv[j].c[w], r0.c[w]);
                    u0.c[w] = cfma(ng[j], uj.c[w], u0.c[w]);
                }
            }
            r0.stv(r, q, d.V, s);
            u0.stv(u, q, d.V, s);
            if (DOT) {
                Ch<R> tv = Ch<R>::ld(rt, q, d.V, s);
#pragma unroll
                for (int w = 0; w < Ch<R>::W; ++w) {
                    dots[0] = cjfma(tv.c[w], r0.c[w], dots[0]);
                    dots[1].r = fmaR(r0.c[w].r, r0.c[w].r, dots[1].r);
                    dots[1].r = fmaR(r0.c[w].i, r0.c[w].i, dots[1].r);
                }
            }
        }
    }
    if (DOT) {
        block_reduce_store<2, R>(dots, partials, nbx, bx);
        run_step<dfp_of<R>()>(d, step, nbx, w.ntk);
    }
}

// <rt, r0> (slot 0) and |r0|^2 (slot 1), grid-stride (start of a solve)
template <typename R>
__device__ __forceinline__ void k_dot2_body(int V, const typename Ch<R>::T* rt, const typename Ch<R>::T* r0,
                                            double2* partials, int bx, int nbx) {
    cx<R> dots[2] = {czero<R>(), czero<R>()};
    int s0, s1;
    site_range(V, bx, nbx, s0, s1);
    for (int s = s0 + threadIdx.x; s < s1; s += kThreads) {
#pragma unroll
        for (int q = 0; q < Ch<R>::N; ++q) {
            Ch<R> a = Ch<R>::ld(rt, q, V, s), b = Ch<R>::ld(r0, q, V, s);
#pragma unroll
            for (int w = 0; w < Ch<R>::W; ++w) {
                dots[0] = cjfma(a.c[w], b.c[w], dots[0]);
                dots[1].r = fmaR(b.c[w].r, b.c[w].r, dots[1].r);
                dots[1].r = fmaR(b.c[w].i, b.c[w].i, dots[1].r);
            }
        }
    }
    block_reduce_store<2, R>(dots, partials, nbx, bx);
}

template <typename R>
__global__ void __launch_bounds__(kThreads)
k_dot2(int V, const typename Ch<R>::T* rt, const typename Ch<R>::T* r0, double2* partials) {
    k_dot2_body<R>(V, rt, r0, partials, blockIdx.x, gridDim.x);
}

// start of pass 1: <rt, r0>, |r0|^2 and, in the last block, the initial state
template <typename R>
__global__ void __launch_bounds__(kThreads, kVecBlocks)
k_dot2_sys(const SolverDev* __restrict__ ds, double tol, double theta, const int4* tab) {
    const Where w = where<false>(tab);
    const SolverDev& d = ds[w.sys];
    k_dot2_body<R>(d.V, Vec<R>::rt(d), Vec<R>::r(d), d.part, w.bx, w.nbx);
    if (last_block(d.st, w.ntk) == LB_LAST) sc_init<dfp_of<R>()>(d, w.nbx, tol, theta);
}

// A application inside the solver: out = scale * g5 D in on the system's own
// links, mu and scale (scale = 1 for the first hop of A, c for the second).
// Vector selectors: 0 = u family, 1 = r family, 2 = scratch.  DOT: per-block
// partials of <rt, out> into the system's partial buffer.
template <typename R>
__device__ __forceinline__ typename Ch<R>::T* select_vec(const SolverDev& d, int sel, int j) {
    typename Ch<R>::T* base = sel == 0 ? Vec<R>::u(d) : (sel == 1 ? Vec<R>::r(d) : Vec<R>::tmp(d));
    return base + (size_t)j * vstride<R>(d);
}

template <typename R, bool DOT>
__global__ void __launch_bounds__(kThreads, hop_min_blocks<R>())
k_hop_sys(const SolverDev* __restrict__ ds, int in_sel, int in_j, int out_sel, int out_j, int second, int pass2,
          ScalarStep step, const int4* tab) {
    dep_sync();
    const TraceScope trace_(trace_kind<R>(FA_TK_HOP_SYS, DOT));
    const Where w = where<false>(tab);
    const SolverDev& d = ds[w.sys];
    if (sys_idle(d, pass2)) return;
    const int s = w.bx * kThreads + threadIdx.x;
    cx<R> dres[1] = {czero<R>()};
    if (s < d.V) {
        const double sc = second ? d.scale : 1.0;
        SpinorView<R> in{select_vec<R>(d, in_sel, in_j), d.V};
        SpinorView<R> out{select_vec<R>(d, out_sel, out_j), d.V};
        cx<R> p[12];
        hop_site<R, false, true>(d.g, Vec<R>::links(d), in, s, fromdbl<R>(sc * d.diag), fromdbl<R>(-0.5 * sc),
                                 fromdbl<R>(d.ef), fromdbl<R>(d.eb), fromdbl<R>(d.bc), p);
        out.store(s, p);
        if (DOT) {
            SpinorView<R> rt{Vec<R>::rt(d), d.V};
            cx<R> q[12];
            rt.load(s, q);
            cx<R> a = czero<R>();
#pragma unroll
            for (int k = 0; k < 12; ++k) a = cjfma(q[k], p[k], a);
            dres[0] = a;
        }
    }
    if (DOT) {
        block_reduce_store<1, R>(dres, d.part, 0, w.bx);
        run_step<dfp_of<R>()>(d, step, w.nbx, w.ntk);
    }
}

// Systems that share one gauge field and lattice (the sources of one lattice in
// a batch): the multi-RHS sweep applies D_w to all of them tile by tile.
constexpr int kMaxRhs = 16;
struct GroupDev {
    int nsys;
    int ntile;             // tiles of kHopNarrowThreads sites
    int sys[kMaxRhs];      // descriptor index of each system
};

// FP32 sweep of a batch, several right-hand sides per block.  items[blockIdx.x]
// = (group, tile, first, end): the block applies the sweep to the systems
// first..end-1 of the group on the tile's sites, one after the other, so the
// tile's links (and the neighbours' backward links) come from HBM once and
// from L1 for the other right-hand sides.  Each system's arithmetic, its
// per-tile partials of <rt, out> and its scalar step are those of the
// one-system sweep of the same launch shape (128-thread blocks), so a batched
// solve equals the one-at-a-time solve bit for bit.
template <bool DOT, int MB>
__global__ void __launch_bounds__(kHopNarrowThreads, MB)
k_hop_mrhs(const SolverDev* __restrict__ ds, const GroupDev* __restrict__ groups, const int4* __restrict__ items,
           int in_sel, int in_j, int out_sel, int out_j, int second, int pass2, ScalarStep step) {
    constexpr int NT = kHopNarrowThreads;
    dep_sync();
    const TraceScope trace_(trace_kind<float>(FA_TK_HOP_MRHS, DOT));
    const int4 it = items[blockIdx.x];
    const GroupDev& G = groups[it.x];
    const int tile = it.y;
    for (int r = it.z; r < it.w; ++r) {
        const SolverDev& d = ds[G.sys[r]];
        if (sys_idle(d, pass2)) continue;   // the same for every thread of the block
        const int s = tile * NT + (int)threadIdx.x;
        cx<float> dres[1] = {czero<float>()};
        if (s < d.V) {
            const SpinorView<float> in{select_vec<float>(d, in_sel, in_j), d.V};
            const SpinorView<float> out{select_vec<float>(d, out_sel, out_j), d.V};
            cx<float> p[12];
            hop_site<float, false, true>(d.g, LinkView<float>{d.links32, d.V}, in, s, second ? d.fdiag2 : d.fdiag1,
                                         second ? d.fhop2 : d.fhop1, d.fef, d.feb, d.fbc, p);
            out.store(s, p);
            if (DOT) {
                const SpinorView<float> rt{d.rt32, d.V};
                cx<float> q[12];
                rt.load(s, q);
                cx<float> a = czero<float>();
#pragma unroll
                for (int k = 0; k < 12; ++k) a = cjfma(q[k], p[k], a);
                dres[0] = a;
            }
        }
        if (DOT) {
            block_reduce_store<1, float, NT>(dres, d.part, 0, tile);
            run_step<true>(d, step, G.ntile, G.ntile, r == it.w - 1);   // no dry run before another sweep
        }
    }
}

// double-float batches: the row-split sweep (kRowThreads per block)
template <typename R, bool DOT>
__global__ void __launch_bounds__(kRowThreads, rows_sys_min_blocks<DOT>())
k_hop_sys_rows(const SolverDev* __restrict__ ds, int in_sel, int in_j, int out_sel, int out_j, int second, int pass2,
               ScalarStep step, const int4* tab) {
    dep_sync();
    const TraceScope trace_(trace_kind<R>(FA_TK_HOP_SYS_ROWS, DOT));
    const Where w = where<false>(tab);
    const SolverDev& d = ds[w.sys];
    if (sys_idle(d, pass2)) return;
    const double sc = second ? d.scale : 1.0;
    const Geom g = d.g;
    const SpinorView<R> in{select_vec<R>(d, in_sel, in_j), d.V}, out{select_vec<R>(d, out_sel, out_j), d.V};
    const SpinorView<R> rt{Vec<R>::rt(d), d.V};
    cx<R> dres[1] = {hop_rows_body<R, false, true, DOT>(g, Vec<R>::links(d), in, out,
                                                        fromdbl<R>(sc * d.diag), fromdbl<R>(-0.5 * sc),
                                                        fromdbl<R>(d.ef), fromdbl<R>(d.eb), fromdbl<R>(d.bc), rt,
                                                        w.bx)};
    if (DOT) {
        block_reduce_store<1, R, kRowThreads>(dres, d.part, 0, w.bx);
        run_step<dfp_of<R>()>(d, step, w.nbx, w.ntk, false);   // ALU-bound sweep: no dry runs
    }
}

// The hop of a single solve with its pointers as kernel parameters (the
// descriptor is read only by the scalar step of the last block).  DOT:
// partials of <dotv, out>, then `step`.  Double-float uses the row-split
// sweep (kRowThreads per block, one partial per block).
template <typename R, bool DOT>
__global__ void __launch_bounds__(kRowThreads, rows_min_blocks<DOT>())
k_hop1_rows(Geom g, LinkView<R> U, SpinorView<R> in, SpinorView<R> out, R cdiag, R chop, R ef, R eb, R bc,
            SpinorView<R> dotv, double2* partials, const int* done, const SolverDev* __restrict__ ds,
            ScalarStep step) {
    dep_sync();
    const TraceScope trace_(trace_kind<R>(FA_TK_HOP1_ROWS, DOT));
    if (done != nullptr && *done) return;
    cx<R> dres[1] = {hop_rows_body<R, false, true, DOT>(g, U, in, out, cdiag, chop, ef, eb, bc, dotv, blockIdx.x)};
    if (DOT) {
        block_reduce_store<1, R, kRowThreads>(dres, partials, 0, blockIdx.x);
        run_step<dfp_of<R>()>(ds[0], step, gridDim.x, gridDim.x, false);   // ALU-bound sweep: no dry runs
    }
}

template <typename R, bool DOT, int NT = kThreads, int MB = hop_min_blocks<R>()>
__global__ void __launch_bounds__(NT, MB)
k_hop1(Geom g, LinkView<R> U, SpinorView<R> in, SpinorView<R> out, R cdiag, R chop, R ef, R eb, R bc,
       SpinorView<R> dotv, double2* partials, const int* done, const SolverDev* __restrict__ ds, ScalarStep step) {
    dep_sync();
    const TraceScope trace_(trace_kind<R>(FA_TK_HOP1, DOT));
    if (done != nullptr && *done) return;
    const int s = blockIdx.x * NT + threadIdx.x;
    cx<R> dres[1] = {czero<R>()};
    if (s < g.V) {
        cx<R> p[12];
        hop_site<R, false, true>(g, U, in, s, cdiag, chop, ef, eb, bc, p);
        out.store(s, p);
        if (DOT) {
            cx<R> q[12];
            dotv.load(s, q);
            cx<R> a = czero<R>();
#pragma unroll
            for (int k = 0; k < 12; ++k) a = cjfma(q[k], p[k], a);
            dres[0] = a;
        }
    }
    if (DOT) {
        block_reduce_store<1, R, NT>(dres, partials, 0, blockIdx.x);
        run_step<dfp_of<R>()>(ds[0], step, gridDim.x, gridDim.x);
    }
}

// ------------------------------------------------------------------ reliable update
// r_0 <- b - A x with A x (FP64) already in ax; the new r_0 is rounded to R.
// Rewrites the partials of <rt, r_0> (slot 0) and |r_0|^2 (slot 1) that the
// convergence step reads, grid-stride like k_mr.
template <typename R>
__global__ void __launch_bounds__(kThreads, kVecBlocks)
k_reliable(const SolverDev* __restrict__ ds, const double2* ax, int pass2, ScalarStep step) {
    const TraceScope trace_(trace_kind<R>(FA_TK_RELIABLE));
    const SolverDev& d = ds[blockIdx.y];   // one system (reliable updates are not batched)
    if (sys_idle(d, pass2)) return;
    typename Ch<R>::T* r0 = Vec<R>::r(d);
    const typename Ch<R>::T* rt = Vec<R>::rt(d);
    cx<R> dots[2] = {czero<R>(), czero<R>()};
    int s0, s1;
    site_range(d.V, blockIdx.x, gridDim.x, s0, s1);
    for (int s = s0 + threadIdx.x; s < s1; s += kThreads) {
#pragma unroll
        for (int q = 0; q < Ch<R>::N; ++q) {
            Ch<R> v;
#pragma unroll
            for (int w = 0; w < Ch<R>::W; ++w) {
                const size_t k = (size_t)(q * Ch<R>::W + w) * d.V + s;
                const double2 bb = d.b64[k], aa = ax[k];
                v.c[w] = {fromdbl<R>(__dsub_rn(bb.x, aa.x)), fromdbl<R>(__dsub_rn(bb.y, aa.y))};
            }
            v.stv(r0, q, d.V, s);
            Ch<R> tv = Ch<R>::ld(rt, q, d.V, s);
#pragma unroll
            for (int w = 0; w < Ch<R>::W; ++w) {
                dots[0] = cjfma(tv.c[w], v.c[w], dots[0]);
                dots[1].r = fmaR(v.c[w].r, v.c[w].r, dots[1].r);
                dots[1].r = fmaR(v.c[w].i, v.c[w].i, dots[1].r);
            }
        }
    }
    block_reduce_store<2, R>(dots, d.part, gridDim.x);
    run_step<dfp_of<R>()>(d, step, gridDim.x, gridDim.x);
}

// ------------------------------------------------------------------ pseudo-double-pass gather
// y += sum_{m in [m_begin, m_end)} sum_k coef[m][k] v(m, k), the stored seed-vector
// occurrences of pass 1 (store slot (m - m0) * NC + k).  One thread per site and
// chunk (grid.x = chunks x site blocks), so a thread holds a few accumulators and
// many loads stay in flight.  Terms are summed in R in groups of four; each group
// enters a compensated FP32-pair accumulator (FP64 for an FP64 store), which is
// added to y in FP64 once.
template <typename R> struct GatherAcc {        // FP32 and double-float stores
    df a[2 * Ch<R>::W];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int k = 0; k < 2 * Ch<R>::W; ++k) a[k] = df(0.0f);
    }
    __device__ __forceinline__ static df widen(float x) { return df(x); }
    __device__ __forceinline__ static df widen(df x) { return x; }
    __device__ __forceinline__ void add(const cx<R> (&t)[Ch<R>::W]) {
#pragma unroll
        for (int w = 0; w < Ch<R>::W; ++w) {
            a[2 * w] = addR(a[2 * w], widen(t[w].r));
            a[2 * w + 1] = addR(a[2 * w + 1], widen(t[w].i));
        }
    }
    __device__ __forceinline__ double get(int k) const { return todbl(a[k]); }
};
template <> struct GatherAcc<double> {
    double a[2];
    __device__ __forceinline__ void zero() { a[0] = a[1] = 0.0; }
    __device__ __forceinline__ void add(const cx<double> (&t)[1]) {
        a[0] = __dadd_rn(a[0], t[0].r);
        a[1] = __dadd_rn(a[1], t[0].i);
    }
    __device__ __forceinline__ double get(int k) const { return a[k]; }
};

template <typename R>
__global__ void __launch_bounds__(kThreads)
k_gather(const SolverDev* __restrict__ ds) {
    const TraceScope trace_(trace_kind<R>(FA_TK_GATHER));
    const SolverDev& d = ds[blockIdx.y];
    const int nsb = (d.V + kThreads - 1) / kThreads;
    const int q = blockIdx.x / nsb;
    const int s = (blockIdx.x - q * nsb) * kThreads + threadIdx.x;
    if (q >= Ch<R>::N || s >= d.V) return;
    const int M = d.st->n_outer;
    int m_begin, m_end, m0;
    const typename Ch<R>::T* store;
    if (sizeof(R) == 8) {
        m_begin = 0;
        m_end = min(M, d.cap64);
        if (d.m0_32 >= 0) m_end = min(m_end, d.m0_32);
        m0 = 0;
        store = reinterpret_cast<const typename Ch<R>::T*>(d.store64);
    } else {
        if (d.m0_32 < 0) return;
        m_begin = d.m0_32;
        m_end = min(M, d.m0_32 + d.cap32);
        m0 = d.m0_32;
        store = reinterpret_cast<const typename Ch<R>::T*>(d.store32);
    }
    if (m_end <= m_begin) return;
    const size_t vs = vstride<R>(d);
    const int NC = nc_slots(d.L);
    const int n = (m_end - m_begin) * NC;
    const size_t cf0 = (size_t)m_begin * NC;
    const typename Ch<R>::T* base = store + (size_t)(m_begin - m0) * NC * vs;
    constexpr int W = Ch<R>::W;
    GatherAcc<R> acc;
    acc.zero();
    int k0 = 0;
    for (; k0 + 4 <= n; k0 += 4) {
        Ch<R> v[4];
#pragma unroll
        for (int g = 0; g < 4; ++g) v[g] = Ch<R>::ld_cs(base + (size_t)(k0 + g) * vs, q, d.V, s);
        cx<R> t[W];
#pragma unroll
        for (int w = 0; w < W; ++w) t[w] = czero<R>();
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const cx<R> c = weight<R>(d.coef, d.coef4, cf0 + k0 + g);
#pragma unroll
            for (int w = 0; w < W; ++w) t[w] = cfma(c, v[g].c[w], t[w]);
        }
        acc.add(t);
    }
    if (k0 < n) {
        cx<R> t[W];
#pragma unroll
        for (int w = 0; w < W; ++w) t[w] = czero<R>();
        for (int k = k0; k < n; ++k) {
            const Ch<R> v = Ch<R>::ld_cs(base + (size_t)k * vs, q, d.V, s);
            const cx<R> c = weight<R>(d.coef, d.coef4, cf0 + k);
#pragma unroll
            for (int w = 0; w < W; ++w) t[w] = cfma(c, v.c[w], t[w]);
        }
        acc.add(t);
    }
#pragma unroll
    for (int w = 0; w < W; ++w) {
        double2* p = d.y + (size_t)(q * W + w) * d.V + s;
        double2 a = *p;
        a.x = __dadd_rn(a.x, acc.get(2 * w));
        a.y = __dadd_rn(a.y, acc.get(2 * w + 1));
        *p = a;
    }
}

// pass 2: advance the outer-iteration counter
__global__ void k_advance(const SolverDev* __restrict__ ds) {
    dep_sync();
    const TraceScope trace_(FA_TK_ADVANCE);
    DevState* S = ds[blockIdx.x].st;
    if (S->m < S->n_outer) S->m += 1;
}
// pass 2 starts at outer iteration min(m, M) of each system
__global__ void k_set_m(const SolverDev* __restrict__ ds, int m) {
    DevState* S = ds[blockIdx.x].st;
    S->m = m < S->n_outer ? m : S->n_outer;
    S->done = 0;
}
// done flag of every system (polled by the host)
__global__ void k_flags(const SolverDev* __restrict__ ds, int n, int* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = ds[i].st->done;
}

// ------------------------------------------------------------------ backward sweep
// One thread per shift walks its recorded linear operations backwards
// (adjoint of "dst <- sum a src + sum c v_occ"), starting from the adjoint
// lambda_X = 1 of its final solution; the adjoint of each seed-vector
// occurrence is that occurrence's weight in x_s.  The weighted sum over shifts
// is formed by k_coef_reduce.
template <int L>
__global__ void k_sweep(const SolverDev* __restrict__ ds) {
    const TraceScope trace_(FA_TK_SWEEP);
    const SolverDev& d = ds[blockIdx.y];
    const int sh = blockIdx.x * blockDim.x + threadIdx.x;
    if (sh >= d.ns) return;
    constexpr int NC = nc_slots(L);
    const int Ms = d.iters[sh];
    const double sg = d.sigma[sh];
    dcx lX = mk(1.0);
    dcx lU[L + 1];
#pragma unroll
    for (int i = 0; i <= L; ++i) lU[i] = mk(0.0);
    // fused multiply-adds throughout (the sweep is bound by FP64 issue in one warp)
    for (int m = Ms - 1; m >= 0; --m) {
        const double2* P = d.prec + ((size_t)sh * d.max_outer + m) * ps_stride(L);
        const double2* G = d.rec_gamma + m * (L + 1);
        dcx c[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) c[k] = mk(0.0);
        // MR, reversed: u0 <- (u0 - sum gamma_j u_j)/p_s, then x += sum cx_k r_k
        {
            const dcx t = zmul(lU[0], ld(P[5 * L]));
#pragma unroll
            for (int jj = 1; jj <= L; ++jj) lU[jj] = zfma(zneg(ld(G[jj])), t, lU[jj]);
            lU[0] = t;
#pragma unroll
            for (int k = 0; k < L; ++k) c[slot_mr(L, k)] = zfma(lX, ld(P[5 * L + 1 + k]), c[slot_mr(L, k)]);
        }
#pragma unroll
        for (int j = L - 1; j >= 0; --j) {
            const double2* Q = P + 5 * j;
            // x += alpha_s u_0
            lU[0] = zfma(ld(Q[0]), lX, lU[0]);
            // u_{j+1} <- r_old_j/(alpha_s zeta) - r_j/(alpha_s zeta_new) - sigma u_j
            const dcx lu = lU[j + 1];
            c[slot_old(j, j)] = zfma(lu, ld(Q[3]), c[slot_old(j, j)]);
            const int snew = (j < L - 1) ? slot_old(j + 1, j) : slot_mr(L, L - 1);
            c[snew] = zfma(lu, zneg(ld(Q[4])), c[snew]);
            lU[j] = zrfma(-sg, lu, lU[j]);
            lU[j + 1] = mk(0.0);
            // u_i <- r_old_i/zeta - beta_s u_i
            const dcx iz = ld(Q[2]), nbs = zneg(ld(Q[1]));
#pragma unroll
            for (int i = 0; i <= j; ++i) {
                c[slot_old(j, i)] = zfma(lU[i], iz, c[slot_old(j, i)]);
                lU[i] = zmul(nbs, lU[i]);
            }
        }
        double2* out = d.cs + ((size_t)sh * d.max_outer + m) * NC;
#pragma unroll
        for (int k = 0; k < NC; ++k) out[k] = pk(c[k]);
    }
}

// coef[m][k] = sum_s omega_s cs[s][m][k] for m < M (fixed order over s)
__global__ void k_coef_reduce(const SolverDev* __restrict__ ds) {
    const TraceScope trace_(FA_TK_COEF_REDUCE);
    const SolverDev& d = ds[blockIdx.y];
    const int M = d.st->n_outer;
    const int NC = nc_slots(d.L);
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= M * NC) return;
    const int m = idx / NC, k = idx - m * NC;
    dcx a = mk(0.0);
    for (int sh = 0; sh < d.ns; ++sh) {
        if (m >= d.iters[sh]) continue;
        a = a + d.omega[sh] * ld(d.cs[((size_t)sh * d.max_outer + m) * NC + k]);
    }
    d.coef[(size_t)m * NC + k] = pk(a);
    // the same weight as an FP32 pair per part (hi = FP32 rounding, lo = rest)
    const float hr = __double2float_rn(a.r), hi = __double2float_rn(a.i);
    d.coef4[(size_t)m * NC + k] = make_float4(hr, __double2float_rn(__dsub_rn(a.r, (double)hr)),
                                              hi, __double2float_rn(__dsub_rn(a.i, (double)hi)));
}

// single-pass result y = sum_s omega_s x_s (FP64 [12][V]) of each system
__global__ void k_combine_sys(const SolverDev* __restrict__ ds) {
    const SolverDev& d = ds[blockIdx.y];
    const int idx = blockIdx.x * kThreads + threadIdx.x;
    if (idx >= 12 * d.V) return;
    const size_t svs = (size_t)12 * d.V;
    double a = 0.0, b = 0.0;
    for (int sh = 0; sh < d.ns; ++sh) {
        const double2 v = d.xs[sh * svs + idx];
        a = __fma_rn(d.omega[sh], v.x, a);
        b = __fma_rn(d.omega[sh], v.y, b);
    }
    d.y[idx] = make_double2(a, b);
}

// single-pass result y = sum_s omega_s x_s (FP64 [12][V]); accumulate: y += that sum
__global__ void k_combine(int V, int ns, const double* omega, const double2* xs, size_t svs, double2* y,
                          int accumulate = 0) {
    const int idx = blockIdx.x * kThreads + threadIdx.x;
    if (idx >= 12 * V) return;
    double a = 0.0, b = 0.0;
    if (accumulate) {
        a = y[idx].x;
        b = y[idx].y;
    }
    for (int sh = 0; sh < ns; ++sh) {
        const double2 v = xs[sh * svs + idx];
        a = __fma_rn(omega[sh], v.x, a);
        b = __fma_rn(omega[sh], v.y, b);
    }
    y[idx] = make_double2(a, b);
}

}  // namespace fa
