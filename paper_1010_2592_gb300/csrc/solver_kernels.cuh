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

#include "fa_internal.cuh"

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
    int pad;
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

struct SolverDev {
    DevState* st;
    int ns, L, max_outer, V;
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
    double2* cs;           // [ns][max_outer][nc_slots]   per-shift sweep output
};

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
};

template <typename R> __device__ __forceinline__ cx<R> tocx(double2 v) { return {(R)v.x, (R)v.y}; }
template <typename R> __device__ __forceinline__ cx<R> negcx(double2 v) { return {(R)(-v.x), (R)(-v.y)}; }

// y (FP64, [12][V]) += t for the W complex components of chunk q
template <typename R>
__device__ __forceinline__ void acc_y(double2* y, int q, int V, int s, const cx<R> (&t)[Ch<R>::W]) {
#pragma unroll
    for (int w = 0; w < Ch<R>::W; ++w) {
        double2* p = y + (size_t)(q * Ch<R>::W + w) * V + s;
        double2 a = *p;
        a.x = __dadd_rn(a.x, (double)t[w].r);
        a.y = __dadd_rn(a.y, (double)t[w].i);
        *p = a;
    }
}

// ------------------------------------------------------------------ BiCG sub-step kernels
// u_i <- r_i - beta u_i, i = 0..j (r, u: l+1 spinors each, contiguous, stride vs)
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_update_u(SolverDev d, int j, const typename Ch<R>::T* r, typename Ch<R>::T* u, size_t vs, const int* done) {
    if (done != nullptr && *done) return;
    const int s = blockIdx.x * kThreads + threadIdx.x;
    if (s >= d.V) return;
    const int m = d.st->m;
    const cx<R> nb = negcx<R>(d.rec_beta[m * d.L + j]);
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

// r_i <- r_i - alpha u_{i+1}, i = 0..j.
// ACC (pass 2): y += sum_i coef[m][slot_old(j,i)] r_i(before the update).
// SHIFTS (single-pass, FP64): the shift-vector updates of the BiCG sub-step,
// reading each seed vector once for all active shifts.
template <typename R, bool ACC, bool SHIFTS>
__global__ void __launch_bounds__(kThreads)
k_update_r(SolverDev d, int j, typename Ch<R>::T* r, const typename Ch<R>::T* u, size_t vs, double2* y,
           double2* xs, double2* us, size_t svs, typename Ch<R>::T* store, const int* done) {
    if (done != nullptr && *done) return;
    const int s = blockIdx.x * kThreads + threadIdx.x;
    if (s >= d.V) return;
    const int m = d.st->m;
    const int L = d.L;
    const cx<R> na = negcx<R>(d.rec_alpha[m * L + j]);
    const double2* cf = d.coef + (size_t)m * nc_slots(L);
#pragma unroll
    for (int q = 0; q < Ch<R>::N; ++q) {
        cx<R> t[Ch<R>::W];
#pragma unroll
        for (int w = 0; w < Ch<R>::W; ++w) t[w] = czero<R>();
        for (int i = 0; i <= j; ++i) {
            typename Ch<R>::T* ri = r + i * vs;
            Ch<R> a = Ch<R>::ld(ri, q, d.V, s), b = Ch<R>::ld(u + (i + 1) * vs, q, d.V, s);
            if (store != nullptr) a.stv(store + slot_old(j, i) * vs, q, d.V, s);
            if (ACC) {
                const cx<R> c = tocx<R>(cf[slot_old(j, i)]);
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
    }
}

// ------------------------------------------------------------------ MR part
// Gram matrix <r_i, r_k>, 0 <= i <= k <= L, grid-stride, per-block partials.
template <typename R, int L>
__global__ void __launch_bounds__(kThreads)
k_gram(SolverDev d, const typename Ch<R>::T* r, size_t vs, double2* partials, const int* done) {
    if (done != nullptr && *done) return;
    constexpr int NG = n_gram(L);
    cx<R> acc[NG];
#pragma unroll
    for (int k = 0; k < NG; ++k) acc[k] = czero<R>();
    for (int s = blockIdx.x * kThreads + threadIdx.x; s < d.V; s += gridDim.x * kThreads) {
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
    block_reduce_store<NG, R>(acc, partials, gridDim.x);
}

// MR update: r_0 -= sum gamma_j r_j, u_0 -= sum gamma_j u_j.
// ACC: y += sum_k coef[m][slot_mr(k)] r_k (before the update).
// SHIFTS: x_s += sum_k c_k/(zeta p_s) r_k, u^s_0 <- (u^s_0 - sum gamma_j u^s_j)/p_s.
// DOT: per-block partials of <rt, r_0> (slot 0) and |r_0|^2 (slot 1), grid-stride.
template <typename R, int L, bool ACC, bool SHIFTS, bool DOT>
__global__ void __launch_bounds__(kThreads)
k_mr(SolverDev d, typename Ch<R>::T* r, typename Ch<R>::T* u, const typename Ch<R>::T* rt, size_t vs,
     double2* y, double2* xs, double2* us, size_t svs, typename Ch<R>::T* store, double2* partials,
     const int* done) {
    if (done != nullptr && *done) return;
    const int m = d.st->m;
    cx<R> ng[L + 1];
    ng[0] = czero<R>();
#pragma unroll
    for (int j = 1; j <= L; ++j) ng[j] = negcx<R>(d.rec_gamma[m * (L + 1) + j]);
    const double2* cf = d.coef + (size_t)m * nc_slots(L);
    cx<R> dots[2] = {czero<R>(), czero<R>()};
    for (int s = blockIdx.x * kThreads + threadIdx.x; s < d.V; s += gridDim.x * kThreads) {
#pragma unroll
        for (int q = 0; q < Ch<R>::N; ++q) {
            Ch<R> rv[L + 1];
#pragma unroll
            for (int i = 0; i <= L; ++i) rv[i] = Ch<R>::ld(r + i * vs, q, d.V, s);
            if (store != nullptr) {
#pragma unroll
                for (int k = 0; k < L; ++k) rv[k].stv(store + slot_mr(L, k) * vs, q, d.V, s);
            }
            if (ACC) {
                cx<R> t[Ch<R>::W];
#pragma unroll
                for (int w = 0; w < Ch<R>::W; ++w) t[w] = czero<R>();
#pragma unroll
                for (int k = 0; k < L; ++k) {
                    const cx<R> c = tocx<R>(cf[slot_mr(L, k)]);
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
    if (DOT) block_reduce_store<2, R>(dots, partials, gridDim.x);
}

// <rt, r0> (slot 0) and |r0|^2 (slot 1), grid-stride (start of a solve)
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_dot2(int V, const typename Ch<R>::T* rt, const typename Ch<R>::T* r0, double2* partials) {
    cx<R> dots[2] = {czero<R>(), czero<R>()};
    for (int s = blockIdx.x * kThreads + threadIdx.x; s < V; s += gridDim.x * kThreads) {
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
    block_reduce_store<2, R>(dots, partials, gridDim.x);
}

// ------------------------------------------------------------------ single-block scalar kernels
// Deterministic reduction of nblk partials of slot `slot` by the whole block.
__device__ __forceinline__ dcx reduce_partials(const double2* part, int slot, int nblk) {
    __shared__ double2 red[kScalarThreads];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
        double2 v = part[(size_t)slot * nblk + i];
        a += v.x;
        b += v.y;
    }
    red[threadIdx.x] = make_double2(a, b);
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            red[threadIdx.x].x += red[threadIdx.x + o].x;
            red[threadIdx.x].y += red[threadIdx.x + o].y;
        }
        __syncthreads();
    }
    dcx r = ld(red[0]);
    __syncthreads();
    return r;
}

__device__ __forceinline__ void fail(DevState* S, int code) {
    if (S->status == FA_OK) S->status = code;
    S->done = 1;
}

// start of pass 1: partials hold <rt, r0> and |r0|^2 with r0 = rt = b
__global__ void k_sc_init(SolverDev d, const double2* part, int nblk, double tol, double theta) {
    DevState* S = d.st;
    const dcx rtr = reduce_partials(part, 0, nblk);
    const dcx bb = reduce_partials(part, 1, nblk);
    for (int sh = threadIdx.x; sh < d.ns; sh += blockDim.x) {
        d.zeta[sh] = pk(mk(1.0));
        d.zeta_p[sh] = pk(mk(1.0));
        d.active[sh] = 1;
        d.iters[sh] = 0;
    }
    if (threadIdx.x == 0) {
        S->bnorm2 = bb.r;
        S->tol2b = tol * tol * bb.r;
        S->theta2b = theta * theta * bb.r;
        S->rnorm2 = bb.r;
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
        if (!(bb.r > 0.0) || !isfinite(bb.r)) fail(S, FA_EINVAL);
    }
}

// beta of BiCG sub-step j >= 1 from partials of <rt, r_j>
__global__ void k_sc_beta(SolverDev d, int j, const double2* part, int nblk) {
    DevState* S = d.st;
    if (S->done) return;
    const dcx rho1 = reduce_partials(part, 0, nblk);
    if (threadIdx.x == 0) {
        const dcx rho0 = ld(S->rho0);
        if (abs2(rho0) == 0.0) { fail(S, FA_EBREAKDOWN); return; }
        const dcx beta = ld(S->alpha) * rho1 / rho0;
        if (!finite(beta)) { fail(S, FA_ENONFINITE); return; }
        S->rho0 = pk(rho1);
        d.rec_beta[S->m * d.L + j] = pk(beta);
    }
}

// alpha of BiCG sub-step j from partials of <rt, u_{j+1}>, and the shift scalars
__global__ void k_sc_alpha(SolverDev d, int j, const double2* part, int nblk) {
    DevState* S = d.st;
    if (S->done) return;
    const dcx den = reduce_partials(part, 0, nblk);
    __shared__ int bad;
    if (threadIdx.x == 0) bad = (abs2(den) == 0.0) ? FA_EBREAKDOWN : 0;
    __syncthreads();
    if (bad) { if (threadIdx.x == 0) fail(S, bad); return; }
    const int m = S->m;
    const dcx alpha = ld(S->rho0) / den;
    const dcx beta = ld(d.rec_beta[m * d.L + j]);
    const dcx aprev = ld(S->alpha_prev);
    for (int sh = threadIdx.x; sh < d.ns; sh += blockDim.x) {
        if (!d.active[sh]) continue;
        const double sg = d.sigma[sh];
        const dcx z = ld(d.zeta[sh]), zp = ld(d.zeta_p[sh]);
        const dcx zn = (mk(1.0) + sg * alpha) * z + (alpha * beta / aprev) * (zp - z);
        const dcx as = alpha * z / zn;
        const dcx r = zp / z;
        const dcx bs = beta * r * r;
        double2* P = d.prec + ((size_t)sh * d.max_outer + m) * ps_stride(d.L) + 5 * j;
        P[0] = pk(as);
        P[1] = pk(bs);
        P[2] = pk(mk(1.0) / z);
        P[3] = pk(mk(1.0) / (as * z));
        P[4] = pk(mk(1.0) / (as * zn));
        if (!finite(zn) || abs2(zn) == 0.0 || !finite(as)) fail(S, FA_ENONFINITE);
        d.zeta_p[sh] = pk(z);
        d.zeta[sh] = pk(zn);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!finite(alpha)) { fail(S, FA_ENONFINITE); return; }
        d.rec_alpha[m * d.L + j] = pk(alpha);
        S->alpha = pk(alpha);
        S->alpha_prev = pk(alpha);
    }
}

// MR coefficients: gamma from the Gram partials (diagonally scaled normal
// equations, pivoted elimination), then the shift polynomials p_s(-sigma), c_k.
template <int L>
__global__ void k_sc_mr(SolverDev d, const double2* part, int nblk) {
    DevState* S = d.st;
    if (S->done) return;
    constexpr int NG = n_gram(L);
    __shared__ dcx G[NG];
    __shared__ dcx gam[L + 1];
    __shared__ int bad;
    for (int k = 0; k < NG; ++k) {
        dcx v = reduce_partials(part, k, nblk);
        if (threadIdx.x == 0) G[k] = v;
    }
    if (threadIdx.x == 0) {
        bad = 0;
        // slot of (i, k), i <= k, in the row-major upper triangle
        auto slot = [](int i, int k) { return i * (L + 1) - i * (i - 1) / 2 + (k - i); };
        dcx M[L][L], rhs[L];
        double dsc[L];
        for (int i = 1; i <= L; ++i) {
            const double gii = G[slot(i, i)].r;
            if (!(gii > 0.0) || !isfinite(gii)) bad = FA_EBREAKDOWN;
            dsc[i - 1] = (gii > 0.0) ? 1.0 / sqrt(gii) : 1.0;
        }
        for (int i = 1; i <= L; ++i) {
            for (int k = 1; k <= L; ++k) {
                const dcx gik = (i <= k) ? G[slot(i, k)] : conjd(G[slot(k, i)]);
                M[i - 1][k - 1] = (dsc[i - 1] * dsc[k - 1]) * gik;
            }
            rhs[i - 1] = dsc[i - 1] * conjd(G[slot(0, i)]);   // <r_i, r_0>
        }
        // Gaussian elimination with partial pivoting on the scaled normal
        // equations (the power basis r_1..r_l can make them numerically
        // indefinite for large l; any solution is a valid MR polynomial)
        dcx Ab[L][L + 1];
        for (int i = 0; i < L; ++i) {
            for (int k = 0; k < L; ++k) Ab[i][k] = M[i][k];
            Ab[i][L] = rhs[i];
        }
        for (int k = 0; k < L && !bad; ++k) {
            int pr = k;
            double best = abs2(Ab[k][k]);
            for (int i = k + 1; i < L; ++i)
                if (abs2(Ab[i][k]) > best) { best = abs2(Ab[i][k]); pr = i; }
            if (!(best > 0.0)) { bad = FA_EBREAKDOWN; break; }
            if (pr != k)
                for (int q = k; q <= L; ++q) { dcx t = Ab[k][q]; Ab[k][q] = Ab[pr][q]; Ab[pr][q] = t; }
            for (int i = k + 1; i < L; ++i) {
                const dcx f = Ab[i][k] / Ab[k][k];
                for (int q = k; q <= L; ++q) Ab[i][q] = Ab[i][q] - f * Ab[k][q];
            }
        }
        if (!bad) {
            dcx z[L];
            for (int i = L - 1; i >= 0; --i) {
                dcx v = Ab[i][L];
                for (int q = i + 1; q < L; ++q) v = v - Ab[i][q] * z[q];
                z[i] = v / Ab[i][i];
            }
            gam[0] = mk(-1.0);
            for (int j = 1; j <= L; ++j) {
                gam[j] = dsc[j - 1] * z[j - 1];
                if (!finite(gam[j])) bad = FA_ENONFINITE;
            }
        }
        if (bad) fail(S, bad);
    }
    __syncthreads();
    if (bad) return;
    const int m = S->m;
    for (int sh = threadIdx.x; sh < d.ns; sh += blockDim.x) {
        if (!d.active[sh]) continue;
        const dcx ms = mk(-d.sigma[sh]);
        dcx pw[L + 1];
        pw[0] = mk(1.0);
        for (int j = 1; j <= L; ++j) pw[j] = pw[j - 1] * ms;
        dcx ps = mk(1.0);
        for (int j = 1; j <= L; ++j) ps = ps - gam[j] * pw[j];
        const dcx z = ld(d.zeta[sh]);
        double2* P = d.prec + ((size_t)sh * d.max_outer + m) * ps_stride(L) + 5 * L;
        const dcx zps = z * ps;
        P[0] = pk(mk(1.0) / ps);
        for (int k = 0; k < L; ++k) {
            dcx c = mk(0.0);
            for (int j = k + 1; j <= L; ++j) c = c + gam[j] * pw[j - 1 - k];
            P[1 + k] = pk(c / zps);
        }
        if (abs2(ps) == 0.0 || !finite(ps)) fail(S, FA_ENONFINITE);
        d.zeta[sh] = pk(zps);
        d.zeta_p[sh] = pk(ld(d.zeta_p[sh]) * ps);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int j = 0; j <= L; ++j) d.rec_gamma[m * (L + 1) + j] = pk(gam[j]);
        S->omega = pk(gam[L]);
    }
}

// end of an outer iteration: convergence and freezing of shifts, next beta
__global__ void k_sc_conv(SolverDev d, const double2* part, int nblk, int head) {
    DevState* S = d.st;
    if (S->done) return;
    const dcx rtr = reduce_partials(part, 0, nblk);
    const double rn2 = reduce_partials(part, 1, nblk).r;
    const int m = S->m;
    __shared__ int n_act, all_small;
    if (threadIdx.x == 0) { n_act = 0; all_small = 1; }
    __syncthreads();
    for (int sh = threadIdx.x; sh < d.ns; sh += blockDim.x) {
        if (!d.active[sh]) continue;
        const double z2 = abs2(ld(d.zeta[sh]));
        if (rn2 <= S->tol2b * z2) {
            d.active[sh] = 0;
            d.iters[sh] = m + 1;
        } else {
            atomicAdd(&n_act, 1);
            if (rn2 > S->theta2b * z2) atomicAnd(&all_small, 0);
        }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    S->rnorm2 = rn2;
    S->m = m + 1;
    S->n_active = n_act;
    if (!isfinite(rn2) || !finite(rtr)) { fail(S, FA_ENONFINITE); S->n_outer = m + 1; return; }
    if (head && all_small) S->switch_req = 1;
    if (n_act == 0) { S->done = 1; S->n_outer = m + 1; return; }
    if (m + 1 >= d.max_outer) { fail(S, FA_ENOCONV); S->n_outer = m + 1; return; }
    const dcx rho0 = -1.0 * (ld(S->omega) * ld(S->rho0));
    if (abs2(rho0) == 0.0) { fail(S, FA_EBREAKDOWN); S->n_outer = m + 1; return; }
    const dcx beta = ld(S->alpha) * rtr / rho0;
    S->rho0 = pk(rtr);
    d.rec_beta[(m + 1) * d.L] = pk(beta);
}

// ------------------------------------------------------------------ pseudo-double-pass gather
// y += sum_{m in [m_begin, m_end)} sum_k coef[m][k] v(m, k), the stored seed-vector
// occurrences of pass 1 (store slot (m - m0) * NC + k).  Terms are summed in R
// in groups of four, each group added to y in FP64.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_gather(SolverDev d, const typename Ch<R>::T* store, size_t vs, int m_begin, int m_end, int m0, double2* y) {
    const int s = blockIdx.x * kThreads + threadIdx.x;
    if (s >= d.V) return;
    const int NC = nc_slots(d.L);
    const int n = (m_end - m_begin) * NC;
    const double2* cf = d.coef + (size_t)m_begin * NC;
    const typename Ch<R>::T* base = store + (size_t)(m_begin - m0) * NC * vs;
    double acc[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) acc[k] = 0.0;
    for (int k0 = 0; k0 < n; k0 += 4) {
        cx<R> t[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) t[k] = czero<R>();
        const int k1 = min(n, k0 + 4);
        for (int k = k0; k < k1; ++k) {
            const cx<R> c = tocx<R>(cf[k]);
            const typename Ch<R>::T* v = base + (size_t)k * vs;
#pragma unroll
            for (int q = 0; q < Ch<R>::N; ++q) {
                Ch<R> a = Ch<R>::ld(v, q, d.V, s);
#pragma unroll
                for (int w = 0; w < Ch<R>::W; ++w) t[q * Ch<R>::W + w] = cfma(c, a.c[w], t[q * Ch<R>::W + w]);
            }
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            acc[2 * k] = __dadd_rn(acc[2 * k], (double)t[k].r);
            acc[2 * k + 1] = __dadd_rn(acc[2 * k + 1], (double)t[k].i);
        }
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        double2* p = y + (size_t)k * d.V + s;
        double2 a = *p;
        a.x = __dadd_rn(a.x, acc[2 * k]);
        a.y = __dadd_rn(a.y, acc[2 * k + 1]);
        *p = a;
    }
}

// pass 2: advance the outer-iteration counter
__global__ void k_advance(SolverDev d) { d.st->m += 1; }
__global__ void k_set_m(SolverDev d, int m) { d.st->m = m; d.st->done = 0; }

// ------------------------------------------------------------------ backward sweep
// One thread per shift walks its recorded linear operations backwards
// (adjoint of "dst <- sum a src + sum c v_occ"), starting from the adjoint
// lambda_X = 1 of its final solution; the adjoint of each seed-vector
// occurrence is that occurrence's weight in x_s.  The weighted sum over shifts
// is formed by k_coef_reduce.
template <int L>
__global__ void k_sweep(SolverDev d) {
    const int sh = blockIdx.x * blockDim.x + threadIdx.x;
    if (sh >= d.ns) return;
    constexpr int NC = nc_slots(L);
    const int Ms = d.iters[sh];
    const double sg = d.sigma[sh];
    dcx lX = mk(1.0);
    dcx lU[L + 1];
#pragma unroll
    for (int i = 0; i <= L; ++i) lU[i] = mk(0.0);
    for (int m = Ms - 1; m >= 0; --m) {
        const double2* P = d.prec + ((size_t)sh * d.max_outer + m) * ps_stride(L);
        const double2* G = d.rec_gamma + m * (L + 1);
        dcx c[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) c[k] = mk(0.0);
        // MR, reversed: u0 <- (u0 - sum gamma_j u_j)/p_s, then x += sum cx_k r_k
        {
            const dcx t = lU[0] * ld(P[5 * L]);
#pragma unroll
            for (int jj = 1; jj <= L; ++jj) lU[jj] = lU[jj] - ld(G[jj]) * t;
            lU[0] = t;
#pragma unroll
            for (int k = 0; k < L; ++k) c[slot_mr(L, k)] = c[slot_mr(L, k)] + lX * ld(P[5 * L + 1 + k]);
        }
#pragma unroll
        for (int j = L - 1; j >= 0; --j) {
            const double2* Q = P + 5 * j;
            // x += alpha_s u_0
            lU[0] = lU[0] + ld(Q[0]) * lX;
            // u_{j+1} <- r_old_j/(alpha_s zeta) - r_j/(alpha_s zeta_new) - sigma u_j
            const dcx lu = lU[j + 1];
            c[slot_old(j, j)] = c[slot_old(j, j)] + lu * ld(Q[3]);
            const int snew = (j < L - 1) ? slot_old(j + 1, j) : slot_mr(L, L - 1);
            c[snew] = c[snew] - lu * ld(Q[4]);
            lU[j] = lU[j] - sg * lu;
            lU[j + 1] = mk(0.0);
            // u_i <- r_old_i/zeta - beta_s u_i
            const dcx iz = ld(Q[2]), bs = ld(Q[1]);
#pragma unroll
            for (int i = 0; i <= j; ++i) {
                c[slot_old(j, i)] = c[slot_old(j, i)] + lU[i] * iz;
                lU[i] = -1.0 * (bs * lU[i]);
            }
        }
        double2* out = d.cs + ((size_t)sh * d.max_outer + m) * NC;
#pragma unroll
        for (int k = 0; k < NC; ++k) out[k] = pk(c[k]);
    }
}

// coef[m][k] = sum_s omega_s cs[s][m][k] for m < M (fixed order over s)
__global__ void k_coef_reduce(SolverDev d, int M) {
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
}

// single-pass result y = sum_s omega_s x_s (FP64 [12][V])
__global__ void k_combine(int V, int ns, const double* omega, const double2* xs, size_t svs, double2* y) {
    const int idx = blockIdx.x * kThreads + threadIdx.x;
    if (idx >= 12 * V) return;
    double a = 0.0, b = 0.0;
    for (int sh = 0; sh < ns; ++sh) {
        const double2 v = xs[sh * svs + idx];
        a = __fma_rn(omega[sh], v.x, a);
        b = __fma_rn(omega[sh], v.y, b);
    }
    y[idx] = make_double2(a, b);
}

}  // namespace fa
