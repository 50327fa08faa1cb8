// Per-site arithmetic of one Wilson-Dirac sweep D_w(mu), shared by the
// stand-alone hop kernel (dslash.cu) and the solver's descriptor-driven hop
// (solver.cu), so that every application of the operator rounds identically.
//
//   (D psi)(x) = (4+m) psi(x) - 1/2 sum_nu [ f+ (1 - g_nu) U_nu(x) psi(x+nu)
//                                          + f- (1 + g_nu) U_nu(x-nu)^H psi(x-nu) ]
// (the Wilson-Dirac operator named in Sec. 1, mass form, e^{+-mu} on time hops,
// boundary sign on hops across t = T-1 <-> 0, DeGrand-Rossi projectors).
#pragma once

#include <type_traits>

#include "fa_internal.cuh"

namespace fa {

// projector P = 1 - S g_MU (S = +1 forward hop, -1 backward hop) applied to
// the 4 spin x 3 colour spinor p, as the two independent spin rows h0, h1.
// i*a = (-a.i, a.r).
template <int MU, int S, typename R>
__device__ __forceinline__ void project(const cx<R> p[12], cx<R> h[6]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cx<R> a0 = p[c], a1 = p[3 + c], a2 = p[6 + c], a3 = p[9 + c];
        if (MU == 0) {        // h0 = a0 - S i a3, h1 = a1 - S i a2
            h[c] = {a0.r + S * a3.i, a0.i - S * a3.r};
            h[3 + c] = {a1.r + S * a2.i, a1.i - S * a2.r};
        } else if (MU == 1) { // h0 = a0 + S a3, h1 = a1 - S a2
            h[c] = {a0.r + S * a3.r, a0.i + S * a3.i};
            h[3 + c] = {a1.r - S * a2.r, a1.i - S * a2.i};
        } else if (MU == 2) { // h0 = a0 - S i a2, h1 = a1 + S i a3
            h[c] = {a0.r + S * a2.i, a0.i - S * a2.r};
            h[3 + c] = {a1.r - S * a3.i, a1.i + S * a3.r};
        } else {              // h0 = a0 - S a2, h1 = a1 - S a3
            h[c] = {a0.r - S * a2.r, a0.i - S * a2.i};
            h[3 + c] = {a1.r - S * a3.r, a1.i - S * a3.i};
        }
    }
}

// acc += P psi given the projected, link-multiplied half spinor h.
template <int MU, int S, typename R>
__device__ __forceinline__ void recon_add(cx<R> acc[12], const cx<R> h[6]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cx<R> h0 = h[c], h1 = h[3 + c];
        acc[c] = cadd(acc[c], h0);
        acc[3 + c] = cadd(acc[3 + c], h1);
        if (MU == 0) {        // rows 2,3: S i h1, S i h0
            acc[6 + c] = {acc[6 + c].r - S * h1.i, acc[6 + c].i + S * h1.r};
            acc[9 + c] = {acc[9 + c].r - S * h0.i, acc[9 + c].i + S * h0.r};
        } else if (MU == 1) { // rows 2,3: -S h1, S h0
            acc[6 + c] = {acc[6 + c].r - S * h1.r, acc[6 + c].i - S * h1.i};
            acc[9 + c] = {acc[9 + c].r + S * h0.r, acc[9 + c].i + S * h0.i};
        } else if (MU == 2) { // rows 2,3: S i h0, -S i h1
            acc[6 + c] = {acc[6 + c].r - S * h0.i, acc[6 + c].i + S * h0.r};
            acc[9 + c] = {acc[9 + c].r + S * h1.i, acc[9 + c].i - S * h1.r};
        } else {              // rows 2,3: -S h0, -S h1
            acc[6 + c] = {acc[6 + c].r - S * h0.r, acc[6 + c].i - S * h0.i};
            acc[9 + c] = {acc[9 + c].r - S * h1.r, acc[9 + c].i - S * h1.i};
        }
    }
}

template <typename R, bool G5IN>
__device__ __forceinline__ void load_in(const SpinorView<R>& in, int s, cx<R> p[12]) {
    in.load(s, p);
    if (G5IN) {
#pragma unroll
        for (int k = 6; k < 12; ++k) p[k] = {-p[k].r, -p[k].i};
    }
}

// forward hop from site s to neighbour nb: acc += w (1 - g_MU) U_MU(s) psi(nb)
template <int MU, bool WEIGHT, bool G5IN, typename R>
__device__ __forceinline__ void hop_fwd(cx<R> acc[12], const SpinorView<R>& in, const LinkView<R>& U,
                                        int s, int nb, R w) {
    cx<R> p[12], h[6], L[3][3], c[6];
    load_in<R, G5IN>(in, nb, p);
    project<MU, +1>(p, h);
    U.load(MU, s, L);
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cx<R> t = cmul(L[a][0], h[3 * sp]);
            t = cfma(L[a][1], h[3 * sp + 1], t);
            t = cfma(L[a][2], h[3 * sp + 2], t);
            c[3 * sp + a] = WEIGHT ? cscale(w, t) : t;
        }
    recon_add<MU, +1>(acc, c);
}

// backward hop: acc += w (1 + g_MU) U_MU(nb)^H psi(nb), nb = s - MU
template <int MU, bool WEIGHT, bool G5IN, typename R>
__device__ __forceinline__ void hop_bwd(cx<R> acc[12], const SpinorView<R>& in, const LinkView<R>& U,
                                        int nb, R w) {
    cx<R> p[12], h[6], L[3][3], c[6];
    load_in<R, G5IN>(in, nb, p);
    project<MU, -1>(p, h);
    U.load(MU, nb, L);
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cx<R> t = cmul(cx<R>{L[0][a].r, -L[0][a].i}, h[3 * sp]);
            t = cjfma(L[1][a], h[3 * sp + 1], t);
            t = cjfma(L[2][a], h[3 * sp + 2], t);
            c[3 * sp + a] = WEIGHT ? cscale(w, t) : t;
        }
    recon_add<MU, -1>(acc, c);
}

// out = scale * G5OUT * ((4+m) in'(s) - 1/2 sum hops(in')), in' = G5IN ? g5 in : in;
// cdiag = scale*(4+m), chop = -scale/2, ef/eb = e^{+-mu}, bc = time-boundary sign.
template <typename R, bool G5IN, bool G5OUT>
__device__ __forceinline__ void hop_site(const Geom& g, const LinkView<R>& U, const SpinorView<R>& in, int s,
                                         R cdiag, R chop, R ef, R eb, R bc, cx<R> p[12]) {
    const int X = g.X, Y = g.Y, Z = g.Z, T = g.T;
    const int x = s % X;
    const int r1 = s / X;
    const int y = r1 % Y;
    const int r2 = r1 / Y;
    const int z = r2 % Z;
    const int t = r2 / Z;
    const int sY = X, sZ = X * Y, sT = X * Y * Z;
    cx<R> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = czero<R>();
    hop_fwd<0, false, G5IN>(acc, in, U, s, (x == X - 1) ? s - (X - 1) : s + 1, R(1));
    hop_bwd<0, false, G5IN>(acc, in, U, (x == 0) ? s + (X - 1) : s - 1, R(1));
    hop_fwd<1, false, G5IN>(acc, in, U, s, (y == Y - 1) ? s - (Y - 1) * sY : s + sY, R(1));
    hop_bwd<1, false, G5IN>(acc, in, U, (y == 0) ? s + (Y - 1) * sY : s - sY, R(1));
    hop_fwd<2, false, G5IN>(acc, in, U, s, (z == Z - 1) ? s - (Z - 1) * sZ : s + sZ, R(1));
    hop_bwd<2, false, G5IN>(acc, in, U, (z == 0) ? s + (Z - 1) * sZ : s - sZ, R(1));
    const R wf = (t == T - 1) ? mulR(ef, bc) : ef;
    const R wb = (t == 0) ? mulR(eb, bc) : eb;
    hop_fwd<3, true, G5IN>(acc, in, U, s, (t == T - 1) ? s - (T - 1) * sT : s + sT, wf);
    hop_bwd<3, true, G5IN>(acc, in, U, (t == 0) ? s + (T - 1) * sT : s - sT, wb);
    load_in<R, G5IN>(in, s, p);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const bool neg = G5OUT && k >= 6;
        const R a = neg ? -cdiag : cdiag;
        const R b = neg ? -chop : chop;
        cx<R> o = cscale(a, p[k]);
        o = crfma(b, acc[k], o);
        p[k] = o;
    }
}

// FP32: the kernel is bound by load latency (long-scoreboard stalls); the
// register budget is set for FA_HOP_MINB resident blocks per SM.  Measured on
// 32^3 x 64: 3 blocks/SM (79 registers) 5.02 TB/s, 4 blocks/SM (64 registers,
// 132 B spilled) 4.78 TB/s.
#ifndef FA_HOP_MINB
#define FA_HOP_MINB 3
#endif
// double-float: register budget for FA_HOP_MINB_DF resident blocks per SM.  The
// kernel is bound by dependent FP32 instruction chains; measured on 16^3 x 32:
// 1 block/SM (160 registers) 0.219 ms, 2 blocks/SM (128 registers, 40 B
// spilled) 0.169 ms per sweep.
#ifndef FA_HOP_MINB_DF
#define FA_HOP_MINB_DF 2
#endif
template <typename R> constexpr int hop_min_blocks() {
    return sizeof(R) == 4 ? FA_HOP_MINB : (std::is_same<R, df>::value ? FA_HOP_MINB_DF : 1);
}

}  // namespace fa
