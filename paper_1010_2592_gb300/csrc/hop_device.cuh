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
// one colour of the spinor (spins a0..a3), as the two independent spin rows
// h0, h1.  i*a = (-a.i, a.r).
template <int MU, int S, typename R>
__device__ __forceinline__ void project1(cx<R> a0, cx<R> a1, cx<R> a2, cx<R> a3, cx<R>& h0, cx<R>& h1) {
    if (MU == 0) {        // h0 = a0 - S i a3, h1 = a1 - S i a2
        h0 = {a0.r + S * a3.i, a0.i - S * a3.r};
        h1 = {a1.r + S * a2.i, a1.i - S * a2.r};
    } else if (MU == 1) { // h0 = a0 + S a3, h1 = a1 - S a2
        h0 = {a0.r + S * a3.r, a0.i + S * a3.i};
        h1 = {a1.r - S * a2.r, a1.i - S * a2.i};
    } else if (MU == 2) { // h0 = a0 - S i a2, h1 = a1 + S i a3
        h0 = {a0.r + S * a2.i, a0.i - S * a2.r};
        h1 = {a1.r - S * a3.i, a1.i + S * a3.r};
    } else {              // h0 = a0 - S a2, h1 = a1 - S a3
        h0 = {a0.r - S * a2.r, a0.i - S * a2.i};
        h1 = {a1.r - S * a3.r, a1.i - S * a3.i};
    }
}

// the 4 spin x 3 colour spinor p -> h[c] = h0, h[3 + c] = h1 for every colour
template <int MU, int S, typename R>
__device__ __forceinline__ void project(const cx<R> p[12], cx<R> h[6]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) project1<MU, S>(p[c], p[3 + c], p[6 + c], p[9 + c], h[c], h[3 + c]);
}

// one colour of acc += P psi given the link-multiplied spin rows h0, h1
template <int MU, int S, typename R>
__device__ __forceinline__ void recon1(cx<R>& c0, cx<R>& c1, cx<R>& c2, cx<R>& c3, cx<R> h0, cx<R> h1) {
    c0 = cadd(c0, h0);
    c1 = cadd(c1, h1);
    if (MU == 0) {        // rows 2,3: S i h1, S i h0
        c2 = {c2.r - S * h1.i, c2.i + S * h1.r};
        c3 = {c3.r - S * h0.i, c3.i + S * h0.r};
    } else if (MU == 1) { // rows 2,3: -S h1, S h0
        c2 = {c2.r - S * h1.r, c2.i - S * h1.i};
        c3 = {c3.r + S * h0.r, c3.i + S * h0.i};
    } else if (MU == 2) { // rows 2,3: S i h0, -S i h1
        c2 = {c2.r - S * h0.i, c2.i + S * h0.r};
        c3 = {c3.r + S * h1.i, c3.i - S * h1.r};
    } else {              // rows 2,3: -S h0, -S h1
        c2 = {c2.r - S * h0.r, c2.i - S * h0.i};
        c3 = {c3.r - S * h1.r, c3.i - S * h1.i};
    }
}

// acc += P psi given the projected, link-multiplied half spinor h
template <int MU, int S, typename R>
__device__ __forceinline__ void recon_add(cx<R> acc[12], const cx<R> h[6]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) recon1<MU, S>(acc[c], acc[3 + c], acc[6 + c], acc[9 + c], h[c], h[3 + c]);
}

// `in` is any spinor view with load(site, cx<R>[12]): a stored spinor, or a
// linear combination of two formed as it is read (the solver's fused sweeps)
template <typename R, bool G5IN, typename SV>
__device__ __forceinline__ void load_in(const SV& in, int s, cx<R> p[12]) {
    in.load(s, p);
    if (G5IN) {
#pragma unroll
        for (int k = 6; k < 12; ++k) p[k] = {-p[k].r, -p[k].i};
    }
}

// forward hop from site s to neighbour nb: acc += w (1 - g_MU) U_MU(s) psi(nb)
template <int MU, bool WEIGHT, bool G5IN, typename R, typename SV>
__device__ __forceinline__ void hop_fwd(cx<R> acc[12], const SV& in, const LinkView<R>& U,
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
template <int MU, bool WEIGHT, bool G5IN, typename R, typename SV>
__device__ __forceinline__ void hop_bwd(cx<R> acc[12], const SV& in, const LinkView<R>& U,
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
// PIN: pin receives in'(s), the input at the site itself.
template <typename R, bool G5IN, bool G5OUT, bool PIN = false, typename SV>
__device__ __forceinline__ void hop_site(const Geom& g, const LinkView<R>& U, const SV& in, int s,
                                         R cdiag, R chop, R ef, R eb, R bc, cx<R> p[12], cx<R>* pin = nullptr) {
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
    if constexpr (PIN) {
#pragma unroll
        for (int k = 0; k < 12; ++k) pin[k] = p[k];
    }
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

// ------------------------------------------------------------------ colour-row split (double-float)
// The double-float sweep with one thread per site and output colour row a: for
// each hop the thread of row a projects colour a of the neighbour spinor and
// shares the two spin rows through shared memory, then multiplies the three
// colours by row a of U (column a of U^H), so it holds two partial products and
// four accumulators instead of whole spinors.
//
// Its arithmetic is compensated rather than renormalised after every
// operation: each row of U h is one compensated dot product (the Dot2 scheme of
// Ogita, Rump and Oishi, SIAM J. Sci. Comput. 26 (2005), with FP32-pair
// inputs).  A value is carried as an FP32 sum s and an FP32 term e; a product
// adds its rounded value to s by TwoSum and its exact error (FMA), the two
// hi*lo cross terms and the TwoSum error to e.  Projections and the sum over
// the eight directions carry (s, e) the same way, and each output component is
// renormalised once (TwoSum of s and e).  The result has the accuracy of a
// product in twice the working precision, rounded to an FP32 pair (relative
// error a few times 2^-44 at most here), at about 70% of the instructions.
struct dsum {
    float s, e;
};
__device__ __forceinline__ dsum dsum_of(df a) { return {a.hi, a.lo}; }
__device__ __forceinline__ dsum dneg(dsum a) { return {-a.s, -a.e}; }
// a + b: TwoSum of the leading parts, the lower parts added to the error term
__device__ __forceinline__ dsum dadd(dsum a, dsum b) {
    const float s = __fadd_rn(a.s, b.s);
    const float bb = __fsub_rn(s, a.s);
    const float t = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, bb)), __fsub_rn(b.s, bb));
    return {s, __fadd_rn(t, __fadd_rn(a.e, b.e))};
}
// a * b: the rounded product and its exact error plus the cross terms
__device__ __forceinline__ dsum dmul(dsum a, dsum b) {
    const float p = __fmul_rn(a.s, b.s);
    float err = __fmaf_rn(a.s, b.s, -p);
    err = __fmaf_rn(a.s, b.e, err);
    err = __fmaf_rn(a.e, b.s, err);
    return {p, err};
}
// A + a * b
__device__ __forceinline__ dsum dfma(dsum a, dsum b, dsum A) {
    const float p = __fmul_rn(a.s, b.s);
    float err = __fmaf_rn(a.s, b.s, -p);
    err = __fmaf_rn(a.s, b.e, err);
    err = __fmaf_rn(a.e, b.s, err);
    const float s = __fadd_rn(A.s, p);
    const float bb = __fsub_rn(s, A.s);
    const float t = __fadd_rn(__fsub_rn(A.s, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    return {s, __fadd_rn(A.e, __fadd_rn(err, t))};
}
// renormalised FP32 pair (TwoSum: |e| may exceed |s| after cancellation)
__device__ __forceinline__ df dnorm(dsum a) { return two_sum(a.s, a.e); }

struct dcs {     // complex (s, e) pairs
    dsum r, i;
};
__device__ __forceinline__ dcs dcs_of(cx<df> a) { return {dsum_of(a.r), dsum_of(a.i)}; }

// projector rows of one colour in (s, e) form (project1 with compensated sums)
template <int MU, int S>
__device__ __forceinline__ void project1_c(dcs a0, dcs a1, dcs a2, dcs a3, dcs& h0, dcs& h1) {
    auto sg = [](dsum x) { return S > 0 ? x : dneg(x); };
    if (MU == 0) {        // h0 = a0 - S i a3, h1 = a1 - S i a2
        h0 = {dadd(a0.r, sg(a3.i)), dadd(a0.i, dneg(sg(a3.r)))};
        h1 = {dadd(a1.r, sg(a2.i)), dadd(a1.i, dneg(sg(a2.r)))};
    } else if (MU == 1) { // h0 = a0 + S a3, h1 = a1 - S a2
        h0 = {dadd(a0.r, sg(a3.r)), dadd(a0.i, sg(a3.i))};
        h1 = {dadd(a1.r, dneg(sg(a2.r))), dadd(a1.i, dneg(sg(a2.i)))};
    } else if (MU == 2) { // h0 = a0 - S i a2, h1 = a1 + S i a3
        h0 = {dadd(a0.r, sg(a2.i)), dadd(a0.i, dneg(sg(a2.r)))};
        h1 = {dadd(a1.r, dneg(sg(a3.i))), dadd(a1.i, sg(a3.r))};
    } else {              // h0 = a0 - S a2, h1 = a1 - S a3
        h0 = {dadd(a0.r, dneg(sg(a2.r))), dadd(a0.i, dneg(sg(a2.i)))};
        h1 = {dadd(a1.r, dneg(sg(a3.r))), dadd(a1.i, dneg(sg(a3.i)))};
    }
}

// acc (4 spins of one colour) += P psi given the link-multiplied rows h0, h1
template <int MU, int S>
__device__ __forceinline__ void recon1_c(dcs acc[4], dcs h0, dcs h1) {
    auto sg = [](dsum x) { return S > 0 ? x : dneg(x); };
    acc[0] = {dadd(acc[0].r, h0.r), dadd(acc[0].i, h0.i)};
    acc[1] = {dadd(acc[1].r, h1.r), dadd(acc[1].i, h1.i)};
    if (MU == 0) {        // rows 2,3: S i h1, S i h0
        acc[2] = {dadd(acc[2].r, dneg(sg(h1.i))), dadd(acc[2].i, sg(h1.r))};
        acc[3] = {dadd(acc[3].r, dneg(sg(h0.i))), dadd(acc[3].i, sg(h0.r))};
    } else if (MU == 1) { // rows 2,3: -S h1, S h0
        acc[2] = {dadd(acc[2].r, dneg(sg(h1.r))), dadd(acc[2].i, dneg(sg(h1.i)))};
        acc[3] = {dadd(acc[3].r, sg(h0.r)), dadd(acc[3].i, sg(h0.i))};
    } else if (MU == 2) { // rows 2,3: S i h0, -S i h1
        acc[2] = {dadd(acc[2].r, dneg(sg(h0.i))), dadd(acc[2].i, sg(h0.r))};
        acc[3] = {dadd(acc[3].r, sg(h1.i)), dadd(acc[3].i, dneg(sg(h1.r)))};
    } else {              // rows 2,3: -S h0, -S h1
        acc[2] = {dadd(acc[2].r, dneg(sg(h0.r))), dadd(acc[2].i, dneg(sg(h0.i)))};
        acc[3] = {dadd(acc[3].r, dneg(sg(h1.r))), dadd(acc[3].i, dneg(sg(h1.i)))};
    }
}

// Thread layout of the row-split sweep: blocks of kRowThreads = 3 colour rows x
// 64 sites; warps 2a and 2a+1 take row a of 32 consecutive sites each, so the
// three rows of a site run on one SM and share its neighbour loads in L1.
constexpr int kRowSites = 64;
constexpr int kRowThreads = 3 * kRowSites;
__device__ __forceinline__ int row_of_thread() { return (int)(threadIdx.x >> 6); }
// site of the thread in block bx of the sweep
__device__ __forceinline__ int site_of_thread(int bx) {
    return bx * kRowSites + (int)(threadIdx.x & (kRowSites - 1));
}
inline int row_blocks(int V) { return (V + kRowSites - 1) / kRowSites; }

// The projection is shared through shared memory: for each hop the thread of
// row a projects colour a of the neighbour spinor (four loads instead of
// twelve) and stores the two spin rows; after a barrier every row reads the
// three colours.  Double-buffered, one barrier per hop.
__device__ __forceinline__ float4 dcs_pack(dcs v) { return make_float4(v.r.s, v.r.e, v.i.s, v.i.e); }
__device__ __forceinline__ dcs dcs_unpack(float4 t) { return {{t.x, t.y}, {t.z, t.w}}; }

// project colour a of psi(nb) and store the spin rows: buf[(2a + r) * kRowSites + i]
template <int MU, int S, bool G5IN>
__device__ __forceinline__ void proj_store(const SpinorView<df>& in, int nb, int a, float4* buf, int i, bool valid) {
    dcs h0{{0.0f, 0.0f}, {0.0f, 0.0f}}, h1 = h0;
    if (valid) {
        dcs p0 = dcs_of(in.ld1(nb, a)), p1 = dcs_of(in.ld1(nb, 3 + a));
        dcs p2 = dcs_of(in.ld1(nb, 6 + a)), p3 = dcs_of(in.ld1(nb, 9 + a));
        if (G5IN) {
            p2 = {dneg(p2.r), dneg(p2.i)};
            p3 = {dneg(p3.r), dneg(p3.i)};
        }
        project1_c<MU, S>(p0, p1, p2, p3, h0, h1);
    }
    buf[(2 * a) * kRowSites + i] = dcs_pack(h0);
    buf[(2 * a + 1) * kRowSites + i] = dcs_pack(h1);
}

// acc += w P (U or U^H) psi(nb) for row a, from the stored spin rows of all colours
template <int MU, int S, bool WEIGHT>
__device__ __forceinline__ void mul_recon(dcs acc[4], const LinkView<df>& U, int ls, int a, df w, const float4* buf,
                                          int i) {
    dcs t0, t1;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const dcs h0 = dcs_unpack(buf[(2 * c) * kRowSites + i]), h1 = dcs_unpack(buf[(2 * c + 1) * kRowSites + i]);
        const dcs L = dcs_of(U.ld1(MU, ls, S > 0 ? a * 3 + c : c * 3 + a));
        const dsum li = S > 0 ? L.i : dneg(L.i);
        if (c == 0) {
            t0 = {dfma(dneg(li), h0.i, dmul(L.r, h0.r)), dfma(li, h0.r, dmul(L.r, h0.i))};
            t1 = {dfma(dneg(li), h1.i, dmul(L.r, h1.r)), dfma(li, h1.r, dmul(L.r, h1.i))};
        } else {
            t0 = {dfma(dneg(li), h0.i, dfma(L.r, h0.r, t0.r)), dfma(li, h0.r, dfma(L.r, h0.i, t0.i))};
            t1 = {dfma(dneg(li), h1.i, dfma(L.r, h1.r, t1.r)), dfma(li, h1.r, dfma(L.r, h1.i, t1.i))};
        }
    }
    if (WEIGHT) {
        const dsum ws = dsum_of(w);
        t0 = {dmul(dsum_of(dnorm(t0.r)), ws), dmul(dsum_of(dnorm(t0.i)), ws)};
        t1 = {dmul(dsum_of(dnorm(t1.r)), ws), dmul(dsum_of(dnorm(t1.i)), ws)};
    }
    recon1_c<MU, S>(acc, t0, t1);
}

template <bool G5IN, bool G5OUT>
__device__ __forceinline__ void hop_site_row_sh(const Geom& g, const LinkView<df>& U, const SpinorView<df>& in, int s,
                                                int a, bool valid, df cdiag, df chop, df ef, df eb, df bc, cx<df> o[4]) {
    __shared__ float4 hs[2][6 * kRowSites];
    const int i = (int)(threadIdx.x & (kRowSites - 1));
    const int X = g.X, Y = g.Y, Z = g.Z, T = g.T;
    const int sv = valid ? s : 0;
    const int x = sv % X;
    const int r1 = sv / X;
    const int y = r1 % Y;
    const int r2 = r1 / Y;
    const int z = r2 % Z;
    const int t = r2 / Z;
    const int sY = X, sZ = X * Y, sT = X * Y * Z;
    dcs acc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
    const df one(1.0f);
    int nb = (x == X - 1) ? sv - (X - 1) : sv + 1;
    proj_store<0, +1, G5IN>(in, nb, a, hs[0], i, valid);
    __syncthreads();
    mul_recon<0, +1, false>(acc, U, sv, a, one, hs[0], i);
    nb = (x == 0) ? sv + (X - 1) : sv - 1;
    proj_store<0, -1, G5IN>(in, nb, a, hs[1], i, valid);
    __syncthreads();
    mul_recon<0, -1, false>(acc, U, nb, a, one, hs[1], i);
    nb = (y == Y - 1) ? sv - (Y - 1) * sY : sv + sY;
    proj_store<1, +1, G5IN>(in, nb, a, hs[0], i, valid);
    __syncthreads();
    mul_recon<1, +1, false>(acc, U, sv, a, one, hs[0], i);
    nb = (y == 0) ? sv + (Y - 1) * sY : sv - sY;
    proj_store<1, -1, G5IN>(in, nb, a, hs[1], i, valid);
    __syncthreads();
    mul_recon<1, -1, false>(acc, U, nb, a, one, hs[1], i);
    nb = (z == Z - 1) ? sv - (Z - 1) * sZ : sv + sZ;
    proj_store<2, +1, G5IN>(in, nb, a, hs[0], i, valid);
    __syncthreads();
    mul_recon<2, +1, false>(acc, U, sv, a, one, hs[0], i);
    nb = (z == 0) ? sv + (Z - 1) * sZ : sv - sZ;
    proj_store<2, -1, G5IN>(in, nb, a, hs[1], i, valid);
    __syncthreads();
    mul_recon<2, -1, false>(acc, U, nb, a, one, hs[1], i);
    const df wf = (t == T - 1) ? mulR(ef, bc) : ef;
    const df wb = (t == 0) ? mulR(eb, bc) : eb;
    nb = (t == T - 1) ? sv - (T - 1) * sT : sv + sT;
    proj_store<3, +1, G5IN>(in, nb, a, hs[0], i, valid);
    __syncthreads();
    mul_recon<3, +1, true>(acc, U, sv, a, wf, hs[0], i);
    nb = (t == 0) ? sv + (T - 1) * sT : sv - sT;
    proj_store<3, -1, G5IN>(in, nb, a, hs[1], i, valid);
    __syncthreads();
    mul_recon<3, -1, true>(acc, U, nb, a, wb, hs[1], i);
    if (!valid) return;
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) {
        cx<df> p = in.ld1(s, sp * 3 + a);
        if (G5IN && sp >= 2) p = {-p.r, -p.i};
        const bool neg = G5OUT && sp >= 2;
        const df ca = neg ? -cdiag : cdiag;
        const df cb = neg ? -chop : chop;
        const cx<df> h{dnorm(acc[sp].r), dnorm(acc[sp].i)};
        cx<df> v = cscale(ca, p);
        v = crfma(cb, h, v);
        o[sp] = v;
    }
}

// out(s, row) = hop_site(s) row; DOT: returns <dotv, out> over the thread's 4 components
// (every thread of the block takes part: the sweep has block barriers)
template <typename R, bool G5IN, bool G5OUT, bool DOT>
__device__ __forceinline__ cx<R> hop_rows_body(const Geom& g, const LinkView<R>& U, const SpinorView<R>& in,
                                               const SpinorView<R>& out, R cdiag, R chop, R ef, R eb, R bc,
                                               const SpinorView<R>& dotv, int bx) {
    const int a = row_of_thread(), s = site_of_thread(bx);
    cx<R> dres = czero<R>();
    cx<R> o[4];
    hop_site_row_sh<G5IN, G5OUT>(g, U, in, s, a, s < g.V, cdiag, chop, ef, eb, bc, o);
    if (s < g.V) {
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) out.st1(s, sp * 3 + a, o[sp]);
        if (DOT) {
#pragma unroll
            for (int sp = 0; sp < 4; ++sp) dres = cjfma(dotv.ld1(s, sp * 3 + a), o[sp], dres);
        }
    }
    return dres;
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
// row-split double-float sweep: resident blocks of kRowThreads per SM.  Measured
// per sweep (16^3 x 32 / 32^3 x 64) with the first, renormalised row split:
// 3 blocks/SM 0.099 / 1.416 ms, 4 (80 registers) 0.099 / 1.409 ms, 5 (64
// registers) 0.098 / 1.377 ms; the whole-site double-float sweep took 0.169 /
// 2.65 ms.  The compensated sweep with the shared projection (64 registers, no
// spill) takes 0.068 / 0.934 ms.
// The batched variant that also forms <dotv, out> and runs a scalar step keeps
// one block less (the descriptor fields cost registers).
#ifndef FA_HOP_ROWS_MINB
#define FA_HOP_ROWS_MINB 5
#endif
template <bool DOT> constexpr int rows_min_blocks() { return FA_HOP_ROWS_MINB; }
template <bool DOT> constexpr int rows_sys_min_blocks() { return DOT ? FA_HOP_ROWS_MINB - 1 : FA_HOP_ROWS_MINB; }
// FP32 narrow launch shape: 128-thread blocks, 7 per SM (72 registers), used
// when the whole lattice then fits in one wave (7 x 128 x SMs sites); a lattice
// a little larger than one wave of the 3 x 256 shape otherwise runs a second,
// nearly empty wave.
#ifndef FA_HOP_NARROW_BLOCKS
#define FA_HOP_NARROW_BLOCKS 7
#endif
constexpr int kHopNarrowThreads = 128;
constexpr int kHopNarrowBlocks = FA_HOP_NARROW_BLOCKS;   // 0: never narrow
template <typename R> constexpr int hop_min_blocks() {
    return sizeof(R) == 4 ? FA_HOP_MINB : (std::is_same<R, df>::value ? FA_HOP_MINB_DF : 1);
}

}  // namespace fa
