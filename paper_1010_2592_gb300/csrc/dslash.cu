// Wilson-Dirac hop kernels D_w(mu) for sm_103a, FP64 (18-real links) and
// FP32 (12-real links), plus layout conversions.
//
// D_w(mu) is named in Sec. 1 (the kernel of the overlap operator at nonzero
// chemical potential); the definition implemented is the standard mass form
//   (D psi)(x) = (4+m) psi(x) - 1/2 sum_nu [ f+ (1 - g_nu) U_nu(x) psi(x+nu)
//                                          + f- (1 + g_nu) U_nu(x-nu)^H psi(x-nu) ]
// with f+- = e^{+-mu} on time hops and the time-boundary sign on hops that
// cross t = T-1 <-> 0.  Each hop projects the neighbour spinor to a half
// spinor with the DeGrand-Rossi projector (1 -+ g_nu), multiplies the two
// colour vectors by the link and rebuilds the lower spin components.
//
// One thread per site; the nearest-neighbour reuse of spinors and links is
// left to L1/L2 (the 126 MB L2 holds several time slices of every field even
// on 32^3 x 64).  Memory traffic floor per site and sweep: one spinor in, one
// out, four links (FP32: 96 + 96 + 4 * 48 = 384 B).
#include "hop_device.cuh"

namespace fa {

template <typename R, bool G5IN, bool G5OUT, bool DOT, int NT = kThreads, int MB = hop_min_blocks<R>()>
__global__ void __launch_bounds__(NT, MB)
hop_kernel(Geom g, LinkView<R> U, SpinorView<R> in, SpinorView<R> out, R cdiag, R chop, R ef, R eb,
           R bc, SpinorView<R> dotv, double2* partials, const int* done) {
    if (done != nullptr && *done) return;
    const int s = blockIdx.x * NT + threadIdx.x;
    cx<R> dres[1] = {czero<R>()};
    if (s < g.V) {
        cx<R> p[12];
        hop_site<R, G5IN, G5OUT>(g, U, in, s, cdiag, chop, ef, eb, bc, p);
        out.store(s, p);
        if (DOT) {
            cx<R> d[12];
            dotv.load(s, d);
            cx<R> a = czero<R>();
#pragma unroll
            for (int k = 0; k < 12; ++k) a = cjfma(d[k], p[k], a);
            dres[0] = a;
        }
    }
    if (DOT) block_reduce_store<1, R, NT>(dres, partials, 0, blockIdx.x);
}

// Number of SMs of the current device (cached per device).
int sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (cache[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        cache[dev] = n;
    }
    return cache[dev];
}

bool hop_narrow(int V) {
    const int n = sm_count();
    return n > 0 && kHopNarrowBlocks > 0 && (V + kHopNarrowThreads - 1) / kHopNarrowThreads <= kHopNarrowBlocks * n;
}

// the same sweep split by colour row (double-float)
template <typename R, bool G5IN, bool G5OUT, bool DOT>
__global__ void __launch_bounds__(kRowThreads, rows_min_blocks<DOT>())
hop_rows_kernel(Geom g, LinkView<R> U, SpinorView<R> in, SpinorView<R> out, R cdiag, R chop, R ef, R eb,
                R bc, SpinorView<R> dotv, double2* partials, const int* done) {
    if (done != nullptr && *done) return;
    cx<R> dres[1] = {hop_rows_body<R, G5IN, G5OUT, DOT>(g, U, in, out, cdiag, chop, ef, eb, bc, dotv, blockIdx.x)};
    if (DOT) block_reduce_store<1, R, kRowThreads>(dres, partials, 0, blockIdx.x);
}

template <typename R, typename LP, typename SP>
static int launch_hop_t(const Geom& g, const LP* links, const SP* in, SP* out, double diag, double ef,
                        double eb, double t_bc, double scale, bool g5in, bool g5out, const SP* dot_with,
                        double2* partials, const int* done, cudaStream_t st, int shape = 0) {
    LinkView<R> U{links, g.V};
    SpinorView<R> vin{const_cast<SP*>(in), g.V};
    SpinorView<R> vout{out, g.V};
    SpinorView<R> vd{const_cast<SP*>(dot_with), g.V};
    const R cdiag = (R)(scale * diag), chop = (R)(-0.5 * scale);
    const R ref = (R)ef, reb = (R)eb, rbc = (R)t_bc;
    const bool dot = dot_with != nullptr;
    if constexpr (std::is_same<R, float>::value) {
      if (hop_use_narrow(shape, g.V)) {
        constexpr int NT = kHopNarrowThreads, MB = kHopNarrowBlocks;
        const int nb = (g.V + NT - 1) / NT;
#define FA_HOPN(A, B, C) hop_kernel<R, A, B, C, NT, MB><<<nb, NT, 0, st>>>(g, U, vin, vout, cdiag, chop, ref, reb, rbc, vd, partials, done)
        if (!g5in && !g5out && !dot) FA_HOPN(false, false, false);
        else if (!g5in && g5out && !dot) FA_HOPN(false, true, false);
        else if (!g5in && g5out && dot) FA_HOPN(false, true, true);
        else if (g5in && g5out && !dot) FA_HOPN(true, true, false);
        else if (!g5in && !g5out && dot) FA_HOPN(false, false, true);
        else return FA_EINVAL;
#undef FA_HOPN
        return launch_status("hop kernel");
      }
    }
    const int nb = nblocks(g.V);
#define FA_HOP(A, B, C) hop_kernel<R, A, B, C><<<nb, kThreads, 0, st>>>(g, U, vin, vout, cdiag, chop, ref, reb, rbc, vd, partials, done)
    if (!g5in && !g5out && !dot) FA_HOP(false, false, false);
    else if (!g5in && g5out && !dot) FA_HOP(false, true, false);
    else if (!g5in && g5out && dot) FA_HOP(false, true, true);
    else if (g5in && g5out && !dot) FA_HOP(true, true, false);
    else if (!g5in && !g5out && dot) FA_HOP(false, false, true);
    else return FA_EINVAL;
#undef FA_HOP
    return launch_status("hop kernel");
}

int launch_hop_f64(const Geom& g, const double2* links, const double2* in, double2* out, double diag,
                   double ef, double eb, double t_bc, double scale, bool g5in, bool g5out,
                   const double2* dot_with, double2* partials, const int* done, cudaStream_t st) {
    return launch_hop_t<double>(g, links, in, out, diag, ef, eb, t_bc, scale, g5in, g5out, dot_with,
                                partials, done, st);
}

int launch_hop_df(const Geom& g, const float4* links, const float4* in, float4* out, double diag, double ef,
                  double eb, double t_bc, double scale, bool g5in, bool g5out, const float4* dot_with,
                  double2* partials, const int* done, cudaStream_t st) {
    LinkView<df> U{links, g.V};
    SpinorView<df> vin{const_cast<float4*>(in), g.V};
    SpinorView<df> vout{out, g.V};
    SpinorView<df> vd{const_cast<float4*>(dot_with), g.V};
    const df cdiag = host_cvt<df>(scale * diag), chop = host_cvt<df>(-0.5 * scale);
    const df ref = host_cvt<df>(ef), reb = host_cvt<df>(eb), rbc = host_cvt<df>(t_bc);
    const int nb = row_blocks(g.V);
    const bool dot = dot_with != nullptr;
#define FA_HOPD(A, B, C) hop_rows_kernel<df, A, B, C><<<nb, kRowThreads, 0, st>>>(g, U, vin, vout, cdiag, chop, ref, reb, rbc, vd, partials, done)
    if (!g5in && !g5out && !dot) FA_HOPD(false, false, false);
    else if (!g5in && g5out && !dot) FA_HOPD(false, true, false);
    else if (!g5in && g5out && dot) FA_HOPD(false, true, true);
    else if (g5in && g5out && !dot) FA_HOPD(true, true, false);
    else if (!g5in && !g5out && dot) FA_HOPD(false, false, true);
    else return FA_EINVAL;
#undef FA_HOPD
    return launch_status("hop kernel");
}

int launch_hop_f32(const Geom& g, const float4* links, const float4* in, float4* out, double diag,
                   double ef, double eb, double t_bc, double scale, bool g5in, bool g5out,
                   const float4* dot_with, double2* partials, const int* done, cudaStream_t st, int shape) {
    return launch_hop_t<float>(g, links, in, out, diag, ef, eb, t_bc, scale, g5in, g5out, dot_with,
                               partials, done, st, shape);
}

// ------------------------------------------------------------------ link force (adjoint)
// For the bilinears B_p = <a_p, D_w(mu) b_p> (p = 1, 2) the variation under a
// link change dU_nu(x) is sum_ij [dU_ij M_ij + conj(dU_ji) K_ij] with
//   M_ij = -1/2 f+ sum_s conj(a_si(x))      ((1 - g_nu) b(x+nu))_sj   (forward hop at x)
//   K_ij = -1/2 f- sum_s conj(a_si(x+nu))   ((1 + g_nu) b(x))_sj      (backward hop at x+nu)
// so Re dB = Re tr(G^H dU) with G = conj(M) + K^T.  The kernel adds
// w * (G_1 + G_2) to the canonical gradient array and writes per-block partials
// of w * (dB_1/dmu + dB_2/dmu), dB/dmu = sum M_ij U_ij - sum K_ij conj(U_ji) on
// time links.  a_1 enters as gamma_5 a_1 when G5A1 is set.
template <int MU>
__device__ __forceinline__ void force_dir(int s, int nb, double fp, double fm, const LinkView<double>& U,
                                          const SpinorView<double> a[2], const SpinorView<double> b[2],
                                          double w, double2* Gout, cx<double>& dmu) {
    cx<double> Gm[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Gm[i][j] = czero<double>();
    cx<double> Uc[3][3];
    if (MU == 3) U.load(3, s, Uc);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        cx<double> ax[12], an[12], bx[12], bn[12], Pb[12], Qb[12], h[6];
        a[p].load(s, ax);
        a[p].load(nb, an);
        b[p].load(s, bx);
        b[p].load(nb, bn);
        if (p == 0) {
#pragma unroll
            for (int k = 6; k < 12; ++k) { ax[k] = {-ax[k].r, -ax[k].i}; an[k] = {-an[k].r, -an[k].i}; }
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) { Pb[k] = czero<double>(); Qb[k] = czero<double>(); }
        project<MU, +1>(bn, h);
        recon_add<MU, +1>(Pb, h);
        project<MU, -1>(bx, h);
        recon_add<MU, -1>(Qb, h);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                cx<double> m = czero<double>(), k = czero<double>();
#pragma unroll
                for (int sp = 0; sp < 4; ++sp) {
                    m = cjfma(ax[3 * sp + i], Pb[3 * sp + j], m);
                    k = cjfma(an[3 * sp + i], Qb[3 * sp + j], k);
                }
                m = cscale(-0.5 * fp, m);
                k = cscale(-0.5 * fm, k);
                // G_ij += conj(M_ij); G_ji += K_ij
                Gm[i][j] = cadd(Gm[i][j], cx<double>{m.r, -m.i});
                Gm[j][i] = cadd(Gm[j][i], k);
                if (MU == 3) {
                    dmu = cfma(m, Uc[i][j], dmu);                                     // + M_ij U_ij
                    dmu = cfma(cx<double>{-k.r, -k.i}, cx<double>{Uc[j][i].r, -Uc[j][i].i}, dmu);  // - K_ij conj(U_ji)
                }
            }
    }
    double2* g = Gout + ((size_t)s * 4 + MU) * 9;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        double2 v = g[e];
        v.x = __fma_rn(w, Gm[e / 3][e % 3].r, v.x);
        v.y = __fma_rn(w, Gm[e / 3][e % 3].i, v.y);
        g[e] = v;
    }
}

__global__ void __launch_bounds__(kThreads)
k_force(Geom g, LinkView<double> U, SpinorView<double> a1, SpinorView<double> b1, SpinorView<double> a2,
        SpinorView<double> b2, double2* G, double w, double ef, double eb, double bc, double2* partials) {
    const int s = blockIdx.x * kThreads + threadIdx.x;
    cx<double> dm[1] = {czero<double>()};
    if (s < g.V) {
        const int X = g.X, Y = g.Y, Z = g.Z, T = g.T;
        const int x = s % X, r1 = s / X, y = r1 % Y, r2 = r1 / Y, z = r2 % Z, t = r2 / Z;
        const int sY = X, sZ = X * Y, sT = X * Y * Z;
        const SpinorView<double> a[2] = {a1, a2};
        const SpinorView<double> b[2] = {b1, b2};
        force_dir<0>(s, (x == X - 1) ? s - (X - 1) : s + 1, 1.0, 1.0, U, a, b, w, G, dm[0]);
        force_dir<1>(s, (y == Y - 1) ? s - (Y - 1) * sY : s + sY, 1.0, 1.0, U, a, b, w, G, dm[0]);
        force_dir<2>(s, (z == Z - 1) ? s - (Z - 1) * sZ : s + sZ, 1.0, 1.0, U, a, b, w, G, dm[0]);
        // forward hop at x crosses the boundary from t = T-1; so does the backward hop at x + t_hat
        const double fp = (t == T - 1) ? ef * bc : ef;
        const double fm = (t == T - 1) ? eb * bc : eb;
        force_dir<3>(s, (t == T - 1) ? s - (T - 1) * sT : s + sT, fp, fm, U, a, b, w, G, dm[0]);
        dm[0] = cscale(w, dm[0]);
    }
    block_reduce_store<1, double>(dm, partials, 0);
}

int launch_force(const Geom& g, const double2* links, const double2* a1, const double2* b1, const double2* a2,
                 const double2* b2, double* G_canon, double w, double ef, double eb, double t_bc,
                 double2* partials, cudaStream_t st) {
    LinkView<double> U{links, g.V};
    SpinorView<double> va1{const_cast<double2*>(a1), g.V}, vb1{const_cast<double2*>(b1), g.V};
    SpinorView<double> va2{const_cast<double2*>(a2), g.V}, vb2{const_cast<double2*>(b2), g.V};
    k_force<<<nblocks(g.V), kThreads, 0, st>>>(g, U, va1, vb1, va2, vb2, (double2*)G_canon, w, ef, eb, t_bc,
                                                partials);
    return launch_status("hop kernel");
}

// ------------------------------------------------------------------ layout conversions
// canonical spinor: double [V][12][2]; element (s, k) at 2*(12 s + k)
__global__ void pack_f64_kernel(int V, const double2* __restrict__ canon, double2* __restrict__ out) {
    const int idx = blockIdx.x * kThreads + threadIdx.x;   // idx = k*V + s
    if (idx >= 12 * V) return;
    const int k = idx / V, s = idx - k * V;
    out[idx] = canon[(size_t)s * 12 + k];
}

__global__ void unpack_f64_kernel(int V, const double2* __restrict__ in, double2* __restrict__ canon) {
    const int idx = blockIdx.x * kThreads + threadIdx.x;   // idx = 12*s + k
    if (idx >= 12 * V) return;
    const int s = idx / 12, k = idx - s * 12;
    canon[idx] = in[(size_t)k * V + s];
}

__global__ void pack_f32_kernel(int V, const double2* __restrict__ canon, float4* __restrict__ out) {
    const int idx = blockIdx.x * kThreads + threadIdx.x;   // idx = q*V + s
    if (idx >= 6 * V) return;
    const int q = idx / V, s = idx - q * V;
    const double2 a = canon[(size_t)s * 12 + 2 * q], b = canon[(size_t)s * 12 + 2 * q + 1];
    out[idx] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
}

__global__ void unpack_f32_kernel(int V, const float4* __restrict__ in, double2* __restrict__ canon) {
    const int idx = blockIdx.x * kThreads + threadIdx.x;   // idx = 6*s + q
    if (idx >= 6 * V) return;
    const int s = idx / 6, q = idx - s * 6;
    const float4 a = in[(size_t)q * V + s];
    canon[(size_t)s * 12 + 2 * q] = make_double2(a.x, a.y);
    canon[(size_t)s * 12 + 2 * q + 1] = make_double2(a.z, a.w);
}

__global__ void convert_f64_f32_kernel(int V, const double2* __restrict__ in, float4* __restrict__ out) {
    const int idx = blockIdx.x * kThreads + threadIdx.x;   // idx = q*V + s
    if (idx >= 6 * V) return;
    const int q = idx / V, s = idx - q * V;
    const double2 a = in[(size_t)(2 * q) * V + s], b = in[(size_t)(2 * q + 1) * V + s];
    out[idx] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
}

// canonical links: double [V][4][3][3][2]
__device__ __forceinline__ float4 to_df4(double2 v) {
    const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
    return make_float4(rh, __double2float_rn(__dsub_rn(v.x, (double)rh)), ih,
                       __double2float_rn(__dsub_rn(v.y, (double)ih)));
}

__global__ void pack_links_kernel(int V, const double2* __restrict__ canon, double2* __restrict__ l64,
                                  float4* __restrict__ l32, float4* __restrict__ ldf) {
    const int idx = blockIdx.x * kThreads + threadIdx.x;   // idx = mu*V + s
    if (idx >= 4 * V) return;
    const int mu = idx / V, s = idx - mu * V;
    const double2* src = canon + ((size_t)s * 4 + mu) * 9;
    double2 e[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) e[k] = src[k];
#pragma unroll
    for (int k = 0; k < 9; ++k) l64[((size_t)mu * 9 + k) * V + s] = e[k];
    if (ldf != nullptr) {
#pragma unroll
        for (int k = 0; k < 9; ++k) ldf[((size_t)mu * 9 + k) * V + s] = to_df4(e[k]);
    }
    if (l32 != nullptr) {
#pragma unroll
        for (int q = 0; q < 3; ++q)
            l32[((size_t)mu * 3 + q) * V + s] =
                make_float4((float)e[2 * q].x, (float)e[2 * q].y, (float)e[2 * q + 1].x, (float)e[2 * q + 1].y);
    }
}

static int grid_for(size_t n) { return (int)((n + kThreads - 1) / kThreads); }

int launch_pack_spinor_f64(const Geom& g, const double* canon, double2* out, cudaStream_t st) {
    pack_f64_kernel<<<grid_for((size_t)12 * g.V), kThreads, 0, st>>>(g.V, (const double2*)canon, out);
    return launch_status("layout conversion kernel");
}
int launch_unpack_spinor_f64(const Geom& g, const double2* in, double* canon, cudaStream_t st) {
    unpack_f64_kernel<<<grid_for((size_t)12 * g.V), kThreads, 0, st>>>(g.V, in, (double2*)canon);
    return launch_status("layout conversion kernel");
}
int launch_pack_spinor_f32(const Geom& g, const double* canon, float4* out, cudaStream_t st) {
    pack_f32_kernel<<<grid_for((size_t)6 * g.V), kThreads, 0, st>>>(g.V, (const double2*)canon, out);
    return launch_status("layout conversion kernel");
}
int launch_unpack_spinor_f32(const Geom& g, const float4* in, double* canon, cudaStream_t st) {
    unpack_f32_kernel<<<grid_for((size_t)6 * g.V), kThreads, 0, st>>>(g.V, in, (double2*)canon);
    return launch_status("layout conversion kernel");
}
int launch_pack_links(const Geom& g, const double* canon, double2* l64, float4* l32, float4* ldf, cudaStream_t st) {
    pack_links_kernel<<<grid_for((size_t)4 * g.V), kThreads, 0, st>>>(g.V, (const double2*)canon, l64, l32, ldf);
    return launch_status("layout conversion kernel");
}

__global__ void pack_df_kernel(int V, const double2* __restrict__ canon, float4* __restrict__ out) {
    const int idx = blockIdx.x * kThreads + threadIdx.x;   // idx = k*V + s
    if (idx >= 12 * V) return;
    const int k = idx / V, s = idx - k * V;
    out[idx] = to_df4(canon[(size_t)s * 12 + k]);
}

__global__ void unpack_df_kernel(int V, const float4* __restrict__ in, double2* __restrict__ canon) {
    const int idx = blockIdx.x * kThreads + threadIdx.x;   // idx = 12*s + k
    if (idx >= 12 * V) return;
    const int s = idx / 12, k = idx - s * 12;
    const float4 a = in[(size_t)k * V + s];
    canon[idx] = make_double2(__dadd_rn((double)a.x, (double)a.y), __dadd_rn((double)a.z, (double)a.w));
}

// double-float -> FP32 ([12][V] float4 -> [6][V] float4): hi + lo rounded once
__global__ void convert_df_f32_kernel(int V, const float4* __restrict__ in, float4* __restrict__ out) {
    const int idx = blockIdx.x * kThreads + threadIdx.x;   // idx = q*V + s
    if (idx >= 6 * V) return;
    const int q = idx / V, s = idx - q * V;
    const float4 a = in[(size_t)(2 * q) * V + s], b = in[(size_t)(2 * q + 1) * V + s];
    out[idx] = make_float4(__fadd_rn(a.x, a.y), __fadd_rn(a.z, a.w), __fadd_rn(b.x, b.y), __fadd_rn(b.z, b.w));
}

int launch_pack_spinor_df(const Geom& g, const double* canon, float4* out, cudaStream_t st) {
    pack_df_kernel<<<grid_for((size_t)12 * g.V), kThreads, 0, st>>>(g.V, (const double2*)canon, out);
    return launch_status("layout conversion kernel");
}
int launch_unpack_spinor_df(const Geom& g, const float4* in, double* canon, cudaStream_t st) {
    unpack_df_kernel<<<grid_for((size_t)12 * g.V), kThreads, 0, st>>>(g.V, in, (double2*)canon);
    return launch_status("layout conversion kernel");
}
int launch_convert_df_to_f32(const Geom& g, const float4* in, float4* out, cudaStream_t st) {
    convert_df_f32_kernel<<<grid_for((size_t)6 * g.V), kThreads, 0, st>>>(g.V, in, out);
    return launch_status("layout conversion kernel");
}
int launch_convert_f64_to_f32(const Geom& g, const double2* in, float4* out, cudaStream_t st) {
    convert_f64_f32_kernel<<<grid_for((size_t)6 * g.V), kThreads, 0, st>>>(g.V, in, out);
    return launch_status("layout conversion kernel");
}

}  // namespace fa
