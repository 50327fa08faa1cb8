// C-ABI entry points of libfapath (declared in include/fapath.h).
#include <cmath>
#include <cstdarg>
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "fa_context.h"

namespace fa {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int cuda_fail(cudaError_t e, const char* what) {
    set_error("%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    return FA_ECUDA;
}

}  // namespace fa

using namespace fa;

#define CUDA_OR(x, what)                                   \
    do {                                                   \
        cudaError_t _e = (x);                              \
        if (_e != cudaSuccess) return cuda_fail(_e, what); \
    } while (0)
#define TRY(x)                        \
    do {                              \
        int _rc = (x);                \
        if (_rc != FA_OK) return _rc; \
    } while (0)

extern "C" {

const char* fa_version(void) { return "fapath 0.1 (sm_103a)"; }

const char* fa_last_error(void) { return g_err; }

const char* fa_status_string(int s) {
    switch (s) {
        case FA_OK: return "ok";
        case FA_EINVAL: return "invalid argument";
        case FA_ENOMEM: return "out of memory";
        case FA_ECUDA: return "CUDA error";
        case FA_EBREAKDOWN: return "Krylov breakdown";
        case FA_ENOCONV: return "not converged within max_outer";
        case FA_ENONFINITE: return "non-finite recurrence scalar";
        case FA_ETIMEOUT: return "device wait timed out";
        case FA_ESTATE: return "call out of order (gauge field, parameters or poles missing)";
        default: return "unknown status";
    }
}

int fa_create(fa_ctx** out, const int dims[4], void* cuda_stream) {
    if (!out || !dims) return FA_EINVAL;
    *out = nullptr;
    for (int k = 0; k < 4; ++k)
        if (dims[k] < 2 || dims[k] > 4096) {
            set_error("fa_create: extent %d out of range", dims[k]);
            return FA_EINVAL;
        }
    const long long V = (long long)dims[0] * dims[1] * dims[2] * dims[3];
    if (V > (1LL << 26)) {
        set_error("fa_create: volume %lld above 2^26 sites", V);
        return FA_EINVAL;
    }
    fa_ctx* c = new (std::nothrow) fa_ctx();
    if (!c) return FA_ENOMEM;
    c->g = Geom{dims[0], dims[1], dims[2], dims[3], (int)V};
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "fa_create: cudaGetDevice");
    }
    *out = c;
    return FA_OK;
}

int fa_destroy(fa_ctx* c) {
    if (!c) return FA_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    for (cudaEvent_t e : c->hop_ev) cudaEventDestroy(e);
    for (auto& g : c->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (c->pinned) cudaFreeHost(c->pinned);
    delete c;
    return FA_OK;
}

int fa_set_gauge(fa_ctx* c, const double* U, int on_device) {
    if (!c || !U) return FA_EINVAL;
    const int V = c->g.V;
    const size_t canon_bytes = (size_t)V * 72 * sizeof(double);
    CUDA_OR(c->links64.ensure((size_t)36 * V * sizeof(double2)), "fa_set_gauge: alloc FP64 links");
    CUDA_OR(c->links32.ensure((size_t)12 * V * sizeof(float4)), "fa_set_gauge: alloc FP32 links");
    CUDA_OR(c->linksdf.ensure((size_t)36 * V * sizeof(float4)), "fa_set_gauge: alloc double-float links");
    const double* src = U;
    DevBuf stage;
    if (!on_device) {
        CUDA_OR(stage.ensure(canon_bytes), "fa_set_gauge: alloc staging");
        CUDA_OR(cudaMemcpyAsync(stage.p, U, canon_bytes, cudaMemcpyHostToDevice, c->stream), "fa_set_gauge: copy");
        src = stage.as<double>();
    }
    TRY(launch_pack_links(c->g, src, c->links64.as<double2>(), c->links32.as<float4>(), c->linksdf.as<float4>(),
                          c->stream));
    c->launches++;
    CUDA_OR(cudaStreamSynchronize(c->stream), "fa_set_gauge: sync");
    c->links_owner = nullptr;
    c->have_gauge = true;
    return FA_OK;
}

int fa_share_gauge(fa_ctx* c, const fa_ctx* owner) {
    if (!c || !owner || c == owner || owner->links_owner) return FA_EINVAL;
    if (!owner->have_gauge) return FA_ESTATE;
    if (c->g.X != owner->g.X || c->g.Y != owner->g.Y || c->g.Z != owner->g.Z || c->g.T != owner->g.T ||
        c->device != owner->device)
        return FA_EINVAL;
    c->links64.release();
    c->links32.release();
    c->linksdf.release();
    c->links_owner = owner;
    c->have_gauge = true;
    return FA_OK;
}

int fa_set_params(fa_ctx* c, double wilson_mass, double mu, int t_bc, double scale_c) {
    if (!c) return FA_EINVAL;
    if (!std::isfinite(wilson_mass) || !std::isfinite(mu) || !(t_bc == 1 || t_bc == -1) ||
        !(scale_c > 0.0) || !std::isfinite(scale_c) || std::fabs(mu) > 20.0)
        return FA_EINVAL;
    c->mass = wilson_mass;
    c->mu = mu;
    c->t_bc = (double)t_bc;
    c->scale_c = scale_c;
    c->have_params = true;
    return FA_OK;
}

int fa_set_poles(fa_ctx* c, int ns, const double* omega, const double* sigma) {
    if (!c || !omega || !sigma || ns < 1 || ns > kMaxShifts) return FA_EINVAL;
    for (int s = 0; s < ns; ++s)
        if (!(sigma[s] > 0.0) || !std::isfinite(sigma[s]) || !std::isfinite(omega[s])) return FA_EINVAL;
    c->ns = ns;
    for (int s = 0; s < ns; ++s) {
        c->omega[s] = omega[s];
        c->sigma[s] = sigma[s];
    }
    c->have_poles = true;
    return FA_OK;
}

int fa_neuberger_poles(int ns, double* omega, double* sigma) {
    if (ns < 1 || ns > kMaxShifts || !omega || !sigma) return FA_EINVAL;
    const double pi = 3.14159265358979323846;
    for (int s = 1; s <= ns; ++s) {
        const double th = pi * (s - 0.5) / (2.0 * ns);
        const double cth = std::cos(th);
        omega[s - 1] = (1.0 / ns) / (cth * cth);
        const double t = std::tan(th);
        sigma[s - 1] = t * t;
    }
    return FA_OK;
}

// Elliptic functions for Zolotarev's expansion.  K(k) = pi / (2 AGM(1, k')) with
// k' the complementary modulus (Abramowitz & Stegun 17.6).  The expansion needs
// sc(u | kappa') and dn(u | kappa') for kappa' = sqrt(1 - eps^2), a modulus close
// to 1 where cn(u) is small and amplitude-based methods lose digits.  Jacobi's
// imaginary transformation (A&S 16.20) turns them into functions of the small
// modulus eps at the imaginary argument iu: sc(u | kappa') = -i sn(iu | eps) and
// dn(u | kappa') = dn(iu | eps) / cn(iu | eps), evaluated by the theta series
// (A&S 16.36) of nome q = exp(-pi K(kappa') / K(eps)) at v = i w,
// w = pi u / (2 K(eps)):
//   sc = (th3(0) / th2(0)) * 2 sum_n (-1)^n q^{(n+1/2)^2} sinh((2n+1) w) / th4(iw),
//   dn = (th2(0) / th3(0)) * th3(iw) / th2(iw),
// th3(iw) = 1 + 2 sum q^{n^2} cosh(2nw), th4(iw) = 1 + 2 sum (-1)^n q^{n^2} cosh(2nw),
// th2(iw) = 2 sum q^{(n+1/2)^2} cosh((2n+1)w).  For u <= K(kappa')/2 the terms
// fall like q^{n^2 - n} and th4(iw) >= 1 - 2 sqrt(q).
namespace {
double ellip_K_of_complement(double kc) {
    double a = 1.0, b = kc;
    for (int it = 0; it < 64 && std::fabs(a - b) > 1e-17 * a; ++it) {
        const double an = 0.5 * (a + b);
        b = std::sqrt(a * b);
        a = an;
    }
    return 3.14159265358979323846 / (2.0 * a);
}
struct ZoloElliptic {
    double K_eps, K_kp, log_q, th2_0, th3_0;
    explicit ZoloElliptic(double eps) {
        const double kp = std::sqrt((1.0 - eps) * (1.0 + eps));
        K_eps = ellip_K_of_complement(kp);   // K(eps)
        K_kp = ellip_K_of_complement(eps);   // K(kappa')
        log_q = -3.14159265358979323846 * K_kp / K_eps;
        th2_0 = 0.0;
        th3_0 = 1.0;
        for (int n = 0; n < 64; ++n) {
            const double e = std::exp(log_q * (n + 0.5) * (n + 0.5));
            th2_0 += 2.0 * e;
            if (n >= 1) th3_0 += 2.0 * std::exp(log_q * n * n);
            if (e < 1e-300) break;
        }
    }
    // sc(u | kappa') and dn(u | kappa') for 0 <= u <= K(kappa') / 2
    void sc_dn(double u, double* sc, double* dn) const {
        const double w = 3.14159265358979323846 * u / (2.0 * K_eps);
        double t1 = 0.0, t2 = 0.0, th3 = 1.0, th4 = 1.0;
        for (int n = 0; n < 64; ++n) {
            const double e = std::exp(log_q * (n + 0.5) * (n + 0.5));
            const double sgn = (n % 2) ? -1.0 : 1.0;
            t1 += 2.0 * sgn * e * std::sinh((2 * n + 1) * w);
            t2 += 2.0 * e * std::cosh((2 * n + 1) * w);
            if (n >= 1) {
                const double f = 2.0 * std::exp(log_q * n * n) * std::cosh(2.0 * n * w);
                th3 += f;
                th4 += sgn * f;
            }
            if (e * std::cosh((2 * n + 1) * w) < 1e-300) break;
        }
        *sc = (th3_0 / th2_0) * t1 / th4;
        *dn = (th2_0 / th3_0) * th3 / t2;
    }
};
}  // namespace

int fa_zolotarev_poles(int ns, double eps, double* omega, double* sigma, double* delta) {
    if (ns < 1 || ns > kMaxShifts || !omega || !sigma || !(eps > 0.0) || !(eps < 1.0)) return FA_EINVAL;
    // modulus kappa' = sqrt(1 - eps^2); u_l = l K(kappa') / (2 ns).  Past K/2 the
    // reflection u -> K - u: sc(K - u) = cs(u) / eps and dn(K - u) = eps / dn(u).
    const ZoloElliptic z(eps);
    const double Kp = z.K_kp;
    double c[2 * kMaxShifts];
    for (int l = 1; l <= 2 * ns - 1; ++l) {
        double sc, dn;
        if (2 * l <= 2 * ns) {
            z.sc_dn(l * Kp / (2.0 * ns), &sc, &dn);
            c[l] = eps * eps * sc * sc;
        } else {
            z.sc_dn((2 * ns - l) * Kp / (2.0 * ns), &sc, &dn);
            c[l] = 1.0 / (sc * sc);
        }
    }
    // sigma_s = c_{2s-1}; residues of prod_{i<ns} (z + c_{2i}) / prod_s (z + c_{2s-1}).
    // Zeros and poles interlace, so each zero is paired with the neighbouring pole
    // on the far side from sigma_s: every factor lies in (0, 1) and the product
    // neither overflows nor underflows to 0/0 when the c span many decades.
    for (int s = 0; s < ns; ++s) {
        const double sg = c[2 * s + 1];
        double r = 1.0;
        for (int i = 1; i < ns; ++i) {
            const double pole = i <= s ? c[2 * (i - 1) + 1] : c[2 * i + 1];
            r *= (c[2 * i] - sg) / (pole - sg);
        }
        sigma[s] = sg;
        omega[s] = r;
    }
    // the error alternates at x_j = eps / dn(j K / (2 ns)), j = 0..2 ns (past K/2:
    // x_j = dn(K - u_j)); D centres it at x_0 and x_1
    double p[2 * kMaxShifts + 1];
    for (int j = 0; j <= 2 * ns; ++j) {
        double sc, dn, x;
        if (2 * j <= 2 * ns) {
            z.sc_dn(j * Kp / (2.0 * ns), &sc, &dn);
            x = eps / dn;
        } else {
            z.sc_dn((2 * ns - j) * Kp / (2.0 * ns), &sc, &dn);
            x = dn;
        }
        double acc = 0.0;
        for (int s = 0; s < ns; ++s) acc += omega[s] / (x * x + sigma[s]);
        p[j] = x * acc;
    }
    const double D = 2.0 / (p[0] + p[1]);
    const double d0 = std::fabs(D * p[0] - 1.0);
    // self-check: residues positive, and the error equal in size (to 1 % above the
    // rounding level of about 1e-12) with alternating signs at every alternation
    // point.  A pole set that double precision does not resolve fails it.
    const double floor_err = 1e-12;
    bool ok = std::isfinite(D) && D > 0.0;
    for (int s = 0; s < ns; ++s) ok = ok && omega[s] > 0.0 && std::isfinite(omega[s]);
    double dmax = 0.0;
    for (int j = 0; j <= 2 * ns; ++j) {
        const double e = D * p[j] - 1.0;
        dmax = std::max(dmax, std::fabs(e));
        ok = ok && std::fabs(std::fabs(e) - d0) <= 0.01 * d0 + floor_err;
        if (d0 > 100.0 * floor_err) ok = ok && (e > 0.0) == (j % 2 == 1);
    }
    if (!ok) {
        set_error("fa_zolotarev_poles: %d poles exceed what double precision resolves at eps = %g; "
                  "fewer poles reach the rounding floor", ns, eps);
        return FA_EINVAL;
    }
    for (int s = 0; s < ns; ++s) omega[s] *= D;
    if (delta) *delta = dmax;
    return FA_OK;
}

int fa_estimate_scale(fa_ctx* c, const double* v0, int iters, double* scale_out) {
    if (!c) return FA_EINVAL;
    return estimate_scale(c, v0, iters, scale_out);
}

// canonical in -> internal (FP64 or FP32), one or two hops, -> canonical out
static int apply_op(fa_ctx* c, const double* in, double* out, int dagger, int precision, bool is_A) {
    if (!c || !in || !out || in == out) return FA_EINVAL;
    if (!c->have_gauge || !c->have_params) return FA_ESTATE;
    const int V = c->g.V;
    cudaStream_t st = c->stream;
    const bool dg = dagger != 0;
    if (precision == FA_F64) {
        const size_t b = (size_t)12 * V * sizeof(double2);
        CUDA_OR(c->io64a.ensure(b), "alloc");
        CUDA_OR(c->io64b.ensure(b), "alloc");
        double2 *a = c->io64a.as<double2>(), *o = c->io64b.as<double2>();
        TRY(launch_pack_spinor_f64(c->g, in, a, st));
        if (is_A) {
            CUDA_OR(c->tmp64.ensure(b), "alloc");
            double2* t = c->tmp64.as<double2>();
            TRY(hop_f64(c, a, t, 1.0, false, true, dg, nullptr, nullptr, nullptr));
            TRY(hop_f64(c, t, o, c->scale_c, false, true, dg, nullptr, nullptr, nullptr));
        } else {
            TRY(hop_f64(c, a, o, 1.0, dg, dg, dg, nullptr, nullptr, nullptr));
        }
        TRY(launch_unpack_spinor_f64(c->g, o, out, st));
    } else if (precision == FA_F32) {
        const size_t b = (size_t)6 * V * sizeof(float4);
        CUDA_OR(c->io32a.ensure(b), "alloc");
        CUDA_OR(c->io32b.ensure(b), "alloc");
        float4 *a = c->io32a.as<float4>(), *o = c->io32b.as<float4>();
        TRY(launch_pack_spinor_f32(c->g, in, a, st));
        if (is_A) {
            CUDA_OR(c->tmp32.ensure(b), "alloc");
            float4* t = c->tmp32.as<float4>();
            TRY(hop_f32(c, a, t, 1.0, false, true, dg, nullptr, nullptr, nullptr));
            TRY(hop_f32(c, t, o, c->scale_c, false, true, dg, nullptr, nullptr, nullptr));
        } else {
            TRY(hop_f32(c, a, o, 1.0, dg, dg, dg, nullptr, nullptr, nullptr));
        }
        TRY(launch_unpack_spinor_f32(c->g, o, out, st));
    } else if (precision == FA_DF) {
        const size_t b = (size_t)12 * V * sizeof(float4);
        CUDA_OR(c->io64a.ensure(b), "alloc");
        CUDA_OR(c->io64b.ensure(b), "alloc");
        float4 *a = c->io64a.as<float4>(), *o = c->io64b.as<float4>();
        TRY(launch_pack_spinor_df(c->g, in, a, st));
        if (is_A) {
            CUDA_OR(c->tmp64.ensure(b), "alloc");
            float4* t = c->tmp64.as<float4>();
            TRY(hop_df(c, a, t, 1.0, false, true, dg, nullptr, nullptr, nullptr));
            TRY(hop_df(c, t, o, c->scale_c, false, true, dg, nullptr, nullptr, nullptr));
        } else {
            TRY(hop_df(c, a, o, 1.0, dg, dg, dg, nullptr, nullptr, nullptr));
        }
        TRY(launch_unpack_spinor_df(c->g, o, out, st));
    } else {
        return FA_EINVAL;
    }
    c->launches += 2;
    return FA_OK;
}

int fa_apply_dw(fa_ctx* c, const double* in, double* out, int dagger, int precision) {
    return apply_op(c, in, out, dagger, precision, false);
}

int fa_apply_A(fa_ctx* c, const double* in, double* out, int dagger, int precision) {
    return apply_op(c, in, out, dagger, precision, true);
}

int fa_solve_multishift(fa_ctx* c, const double* b, double* const* x_s, const fa_solver_params* p,
                        fa_solver_stats* stats) {
    if (!c || !b || !x_s || !p) return FA_EINVAL;
    if (p->mode != FA_SINGLE || p->precision != FA_F64) return FA_EINVAL;
    for (int s = 0; s < c->ns; ++s)
        if (!x_s[s]) return FA_EINVAL;
    return solve(c, b, nullptr, x_s, p, stats);
}

int fa_apply_f(fa_ctx* c, const double* b, double* y, const fa_solver_params* p, fa_solver_stats* stats) {
    if (!c || !b || !y || !p || b == y) return FA_EINVAL;
    return solve(c, b, y, nullptr, p, stats);
}

int fa_apply_sign(fa_ctx* c, const double* b, double* out, const fa_solver_params* p, fa_solver_stats* stats) {
    if (!c || !b || !out || !p || b == out) return FA_EINVAL;
    return apply_sign(c, b, out, p, stats, false);
}

int fa_apply_overlap(fa_ctx* c, const double* b, double* out, const fa_solver_params* p,
                     fa_solver_stats* stats) {
    if (!c || !b || !out || !p || b == out) return FA_EINVAL;
    return apply_sign(c, b, out, p, stats, true);
}

int fa_apply_sign_deflated(fa_ctx* c, const double* b, double* out, int k, const double* lambda, const double* R,
                           const double* Lv, int overlap, const fa_solver_params* p, fa_solver_stats* stats) {
    if (!c || !b || !out || !p || b == out || k < 0 || k > 1024) return FA_EINVAL;
    if (k > 0 && (!lambda || !R || !Lv || R == out || Lv == out)) return FA_EINVAL;
    return apply_sign_deflated(c, b, out, k, lambda, R, Lv, overlap != 0, p, stats);
}

int fa_eigs_smallest(fa_ctx* c, int k, int m, double tol, int max_restarts, const fa_solver_params* p,
                     unsigned long long seed, double* lambda, double* R, double* Lv, int* n_converged,
                     int* n_solves) {
    if (!c || !p || !lambda || !R || !Lv || !n_converged || !n_solves || R == Lv) return FA_EINVAL;
    return eigs_smallest(c, k, m, tol, max_restarts, p, seed, lambda, R, Lv, n_converged, n_solves);
}

int fa_apply_f_batched(fa_ctx* const* ctxs, int n, const double* const* b, double* const* y,
                       const fa_solver_params* p, fa_solver_stats* stats) {
    if (!ctxs || !b || !y || !p || n < 1 || n > 4096) return FA_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!ctxs[i] || !b[i] || !y[i]) return FA_EINVAL;
    // every system in one solve: each kernel launch serves all of them, whatever
    // their lattice shapes (work tables), and the FP32 sweeps read a lattice's
    // links once per tile for all the sources that share its gauge field
    std::vector<fa_solver_stats> st(n);
    const int rc = solve_batch(ctxs, n, b, y, nullptr, p, st.data());
    if (stats)
        for (int i = 0; i < n; ++i) stats[i] = st[i];
    return rc;
}

int fa_autotune_batched(fa_ctx* const* ctxs, int n, int reps, int* rhs_per_block, int* min_blocks, double* times_ms,
                        int ntimes) {
    if (!ctxs || n < 1 || n > 4096 || reps < 1 || !rhs_per_block || !min_blocks) return FA_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!ctxs[i]) return FA_EINVAL;
    return autotune_batch(ctxs, n, reps, rhs_per_block, min_blocks, times_ms, ntimes);
}

int fa_apply_f_host(fa_ctx* c, const double* b_host, double* y_host, const fa_solver_params* p,
                    fa_solver_stats* stats) {
    if (!c || !b_host || !y_host || !p) return FA_EINVAL;
    const size_t bytes = (size_t)c->g.V * 24 * sizeof(double);
    CUDA_OR(c->bhost_dev.ensure(bytes), "alloc staging");
    CUDA_OR(c->yhost_dev.ensure(bytes), "alloc staging");
    CUDA_OR(cudaMemcpyAsync(c->bhost_dev.p, b_host, bytes, cudaMemcpyHostToDevice, c->stream), "copy b");
    const int rc = solve(c, c->bhost_dev.as<double>(), c->yhost_dev.as<double>(), nullptr, p, stats);
    if (rc != FA_OK) return rc;
    CUDA_OR(cudaMemcpyAsync(y_host, c->yhost_dev.p, bytes, cudaMemcpyDeviceToHost, c->stream), "copy y");
    CUDA_OR(cudaStreamSynchronize(c->stream), "sync");
    return FA_OK;
}

int fa_grad(fa_ctx* c, const double* b, const double* eta, double* dLdU, double* dLdmu, double* L, double* dLdb,
            const fa_solver_params* p, fa_solver_stats* stats) {
    if (!c) return FA_EINVAL;
    return grad(c, b, eta, dLdU, dLdmu, L, dLdb, p, stats);
}

int fa_sync(fa_ctx* c) {
    if (!c) return FA_EINVAL;
    CUDA_OR(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize(), "fa_sync");
    CUDA_OR(cudaGetLastError(), "fa_sync");
    return FA_OK;
}

long long fa_launch_count(const fa_ctx* c) { return c ? c->launches : -1; }

namespace fa {
// FP32 issue-rate probe: eight independent FMA chains per thread, kFmaIters
// steps of eight FMAs each; the sums leave the kernel only if a runtime value
// says so (never), which keeps the chains alive.
constexpr int kFmaIters = 4096;
static __device__ float g_fma_sink;
__global__ void __launch_bounds__(256) k_fma_probe(float b, float c, int never) {
    float a0 = threadIdx.x * 1e-3f, a1 = a0 + 1.f, a2 = a0 + 2.f, a3 = a0 + 3.f;
    float a4 = a0 + 4.f, a5 = a0 + 5.f, a6 = a0 + 6.f, a7 = a0 + 7.f;
    for (int i = 0; i < kFmaIters; ++i) {
        a0 = __fmaf_rn(a0, b, c); a1 = __fmaf_rn(a1, b, c); a2 = __fmaf_rn(a2, b, c); a3 = __fmaf_rn(a3, b, c);
        a4 = __fmaf_rn(a4, b, c); a5 = __fmaf_rn(a5, b, c); a6 = __fmaf_rn(a6, b, c); a7 = __fmaf_rn(a7, b, c);
    }
    if (never) g_fma_sink = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}
}  // namespace fa

int fa_fp32_issue_rate(int reps, double* rate, double* ms_out) {
    using namespace fa;
    if (reps < 1 || !rate || !ms_out) return FA_EINVAL;
    int dev = 0, nsm = 0;
    CUDA_OR(cudaGetDevice(&dev), "fa_fp32_issue_rate: device");
    CUDA_OR(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "fa_fp32_issue_rate: SMs");
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_OR(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "fa_fp32_issue_rate: stream");
    cudaError_t err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    const int blocks = 8 * nsm;   // 2048 threads per SM
    float best = 0.f;
    for (int r = 0; r <= reps && err == cudaSuccess; ++r) {   // launch 0: warm-up
        cudaEventRecord(e0, st);
        k_fma_probe<<<blocks, 256, 0, st>>>(0.999f, 1e-3f, 0);
        cudaEventRecord(e1, st);
        err = cudaEventSynchronize(e1);
        if (err == cudaSuccess) err = cudaGetLastError();
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err == cudaSuccess && r > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    if (err != cudaSuccess) return cuda_fail(err, "fa_fp32_issue_rate");
    *ms_out = best;
    *rate = (double)blocks * 256.0 * 8.0 * (double)kFmaIters / (best * 1e-3);
    return FA_OK;
}

int fa_device_bytes(const fa_ctx* c, unsigned long long* field_bytes, unsigned long long* scalar_bytes) {
    if (!c || !field_bytes || !scalar_bytes) return FA_EINVAL;
    // lattice-sized buffers: links, spinors, stores, staging, reduction partials
    const fa::DevBuf* field[] = {&c->links64, &c->links32, &c->linksdf, &c->io64a, &c->io64b, &c->io32a,
                                 &c->io32b, &c->tmp64, &c->tmp32, &c->partials, &c->r64, &c->u64, &c->rt64,
                                 &c->r32, &c->u32, &c->rt32, &c->y64, &c->xs64, &c->us64, &c->bhost_dev,
                                 &c->yhost_dev, &c->gx, &c->gpart, &c->store64, &c->store32, &c->snap64,
                                 &c->snap32, &c->xrel, &c->brel, &c->snapx, &c->defl, &c->eig};
    // scalars: solver state, shifts, records, pass-2 weights, batch descriptors
    const fa::DevBuf* scal[] = {&c->state, &c->shiftbuf, &c->rec, &c->prec, &c->coef, &c->cs, &c->coef4,
                                &c->descbuf, &c->flagbuf};
    unsigned long long f = 0, s = 0;
    for (const fa::DevBuf* b : field) f += b->bytes;
    for (const fa::DevBuf* b : scal) s += b->bytes;
    *field_bytes = f;
    *scalar_bytes = s;
    return FA_OK;
}

int fa_hop_timing_split(const fa_ctx* c, int precision, int with_dot, double* mean_ms, long long* count) {
    if (!c || !mean_ms || !count || (precision != FA_F64 && precision != FA_F32 && precision != FA_DF) ||
        with_dot < -1 || with_dot > 2 || (with_dot == 2 && precision != FA_F32))
        return FA_EINVAL;
    const int k = precision == FA_F64 ? 0 : (precision == FA_F32 ? 1 : 2);
    double ms = 0.0;
    long long n = 0;
    // index of each selector: plain k, with the inner product k + 3, FP32 Gram sweep 6
    for (int d = 0; d < 3; ++d) {
        if (with_dot >= 0 && d != with_dot) continue;
        if (d == 2 && precision != FA_F32) continue;
        const int idx = d == 2 ? 6 : k + 3 * d;
        ms += c->hop_ms[idx];
        n += c->hop_count[idx];
    }
    *count = n;
    *mean_ms = n ? ms / (double)n : 0.0;
    return FA_OK;
}

int fa_hop_timing(const fa_ctx* c, int precision, double* mean_ms, long long* count) {
    return fa_hop_timing_split(c, precision, -1, mean_ms, count);
}

int fa_hop_timing_reset(fa_ctx* c) {
    if (!c) return FA_EINVAL;
    for (int k = 0; k < 7; ++k) {
        c->hop_ms[k] = 0.0;
        c->hop_count[k] = 0;
    }
    return FA_OK;
}

int fa_set_hop_shape(fa_ctx* c, int shape) {
    if (!c || shape < FA_SHAPE_AUTO || shape > FA_SHAPE_NARROW) {
        set_error("fa_set_hop_shape: unknown shape %d", shape);
        return FA_EINVAL;
    }
    c->hop_shape = shape;
    return FA_OK;
}

int fa_get_hop_shape(const fa_ctx* c) { return c ? c->hop_shape : FA_EINVAL; }

// Time each FP32 sweep launch shape on the context's lattice: chains of sweeps
// g5 D_w(mu) that read the previous sweep's output (as in a solve), `reps`
// launches between two CUDA events on the context's stream, three rounds with
// the shapes interleaved, the best round per shape.  The automatic choice is
// kept unless the other shape is faster by more than 3 % (single-launch timings
// of the two shapes are close; inside a solve the automatic choice measured
// better).
int fa_autotune(fa_ctx* c, int reps, double* times_ms) {
    if (!c || reps < 1 || !times_ms) return FA_EINVAL;
    if (!c->have_gauge || !c->have_params) return FA_ESTATE;
    const int V = c->g.V;
    const size_t b = (size_t)6 * V * sizeof(float4);
    CUDA_OR(c->io32a.ensure(b), "fa_autotune: alloc");
    CUDA_OR(c->io32b.ensure(b), "fa_autotune: alloc");
    CUDA_OR(cudaMemsetAsync(c->io32a.p, 0, b, c->stream), "fa_autotune: clear");
    CUDA_OR(cudaMemsetAsync(c->io32b.p, 0, b, c->stream), "fa_autotune: clear");
    float4* buf[2] = {c->io32a.as<float4>(), c->io32b.as<float4>()};
    const int saved = c->hop_shape;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_OR(cudaEventCreate(&e0), "fa_autotune: event");
    CUDA_OR(cudaEventCreate(&e1), "fa_autotune: event");
    double best_ms[2] = {1e30, 1e30};
    int rc = FA_OK;
    const bool saved_timing = c->hop_timing;
    c->hop_timing = false;
    auto chain = [&](int n) {
        for (int k = 0; k < n && rc == FA_OK; ++k)
            rc = hop_f32(c, buf[k & 1], buf[(k + 1) & 1], 1.0, false, true, false, nullptr, nullptr, nullptr);
    };
    // The solver replays its outer iterations from CUDA graphs, so the chains are
    // timed the same way where the stream can be captured (not the legacy or
    // per-thread default stream); else as direct launches.
    const bool capturable = c->stream != nullptr && c->stream != cudaStreamLegacy && c->stream != cudaStreamPerThread;
    cudaGraphExec_t ge[2] = {nullptr, nullptr};
    for (int shape = FA_SHAPE_WIDE; capturable && shape <= FA_SHAPE_NARROW && rc == FA_OK; ++shape) {
        c->hop_shape = shape;
        cudaGraph_t gr = nullptr;
        if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "fa_autotune: begin capture");
            break;
        }
        chain(reps);
        const cudaError_t ee = cudaStreamEndCapture(c->stream, &gr);
        if (rc == FA_OK && ee != cudaSuccess) rc = cuda_fail(ee, "fa_autotune: end capture");
        if (rc == FA_OK) {
            const cudaError_t ei = cudaGraphInstantiate(&ge[shape - 1], gr, 0);
            if (ei != cudaSuccess) rc = cuda_fail(ei, "fa_autotune: instantiate");
        }
        if (gr) cudaGraphDestroy(gr);
    }
    for (int round = 0; round < 3 && rc == FA_OK; ++round) {
        for (int shape = FA_SHAPE_WIDE; shape <= FA_SHAPE_NARROW && rc == FA_OK; ++shape) {
            c->hop_shape = shape;
            cudaGraphExec_t x = ge[shape - 1];
            if (x) {
                if (round == 0) cudaGraphLaunch(x, c->stream);   // first replay uploads the graph
                cudaEventRecord(e0, c->stream);
                cudaGraphLaunch(x, c->stream);
                cudaEventRecord(e1, c->stream);
                const cudaError_t el = cudaGetLastError();
                if (el != cudaSuccess) { rc = cuda_fail(el, "fa_autotune: graph launch"); break; }
            } else {
                chain(3);
                cudaEventRecord(e0, c->stream);
                chain(reps);
                cudaEventRecord(e1, c->stream);
                if (rc != FA_OK) break;
            }
            if (cudaEventSynchronize(e1) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "fa_autotune: timing"); break; }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            best_ms[shape - 1] = std::min(best_ms[shape - 1], (double)ms / reps);
        }
    }
    for (auto x : ge)
        if (x) cudaGraphExecDestroy(x);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->hop_timing = saved_timing;
    if (rc != FA_OK) {
        c->hop_shape = saved;
        return rc;
    }
    times_ms[0] = best_ms[0];
    times_ms[1] = best_ms[1];
    const int deflt = hop_narrow(V) ? FA_SHAPE_NARROW : FA_SHAPE_WIDE, other = 3 - deflt;
    c->hop_shape = best_ms[other - 1] < 0.97 * best_ms[deflt - 1] ? other : deflt;
    return c->hop_shape;
}

}  // extern "C"
