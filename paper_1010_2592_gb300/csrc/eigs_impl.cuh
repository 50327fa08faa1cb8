// Eigenpairs of H = gamma_5 D_w(mu) smallest in magnitude, with left and right
// eigenvectors: the deflation subspace of the sign function (Sec. 3 and the
// captions of Figs. 3, 4: the eigenvalues of gamma_5 D_w smallest in magnitude
// are treated exactly).
//
// Krylov-Schur iteration (Stewart's restarted Arnoldi with a Schur-form
// restart) on the shift-and-invert operator T = H^{-1} = c H A^{-1}: its
// largest eigenvalues in magnitude are the inverses of the wanted ones.  Each
// application of T is one solve of the library (A^{-1} v: the multi-shift
// solver with the single pole omega = 1, sigma = 0) and one FP64 D_w sweep.
// Left eigenvectors of H are right eigenvectors of H^H = gamma_5 D_w(-mu) =
// H(-mu) for the conjugate eigenvalues, found by the same iteration at -mu and
// paired with the right ones, then scaled so that l_i^H r_j = delta_ij.
//
// The basis vectors are canonical device spinors; Gram-Schmidt runs on the
// device (k_dots_canon, k_lincomb_canon, twice per step), the small dense
// problem (Hessenberg reduction, shifted QR to Schur form, reordering) on the
// host in FP64 complex arithmetic.
// (Included by solver.cu: it uses that file's solve(), FP64 sweep and
// canonical-spinor kernels k_dots_canon / k_lincomb_canon.)
#pragma once

#include <complex>

namespace fa {

#define FA_TRY_E(x)                    \
    do {                               \
        int _rc = (x);                 \
        if (_rc != FA_OK) return _rc;  \
    } while (0)
#define FA_CUDA_E(x, what)                                   \
    do {                                                     \
        cudaError_t _e = (x);                                \
        if (_e != cudaSuccess) return cuda_fail(_e, what);   \
    } while (0)

namespace {

using zc = std::complex<double>;

// ------------------------------------------------------------------ small dense complex linear algebra
// column-major n x n matrices, a(i, j) = a[i + n j]
struct Mat {
    int n = 0;
    std::vector<zc> a;
    explicit Mat(int n_ = 0) : n(n_), a((size_t)n_ * n_) {}
    zc& operator()(int i, int j) { return a[i + (size_t)n * j]; }
    zc operator()(int i, int j) const { return a[i + (size_t)n * j]; }
    static Mat eye(int n) {
        Mat m(n);
        for (int i = 0; i < n; ++i) m(i, i) = 1.0;
        return m;
    }
};

// Givens rotation [c s; -conj(s) c] (c real) with  G [x; y] = [r; 0]
struct Givens {
    double c;
    zc s;
};
Givens givens(zc x, zc y) {
    const double ax = std::abs(x), ay = std::abs(y);
    if (ay == 0.0) return {1.0, 0.0};
    if (ax == 0.0) return {0.0, std::conj(y) / ay};
    const double nrm = std::hypot(ax, ay);
    const zc ph = x / ax;
    return {ax / nrm, ph * std::conj(y) / nrm};
}
// rows p, q of A (columns lo..hi-1):  [Ap; Aq] <- G [Ap; Aq]
void rot_rows(Mat& A, int p, int q, const Givens& g, int lo, int hi) {
    for (int j = lo; j < hi; ++j) {
        const zc x = A(p, j), y = A(q, j);
        A(p, j) = g.c * x + g.s * y;
        A(q, j) = -std::conj(g.s) * x + g.c * y;
    }
}
// columns p, q of A (rows lo..hi-1):  [Ap Aq] <- [Ap Aq] G^H
void rot_cols(Mat& A, int p, int q, const Givens& g, int lo, int hi) {
    for (int i = lo; i < hi; ++i) {
        const zc x = A(i, p), y = A(i, q);
        A(i, p) = g.c * x + std::conj(g.s) * y;
        A(i, q) = -g.s * x + g.c * y;
    }
}

// A <- Q^H A Q upper Hessenberg by Givens rotations, Q accumulated (Q <- Q G^H)
void hessenberg(Mat& A, Mat& Q) {
    const int n = A.n;
    for (int j = 0; j + 2 < n; ++j)
        for (int i = n - 1; i > j + 1; --i) {
            const Givens g = givens(A(i - 1, j), A(i, j));
            rot_rows(A, i - 1, i, g, 0, n);
            rot_cols(A, i - 1, i, g, 0, n);
            rot_cols(Q, i - 1, i, g, 0, n);
            A(i, j) = 0.0;
        }
}

// Hessenberg A -> upper triangular Schur form T = Q^H A Q by single-shift QR
// sweeps with Wilkinson shifts and deflation; false if it does not converge
bool schur(Mat& A, Mat& Q) {
    const int n = A.n;
    int hi = n - 1, iter = 0;
    while (hi > 0) {
        if (++iter > 200 * n) return false;
        // deflate at the smallest negligible subdiagonal entry
        int lo = hi;
        while (lo > 0) {
            const double s = std::abs(A(lo - 1, lo - 1)) + std::abs(A(lo, lo));
            if (std::abs(A(lo, lo - 1)) <= 1e-15 * (s > 0.0 ? s : 1.0)) {
                A(lo, lo - 1) = 0.0;
                break;
            }
            --lo;
        }
        if (lo == hi) {
            --hi;
            iter = 0;
            continue;
        }
        // Wilkinson shift from the trailing 2 x 2 block
        const zc a = A(hi - 1, hi - 1), b = A(hi - 1, hi), c = A(hi, hi - 1), d = A(hi, hi);
        const zc tr = a + d, det = a * d - b * c;
        const zc disc = std::sqrt(tr * tr - 4.0 * det);
        const zc l1 = 0.5 * (tr + disc), l2 = 0.5 * (tr - disc);
        zc mu = std::abs(l1 - d) < std::abs(l2 - d) ? l1 : l2;
        if (iter % 11 == 10) mu = d + std::abs(A(hi, hi - 1));   // exceptional shift
        // implicit single-shift QR sweep on rows/cols lo..hi (bulge chase)
        zc x = A(lo, lo) - mu, y = A(lo + 1, lo);
        for (int k = lo; k < hi; ++k) {
            const Givens g = givens(x, y);
            rot_rows(A, k, k + 1, g, k > lo ? k - 1 : lo, n);
            rot_cols(A, k, k + 1, g, 0, std::min(k + 3, hi + 1));
            rot_cols(Q, k, k + 1, g, 0, n);
            if (k > lo) A(k + 1, k - 1) = 0.0;
            if (k + 1 < hi) {
                x = A(k + 1, k);
                y = A(k + 2, k);
            }
        }
    }
    for (int j = 0; j < n; ++j)
        for (int i = j + 1; i < n; ++i) A(i, j) = 0.0;
    return true;
}

// swap the adjacent diagonal entries p, p+1 of the upper triangular T (Q updated)
void swap_schur(Mat& T, Mat& Q, int p) {
    const int n = T.n;
    const zc a = T(p, p), b = T(p, p + 1), c = T(p + 1, p + 1);
    // x = [b, c - a] spans the eigenvector of c within the 2 x 2 block
    const Givens g = givens(b, c - a);
    rot_rows(T, p, p + 1, g, 0, n);
    rot_cols(T, p, p + 1, g, 0, n);
    rot_cols(Q, p, p + 1, g, 0, n);
    T(p + 1, p) = 0.0;
}

// eigenvector of the upper triangular T for its diagonal entry j (back substitution)
std::vector<zc> tri_eigvec(const Mat& T, int j) {
    std::vector<zc> x(T.n, 0.0);
    x[j] = 1.0;
    const zc lam = T(j, j);
    const double scale = std::max(std::abs(lam), 1e-300);
    for (int i = j - 1; i >= 0; --i) {
        zc s = 0.0;
        for (int k = i + 1; k <= j; ++k) s += T(i, k) * x[k];
        zc den = T(i, i) - lam;
        if (std::abs(den) < 1e-14 * scale) den = 1e-14 * scale;
        x[i] = -s / den;
    }
    return x;
}

// ------------------------------------------------------------------ device helpers
struct Dev {
    fa_ctx* c;
    int n;          // complex entries of a spinor (12 V)
    int nb;         // blocks of the reductions
    double2* part;  // partials
    std::vector<double2> hp;
};

// out[i] = V_i^H b for i < k (V: k spinors, contiguous), summed on the host in a fixed order
int dots(Dev& D, const double2* V, int k, const double2* b, std::vector<zc>& out) {
    cudaStream_t st = D.c->stream;
    k_dots_canon<<<dim3(D.nb, k), kThreads, 0, st>>>(D.n, V, b, D.part);
    D.c->launches++;
    D.hp.resize((size_t)k * D.nb);
    cudaError_t e = cudaMemcpyAsync(D.hp.data(), D.part, D.hp.size() * sizeof(double2), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "eigensolver: inner products");
    out.assign(k, 0.0);
    for (int i = 0; i < k; ++i) {
        double re = 0.0, im = 0.0;
        for (int j = 0; j < D.nb; ++j) {
            re += D.hp[(size_t)i * D.nb + j].x;
            im += D.hp[(size_t)i * D.nb + j].y;
        }
        out[i] = zc(re, im);
    }
    return FA_OK;
}

// out = base + sum_i coef_i V_i (coef on the host, staged through the device)
int lincomb(Dev& D, const double2* V, int k, const std::vector<zc>& coef, const double2* base, double2* out,
            double2* coef_dev) {
    cudaStream_t st = D.c->stream;
    std::vector<double2> h(k);
    for (int i = 0; i < k; ++i) h[i] = make_double2(coef[i].real(), coef[i].imag());
    cudaError_t e = cudaMemcpyAsync(coef_dev, h.data(), k * sizeof(double2), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // h is a local
    if (e != cudaSuccess) return cuda_fail(e, "eigensolver: coefficients");
    k_lincomb_canon<<<D.nb, kThreads, 0, st>>>(D.n, k, coef_dev, V, base, out, 0);
    D.c->launches++;
    return launch_status("eigensolver: linear combination");
}

}  // namespace

static int ok_alloc(fa_ctx* c, size_t sb);

// w = T v = c H A^{-1} v at chemical potential `mu` (canonical spinors); y is scratch
static int apply_T(fa_ctx* c, double mu, const double* v, double* w, double* y, const fa_solver_params* ps) {
    const double mu0 = c->mu;
    c->mu = mu;
    fa_solver_stats st{};
    int rc = solve(c, v, y, nullptr, ps, &st);   // A^{-1} v (poles: omega = 1, sigma = 0)
    if (rc == FA_OK) {
        const size_t sb = (size_t)12 * c->g.V * sizeof(double2);
        rc = ok_alloc(c, sb);
        if (rc == FA_OK) rc = launch_pack_spinor_f64(c->g, y, c->io64a.as<double2>(), c->stream);
        if (rc == FA_OK)
            rc = hop_f64(c, c->io64a.as<double2>(), c->io64b.as<double2>(), c->scale_c, false, true, false, nullptr,
                         nullptr, nullptr);
        if (rc == FA_OK) rc = launch_unpack_spinor_f64(c->g, c->io64b.as<double2>(), w, c->stream);
    }
    c->mu = mu0;
    return rc;
}

static int ok_alloc(fa_ctx* c, size_t sb) {
    cudaError_t e = c->io64a.ensure(sb);
    if (e == cudaSuccess) e = c->io64b.ensure(sb);
    return e == cudaSuccess ? FA_OK : cuda_fail(e, "alloc");
}

// Krylov-Schur on T at chemical potential mu: the k eigenvalues of T largest in
// magnitude (theta) and their Ritz vectors (X: k canonical spinors)
static int krylov_schur(fa_ctx* c, double mu, int k, int m, double tol, int max_restarts,
                        const fa_solver_params* ps, unsigned long long seed, std::vector<zc>& theta, double2* X,
                        int* nconv, int* nsolve) {
    const int V = c->g.V;
    const int n = 12 * V;
    const size_t sb = (size_t)n * sizeof(double2);
    Dev D{c, n, std::min((n + kThreads - 1) / kThreads, 4 * std::max(1, sm_count())), nullptr, {}};
    // device memory: basis (m + 1), w, y, new basis (k), partials, coefficients
    FA_CUDA_E(c->eig.ensure((size_t)(m + 1 + 2 + k) * sb + (size_t)(m + 2) * D.nb * sizeof(double2) +
                            (size_t)(m + 2) * sizeof(double2)),
              "eigensolver: alloc");
    double2* Vb = c->eig.as<double2>();
    double2* w = Vb + (size_t)(m + 1) * n;
    double2* y = w + n;
    double2* Vn = y + n;
    D.part = Vn + (size_t)k * n;
    double2* coef_dev = D.part + (size_t)(m + 2) * D.nb;
    cudaStream_t st = c->stream;
    // start vector: complex Gaussian from a counter-based generator (splitmix64 + Box-Muller)
    {
        std::vector<double2> h(n);
        unsigned long long s = seed;
        auto next = [&]() {
            s += 0x9E3779B97F4A7C15ULL;
            unsigned long long z = s;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
            z ^= z >> 31;
            return ((z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        };
        for (int i = 0; i < n; ++i) {
            const double r = std::sqrt(-2.0 * std::log(next())), a = 6.283185307179586 * next();
            h[i] = make_double2(r * std::cos(a), r * std::sin(a));
        }
        FA_CUDA_E(cudaMemcpyAsync(Vb, h.data(), sb, cudaMemcpyHostToDevice, st), "eigensolver: start vector");
        FA_CUDA_E(cudaStreamSynchronize(st), "eigensolver: sync");
    }
    std::vector<zc> hv;
    FA_TRY_E(dots(D, Vb, 1, Vb, hv));
    FA_TRY_E(lincomb(D, Vb, 1, {zc(1.0 / std::sqrt(hv[0].real()) - 1.0)}, Vb, Vb, coef_dev));
    // (m + 1) x m projected matrix, column-major with leading dimension m + 1
    std::vector<zc> Hb((size_t)(m + 1) * m, 0.0);
    auto H = [&](int i, int j) -> zc& { return Hb[i + (size_t)(m + 1) * j]; };
    int p = 0;   // basis vectors kept from the last restart
    *nsolve = 0;
    for (int restart = 0; restart <= max_restarts; ++restart) {
        // Arnoldi expansion from column p to m - 1
        for (int j = p; j < m; ++j) {
            double2* vj = Vb + (size_t)j * n;
            FA_TRY_E(apply_T(c, mu, reinterpret_cast<double*>(vj), reinterpret_cast<double*>(w),
                             reinterpret_cast<double*>(y), ps));
            ++*nsolve;
            std::vector<zc> h(j + 1, 0.0);
            for (int pass = 0; pass < 2; ++pass) {   // classical Gram-Schmidt, twice
                std::vector<zc> g;
                FA_TRY_E(dots(D, Vb, j + 1, w, g));
                std::vector<zc> neg(j + 1);
                for (int i = 0; i <= j; ++i) {
                    h[i] += g[i];
                    neg[i] = -g[i];
                }
                FA_TRY_E(lincomb(D, Vb, j + 1, neg, w, w, coef_dev));
            }
            std::vector<zc> nn;
            FA_TRY_E(dots(D, w, 1, w, nn));
            const double beta = std::sqrt(std::max(nn[0].real(), 0.0));
            for (int i = 0; i <= j; ++i) H(i, j) = h[i];
            H(j + 1, j) = beta;
            if (!(beta > 0.0) || !std::isfinite(beta)) {
                set_error("eigensolver: Krylov space exhausted or non-finite at step %d", j);
                return FA_EBREAKDOWN;
            }
            FA_TRY_E(lincomb(D, w, 1, {zc(1.0 / beta)}, nullptr, Vb + (size_t)(j + 1) * n, coef_dev));
        }
        // Schur form of the m x m projected matrix, wanted (largest |theta|) first
        Mat S(m), Q = Mat::eye(m);
        for (int j = 0; j < m; ++j)
            for (int i = 0; i < m; ++i) S(i, j) = H(i, j);
        hessenberg(S, Q);
        if (!schur(S, Q)) {
            set_error("eigensolver: QR iteration of the projected matrix did not converge");
            return FA_ENOCONV;
        }
        for (int sel = 0; sel < k; ++sel) {   // selection sort by bubbling with swaps
            int best = sel;
            for (int i = sel + 1; i < m; ++i)
                if (std::abs(S(i, i)) > std::abs(S(best, best))) best = i;
            for (int i = best - 1; i >= sel; --i) swap_schur(S, Q, i);
        }
        // residual row b^T = (row m of Hb) Q; Ritz residuals of the k wanted
        std::vector<zc> b(m, 0.0);
        for (int j = 0; j < m; ++j)
            for (int i = 0; i < m; ++i) b[j] += H(m, i) * Q(i, j);
        int conv = 0;
        theta.assign(k, 0.0);
        std::vector<std::vector<zc>> Y(k);
        for (int i = 0; i < k; ++i) {
            Y[i] = tri_eigvec(S, i);
            zc r = 0.0;
            double ny = 0.0;
            for (int j = 0; j <= i; ++j) {
                r += b[j] * Y[i][j];
                ny += std::norm(Y[i][j]);
            }
            theta[i] = S(i, i);
            if (std::abs(r) <= tol * std::abs(theta[i]) * std::sqrt(ny)) ++conv;
        }
        *nconv = conv;
        const bool done = conv == k || restart == max_restarts;
        if (done) {
            // Ritz vectors x_i = V_m Q Y_i, normalised
            for (int i = 0; i < k; ++i) {
                std::vector<zc> cf(m, 0.0);
                for (int j = 0; j < m; ++j)
                    for (int l = 0; l <= i; ++l) cf[j] += Q(j, l) * Y[i][l];
                FA_TRY_E(lincomb(D, Vb, m, cf, nullptr, X + (size_t)i * n, coef_dev));
                std::vector<zc> nr;
                FA_TRY_E(dots(D, X + (size_t)i * n, 1, X + (size_t)i * n, nr));
                FA_TRY_E(lincomb(D, X + (size_t)i * n, 1, {zc(1.0 / std::sqrt(nr[0].real()) - 1.0)},
                                 X + (size_t)i * n, X + (size_t)i * n, coef_dev));
            }
            return conv == k ? FA_OK : FA_ENOCONV;
        }
        // restart: keep the k wanted Schur vectors, then the residual vector
        for (int i = 0; i < k; ++i) {
            std::vector<zc> cf(m);
            for (int j = 0; j < m; ++j) cf[j] = Q(j, i);
            FA_TRY_E(lincomb(D, Vb, m, cf, nullptr, Vn + (size_t)i * n, coef_dev));
        }
        FA_CUDA_E(cudaMemcpyAsync(Vb, Vn, (size_t)k * sb, cudaMemcpyDeviceToDevice, st), "eigensolver: restart");
        FA_CUDA_E(cudaMemcpyAsync(Vb + (size_t)k * n, Vb + (size_t)m * n, sb, cudaMemcpyDeviceToDevice, st),
                  "eigensolver: restart");
        std::fill(Hb.begin(), Hb.end(), zc(0.0));
        for (int j = 0; j < k; ++j) {
            for (int i = 0; i < k; ++i) H(i, j) = S(i, j);
            H(k, j) = b[j];
        }
        p = k;
    }
    return FA_ENOCONV;
}

int eigs_smallest(fa_ctx* c, int k, int m, double tol, int max_restarts, const fa_solver_params* p,
                  unsigned long long seed, double* lambda, double* R, double* Lv, int* nconv, int* nsolve) {
    if (!c->have_gauge || !c->have_params) return FA_ESTATE;
    const int V = c->g.V, n = 12 * V;
    if (k < 1 || m < k + 2 || m > 512 || m > n || !(tol > 0.0) || max_restarts < 0) return FA_EINVAL;
    // the inner solves: one pole omega = 1 at sigma = 0 (A^{-1}); the context's
    // own poles are restored afterwards
    const int ns0 = c->ns;
    const bool hp0 = c->have_poles;
    std::vector<double> om0(c->omega, c->omega + kMaxShifts), sg0(c->sigma, c->sigma + kMaxShifts);
    c->ns = 1;
    c->omega[0] = 1.0;
    c->sigma[0] = 0.0;
    c->have_poles = true;
    fa_solver_params ps = *p;
    if (ps.mode == FA_SINGLE) ps.mode = FA_DOUBLE;
    std::vector<zc> th_r, th_l;
    double2* Rd = reinterpret_cast<double2*>(R);
    double2* Ld = reinterpret_cast<double2*>(Lv);
    int nc_r = 0, nc_l = 0, ns_r = 0, ns_l = 0;
    int rc = krylov_schur(c, c->mu, k, m, tol, max_restarts, &ps, seed, th_r, Rd, &nc_r, &ns_r);
    for (int i = 0; i < (int)th_r.size() && i < k; ++i) {   // the current Ritz values, also without convergence
        const zc lam = 1.0 / th_r[i];
        lambda[2 * i] = lam.real();
        lambda[2 * i + 1] = lam.imag();
    }
    if (rc == FA_OK || rc == FA_ENOCONV) {
        const int rc2 = krylov_schur(c, -c->mu, k, m, tol, max_restarts, &ps, seed + 1, th_l, Ld, &nc_l, &ns_l);
        if (rc == FA_OK) rc = rc2;
    }
    c->ns = ns0;
    c->have_poles = hp0;
    std::copy(om0.begin(), om0.end(), c->omega);
    std::copy(sg0.begin(), sg0.end(), c->sigma);
    *nconv = std::min(nc_r, nc_l);
    *nsolve = ns_r + ns_l;
    if (rc != FA_OK) return rc;
    // pair each right eigenvalue lambda_i = 1/theta_i with the left one of
    // eigenvalue conj(lambda_i), and scale l_i so that l_i^H r_i = 1
    std::vector<int> perm(k, -1), used(k, 0);
    for (int i = 0; i < k; ++i) {
        const zc lr = 1.0 / th_r[i];
        int best = -1;
        double bd = 0.0;
        for (int j = 0; j < k; ++j) {
            if (used[j]) continue;
            const double dd = std::abs(std::conj(1.0 / th_l[j]) - lr);
            if (best < 0 || dd < bd) best = j, bd = dd;
        }
        if (best < 0 || bd > 1e-6 * std::abs(lr) + 1e-12) {
            set_error("eigensolver: no left eigenvalue matches the right eigenvalue %g%+gi", lr.real(), lr.imag());
            return FA_ENOCONV;
        }
        used[best] = 1;
        perm[i] = best;
    }
    Dev D{c, n, std::min((n + kThreads - 1) / kThreads, 4 * std::max(1, sm_count())), nullptr, {}};
    const size_t sb = (size_t)n * sizeof(double2);
    double2* Vb = c->eig.as<double2>();   // reuse the basis storage as scratch
    D.part = Vb + (size_t)(k + 1) * n;
    double2* coef_dev = D.part + (size_t)(k + 2) * D.nb;
    cudaStream_t st = c->stream;
    FA_CUDA_E(cudaMemcpyAsync(Vb, Ld, (size_t)k * sb, cudaMemcpyDeviceToDevice, st), "eigensolver: pairing");
    for (int i = 0; i < k; ++i) {
        double2* li = Vb + (size_t)perm[i] * n;
        std::vector<zc> d;
        FA_TRY_E(dots(D, li, 1, Rd + (size_t)i * n, d));   // l^H r
        if (!(std::abs(d[0]) > 1e-14)) {
            set_error("eigensolver: left and right eigenvectors %d nearly orthogonal", i);
            return FA_EBREAKDOWN;
        }
        // l <- l / conj(l^H r): then l^H r = 1
        FA_TRY_E(lincomb(D, li, 1, {1.0 / std::conj(d[0])}, nullptr, Ld + (size_t)i * n, coef_dev));
        const zc lam = 1.0 / th_r[i];
        lambda[2 * i] = lam.real();
        lambda[2 * i + 1] = lam.imag();
    }
    FA_CUDA_E(cudaStreamSynchronize(st), "eigensolver: sync");
    return FA_OK;
}

#undef FA_TRY_E
#undef FA_CUDA_E

}  // namespace fa
