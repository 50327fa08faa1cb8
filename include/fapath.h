/*
 * fapath — f(A) b by multi-shift BiCGstab(l), single-pass and double-pass,
 * on one NVIDIA GB300 (sm_103a).
 *
 * What is computed (Heybrock, "Double-pass variants for multi-shift
 * BiCGstab(l)", Lattice 2010):
 *
 *     y = f(A) b ~= sum_{s=1}^{Ns} omega_s (A + sigma_s)^{-1} b      (Eq. 1)
 *     A = c (gamma_5 D_w(mu))^2                                      (Sec. 1)
 *
 * D_w(mu) is the Wilson-Dirac operator with chemical potential (named in
 * Sec. 1, Eq. for D_ov; the definition used here is the standard mass form)
 *
 *   (D psi)(x) = (4+m) psi(x) - 1/2 sum_nu [ f+ (1-g_nu) U_nu(x) psi(x+nu)
 *                                          + f- (1+g_nu) U_nu(x-nu)^H psi(x-nu) ]
 *
 * with f+- = e^{+-mu} on time hops, 1 on spatial hops, times t_bc on hops that
 * cross the time boundary; gamma matrices in the DeGrand-Rossi basis,
 * gamma_5 = diag(1, 1, -1, -1).
 *
 * Canonical layouts (the only layouts that cross this boundary), C order,
 * interleaved complex128 (re, im):
 *   spinor  [T][Z][Y][X][spin 4][colour 3]             24 doubles per site
 *   gauge   [T][Z][Y][X][mu 4][row 3][col 3]           72 doubles per site
 *           mu = 0,1,2,3 <-> x,y,z,t; U_mu(x) links x to x + mu_hat.
 * Spinor arguments are DEVICE pointers unless the name says host.  The caller
 * owns them; the context owns its packed copies of the gauge field and all
 * work space.  Vectors must not alias unless stated.
 *
 * Errors: every call returns an fa_status (0 = FA_OK).  No call aborts or
 * throws.  A failed CUDA call returns FA_ECUDA and leaves a message for
 * fa_last_error().  Calls on one context are stream-ordered on the stream
 * given to fa_create(); they are not thread-safe on a shared context.
 */
#ifndef FAPATH_H
#define FAPATH_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fa_ctx fa_ctx;

typedef enum {
    FA_OK = 0,
    FA_EINVAL = -1,       /* bad argument (null pointer, size, range)          */
    FA_ENOMEM = -2,       /* device or host allocation failed                  */
    FA_ECUDA = -3,        /* a CUDA runtime call failed; see fa_last_error()   */
    FA_EBREAKDOWN = -4,   /* a Krylov denominator vanished                      */
    FA_ENOCONV = -5,      /* not all shifts converged within max_outer         */
    FA_ENONFINITE = -6,   /* a recurrence scalar became NaN or Inf             */
    FA_ETIMEOUT = -7,     /* a bounded device wait expired                      */
    FA_ESTATE = -8        /* call out of order (no gauge field, no poles, ...) */
} fa_status;

typedef enum { FA_SINGLE = 0, FA_DOUBLE = 1 } fa_mode;

typedef enum {
    FA_F64 = 0,           /* FP64 spinors, FP64 18-real links, FP64 scalars          */
    FA_F32 = 1,           /* FP32 spinors, FP32 12-real links, FP64 scalars/reductions */
    FA_MIXED = 2          /* FP64 head until every live shift residual is below
                             switch_resid |b|, then FP32 bulk (double-pass only)     */
} fa_precision;

typedef struct {
    int ell;              /* BiCGstab(l) degree, 1..8                                  */
    double tol;           /* per shift: stop when |r_0| / |zeta_s| <= tol |b|          */
    int max_outer;        /* outer-iteration cap (also sizes the scalar record)        */
    int mode;             /* fa_mode                                                   */
    int precision;        /* fa_precision                                              */
    double switch_resid;  /* FA_MIXED: head/tail switch threshold; <= 0: 0.04/l^2      */
    int flags;            /* bit 0: time the passes with CUDA events                   */
} fa_solver_params;

typedef struct {
    int status;               /* fa_status of the solve                              */
    int outer_iters;          /* M: outer iterations of pass 1                        */
    int switch_outer;         /* FA_MIXED: first FP32 outer iteration, else -1        */
    int ns;                   /* number of shifts                                     */
    int iters_per_shift[64];  /* M_s: outer iterations until shift s froze            */
    double resid_recurrence;  /* |r_0| / |b| of the seed at the end of pass 1         */
    long long n_mv;           /* matrix-vector products A v (both passes)             */
    long long n_dot;          /* global inner products                                */
    long long n_launch;       /* kernel launches of the solve                         */
    double t_pass1_ms, t_sweep_ms, t_pass2_ms;   /* with flags bit 0, else 0          */
} fa_solver_stats;

/* Create a context for an X*Y*Z*T lattice (each extent >= 2, V = XYZT <=
 * 2^26 sites) whose work runs on `cuda_stream` (a cudaStream_t; NULL = the
 * legacy default stream) of the current device.  *out receives the handle. */
int fa_create(fa_ctx** out, const int dims[4], void* cuda_stream);

/* Release all device memory of the context.  NULL is accepted. */
int fa_destroy(fa_ctx* ctx);

/* Load the gauge field (canonical complex128 layout above) from host memory
 * (on_device = 0) or device memory (on_device = 1).  Packs FP64 18-real links
 * and FP32 12-real links (rows 1-2; row 3 = conj(row1 x row2) is rebuilt in
 * registers, exact for SU(3)).  The boundary sign and e^{+-mu} are kept as
 * separate scalars, never folded into the links. */
int fa_set_gauge(fa_ctx* ctx, const double* U, int on_device);

/* Wilson mass m (diagonal 4+m), chemical potential mu, time-boundary sign
 * t_bc (+1 periodic, -1 antiperiodic) and the scale c of A = c (g5 D)^2. */
int fa_set_params(fa_ctx* ctx, double wilson_mass, double mu, int t_bc, double scale_c);

/* Power iteration for the scale (workload recipe): v = v0/|v0|, then `iters`
 * times v <- A1 v/|A1 v| with A1 = (g5 D)^2 (c = 1), lambda = |A1 v|;
 * *scale_out = 1/lambda.  v0 is a device spinor (canonical), not modified.
 * FP64 throughout.  Does not change the context's c. */
int fa_estimate_scale(fa_ctx* ctx, const double* v0, int iters, double* scale_out);

/* Poles {omega_s, sigma_s} of Eq. (1), 1 <= ns <= 64, sigma_s > 0 (host arrays). */
int fa_set_poles(fa_ctx* ctx, int ns, const double* omega, const double* sigma);

/* Neuberger's poles (captions of Figs. 1, 3): theta_s = pi (s - 1/2)/(2 ns),
 * omega_s = (1/ns)/cos^2 theta_s, sigma_s = tan^2 theta_s (host arrays). */
int fa_neuberger_poles(int ns, double* omega, double* sigma);

/* out = D_w(mu) in (dagger = 0) or D_w(mu)^H in (dagger = 1), canonical
 * complex128 device spinors, computed in `precision` (FA_F64 or FA_F32; FP32
 * rounds in and out through the packed FP32 layout).  in != out. */
int fa_apply_dw(fa_ctx* ctx, const double* in, double* out, int dagger, int precision);

/* out = A in (dagger = 0) or A^H in = A(-mu) in (dagger = 1). */
int fa_apply_A(fa_ctx* ctx, const double* in, double* out, int dagger, int precision);

/* out = A in (dagger = 0) or A^H in (dagger = 1) in FP64, like fa_apply_A
 * with precision FA_F64, but without allocating any device memory: for
 * callers that cannot let the library call cudaMalloc, such as code recording
 * a CUDA graph under global stream-capture mode (where cudaMalloc is refused)
 * or code whose device memory is owned by a framework allocator or a fixed
 * budget.  The paper has no counterpart; this is a library convenience.
 * The two working spinors live in one static device array sized for at most
 * 8192 sites (3 MiB, resident on every GPU that loads the library until the
 * process exits); larger lattices return FA_EINVAL.  The first call on a
 * device looks up that array's device address (make it before any stream
 * capture); the context's device must be current.  All calls share the array,
 * so calls that overlap on one GPU race and must be serialised by the caller.
 * Stream-ordered on the context's stream; in and out are canonical device
 * spinors, in != out. */
int fa_apply_A_noalloc(fa_ctx* ctx, const double* in, double* out, int dagger);

/* Single-pass multi-shift solve (FP64): x_s = (A + sigma_s)^{-1} b for every
 * pole; x_s is an array of ns device spinors (canonical). */
int fa_solve_multishift(fa_ctx* ctx, const double* b, double* const* x_s,
                        const fa_solver_params* params, fa_solver_stats* stats);

/* y = sum_s omega_s (A + sigma_s)^{-1} b by the single-pass (params->mode =
 * FA_SINGLE, FP64) or the double-pass form (FA_DOUBLE; any precision).
 * b, y: device spinors (canonical).  Returns after the result is in y. */
int fa_apply_f(fa_ctx* ctx, const double* b, double* y,
               const fa_solver_params* params, fa_solver_stats* stats);

/* The same as fa_apply_f with b and y in HOST memory: the host<->device
 * copies are part of the call. */
int fa_apply_f_host(fa_ctx* ctx, const double* b_host, double* y_host,
                    const fa_solver_params* params, fa_solver_stats* stats);

/* Wait for all work of the context; returns a deferred device error, if any. */
int fa_sync(fa_ctx* ctx);

/* Kernel launches issued by this context since creation (instrumentation). */
long long fa_launch_count(const fa_ctx* ctx);

/* Mean device time (ms) of the hop kernels (one D_w sweep) issued by solves
 * with params->flags bit 1 set since the last reset, and how many were timed.
 * Reset with fa_hop_timing_reset(). */
int fa_hop_timing(const fa_ctx* ctx, int precision, double* mean_ms, long long* count);
int fa_hop_timing_reset(fa_ctx* ctx);

const char* fa_status_string(int status);
const char* fa_last_error(void);
const char* fa_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FAPATH_H */
