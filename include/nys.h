/*
 * nys.h -- C ABI of the GB300 Nystrom-accelerated primal LS-SVM ODE solver.
 *
 * Method (arXiv 2510.04094): an ODE y^(p) = f(t, y, ..) on a grid t_1..t_n is
 * fitted by y^(t) = omega^T phi(t) + b, where phi(t) = Lambda^{-1/2} U^T k(t)
 * is the explicit Nystrom feature map built from the eigendecomposition
 * Omega_mm = U Lambda U^T of the m x m landmark kernel (Appendix A.3, eq32),
 * k_j(t) = K(t, s_j) = exp(-(t - s_j)^2 / sigma^2) (Section 3, RBF kernel).
 * Linear ODEs: the primal system of Lemma 1 (Section 3.1).  Nonlinear ODEs:
 * Lemma 2 (Section 3.2, Eq. 2.2) solved by Newton's method (Eq. 3.2.1).
 *
 * Conventions for every entry point:
 *  - Return value: NYS_OK (0) or a negative nys_status.  Argument and CUDA
 *    errors are reported synchronously; nys_last_error() then gives a message
 *    (thread-local).  Nothing aborts, traps or throws across the ABI.
 *  - Numerical outcomes are per instance and asynchronous: they are written
 *    to a caller-provided device array status_out (int32, one per instance).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  All device work is enqueued on it; calls return before the
 *    work finishes.  A context must be used from one stream at a time.
 *  - Pointers documented "device" must be device (or managed) memory that
 *    stays valid until the enqueued work completes; "host" pointers are read
 *    before the call returns.  The caller owns all pointers it passes; the
 *    context owns its own workspaces and frees them in nys_destroy.
 *  - Only nys_setup allocates device memory (cudaMalloc); later calls
 *    allocate nothing on the device.
 */
#ifndef NYS_H
#define NYS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NYS_OK = 0,
  NYS_EINVAL = -1,      /* invalid argument (detail in nys_last_error)          */
  NYS_ENOMEM = -2,      /* device or pinned host allocation failed              */
  NYS_ECUDA = -3,       /* a CUDA runtime call failed                           */
  NYS_ENOTSPD = -4,     /* per instance: projected Hessian not positive definite
                           (or fewer kept eigenpairs + 1 than conditions)       */
  NYS_ENOCONV = -5,     /* per instance: Newton iteration cap reached           */
  NYS_ENONFINITE = -6,  /* per instance: NaN/Inf in inputs or results           */
  NYS_ETIMEOUT = -7,    /* per instance: a bounded device wait gave up (the
                           tensor-core assembly); the GPU context stays usable */
  NYS_EPRECISION = -8,  /* per instance, MIXED: landmark kernel too ill-conditioned
                           for the FP32 factor (kept lambda_min < 1e-7 lambda_max),
                           or refinement that leaves an estimated error above
                           1e-4 of (omega, b): rho * d, d the last pass's
                           max|correction| / max|x|, rho the passes' contraction
                           (the first pass's d, else the ratio of the last two
                           d; not checked when refine_steps is 0);
                           solve that instance with NYS_FP64                   */
  NYS_ESTATE = -9,      /* call out of order (e.g. solve before assemble)       */
  NYS_EBOUNDS = -10     /* per instance, library built with NYS_DEBUG_CHECKS
                           only: a kernel's index check failed and the access
                           was skipped (the release build carries no checks)  */
} nys_status;

/* NYS_MIXED: FP32 assembly, FP32 H and Cholesky factor, float-float residual
   refinement.  NYS_MIXED_F64F: the same FP32 assembly and refinement with the
   H = D + gamma B G B^T formation and its Cholesky factor in FP64 (the split
   that keeps the factorisation FP64); everything else as NYS_MIXED.          */
typedef enum { NYS_FP64 = 0, NYS_MIXED = 1, NYS_MIXED_F64F = 2 } nys_precision;

/* Coefficient families of the ODE (Section 2, Eq. 2.1; Section 3.1).       */
typedef enum {
  /* y^(p) - sum_{k=1..p} f_k(t) y^(p-k) = r(t) with f_k, r tabulated on the
     grid: coef_table is (p+1) x n, row-major, rows f_1..f_p then r.        */
  NYS_COEF_TABLE = 0,
  /* y^(p) + sum_k a_k y^(p-k) = c sin(omega t + phi0):
     c[0] = a_1, c[1] = a_2 (p = 2), c[2] = c, c[3] = omega, c[4] = phi0.   */
  NYS_COEF_LIN = 1,
  /* nonlinear (Lemma 2): y^(p) = c0 + c1 y + c2 y^2 + c3 y^3
     - delta y' + beta y'^2 / y [p = 2 only for delta, beta] + g cos(omega t):
     c[0..3] = c0..c3, c[4] = delta, c[5] = g, c[6] = omega, c[7] = beta
     (y'' = -y + 2 y'^2 / y is Problem 15 of Appendix A.6; y must stay
     nonzero on the collocation points when beta != 0).                      */
  NYS_COEF_POLY_NL = 2
} nys_coef_kind;

/* Conditions of an instance (Section 2: initial or boundary conditions).   */
typedef enum {
  /* initial values (Lemma 1): y^(k)(t_1) = v[k], k < p (y(t_1) = v[0],
     y'(t_1) = v[1] for p = 2); collocation rows i = 2..n                   */
  NYS_BC_IVP = 0,
  /* boundary values (Appendix A.4, BVP case; for the nonlinear kind in the
     Lagrangian of its Problem 15 example): p = 2: y(t_1) = v[0],
     y(t_n) = v[1]; p = 4 (Problem 16): y(t_1) = v[0], y'(t_1) = v[1],
     y(t_n) = v[2], y'(t_n) = v[3].  Collocation rows i = 2..n-1.  nys_grad
     refuses such contexts.                                                   */
  NYS_BC_BVP = 1
} nys_conditions;

/* One ODE instance (host struct).  Grid: t_i = t0 + (i-1)(t1-t0)/(n-1),
   i = 1..n.  Conditions per bc: by default at t_1, y(t_1) = v[0],
   y'(t_1) = v[1] (p = 2).                                                   */
typedef struct {
  int32_t p;                 /* ODE order, 1 or 2; 3 or 4 with kind TABLE and
                                NYS_FP64 (higher-order case of Problem 16)         */
  int32_t n;                 /* collocation points, 3 <= n <= 2^24                 */
  int32_t m;                 /* landmarks, 2 <= m <= min(n, NYS_M_MAX); above
                                NYS_M_MAX_MIXED only linear kinds, NYS_FP64     */
  int32_t kind;              /* nys_coef_kind                                      */
  double t0, t1;             /* interval, t1 > t0                                  */
  double sigma;              /* RBF width in exp(-(u-v)^2/sigma^2), > 0            */
  double gamma;              /* regularisation constant, > 0                       */
  double v[4];               /* initial values y^(k)(t_1), k < p, or boundary values
                                (see bc); unused entries ignored                   */
  double c[8];               /* coefficients, layout per kind above                */
  const int32_t* landmarks;  /* host, optional: m increasing 0-based grid indices;
                                NULL = evenly spaced, index round(j(n-1)/(m-1))    */
  const double* coef_table;  /* host, kind TABLE only: (p+1) x n                   */
  int32_t bc;                /* nys_conditions (0 = NYS_BC_IVP)                    */
  int32_t reserved;          /* must be 0                                          */
} nys_instance;

#define NYS_M_MAX 224        /* landmarks per instance (FP64 linear solves)      */
#define NYS_M_MAX_MIXED 112  /* landmarks for MIXED, Newton, gradients and
                                nys_solve_noalloc                                  */

typedef struct {
  int32_t precision;     /* nys_precision.  MIXED: FP32 assembly and FP32 factor,
                            refined against FP64-accurate residuals.             */
  int32_t refine_steps;  /* MIXED: residual passes after the first solve (0..8,
                            every instance).  Default when negative: 1 (2 if
                            any instance has boundary values, NYS_BC_BVP), then
                            one adaptive pass for the instances whose estimated
                            error (rho * d, see NYS_EPRECISION) is above 1e-8;
                            the others skip it                                 */
  double eig_tau;        /* drop eigenpairs with lambda <= tau * lambda_max
                            (default 1e-12 when <= 0)                            */
  int32_t scale_sqrt_m;  /* 1: eq32's sqrt(m) feature scale (== gamma * m)      */
  int32_t assembly;      /* MIXED only, nys_assembly: NYS_ASM_AUTO (0) runs the
                            Gram of every kind-LIN instance whose landmark
                            windows are narrow (at most 14 landmarks per window
                            of 32..512 rows within the band u <= 16) on the CUDA
                            cores, one warp per work unit (FP32 products, 16 x
                            16 window Grams, compensated unit sums), and every
                            other instance on the tensor cores (tcgen05, TF32
                            hi/lo split, FP32 accumulation in tensor memory);
                            NYS_ASM_TC (3) puts every instance on the tensor
                            cores; NYS_ASM_SIMT (1) runs the older CUDA-core
                            kernel (FP32 FMA, 8x8 register blocks)            */
} nys_options;

/* NYS_ASM_TUNE (MIXED): before the first assembly, time NYS_ASM_AUTO,
   NYS_ASM_TC (both on the tensor-core kernel's long work units) and
   NYS_ASM_SIMT (work items of 512 and 1024 rows) on the context's own batch
   (CUDA events, a few launches each) and keep the fastest; see
   nys_assembly_config.  Other precisions ignore it.                         */
typedef enum {
  NYS_ASM_AUTO = 0,
  NYS_ASM_SIMT = 1,
  NYS_ASM_TUNE = 2,
  NYS_ASM_TC = 3
} nys_assembly;

typedef struct nys_ctx nys_ctx;

/* Create a context for `batch` instances (host array `inst`), allocate all
   device workspaces, upload the descriptors and enqueue the Nystrom setup
   (landmark kernel Omega in FP64; W with W^T W = Omega^{-1}: W = L^{-1} from
   Omega = L L^T for NYS_FP64 when m |W|_F^2 <= 1e6 certifies cond(Omega) <= 1e6, else the
   Jacobi eigendecomposition W = Lambda^{-1/2} U^T with truncation; the fit
   does not depend on which; Appendix A.3 and the feature map eq32).  Instances with identical landmark sets
   (same m, grid spacing/sigma and indices) share one factor.  Instances with
   m > NYS_M_MAX_MIXED (FP64, linear kinds only) are factored and solved in a
   device workspace of about 0.85 MB each.
   Errors: NYS_EINVAL (bad instance: message names it; orders 3-4 or
   m > NYS_M_MAX_MIXED with NYS_MIXED; m > NYS_M_MAX_MIXED with a nonlinear
   kind), NYS_ENOMEM, NYS_ECUDA. */
int32_t nys_setup(nys_ctx** out, const nys_instance* inst, int32_t batch,
                  const nys_options* opt, void* stream);

/* Replace the instances of an existing context (same batch size; per
   instance same p, n, m, kind and landmark indices as at setup).  Enqueues
   the host -> device copy of the descriptors; the Nystrom factor is
   recomputed by the next nys_assemble or nys_run.  MIXED with NYS_ASM_AUTO:
   when a new sigma changes an instance's band plan, the assembly work list is
   rebuilt (synchronises the device, drops captured nys_run graphs).
   Errors: NYS_EINVAL (shape changed), NYS_ECUDA.                            */
int32_t nys_update(nys_ctx* c, const nys_instance* inst, void* stream);

/* Fused row pass (Lemma 1, Section 3.1): for every collocation row
   i = 2..n evaluate k, k', k'' at t_i against the landmarks, apply the ODE
   operator and accumulate the Gram of [kappa_i; -f_p(t_i); r(t_i)] without
   storing any n x m matrix.  kappa_i = k^(p)(t_i) - sum f_k k^(p-k)(t_i).  */
int32_t nys_assemble(nys_ctx* c, void* stream);

/* Solve Lemma 1's system [E + A M, -A f_p, C^T; ...] [omega; b; lambda] =
   [A r; V r; v] for every instance: H = D + gamma B G B^T with B = blkdiag(W, 1),
   null-space elimination of the initial-condition rows, Cholesky.  Landmark
   sets whose kept eigenvalues span more than 1e7 are assembled in omega
   coordinates instead (each row projected through W; FP64 only).  MIXED adds
   refine_steps residual passes (the default: its base passes and the adaptive
   pass, see nys_options.refine_steps).  x_out: device, batch x nys_x_stride(c)
   doubles, per instance [omega (m_eff, zero padded to m_max), b, lambda_1,
   lambda_2] (orders 3 and 4 report the first two of their p multipliers).
   status_out: device, batch int32 (NYS_OK / NYS_ENOTSPD /
   NYS_ENONFINITE / NYS_EPRECISION).  Either pointer may be NULL.            */
int32_t nys_solve(nys_ctx* c, void* stream, double* x_out, int32_t* status_out);

/* Nystrom setup + nys_assemble + nys_solve as one CUDA graph (reading the
   descriptors currently on the device), captured on the first call for this
   (x_out, status_out) pair and replayed afterwards.                         */
int32_t nys_run(nys_ctx* c, void* stream, double* x_out, int32_t* status_out);

/* Assembly configuration in use: kernel (NYS_ASM_AUTO, NYS_ASM_TC or
   NYS_ASM_SIMT) and rows per work item (the tensor-core units; band units are
   planned per instance).  With NYS_ASM_TUNE this runs the tuner if it has not
   run yet (synchronises `stream`).                                           */
int32_t nys_assembly_config(nys_ctx* c, void* stream, int32_t* kernel_out, int32_t* rows_out);

/* Work items of the assembly work list in use: band units (NYS_ASM_AUTO's
   CUDA-core kernel for narrow windows) and the other kernel's items.  Host
   only, no device call; the tuner's choice shows after it has run.
   Errors: NYS_EINVAL (NULL context or output).                                */
int32_t nys_assembly_items(const nys_ctx* c, int32_t* band_items, int32_t* other_items);

/* Bounded device waits of the tensor-core assembly (NYS_MIXED with
   NYS_ASM_AUTO): each mbarrier wait gives up after `polls` polls of at most
   1 us (default 4,194,304, about 4 s; a negative value restores it).  A wait
   that gives up makes every instance of the next solve report NYS_ETIMEOUT and
   leaves the GPU context usable.  0 makes every wait give up at once, which
   exercises that path without a fault (tests of the failure handling).
   Synchronises the device and drops the context's captured nys_run graphs,
   which hold the previous limit.  Errors: NYS_EINVAL (NULL context).        */
int32_t nys_set_wait_limit(nys_ctx* c, int32_t polls);

/* Stride (doubles) of one instance in x_out: m_max + 3.                     */
int32_t nys_x_stride(const nys_ctx* c);

/* Bytes copied host -> device by the last nys_setup / nys_update.           */
int64_t nys_upload_bytes(const nys_ctx* c);

/* Number of eigenpairs kept per instance (host array, batch entries).
   Synchronises the context's stream.                                         */
int32_t nys_m_eff(nys_ctx* c, void* stream, int32_t* m_eff_host);

/* Evaluate the fitted model y^(deriv)(t) = omega^T phi^(deriv)(t) + b[deriv==0]
   (Section 3; deriv 0, 1 or 2) of the last solve or Newton call.
   tq: device query times, tq_off: device int64[batch + 1] offsets into tq,
   yq_out: device, same length as tq.                                          */
int32_t nys_eval(nys_ctx* c, void* stream, const double* tq, const int64_t* tq_off,
                 int32_t deriv, double* yq_out);

/* Newton's method (Eq. 3.2.1) on Lemma 2's KKT system for NYS_COEF_POLY_NL
   instances (FP64).  The diagonal y-block of the Jacobian is eliminated per
   row exactly, so each step costs one fused row pass and an (m+1+p) solve.
   Start: omega = 0, b = v_1, lambda = 0, y_i = v_1; or the caller's warm
   start (device, nullable): batch x nys_x_stride doubles in x_out's layout
   (omega in this context's feature basis, b, lambda_1, lambda_2), followed by
   sum_b (n_b - 1) doubles in y_aux_out's layout (the auxiliary unknowns y_i,
   which at a solution differ from the fit y^(t_i)) -- e.g. the outputs of an
   earlier call on a nearby problem, copied one after the other.
   Stop when |dx|_2 <= tol (1 + |x|_2) for x = (omega, b) and
   |F|_2 <= tol max(1, |F0|_2), F0 = F at the default start (also for a warm
   start, so both stop by the same rule); at most max_iter steps (0..1000).
   x_out as in nys_solve; y_aux_out (device, optional): sum_b (n_b - 1)
   doubles, instance after instance; iters_out, status_out: device int32[batch]
   (status NYS_OK or NYS_ENOCONV with the last iterate, NYS_ENOTSPD).
   The whole iteration runs without host synchronisation: every round is
   enqueued (converged instances drop out of the row passes; once none runs,
   the remaining rounds return at once) and captured as one CUDA graph on the
   first call with these (max_iter, tol, warm, output) arguments, replayed by
   later calls.                                                                */
int32_t nys_newton(nys_ctx* c, void* stream, int32_t max_iter, double tol,
                   const double* warm, double* x_out, double* y_aux_out,
                   int32_t* iters_out, int32_t* status_out);

/* Adjoint gradient (parameter estimation; the paper cites the use and prints no
   formula) of a loss on the fitted model of the last nys_solve, for NYS_COEF_LIN
   instances: theta = (a_1, a_2, c, omega, y0, y0', sigma) of
   y^(p) + a_1 y^(p-1) [+ a_2 y] = c sin(omega t + phi0).  The implicit-function
   derivative of Lemma 1's system: one adjoint solve with the stored FP64 factor
   and one fused row pass.  Needs a NYS_FP64 context.
   obs_t: device observation times, obs_off: device int64[batch + 1] offsets,
   dl_dy: device d loss / d y^(obs_t) (same length as obs_t),
   grad_out: device, batch x 7 doubles (a_2 and y0' entries 0 when p = 1).
   Instances whose solve failed get NaN; the sigma entry is NaN when the
   landmark kernel was truncated (m_eff < m), where sigma also moves the
   discarded eigenvectors.  Errors: NYS_EINVAL (NULL pointer, nonlinear batch,
   boundary values, order above 2, m above NYS_M_MAX_MIXED),
   NYS_ESTATE (MIXED context, or no solve yet), NYS_ECUDA.                   */
int32_t nys_grad(nys_ctx* c, void* stream, const double* obs_t, const int64_t* obs_off,
                 const double* dl_dy, double* grad_out);

/* Allocation-free FP64 solve (the paper has no counterpart; this is a library
   facility).  For callers that cannot call cudaMalloc: processes whose device
   memory is reserved up front by another allocator (a framework's caching
   pool, a fixed-budget server) or latency-critical code that cannot accept
   an allocation's implicit device synchronisation.  Computes exactly what
   nys_setup + nys_assemble + nys_solve compute with precision NYS_FP64 (same
   kernels), for a small batch of NYS_COEF_LIN instances; every workspace,
   including the row pass's partial Gram sums, lives in one static device
   array of NYS_NOALLOC_SCRATCH_BYTES (6 MiB) that every GPU loading the
   library holds until exit.  Nothing is allocated on the device or host.
   Limits: batch <= NYS_NOALLOC_MAX_BATCH, m <= NYS_NOALLOC_MAX_M,
   n <= NYS_NOALLOC_MAX_N; larger requests return NYS_EINVAL with a message.
   inst: host array; x_out: device, batch x (m_max + 3) doubles with m_max
   the largest m in this call (layout of nys_solve); status_out: device
   int32[batch].  The first call on a device looks up the array's device
   address (once per device, with that device current): make that first call
   before any stream capture.  Blocks until earlier work on `stream` is done
   and the descriptors are on the device.  All calls share the array, which
   keeps the last call's contents (the work counter is cleared by each call):
   calls whose GPU work overlaps (several streams or host threads) race.   */
#define NYS_NOALLOC_SCRATCH_BYTES (6 * 1024 * 1024)
#define NYS_NOALLOC_MAX_BATCH 32
#define NYS_NOALLOC_MAX_M 64
#define NYS_NOALLOC_MAX_N (1 << 20)
#define NYS_NOALLOC_MAX_CHUNKS 4
int32_t nys_solve_noalloc(const nys_instance* inst, int32_t batch, double* x_out,
                          int32_t* status_out, void* stream);

/* Free every resource of the context (synchronises its last stream).         */
void nys_destroy(nys_ctx* c);

const char* nys_status_str(int32_t status);
const char* nys_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* NYS_H */
