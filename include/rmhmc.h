/*
 * rmhmc.h — C ABI of the GB300 (sm_103a) implementation of the data-parallel hot path of
 * Riemannian manifold HMC for SU(3) lattice gauge theory
 * (Nguyen, Boyle, Christ, Jang, Jung, "Riemannian manifold hybrid Monte Carlo in lattice QCD",
 *  LATTICE2021, arXiv:2112.04556).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  Lattice   periodic 4D, dims = {Lx, Ly, Lz, Lt}, V = Lx Ly Lz Lt sites,
 *            site s = x + Lx*(y + Ly*(z + Lz*t)).
 *  Links     U: complex128 [V][4][3][3] (interleaved re, im doubles, row major), U[s][mu] = U_mu(x).
 *  Fields    su(3)-valued link fields (momenta, forces, Laplacian operands):
 *            float64 [nfield][V][4][8] (or float32 where `prec` says so): coefficients p^a of
 *            P = sum_a p^a T^a, T^a = lambda^a / 2 (Gell-Mann), a = 1..8 stored at 0..7.
 *            Each of the four components P_mu is an independent operand of the Laplacian.
 *  Inner product  <X,Y> = sum_{x,mu,a} X^a Y^a.
 *  Derivative     left multiplication: U_mu(x) -> exp(i w^a T^a) U_mu(x); a force is F^a = -dS/dw^a
 *                 (Sec. 2, the sentence defining F_G below Eq. 3).
 *  Operator       A = -Delta_G / 16 (Sec. 2, Eq. 3 with d = 4), spectrum in [0, 1].
 *
 *  Memory   All field and link pointers are DEVICE pointers on the context's device, owned by the
 *           caller; the library never frees them.  Small vectors marked (host) are host memory.
 *           The context owns its workspace: it is allocated by rmhmc_create or on the first call that
 *           needs it, and reused afterwards; nothing is allocated inside an iteration loop.
 *  Streams  Every call takes a cudaStream_t (0 = legacy default stream) and enqueues its work there.
 *           Calls that return host scalars synchronise that stream before returning.
 *  Threads  A context is not thread-safe: use one context per host thread / stream.
 *  Errors   Every entry point returns RMHMC_OK (0) or a negative status.  rmhmc_last_error(ctx) gives
 *           a message.  On error the contents of output buffers are unspecified, except that
 *           rmhmc_trajectory leaves U unchanged.
 *  Links    Compute calls take `const double* U`.  A non-NULL U is imported into the context first
 *           (canonical -> internal layout, FP64 and FP32 copies); NULL reuses the links imported last.
 */
#ifndef RMHMC_H
#define RMHMC_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* the library is built with hidden visibility; these declarations are its exported interface */
#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

/* status codes */
#define RMHMC_OK        0
#define RMHMC_EINVAL   -1   /* bad argument: NULL pointer, size, shape, alignment, shift <= 0 */
#define RMHMC_ECUDA    -2   /* a CUDA runtime call failed (message in rmhmc_last_error) */
#define RMHMC_ENOCONV  -3   /* an iteration (CG, refinement, fixed point) hit its cap */
#define RMHMC_ENAN     -4   /* NaN or Inf in a reduction (residual, Hamiltonian) */
#define RMHMC_ETIMEOUT -5   /* a bounded device-side wait gave up */
#define RMHMC_ENOMEM   -6   /* workspace allocation failed */

/* arithmetic precision of a call */
#define RMHMC_FP64  0       /* everything in float64 */
#define RMHMC_FP32  1       /* float32 operands and arithmetic, float64 global sums (lap_apply) */
#define RMHMC_MIXED 1       /* float32 Krylov / recurrence with float64 reliable updates and sums */

/* link storage used by the stencil: 18 reals, or 12 reals (two rows) with the third row rebuilt
 * as the complex conjugate of the cross product of the first two */
#define RMHMC_LINK18 18
#define RMHMC_LINK12 12

/* operator selector of lap_apply */
#define RMHMC_OP_A     0    /* A = -Delta_G/16, spectrum in [0,1] */
#define RMHMC_OP_DELTA 1    /* Delta_G itself */

/* damping of the Chebyshev window expansions */
#define RMHMC_KERNEL_NONE    0
#define RMHMC_KERNEL_JACKSON 1

typedef struct rmhmc_ctx rmhmc_ctx;

/* Rational mass term (Sec. 3, Eq. 6): M = R(A)^{-2},
 *   R(lam) = c + sum_{j<npole} alpha[j] / (lam + sigma[j]),  sigma[j] > 0,
 * the partial-fraction form of the bracket of Eq. (6) (each quadratic denominator of Eq. 6 gives two
 * simple poles).  kappa is the slope of the target linear mass m(lam) = (1-kappa) + kappa*lam used by
 * the momentum heatbath P = m(A) R(A) xi (= M^{1/2} xi to the accuracy of the fit).  kappa = 0 with
 * poles marks a general rational mass (e.g. from rmhmc_mass_fit_spectrum; c >= 0, alpha >= 0), whose
 * heatbath is P = R(A)^{-1} xi exactly.  npole = 0 and c = 1 give M = 1 (plain HMC).  alpha and sigma
 * are host arrays. */
typedef struct {
    double c;
    int npole;
    const double* alpha;
    const double* sigma;
    double kappa;
} rmhmc_mass;

/* RMHMC trajectory parameters (Sec. 3). */
typedef struct {
    double beta;        /* gauge coupling */
    double c1;          /* rectangle coefficient (0: Wilson; -0.331: Iwasaki); c0 = 1 - 8 c1 */
    rmhmc_mass mass;    /* mass term */
    double tau;         /* trajectory length */
    int nsteps;         /* leapfrog steps, eps = tau / nsteps */
    double tol_md;      /* relative residual of the base Krylov system inside the MD forces */
    double tol_h;       /* relative residual per shift for the Hamiltonian and the heatbath */
    double fp_tol;      /* max-norm change that ends each implicit fixed-point iteration */
    int fp_maxit;       /* cap on fixed-point iterations (RMHMC_ENOCONV beyond it) */
    int maxiter;        /* cap on Krylov iterations per solve */
    int prec;           /* RMHMC_FP64 or RMHMC_MIXED */
    uint64_t seed;      /* Philox key for the heatbath noise and the Metropolis uniform */
    uint32_t traj_index;/* Philox stream: trajectory number */
    int metropolis;     /* 1: accept/reject with probability min(1, exp(-dH)); 0: always accept */
    int logdet;         /* 1: the log|M| term of Eq. (5) through an auxiliary field phi = R(A) eta (eta from
                           Philox(seed, traj_index, tag 3)), held fixed in the MD, with action
                           1/2 <phi, M phi> = 1/2 |R(A)^{-1} phi|^2 in H and its force in the MD (needs c > 0) */
    int symplectic;     /* 0: the implicit leapfrog of Sec. 3 with group exponentials (momentum half steps
                           P' = P + eps/2 F(U, P'), links U' = exp(i eps/2 V(U',P')) exp(i eps/2 V(U,P')) U);
                           1: its exactly symplectic form on T*SU(3), the same steps with the momenta passed
                           through the right-trivialised derivative of the exponential, per link
                           dexp_X = sum_n ad_X^n/(n+1)!, ad_X Y = coefficients of i[X.T, Y.T], X = eps/2 V:
                             dexp^{-1}_{X1} mu = P + eps/2 F(U, mu), X1 = eps/2 V(U, mu); B = exp(i X1) U;
                             P_h = dexp^{-1}_{-X1} mu;  dexp^{-1}_{X2} mu2 = P_h, X2 = eps/2 V(U', mu2),
                             U' = exp(i X2) B;  P'' = dexp^{-1}_{-X2} mu2 + eps/2 F(U', mu2).
                           It preserves phase-space volume exactly (the first form only to O(eps^3) per step
                           with a link-dependent mass).  Host-driven MD only (no graph); dexp series in float64
                           (float32 corrections on the mixed path).  Any other value: RMHMC_EINVAL. */
    int fp_extra;       /* fixed-point iterations run after the max-norm change first falls to fp_tol (0: stop
                           there; 0 <= fp_extra < fp_maxit, which counts every iteration).  With float32 forces
                           the change cannot fall much below the forces' rounding noise, while the error the
                           iteration has left shrinks by the contraction factor at every further iteration:
                           extra iterations remove that systematic part, so the mixed trajectory follows the
                           float64 one to the noise level. */
    int fg_fp64;        /* gauge force inside the mixed-precision MD: 0 float32 staples from the float32 link
                           copies, 1 float64 staples from the float64 links (the float64 MD always uses float64);
                           any other value: RMHMC_EINVAL */
} rmhmc_params;

typedef struct {
    double dH, H0, H1;  /* Hamiltonian (Eq. 5; the log|M| term through the auxiliary field when logdet) */
    double T0, S0, T1, S1;
    double plaq;        /* average plaquette ReTr/3 of the output configuration */
    double u;           /* the uniform used by the Metropolis test */
    int accepted;
    int md_solves;      /* Krylov runs inside the MD */
    long long md_iters; /* Krylov iterations inside the MD */
    int fp_iters_p;     /* momentum fixed-point iterations, summed over steps */
    int fp_iters_u;     /* link fixed-point iterations, summed over steps */
    double max_fp_change;
    double A0, A1;      /* auxiliary-field action before and after the MD (0 without logdet); H includes it */
} rmhmc_result;

/* ---------------------------------------------------------------------------------------------- */
/* context                                                                                          */
/* ---------------------------------------------------------------------------------------------- */

/* Create a context for a lattice of extents dims[4] (each >= 2) on CUDA device `device`.
 * Allocates the link copies and the reduction scratch.  *out receives the handle. */
int rmhmc_create(const int dims[4], int device, rmhmc_ctx** out);

/* Free all workspace of the context (NULL is allowed). */
int rmhmc_destroy(rmhmc_ctx* ctx);

/* Message of the last failing call on this context ("" if none); valid until the next call. */
const char* rmhmc_last_error(const rmhmc_ctx* ctx);

/* Import links U (device, canonical complex128 [V][4][3][3]) into the context: an FP64
 * structure-of-arrays copy and an FP32 copy (first two rows + third row), Sec. 2 Eq. (3)'s links. */
int rmhmc_set_links(rmhmc_ctx* ctx, const double* U, cudaStream_t stream);

/* Counters of the context (host scalars, each pointer nullable): kernels launched by the library,
 * Krylov iterations, and -- while profiling is on -- the number and summed duration (ms, CUDA events
 * on the caller's stream) of the conjugate-gradient stencil launches that did work (the matvec that
 * dominates the trajectory).  reset != 0 zeroes the counters after reading them. */
int rmhmc_set_profiling(rmhmc_ctx* ctx, int on);
int rmhmc_get_counters(rmhmc_ctx* ctx, long long* launches, long long* krylov_iters, long long* cg_count,
                       double* cg_ms, int reset);

/* Mixed-precision molecular dynamics (rmhmc_md, rmhmc_trajectory) runs as one CUDA graph per parameter set:
 * both implicit fixed points and every Krylov run are conditional WHILE nodes decided on the device, so an
 * MD trajectory is a single graph launch.  The graph is captured on first use (and after a workspace
 * reallocation) on the context's own streams and launched on the caller's stream.  on = 0 selects the
 * host-driven path (the float64 path always uses it); a failed capture falls back to it as well.  Graphs are
 * on by default. */
int rmhmc_set_graphs(rmhmc_ctx* ctx, int on);

/* Text report of the stencil launch shapes the autotuner chose in this context (components per lane and
 * threads per block for each precision and link format, with the measured times of every candidate),
 * written NUL-terminated into buf[len]. */
int rmhmc_tuning(const rmhmc_ctx* ctx, char* buf, int len);

/* Pin a stencil launch shape instead of timing the candidates: kernel = RMHMC_SHAPE_LAP (lap_apply and the
 * float32 recurrence of one field), RMHMC_SHAPE_CG (the conjugate-gradient stencil) or RMHMC_SHAPE_KFORCE (see
 * below), for precision prec
 * (RMHMC_FP64 / RMHMC_FP32) and link format linkfmt (the CG stencil streams 18-real links: 18 only).
 * nmu: components per lane (1, 2, 4), 0 (one component per lane with every neighbour value prefetched) or
 * 8 (the link-centric adjoint kernel: each link's adjoint matrix serves both hops across it, in 4D boxes
 * swept through time; float32 only, block 256); block: 64, 128 or 256 threads.  RMHMC_EINVAL otherwise. */
#define RMHMC_SHAPE_LAP 0
#define RMHMC_SHAPE_CG  1
#define RMHMC_SHAPE_KFORCE 2   /* the mixed kinetic force's basis contraction (prec RMHMC_FP32, linkfmt 18): nmu 0,
                                  block 128 (the default): four lanes per link, the block's own basis rows read
                                  from global memory once per chunk of 4; nmu 1, block 128: the same rows staged
                                  once in shared memory (runs of up to 20 vectors); nmu 2, block 256: eight lanes
                                  per link splitting the rows of the 8x8 accumulator, chunks of 8; nmu 3, block
                                  128: as nmu 0 with the neighbour rows loaded whole by the four lanes of a site
                                  and passed through shared memory */
#define RMHMC_SHAPE_LINKUPDATE 3   /* the float64 link update exp(i eps V) U (prec RMHMC_FP64, linkfmt 18, block
                                      128): nmu 1 (the default) in float-float arithmetic (two float32 numbers per
                                      value, ~2^-48 relative; rotations with Tr Q^2 / 2 >= 0.24 in float64), nmu 0
                                      in float64 throughout.  Applies to rmhmc_link_update and the mixed-precision
                                      trajectories; float64 trajectories and the flow stay in float64 */
#define RMHMC_SHAPE_ADJOINT 4   /* the multi-field adjoint-form stencil (lap_apply of 6 or more float32 fields, the
                                   batched Chebyshev recurrence; prec RMHMC_FP32, linkfmt 12 or 18): nmu = fields
                                   per pass and parity, 2 or 3 (0: timed on first use, the default); block = the
                                   z-extent of the slabs in which the grid sweeps t, 1 .. L2 (0: L2, i.e.
                                   lexicographic order, the default) */
int rmhmc_set_stencil_shape(rmhmc_ctx* ctx, int kernel, int prec, int linkfmt, int nmu, int block);

/* ---------------------------------------------------------------------------------------------- */
/* Sec. 2, Eq. (3): the normalised adjoint covariant Laplacian                                       */
/* ---------------------------------------------------------------------------------------------- */

/* Y = op(X) for nfield fields (device, [nfield][V][4][8], float64 if prec == RMHMC_FP64 else
 * float32; X and Y must not overlap), with
 *   Delta X_mu(x) = sum_nu [ U_nu(x) X_mu(x+nu) U_nu(x)^dag + U_nu(x-nu)^dag X_mu(x-nu) U_nu(x-nu)
 *                            - 2 X_mu(x) ]
 * (the second term as U^dag X U: the gauge-covariant reading of the printed Eq. 3), op = A = -Delta/16
 * (RMHMC_OP_A) or Delta (RMHMC_OP_DELTA).  linkfmt: RMHMC_LINK18 or RMHMC_LINK12. */
int lap_apply(rmhmc_ctx* ctx, const double* U, const void* X, void* Y, int nfield, int prec,
              int linkfmt, int op, cudaStream_t stream);

/* Link derivative of the Laplacian's bilinear form (adjoint of Eq. 3 with respect to the links):
 *   G^a_nu(y) = sum_f w[f] d<Z_f, A X_f>/dw^a,   U_nu(y) -> exp(i w^a T^a) U_nu(y),
 * X, Z device float64 [nfield][V][4][8], w host [nfield], G device float64 [V][4][8] (overwritten).
 * This is the backward kernel behind the kinetic force and the autograd Laplacian. */
int lap_link_grad(rmhmc_ctx* ctx, const double* U, const double* X, const double* Z, int nfield,
                  const double* w, int prec, double* G, cudaStream_t stream);

/* ---------------------------------------------------------------------------------------------- */
/* Sec. 2, Eq. (4): Chebyshev band-pass filters and per-mode power spectra                           */
/* ---------------------------------------------------------------------------------------------- */

/* Moments mu_k(G) = <G, T_k(2A-1) G>, k = 0..degree, of every field G in F (device float64
 * [nF][V][4][8]) and in the noise set (device float64 [nnoise][V][4][8]; NULL: the library draws
 * nnoise N(0,1) fields from Philox with key `seed`), all fields in one batched recurrence.  Window w
 * is [edges[w], edges[w+1]] of eigenvalues of A (host, nwin+1 increasing values in [0,1]); its filter
 * is B_w = sum_k C[w][k] T_k(2A-1) with C the Chebyshev coefficients of the window's indicator,
 * damped by Jackson's kernel if kernel == RMHMC_KERNEL_JACKSON.  Outputs (host):
 *   num[f][w]  = <F_f|B_w|F_f>,
 *   tr[w]      = mean over noise fields of <eta|B_w|eta>  (Hutchinson estimate of Tr B_w over the
 *                full [V][4][8] space),
 *   spec[f][w] = num[f][w] / tr[w]                        (Eq. 4: power per mode),
 *   moments[(nF+nnoise)][degree+1] (nullable).
 * prec: RMHMC_FP64, or RMHMC_MIXED (float32 recurrence, float64 moment sums). */
int cheb_filter_spectrum(rmhmc_ctx* ctx, const double* U, const double* F, int nF,
                         const double* noise, int nnoise, uint64_t seed, int degree, int nwin,
                         const double* edges, int kernel, int prec, double* spec, double* num,
                         double* tr, double* moments, cudaStream_t stream);

/* ---------------------------------------------------------------------------------------------- */
/* Sec. 3, Eq. (6): rational mass term via a multishift Krylov solve                                */
/* ---------------------------------------------------------------------------------------------- */

/* y_f = c b_f + sum_j alpha[j] (A + sigma[j])^{-1} b_f for nfield fields b_f (Sec. 3, Eq. 6: the rational
 * mass term; device float64 [nfield][V][4][8]), nshift shifts (host sigma[], alpha[], every sigma > 0).  For
 * each field all shifts share one Krylov space (multishift CG); the fields are solved one after the other
 * with one workspace.  Stops when every shift of a field has relative true residual
 * |b_f - (A+sigma_j) x_fj| / |b_f| <= tol (checked in float64), or returns RMHMC_ENOCONV once a field's
 * solve exceeds maxiter Krylov iterations.
 * prec = RMHMC_FP64: float64 throughout.  prec = RMHMC_MIXED: float32 Krylov iterations, then
 * float64-accurate reliable updates (true residual per shift) with float32 correction solves until tol.
 * Outputs: y (device float64 [nfield][V][4][8]); xs (device float64 [nfield][nshift][V][4][8], nullable);
 * iters (host, nullable) Krylov iterations summed over the fields; resid (host [nfield][nshift],
 * nullable) final true relative residuals.  nfield = 0 does nothing. */
int rat_mass_solve(rmhmc_ctx* ctx, const double* U, const double* b, int nfield, int nshift,
                   const double* sigma, const double* alpha, double c, double tol, int maxiter,
                   int prec, double* y, double* xs, int* iters, double* resid, cudaStream_t stream);

/* Momentum heatbath (Sec. 3): P = m(A) R(A) xi with m(A) = (1-kappa) + kappa A, so that P has
 * covariance M = R^{-2} up to the fit error.  A general rational mass (kappa = 0 with poles, e.g. from
 * rmhmc_mass_fit_spectrum; c >= 0, alpha_j >= 0) gets P = R(A)^{-1} xi exactly, from the partial fraction
 * 1/R = p0 + p1 lam + sum_j beta_j/(lam + zeta_j) (zeros of R found on the host).  xi, P: device float64
 * [V][4][8]. */
int rmhmc_heatbath(rmhmc_ctx* ctx, const double* U, const double* xi, const rmhmc_mass* mass,
                   double tol, int prec, double* P, cudaStream_t stream);

/* Zolotarev's best relative rational approximation R(lam) ~ m(lam)^{-1/2}, m = (1-kappa) + kappa lam
 * on lam in [0,1] with npole simple poles (host outputs c, alpha[npole], sigma[npole]); max_rel_err
 * (nullable) receives max |R m^{1/2} - 1| on a 4096-point grid. */
int rmhmc_mass_fit(int npole, double kappa, double* c, double* alpha, double* sigma,
                   double* max_rel_err);

/* Mass term fitted to a measured force power spectrum per mode (Sec. 4; e.g. the spec output of
 * cheb_filter_spectrum at the window centres lam): M(lam) proportional to s(lam), normalised to 1 at the largest
 * power, so that every Laplacian mode moves at the same MD rate.  R = M^{-1/2} = c + sum_j alpha_j/(lam + sigma_j)
 * with the npole poles fixed on a geometric grid in [sigma_min, sigma_max] and c, alpha_j >= 0 minimising
 * sum_w (R(lam_w) (s_w / max s)^{1/2} - 1)^2 (non-negative least squares), so M = R^{-2} is positive and
 * increasing.  Host outputs c, alpha[npole], sigma[npole]; max_rel_err (nullable) receives the largest
 * relative error of R at the lam_w.  Use the result with kappa = 0 (a general rational mass: the heatbath is
 * then P = R(A)^{-1} xi).  RMHMC_EINVAL for nwin < 1, npole outside [0, 24], lam outside [0, 1], a
 * non-positive power or a bad pole range. */
int rmhmc_mass_fit_spectrum(int nwin, const double* lam, const double* spec, int npole, double sigma_min,
                            double sigma_max, double* c, double* alpha, double* sigma, double* max_rel_err);

/* Allocation-free gauge action: the paper has no counterpart; this is a service for callers that cannot
 * allocate device memory -- an application whose device memory is entirely handed out by another
 * allocator (a caching pool that reserved the GPU), or code on a latency-critical path that must not call
 * cudaMalloc/cudaFree because they synchronise the device.  No context is needed and nothing is
 * allocated: U (device, canonical complex128 [V][4][3][3]) and out (device, 2 doubles: out[0] = S as in
 * gauge_force, out[1] = average plaquette ReTr P/3) are the caller's; the only scratch is a ~64 KB
 * file-scope device array inside the library (4096 block partials and a counter), kept by every GPU that
 * loads the library until the process exits.  Its device address is looked up by the first call made on
 * each device, so make that first call before any stream capture.  Calls share that array and each call
 * clears its counter: calls that overlap on the GPU (e.g. on two unordered streams) race and must not be
 * issued.  Asynchronous on `stream`.  Returns RMHMC_EINVAL for a NULL or misaligned pointer, an extent
 * < 2 or > 2^26, or more than 2^26 sites. */
int rmhmc_action_noalloc(const int dims[4], const double* U, double beta, double c1, double* out,
                         cudaStream_t stream);

/* ---------------------------------------------------------------------------------------------- */
/* forces (Sec. 2 below Eq. 3; Sec. 3 below Eq. 5)                                                   */
/* ---------------------------------------------------------------------------------------------- */

/* Gauge force F^a_mu(x) = -dS/dw^a (device float64 [V][4][8]) for
 *   S = beta sum_x [ c0 sum_{mu<nu} (1 - ReTr P_{mu nu}/3) + c1 sum_{mu!=nu} (1 - ReTr R_{mu nu}/3) ],
 * c0 = 1 - 8 c1 (c1 = 0: Wilson plaquette action), R the 1x2 rectangles.  action and plaq (host,
 * nullable) receive S and the average plaquette ReTr P/3, both summed in float64.
 * prec: RMHMC_FP64, or RMHMC_FP32 (float32 staples, float64 action). */
int gauge_force(rmhmc_ctx* ctx, const double* U, double beta, double c1, int prec, double* F,
                double* action, double* plaq, cudaStream_t stream);

/* Kinetic (mass-term) force F_K = -dT/dw with T = 1/2 <P, M(U)^{-1} P> = 1/2 |R(A) P|^2 (Sec. 3,
 * the force F_M below Eq. 5).  P device float64 [V][4][8]; F (device, nullable) receives F_K;
 * Vout (device, nullable) the velocity M^{-1} P; T (host, nullable) the kinetic energy.
 * tol: relative residual of the base Krylov system. */
int kinetic_force(rmhmc_ctx* ctx, const double* U, const double* P, const rmhmc_mass* mass,
                  double tol, int prec, double* F, double* Vout, double* T, cudaStream_t stream);

/* ---------------------------------------------------------------------------------------------- */
/* Sec. 3: molecular dynamics and the RMHMC trajectory                                              */
/* ---------------------------------------------------------------------------------------------- */

/* Gaussian su(3) field (device float64 [V][4][8]): coefficient n = 8 mu + a of site s is the
 * (n mod 2)-th output of the Box-Muller pair made from Philox4x32-10 block
 * (counter = {n/2, s, stream_id, tag}, key = {seed lo, seed hi}); uniforms take 53 bits from two words. */
int rmhmc_gauss_field(rmhmc_ctx* ctx, double* out, uint64_t seed, uint32_t stream_id, uint32_t tag,
                      cudaStream_t stream);

/* Uout = exp(i eps V) U per link (device canonical links; Uout may equal U); the exponential is the
 * Cayley-Hamilton form, followed by reunitarisation if reunit != 0.  Computed in float-float arithmetic
 * (~2^-48 relative) unless RMHMC_SHAPE_LINKUPDATE pins float64, as in the mixed-precision trajectories; the
 * float64 trajectories and the gradient flow always update links in float64. */
int rmhmc_link_update(rmhmc_ctx* ctx, const double* U, const double* V, double eps, int reunit,
                      double* Uout, cudaStream_t stream);

/* H = T + S for (U, P) (Eq. 5 without log|M|), with the rational solve at relative residual tol. */
int rmhmc_hamiltonian(rmhmc_ctx* ctx, const double* U, const double* P, const rmhmc_params* p,
                      double* H, double* T, double* S, cudaStream_t stream);

/* Molecular dynamics only: p->nsteps generalised-leapfrog steps of size p->tau / p->nsteps on
 * (U, P) in place (device canonical links, device float64 momenta), with the implicit fixed points
 * of Sec. 3.  r (nullable) receives the iteration counts.  p->logdet is not used here (the auxiliary
 * field belongs to a trajectory: rmhmc_trajectory). */
int rmhmc_md(rmhmc_ctx* ctx, double* U, double* P, const rmhmc_params* p, rmhmc_result* r,
             cudaStream_t stream);

/* One RMHMC trajectory on U in place: heatbath P0 = m(A)R(A) xi (xi device float64 [V][4][8], or
 * NULL: Philox(seed, traj_index, tag 0)), H0, MD, H1, then Metropolis with the uniform from Philox
 * (seed, traj_index, tag 1) unless p->metropolis == 0.  With p->logdet the auxiliary field of the log|M|
 * term is drawn (Philox tag 3), its action enters H0 and H1 (r->A0, r->A1) and its force the MD.  On
 * rejection U is restored.  P_out (device, nullable) receives the final momenta of the MD. */
int rmhmc_trajectory(rmhmc_ctx* ctx, double* U, const double* xi, const rmhmc_params* p,
                     rmhmc_result* r, double* P_out, cudaStream_t stream);

/* Chebyshev coefficients of spectral windows, Sec. 2 Eq. (4): C[w][k], w < nwin, k <= degree, of the indicator of
 * [edges[w], edges[w+1]] (eigenvalues of A in [0, 1]; variable x = 2 lambda - 1), times Jackson's damping when
 * kernel == RMHMC_KERNEL_JACKSON.  Host only.  C: nwin * (degree + 1) doubles (caller's).  RMHMC_EINVAL for
 * edges that do not increase within [0, 1], degree outside [0, 20000] or a bad kernel. */
int cheb_window_coeffs(int nwin, const double* edges, int degree, int kernel, double* C);

/* A band filter applied as a vector (the band-filtered momenta of Sec. 4): Y_f = sum_{k=0}^{degree} coef[k]
 * T_k(2A - 1) F_f for nfield fields, F and Y device float64 [nfield][V][4][8] (16-byte aligned, distinct),
 * coef host (degree + 1 doubles, e.g. a row of cheb_window_coeffs).  degree stencil applications by the
 * three-term recurrence; prec RMHMC_FP64, or RMHMC_MIXED (float32 recurrence, float64 accumulation).
 * U as in lap_apply (NULL: the context's links).  RMHMC_EINVAL for bad sizes, a bad prec or misalignment. */
int cheb_filter_apply(rmhmc_ctx* ctx, const double* U, const double* F, int nfield, int degree, const double* coef,
                      int prec, double* Y, cudaStream_t stream);

/* Wilson gradient flow, the flowed-energy observable of Sec. 4 (the paper takes its definition from
 * Luscher, JHEP 08 (2010) 071): nsteps steps of size eps of Luscher's third-order Runge-Kutta scheme for
 * dV/dt = -g0^2 (dS_W) V, in place on U (device, canonical complex128 [V][4][3][3]).  The flow does not
 * depend on beta (g0^2 F = 6 F at beta = 1).  E (host, nullable, nsteps + 1 doubles) receives the plaquette
 * energy density E = (1/V) sum_x 2 sum_{mu<nu} Re Tr(1 - P_mu,nu(x)) = 36 (1 - <Re Tr P / 3>) at
 * t = 0, eps, ..., nsteps eps; t^2 E(t) is the usual scale-setting combination.  prec RMHMC_FP64 (all
 * float64) or RMHMC_MIXED (float32 force, float64 links and updates).  The context's link copies hold the
 * flowed links afterwards.  Synchronous.  RMHMC_EINVAL for a NULL or misaligned U, nsteps < 0, a
 * non-finite eps or a bad prec. */
int wilson_flow(rmhmc_ctx* ctx, double* U, double eps, int nsteps, int prec, double* E, cudaStream_t stream);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif

#ifdef __cplusplus
}
#endif
#endif /* RMHMC_H */
