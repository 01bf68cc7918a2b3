// Krylov engine for the rational mass term (Sec. 3, Eq. 6).
//
// One conjugate-gradient run on the smallest shift, A0 = A + sigma_0, keeps every residual r_k in
// HBM.  The residuals are the Lanczos vectors of A0 (up to normalisation); the CG coefficients give
// the Lanczos tridiagonal matrix T_n, and every shifted Galerkin solution
//   x_j = (A + sigma_j)^{-1} b ~ |b| V_n (T_n + (sigma_j - sigma_0))^{-1} e_1
// -- identical to what multishift CG produces -- becomes one linear combination of the stored
// residuals.  The same basis yields the nested solves of the kinetic force, Z_j = (A+sigma_j)^{-1} R(A) b,
// and the velocity R(A)^2 b, from one Krylov run instead of two.  All small-matrix work is float64
// on the host; all field work is in the kernels.
#pragma once
#include <vector>

#include "common.cuh"

namespace rm {

// capacity of the stored basis (residual vectors of one run)
constexpr int kBasisCap = 160;
// reduction slots of the Krylov engine (the residual norms use kSlotResid .. kSlotResid + nshift - 1)
constexpr int kSlotGamma = 0, kSlotRho = 1, kSlotNorm = 2, kSlotResid = 8;

struct KrylovResult {
    int n = 0;                      // iterations
    int status = 0;                 // as KScal::done
    std::vector<double> rho, alpha, beta;
};

// what to build from the basis
struct CombineSpec {
    // host coefficients coef[m][k] for outputs m < M on basis vectors k < n
    std::vector<double> coef;
    int M = 0, n = 0;
};

// Lanczos post-processing on the host (float64)
struct Tridiag {
    std::vector<double> d, e;   // diagonal, off-diagonal of T_n
    std::vector<double> inv_norm;  // 1/|r_k|
    double bnorm = 0.0;
    int n = 0;
    void build(const KrylovResult& kr);
    // y = (T + shift)^{-1} rhs
    void solve(double shift, const std::vector<double>& rhs, std::vector<double>& y) const;
    // coefficients on the stored residual vectors of sum_k y_k v_k
    void to_basis(const std::vector<double>& y, double* coef_row) const;
};

// run CG on (A + sigma0) x = b; b (internal precision, [V][4][8]) is copied into basis slot 0
template <typename T>
int krylov_run(rmhmc_ctx* ctx, const T* b, double sigma0, double tol, int maxit, KrylovResult& out, cudaStream_t st);
// basis pointer of the last run
template <typename T> T* krylov_basis(rmhmc_ctx* ctx);
// out[m] = sum_k coef[m][k] r_k for m < M (outputs as float or double)
template <typename T, typename TO>
int krylov_combine(rmhmc_ctx* ctx, const CombineSpec& spec, TO* const* outs, cudaStream_t st);

// per-field residuals r_f = b - (A + sigma_f) x_f in float64 (x_f float64 [nf][V][4][8]), their squared
// norms to host norm2[nf]; r (nullable) stores the residual fields
int resid64(rmhmc_ctx* ctx, const double* b, const double* x, int nf, const double* sigma, double* r, double* norm2,
            cudaStream_t st);

// the same residuals from float32 arithmetic with compensated (float32-pair) sums: tab is the adjoint table
// of the context's links (adjoint_table), r receives the residuals rounded to float32 ([nf][V][4][8])
int adjoint_table(rmhmc_ctx* ctx, float** tab, cudaStream_t st);
int resid_df(rmhmc_ctx* ctx, const float* tab, const double* b, const double* x, int nf, const double* sigma, float* r,
             double* norm2, cudaStream_t st);

// float64 -> float32 field conversion and float32 correction accumulation
int to_float(rmhmc_ctx* ctx, const double* in, float* out, size_t n, cudaStream_t st);
int add_float_to_double(rmhmc_ctx* ctx, const float* in, double* out, size_t n, cudaStream_t st);
int axpby64(rmhmc_ctx* ctx, double a, const double* x, double b, const double* y, double* out, size_t n, cudaStream_t st);
// squared norm of a float64 field (deterministic float64 sum)
int norm2_64(rmhmc_ctx* ctx, const double* x, size_t n, double* out, cudaStream_t st);

// mass-term helper shared by the solve, the kinetic force and the trajectory
struct MassTerm {
    double c = 1.0, kappa = 0.0;
    std::vector<double> alpha, sigma;
    int npole() const { return (int)alpha.size(); }
};
int parse_mass(rmhmc_ctx* ctx, const rmhmc_mass* m, MassTerm& out);

// Solve every shift of the mass term to relative true residual tol (float64 check) for one field b
// (device float64).  prec FP64 or MIXED.  xs: device float64 [npole][V][4][8] (workspace or caller).
int solve_shifts(rmhmc_ctx* ctx, const MassTerm& m, const double* b, double tol, int maxiter, int prec, double* xs,
                 int* iters, double* resid, cudaStream_t st);

// Kinetic pieces from one Krylov run on P: F_K (float64, nullable), velocity M^{-1}P (float64, nullable),
// T = 1/2 |R P|^2 from the same (unrefined) basis (nullable).  Links: the context's current links.
int kinetic_from_krylov(rmhmc_ctx* ctx, const MassTerm& m, const double* P, double tol, int maxiter, int prec,
                        double* F, double* Vel, double* T, int* iters, cudaStream_t st);

// CUDA-graph pieces: handles and WHILE nodes at the capture point of a stream; the captured mixed-precision
// kinetic evaluation (all decisions on the device); kinetic_graph_prepare allocates its buffers and tunes
// the stencil before any capture
int capture_handle(rmhmc_ctx* ctx, cudaStream_t st, unsigned init, cudaGraphConditionalHandle* h);
int capture_while(rmhmc_ctx* ctx, cudaStream_t st, cudaGraphConditionalHandle h, cudaGraph_t* body);
int kinetic_graph_prepare(rmhmc_ctx* ctx, const MassTerm& m, int maxiter);
int kinetic_enqueue(rmhmc_ctx* ctx, const MassTerm& m, const double* P, double tol, int maxiter, double* F, double* Vel,
                    long long* stats, int* status, cudaStream_t st, cudaStream_t aux);

// 1/R(lam) = inv.c + p1 lam + sum_j inv.alpha_j / (lam + inv.sigma_j) for a mass term with c >= 0, alpha_j >= 0
int inverse_rational(rmhmc_ctx* ctx, const MassTerm& m, MassTerm& inv, double& p1);
// momentum heatbath P = m(A) R(A) xi, m(A) = (1-kappa) + kappa A (float64 in and out)
int heatbath_apply(rmhmc_ctx* ctx, const MassTerm& m, const double* xi, double tol, int maxiter, int prec, double* P,
                   cudaStream_t st);
// Y = R(A) b (float64), every shift solved to relative true residual tol
int rational_apply(rmhmc_ctx* ctx, const MassTerm& m, const double* b, double tol, int maxiter, int prec, double* Y,
                   int* iters, cudaStream_t st);

}  // namespace rm
