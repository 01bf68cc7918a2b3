// Internal launchers shared between translation units (not part of the C ABI).
#pragma once
#include "common.cuh"

namespace rm {

// Y = a X + b H(X) + c W for nfield fields (prec: RMHMC_FP64 double, else float); if slot >= 0,
// per-field float64 sums {<Y,Y>, <Y,X>} land in reduction slots slot .. slot+nfield-1.
int launch_lap(rmhmc_ctx* ctx, int prec, int linkfmt, const void* X, void* Y, int nfield, double a, double b,
               const void* W, double c, int slot, cudaStream_t st);

// the same for float32 fields in the adjoint form (lap_ad.cu): each link becomes its 8x8 adjoint matrix once per
// application, shared by all fields; dots as launch_lap
int launch_lap_ad(rmhmc_ctx* ctx, int linkfmt, const float* X, float* Y, int nfield, double a, double b, const float* W,
                  double c, int slot, cudaStream_t st);
// the link-centric adjoint stencil (lap_lc.cu), float32, one field: Y = a X + b H(X); and the CG stencil
// q = diag r_k + (-1/16) H(r_k) + beta q (k from flags[1], as the gather kernel of krylov.cu)
int launch_lap_lc(rmhmc_ctx* ctx, int linkfmt, const float* X, float* Y, double a, double b, cudaStream_t st);
int launch_cg_lc(rmhmc_ctx* ctx, const float* R, float* q, double diag, const int* flags, double* vals, int maxit,
                 double* partials, unsigned* counter, cudaStream_t st);
// fewest fields for which launch_lap takes the adjoint form
constexpr int kAdMinFields = 6;

// gauge force F = -dS/dw (float64 output; arithmetic float64 or float32) from the context's links
int gauge_force_launch(rmhmc_ctx* ctx, double beta, double c1, int prec, double* F, cudaStream_t st);
// action S and average plaquette (float64, deterministic) from the context's float64 links
int action_launch(rmhmc_ctx* ctx, double beta, double c1, double* S, double* plaq, cudaStream_t st);
// G = sum_f w_f d<Z_f, A X_f>/dw (X, Z in the arithmetic precision, [nf][V][4][8]); G float64 [V][4][8]
int link_grad_launch(rmhmc_ctx* ctx, int prec, const void* X, const void* Z, int nf, const double* w, double* G,
                     cudaStream_t st);
// Uout = exp(i eps V) Uin per link (float64, canonical [V][4][3][3]; in place allowed), optionally reunitarised;
// with Wold, max |Uout - Wold| into *dmax; internal refreshes the context's link copies from Uout
// ff: the float-float kernel may be used (when it is enabled, ctx->link_update_ff); the float64 trajectories
// and the gradient flow pass false and stay in float64 throughout
int link_update_launch(rmhmc_ctx* ctx, const double* Uin, const double* V, double eps, bool reunit, double* Uout,
                       const double* Wold, double* dmax, bool internal, bool ff, cudaStream_t st);
// kinetic force G = sum_j alpha_j d<Z_j, A X_j>/dw straight from the float32 Krylov basis R (n vectors), with
// X_j, Z_j given as rows of basis coefficients (rows j and ns + j, row stride ldr, device float64); n is
// read on the device from flags[1] when flags is not null.  G float64 [V][4][8].
int link_grad_krylov_launch(rmhmc_ctx* ctx, const float* R, const double* rows, int ldr, int ns, const double* alpha,
                            const int* flags, int n, double* G, cudaStream_t st);

}  // namespace rm
