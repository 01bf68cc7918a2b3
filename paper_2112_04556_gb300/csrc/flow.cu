// Wilson gradient flow and the flowed energy, the long-distance observable of Sec. 4 (the paper takes its
// definition from Luscher, JHEP 08 (2010) 071).  The flow dV/dt = -g0^2 (dS_W) V is integrated with
// Luscher's third-order Runge-Kutta scheme
//   W1 = exp(Z0/4) W0,  W2 = exp(8/9 Z1 - 17/36 Z0) W1,  W3 = exp(3/4 Z2 - 8/9 Z1 + 17/36 Z0) W2,
// Z_i = eps Z(W_i).  With U -> exp(i w^a T^a) U and F = -dS/dw the flow velocity is i g0^2 F^a T^a, and
// g0^2 F = 6 F(beta = 1): each stage is one gauge-force launch at beta = 1 (Wilson), float64 field
// combinations, and one float64 link update exp(i 6 eps Z) W on the device.  E is the plaquette energy
// density 36 (1 - <Re Tr P / 3>) from the deterministic float64 action reduction.
#include <math.h>

#include "krylov.cuh"
#include "ops.cuh"

using namespace rm;

extern "C" int wilson_flow(rmhmc_ctx* ctx, double* U, double eps, int nsteps, int prec, double* E, cudaStream_t stream) {
    if (!ctx) return RMHMC_EINVAL;
    ctx->err.clear();
    if (!U) return set_err(ctx, RMHMC_EINVAL, "wilson_flow: null links");
    if (nsteps < 0 || !isfinite(eps)) return set_err(ctx, RMHMC_EINVAL, "wilson_flow: bad step size or count");
    if (prec != RMHMC_FP64 && prec != RMHMC_MIXED) return set_err(ctx, RMHMC_EINVAL, "wilson_flow: bad prec");
    if ((uintptr_t)U % 16) return set_err(ctx, RMHMC_EINVAL, "wilson_flow: links must be 16-byte aligned");
    const size_t fs = field_elems(ctx), ls = (size_t)ctx->g.V * 72;
    const int gprec = prec == RMHMC_FP64 ? RMHMC_FP64 : RMHMC_FP32;
    int status = RMHMC_OK;
    double* Z0 = (double*)workspace(ctx, "wf_z0", sizeof(double) * fs, &status);
    double* Z1 = (double*)workspace(ctx, "wf_z1", sizeof(double) * fs, &status);
    double* Z2 = (double*)workspace(ctx, "wf_z2", sizeof(double) * fs, &status);
    double* Zc = (double*)workspace(ctx, "wf_zc", sizeof(double) * fs, &status);
    double* W = (double*)workspace(ctx, "wf_w", sizeof(double) * ls, &status);
    if (!Z0 || !Z1 || !Z2 || !Zc || !W) return status;
    RM_TRY(import_links(ctx, U, stream));
    auto energy = [&](double* out) -> int {
        double S = 0.0, plaq = 0.0;
        RM_TRY(action_launch(ctx, 1.0, 0.0, &S, &plaq, stream));
        *out = 36.0 * (1.0 - plaq);
        return RMHMC_OK;
    };
    if (E) RM_TRY(energy(E));
    const double g2 = 6.0;   // g0^2 F = 6 F(beta = 1)
    for (int n = 0; n < nsteps; n++) {
        RM_TRY(gauge_force_launch(ctx, 1.0, 0.0, gprec, Z0, stream));
        RM_TRY(link_update_launch(ctx, U, Z0, 0.25 * g2 * eps, false, W, nullptr, nullptr, true, false, stream));
        RM_TRY(gauge_force_launch(ctx, 1.0, 0.0, gprec, Z1, stream));
        RM_TRY(axpby64(ctx, 8.0 / 9.0, Z1, -17.0 / 36.0, Z0, Zc, fs, stream));
        RM_TRY(link_update_launch(ctx, W, Zc, g2 * eps, false, W, nullptr, nullptr, true, false, stream));
        RM_TRY(gauge_force_launch(ctx, 1.0, 0.0, gprec, Z2, stream));
        RM_TRY(axpby64(ctx, 0.75, Z2, -8.0 / 9.0, Z1, Zc, fs, stream));
        RM_TRY(axpby64(ctx, 1.0, Zc, 17.0 / 36.0, Z0, Zc, fs, stream));
        RM_TRY(link_update_launch(ctx, W, Zc, g2 * eps, false, U, nullptr, nullptr, true, false, stream));
        if (E) RM_TRY(energy(E + n + 1));
    }
    RM_CHECK(ctx, cudaStreamSynchronize(stream));
    return RMHMC_OK;
}
