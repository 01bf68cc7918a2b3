// Internal launchers shared between translation units (not part of the C ABI).
#pragma once
#include "common.cuh"

namespace rm {

// Y = a X + b H(X) + c W for nfield fields (prec: RMHMC_FP64 double, else float); if slot >= 0,
// per-field float64 sums {<Y,Y>, <Y,X>} land in reduction slots slot .. slot+nfield-1.
int launch_lap(rmhmc_ctx* ctx, int prec, int linkfmt, const void* X, void* Y, int nfield, double a, double b,
               const void* W, double c, int slot, cudaStream_t st);

}  // namespace rm
