"""The accuracy bar of the mixed-precision path at the benchmark's lattice: from the benchmark's thermalised
32^4 links and its trajectory momenta, a mixed trajectory at tau = 1 in 40 steps (the benchmark's mixed
settings) ends within 1e-3 of the float64 one in dH (the Hamiltonian of Sec. 3, Eq. 5), and is faster.
At the workload's own 20 steps the integrator is near its stability edge (dH ~ 196) and amplifies float32
rounding beyond the bar; the benchmark reports that pair too.  Takes about three minutes (the float64
trajectory)."""
import time

import pytest

from gpu_util import torch_cuda
from paper_2112_04556_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_mixed_vs_fp64_dH_bar_32_4():
    import bench
    import paper_2112_04556_gb300 as rm
    torch = torch_cuda()
    L = (32, 32, 32, 32)
    seeds = bench.replica_seeds(0)
    ident = {"c": 1.0, "alpha": [], "sigma": [], "kappa": 0.0}
    out = {}
    with rm.Context(L) as ctx:
        # fixed launch shapes, so that the float32 rounding does not depend on the autotuner's timing
        rm.set_stencil_shape(ctx, rm.SHAPE_LAP, rm.FP32, 18, 1, 256)
        rm.set_stencil_shape(ctx, rm.SHAPE_CG, rm.FP32, 18, 1, 256)
        rm.set_stencil_shape(ctx, rm.SHAPE_ADJOINT, rm.FP32, 18, 3, 0)
        U = torch.from_numpy(inputs.random_links(L, eps=0.3, seed=seeds["links"])).cuda()
        for n in range(20):   # the benchmark's plain-HMC thermalisation
            p = rm.make_params(beta=bench.BETA, mass=ident, tau=1.0, nsteps=20, tol_md=1e-6, tol_h=1e-11,
                               fp_tol=1e-6, prec=rm.MIXED, seed=seeds["therm"], traj_index=1000 + n,
                               metropolis=False)
            rm.rmhmc_trajectory(ctx, U, p)
        mass = rm.mass_fit(bench.NPOLE, bench.KAPPA)
        for prec in (rm.FP64, rm.MIXED):
            mixed = prec == rm.MIXED
            p = rm.make_params(beta=bench.BETA, mass=mass, tau=bench.TAU, nsteps=bench.PAIR_NSTEPS,
                               tol_md=bench.MIXED_TOL_MD if mixed else bench.FP64_TOL, tol_h=1e-12,
                               fp_tol=bench.MIXED_FP_TOL if mixed else bench.FP64_TOL,
                               fp_extra=bench.MIXED_FP_EXTRA if mixed else 0, fp_maxit=50, maxiter=400, prec=prec,
                               seed=seeds["traj"], traj_index=0, metropolis=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = rm.rmhmc_trajectory(ctx, U.clone(), p)
            torch.cuda.synchronize()
            r["seconds"] = time.perf_counter() - t0
            out[prec] = r
    a, b = out[rm.FP64], out[rm.MIXED]
    print("dH float64 %.6f (%.1f s), mixed %.6f (%.2f s)" % (a["dH"], a["seconds"], b["dH"], b["seconds"]))
    assert abs(a["dH"]) < 5.0, a["dH"]                        # an accepting step size
    assert abs(b["dH"] - a["dH"]) <= bench.DH_BAR, (a["dH"], b["dH"])
    assert abs(b["plaq"] - a["plaq"]) <= 1e-6
    assert b["seconds"] < a["seconds"] / 10
