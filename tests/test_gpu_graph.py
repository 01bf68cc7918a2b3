"""The mixed-precision molecular dynamics as one CUDA graph (conditional WHILE nodes for both implicit fixed
points and every Krylov run, decided on the device) against the host-driven path on the same inputs."""
import numpy as np
import pytest

from gpu_util import dev, host, rel_l2, torch_cuda
from paper_2112_04556_gb300 import inputs

pytestmark = pytest.mark.gpu


def _params(rm, m, **kw):
    d = dict(beta=6.0, c1=0.0, mass=m, tau=0.2, nsteps=4, tol_md=1e-6, tol_h=1e-12, fp_tol=1e-6, fp_maxit=50,
             maxiter=400, prec=rm.MIXED, seed=5, traj_index=0, metropolis=False)
    d.update(kw)
    return rm.make_params(**d)


@pytest.mark.parametrize("L,c1", [((8, 8, 8, 8), 0.0), ((6, 4, 6, 8), -0.331)])
def test_md_graph_matches_host_driven(L, c1):
    import paper_2112_04556_gb300 as rm
    U = inputs.random_links(L, eps=0.3, seed=71)
    P = inputs.gaussian_fields(L, 1, seed=72)[0]
    m = rm.mass_fit(12, 0.9)
    out = {}
    for graphs in (False, True):
        with rm.Context(L) as ctx:
            rm.set_graphs(ctx, graphs)
            Ud, Pd = dev(U), dev(P)
            r = rm.md(ctx, Ud, Pd, _params(rm, m, c1=c1))
            out[graphs] = (host(Ud), host(Pd), r, rm.tuning(ctx))
    assert "md graph captured" in out[True][3], out[True][3]
    assert np.abs(out[True][0] - out[False][0]).max() <= 1e-9
    assert rel_l2(out[True][1], out[False][1]) <= 1e-8
    assert out[True][2]["fp_iters_p"] == out[False][2]["fp_iters_p"]
    assert out[True][2]["fp_iters_u"] == out[False][2]["fp_iters_u"]
    assert abs(out[True][2]["md_iters"] - out[False][2]["md_iters"]) <= 2


def test_trajectory_graph_reused_and_reversible():
    """The cached graph is reused across trajectories; forward, momentum flip, forward returns to the start."""
    import paper_2112_04556_gb300 as rm
    L = (8, 8, 8, 8)
    U = inputs.random_links(L, eps=0.3, seed=73)
    P = inputs.gaussian_fields(L, 1, seed=74)[0]
    m = rm.mass_fit(12, 0.9)
    with rm.Context(L) as ctx:
        Ud, Pd = dev(U), dev(P)
        p = _params(rm, m, tol_md=1e-7, fp_tol=1e-7)
        rm.md(ctx, Ud, Pd, p)
        Pd.neg_()
        rm.md(ctx, Ud, Pd, p)
        assert "md graph captured" in rm.tuning(ctx)
        assert np.abs(host(Ud) - U).max() <= 1e-5
        for k in range(3):
            r = rm.rmhmc_trajectory(ctx, Ud, _params(rm, m, traj_index=k))
            assert np.isfinite(r["dH"]) and r["md_iters"] > 0


def test_graph_fixed_point_cap_reports_noconv():
    import paper_2112_04556_gb300 as rm
    L = (4, 4, 4, 4)
    U = inputs.random_links(L, eps=0.3, seed=75)
    P = inputs.gaussian_fields(L, 1, seed=76)[0]
    with rm.Context(L) as ctx:
        with pytest.raises(rm.RmhmcError) as e:
            rm.md(ctx, dev(U), dev(P), _params(rm, rm.mass_fit(12, 0.9), fp_maxit=1, fp_tol=1e-15))
        assert e.value.code == rm.ENOCONV
