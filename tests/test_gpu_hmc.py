"""GPU parity of the RMHMC trajectory pieces: Philox momenta, the exponential link update, the
implicit leapfrog and the full trajectory; reversibility, dH ~ dtau^2, mixed vs float64 dH."""
import numpy as np
import pytest

import oracle
from gpu_util import dev, host, rel_l2, torch_cuda
from oracle import fit
from paper_2112_04556_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_gauss_field_matches_oracle():
    import paper_2112_04556_gb300 as rm
    L = (4, 4, 4, 6)
    ref = oracle.gauss_field(L, 12345, 7, 0)
    with rm.Context(L) as ctx:
        g = host(rm.gauss_field(ctx, 12345, 7, 0))
    assert np.abs(g - ref).max() <= 1e-13


@pytest.mark.parametrize("eps", [1e-3, 0.05, 0.7, 3.0])
def test_link_update_matches_oracle(eps):
    import paper_2112_04556_gb300 as rm
    L = (4, 4, 4, 4)
    U = inputs.random_links(L, eps=0.5, seed=50)
    V = inputs.gaussian_fields(L, 1, seed=51)[0]
    ref = oracle.link_update(L, U, V, eps)
    with rm.Context(L) as ctx:
        out = host(rm.link_update(ctx, dev(U), dev(V), eps, reunit=False))
        assert np.abs(out - ref).max() <= 1e-13
        out2 = host(rm.link_update(ctx, dev(U), dev(V), eps, reunit=True))
        assert np.abs(out2 - ref).max() <= 1e-13


@pytest.mark.parametrize("eps,unit", [(1e-3, False), (0.05, False), (0.2, False), (0.7, False), (0.05, True)])
def test_link_update_float_float_and_float64(eps, unit):
    """The float-float link update (the default) and the float64 one both match the oracle to 1e-13 and each
    other to 2e-14 (float pairs carry 48-49 significant bits, and an update chains a few dozen dependent
    float-float operations), with and without reunitarisation; at eps = 0.7 most links rotate far enough to take the
    float64 branch inside the float-float kernel.  Unit links (exact zeros and ones, whose float pairs come
    from the zero-exponent and exact-power cases of the bit-field split) and momenta with exact zeros and a
    tiny coefficient are included."""
    import paper_2112_04556_gb300 as rm
    L = (6, 4, 4, 5)
    U = inputs.unit_links(L) if unit else inputs.random_links(L, eps=0.5, seed=52)
    V = inputs.gaussian_fields(L, 1, seed=53)[0]
    if unit:
        V[::3, :, 2] = 0.0
        V[1::7, 1, 5] = 3e-30
    ref = oracle.link_update(L, U, V, eps)
    out = {}
    with rm.Context(L) as ctx:
        for mode in (1, 0):
            rm.set_stencil_shape(ctx, rm.SHAPE_LINKUPDATE, rm.FP64, 18, mode, 128)
            for reunit in (False, True):
                out[(mode, reunit)] = host(rm.link_update(ctx, dev(U), dev(V), eps, reunit=reunit))
        with pytest.raises(rm.RmhmcError):
            rm.set_stencil_shape(ctx, rm.SHAPE_LINKUPDATE, rm.FP32, 18, 1, 128)
    for key, o in out.items():
        assert np.abs(o - ref).max() <= 1e-13, key
    for reunit in (False, True):
        assert np.abs(out[(1, reunit)] - out[(0, reunit)]).max() <= 2e-14


def test_float64_trajectory_keeps_float64_link_update():
    """The float-float link update serves the mixed-precision trajectories only: a float64 trajectory gives the
    same bits whether it is enabled (the default) or float64 is pinned; a mixed one stays within the fixed-point
    tolerance of its float64-update twin."""
    import paper_2112_04556_gb300 as rm
    L = (4, 4, 4, 4)
    U = inputs.random_links(L, eps=0.3, seed=61)
    P = inputs.gaussian_fields(L, 1, seed=62)[0]
    m = fit.mass_term(6, 0.9)
    res = {}
    for prec, kw in ((rm.FP64, {}), (rm.MIXED, dict(tol_md=1e-7, fp_tol=1e-6, fp_extra=2))):
        for mode in (1, 0):
            with rm.Context(L) as ctx:
                rm.set_stencil_shape(ctx, rm.SHAPE_LINKUPDATE, rm.FP64, 18, mode, 128)
                Ud, Pd = dev(U), dev(P)
                rm.md(ctx, Ud, Pd, _params(rm, m, nsteps=3, prec=prec, **kw))
                res[(prec, mode)] = (host(Ud), host(Pd))
    for i in range(2):
        assert np.array_equal(res[(rm.FP64, 1)][i], res[(rm.FP64, 0)][i])
        assert np.abs(res[(rm.MIXED, 1)][i] - res[(rm.MIXED, 0)][i]).max() <= 1e-5


def _params(rm, mass, **kw):
    d = dict(beta=6.0, c1=0.0, mass=mass, tau=0.2, nsteps=4, tol_md=1e-13, tol_h=1e-13, fp_tol=1e-13,
             fp_maxit=100, maxiter=2000, prec=rm.FP64, seed=3, traj_index=0, metropolis=True)
    d.update(kw)
    return rm.make_params(**d)


@pytest.mark.parametrize("L,npole,c1", [((2, 2, 2, 4), 12, 0.0), ((4, 4, 4, 4), 6, -0.331)])
def test_md_parity(L, npole, c1):
    import paper_2112_04556_gb300 as rm
    U = inputs.random_links(L, eps=0.3, seed=52)
    P = inputs.gaussian_fields(L, 1, seed=53)[0]
    m = fit.mass_term(npole, 0.9)
    U_ref, P_ref, its = oracle.md_trajectory(L, U, P, 0.2, 3, 6.0, c1, m, tol=1e-14, fp_tol=1e-13)
    with rm.Context(L) as ctx:
        Ud, Pd = dev(U), dev(P)
        r = rm.md(ctx, Ud, Pd, _params(rm, m, c1=c1, nsteps=3))
    assert np.abs(host(Ud) - U_ref).max() <= 1e-11
    assert rel_l2(host(Pd), P_ref) <= 1e-10
    assert r["fp_iters_p"] > 0 and r["fp_iters_u"] > 0


def test_trajectory_parity():
    import paper_2112_04556_gb300 as rm
    L = (4, 4, 4, 4)
    U = inputs.random_links(L, eps=0.3, seed=54)
    xi = inputs.gaussian_fields(L, 1, seed=55)[0]
    m = fit.mass_term(8, 0.9)
    ref = oracle.trajectory(L, U, xi, 0.5, 0.2, 4, 6.0, 0.0, m, tol_md=1e-14, tol_h=1e-14, fp_tol=1e-13)
    with rm.Context(L) as ctx:
        Ud = dev(U)
        r = rm.rmhmc_trajectory(ctx, Ud, _params(rm, m), xi=dev(xi))
    assert abs(r["H0"] - ref["H0"]) <= 1e-12 * abs(ref["H0"])
    assert abs(r["dH"] - ref["dH"]) <= 1e-8
    assert abs(r["plaq"] - ref["plaq"]) <= 1e-12
    if r["accepted"] == ref["accepted"]:
        assert np.abs(host(Ud) - ref["U"]).max() <= 1e-11


def test_identity_mass_trajectory_is_plain_hmc():
    import paper_2112_04556_gb300 as rm
    L = (4, 4, 4, 4)
    U = inputs.random_links(L, eps=0.3, seed=56)
    xi = oracle.gauss_field(L, 3, 0, 0)
    ref = oracle.trajectory(L, U, xi, oracle.uniform(3, 0), 1.0, 10, 6.0, 0.0, oracle.identity_mass())
    with rm.Context(L) as ctx:
        Ud = dev(U)
        r = rm.rmhmc_trajectory(ctx, Ud, _params(rm, {"c": 1.0, "alpha": [], "sigma": []}, tau=1.0, nsteps=10))
    assert abs(r["u"] - oracle.uniform(3, 0)) == 0.0
    assert abs(r["dH"] - ref["dH"]) <= 1e-9 and r["accepted"] == ref["accepted"]
    assert np.abs(host(Ud) - ref["U"]).max() <= 1e-11


def test_reversibility_gpu():
    import paper_2112_04556_gb300 as rm
    L = (6, 6, 6, 6)
    U = inputs.random_links(L, eps=0.3, seed=57)
    P = inputs.gaussian_fields(L, 1, seed=58)[0]
    m = rm.mass_fit(12, 0.9)
    with rm.Context(L) as ctx:
        Ud, Pd = dev(U), dev(P)
        p = _params(rm, m, tau=0.3, nsteps=3)
        rm.md(ctx, Ud, Pd, p)
        Pd.neg_()
        rm.md(ctx, Ud, Pd, p)
    assert np.abs(host(Ud) - U).max() <= 1e-10
    assert np.abs(host(Pd) + P).max() <= 1e-9


def test_dH_scales_with_step_squared():
    import paper_2112_04556_gb300 as rm
    L = (6, 6, 6, 6)
    U = inputs.random_links(L, eps=0.3, seed=59)
    xi = inputs.gaussian_fields(L, 1, seed=60)[0]
    m = rm.mass_fit(12, 0.9)
    dH = []
    with rm.Context(L) as ctx:
        for n in (4, 8):
            r = rm.rmhmc_trajectory(ctx, dev(U), _params(rm, m, tau=0.4, nsteps=n, tol_md=1e-12, fp_tol=1e-12,
                                                          metropolis=False), xi=dev(xi))
            dH.append(r["dH"])
    assert 3.0 < dH[0] / dH[1] < 5.0, dH


def test_mixed_vs_fp64_dH_16_4():
    """16^4 oracle-HMC links (beta = 6.0), step size with dH = O(1): the mixed-precision trajectory
    reproduces the float64 one, |dH_mixed - dH_fp64| <= 1e-3, from the same links and momenta."""
    import paper_2112_04556_gb300 as rm
    from conftest import config2_links
    L = (16, 16, 16, 16)
    U = config2_links()
    m = rm.mass_fit(12, 0.9)
    out = {}
    with rm.Context(L) as ctx:
        for prec in (rm.FP64, rm.MIXED):
            Ud = dev(U)
            r = rm.rmhmc_trajectory(ctx, Ud, _params(rm, m, tau=0.5, nsteps=40, prec=prec, tol_md=1e-10 if prec == 0 else 1e-6,
                                                     tol_h=1e-12, fp_tol=1e-10 if prec == 0 else 1e-6, metropolis=False))
            out[prec] = (r, host(Ud))
    assert abs(out[1][0]["dH"] - out[0][0]["dH"]) <= 1e-3, (out[0][0]["dH"], out[1][0]["dH"])
    assert abs(out[0][0]["dH"]) < 10.0, out[0][0]["dH"]      # thermalised links, small steps: dH = O(1)
    assert abs(out[1][0]["plaq"] - out[0][0]["plaq"]) <= 1e-6
    assert abs(out[1][0]["H0"] - out[0][0]["H0"]) <= 1e-9 * abs(out[0][0]["H0"])


def test_fp_extra_iterations_graph_and_host():
    """fp_extra: each fixed point runs exactly fp_extra iterations past its first convergence (the iterates are
    deterministic, so the counts add 2 x fp_extra per step), the graph and host-driven MD agree bit for bit with
    and without it and with the float64 gauge force, and the extra iterations bring the mixed trajectory closer
    to the oracle's converged float64 one."""
    import paper_2112_04556_gb300 as rm
    L = (6, 4, 4, 8)
    U = inputs.random_links(L, eps=0.3, seed=71)
    m = fit.mass_term(12, 0.9)
    xi = oracle.gauss_field(L, 3, 0, 0)
    ref = oracle.trajectory(L, U, xi, oracle.uniform(3, 0), 0.3, 3, 6.0, 0.0, m, tol_md=1e-13, tol_h=1e-13,
                            fp_tol=1e-13, metropolis=False)
    out = {}
    with rm.Context(L) as ctx:
        for extra in (0, 2):
            for fg in (False, True):
                for graphs in (True, False):
                    rm.set_graphs(ctx, graphs)
                    Ud = dev(U)
                    r = rm.rmhmc_trajectory(ctx, Ud, _params(rm, m, tau=0.3, nsteps=3, prec=rm.MIXED, tol_md=1e-6,
                                                             tol_h=1e-12, fp_tol=1e-6, fp_extra=extra, fg_fp64=fg,
                                                             metropolis=False))
                    out[(extra, fg, graphs)] = (r, host(Ud))
        rm.set_graphs(ctx, True)
        with pytest.raises(rm.RmhmcError):
            rm.rmhmc_trajectory(ctx, dev(U), _params(rm, m, prec=rm.MIXED, fp_extra=100, fp_maxit=100))
    for extra in (0, 2):
        for fg in (False, True):
            a, b = out[(extra, fg, True)], out[(extra, fg, False)]
            assert a[0]["dH"] == b[0]["dH"] and np.array_equal(a[1], b[1])
            assert a[0]["fp_iters_p"] == b[0]["fp_iters_p"] and a[0]["fp_iters_u"] == b[0]["fp_iters_u"]
    for fg in (False, True):
        r0, r2 = out[(0, fg, True)][0], out[(2, fg, True)][0]
        assert r2["fp_iters_p"] == r0["fp_iters_p"] + 2 * 3 and r2["fp_iters_u"] == r0["fp_iters_u"] + 2 * 3
    for key in out:
        assert np.abs(out[key][1] - ref["U1"]).max() < 2e-6, key
        assert abs(out[key][0]["dH"] - ref["dH"]) < 1e-4, key


def test_trajectory_errors_leave_links_unchanged():
    import paper_2112_04556_gb300 as rm
    L = (4, 4, 4, 4)
    U = inputs.random_links(L, eps=0.3, seed=61)
    with rm.Context(L) as ctx:
        Ud = dev(U)
        with pytest.raises(rm.RmhmcError) as e:
            rm.rmhmc_trajectory(ctx, Ud, _params(rm, rm.mass_fit(12, 0.9), fp_maxit=1, fp_tol=1e-15))
        assert e.value.code == rm.ENOCONV
        assert np.abs(host(Ud) - U).max() == 0.0
        with pytest.raises(rm.RmhmcError):
            rm.rmhmc_trajectory(ctx, Ud, _params(rm, rm.mass_fit(12, 0.9), nsteps=0))


def _logdet_params(rm, m, prec, **kw):
    d = dict(beta=6.0, c1=0.0, mass=m, tau=0.2, nsteps=4, tol_md=1e-13 if prec == 0 else 1e-6,
             tol_h=1e-13 if prec == 0 else 1e-12, fp_tol=1e-13 if prec == 0 else 1e-6, fp_maxit=100,
             maxiter=2000, prec=prec, seed=5, traj_index=2, metropolis=False, logdet=True)
    d.update(kw)
    return rm.make_params(**d)


def test_logdet_trajectory_parity():
    """The log|M| term through the auxiliary field: float64 trajectory against the oracle's with the same
    Philox noise (xi tag 0, eta tag 3); A0 = |eta|^2 / 2."""
    import paper_2112_04556_gb300 as rm
    L = (4, 4, 4, 4)
    U = inputs.random_links(L, eps=0.3, seed=65)
    m = fit.mass_term(8, 0.9)
    xi = oracle.gauss_field(L, 5, 2, 0)
    eta = oracle.gauss_field(L, 5, 2, 3)
    ref = oracle.trajectory(L, U, xi, oracle.uniform(5, 2), 0.2, 4, 6.0, 0.0, m, tol_md=1e-13, tol_h=1e-13,
                            fp_tol=1e-13, metropolis=False, eta=eta)
    with rm.Context(L) as ctx:
        Ud = dev(U)
        r = rm.rmhmc_trajectory(ctx, Ud, _logdet_params(rm, m, rm.FP64))
        Uo = host(Ud)
    assert abs(r["A0"] - 0.5 * np.sum(eta * eta)) <= 1e-10 * r["A0"]
    assert abs(r["A0"] - ref["A0"]) <= 1e-10 * ref["A0"] and abs(r["A1"] - ref["A1"]) <= 1e-10 * ref["A1"]
    assert abs(r["dH"] - ref["dH"]) <= 1e-8
    assert np.abs(Uo - ref["U1"]).max() <= 1e-10


def test_logdet_mixed_graph_and_host_agree_with_fp64():
    """8^4: the mixed trajectory with the auxiliary field, captured as a graph and host-driven, against
    float64 (small step: dH = O(1e-2))."""
    import paper_2112_04556_gb300 as rm
    L = (8, 8, 8, 8)
    U = inputs.random_links(L, eps=0.3, seed=66)
    m = rm.mass_fit(12, 0.9)
    out = {}
    with rm.Context(L) as ctx:
        out["fp64"] = rm.rmhmc_trajectory(ctx, dev(U), _logdet_params(rm, m, rm.FP64, tol_md=1e-10, fp_tol=1e-10))
        out["graph"] = rm.rmhmc_trajectory(ctx, dev(U), _logdet_params(rm, m, rm.MIXED))
        note = rm.tuning(ctx)
        rm.set_graphs(ctx, False)
        out["host"] = rm.rmhmc_trajectory(ctx, dev(U), _logdet_params(rm, m, rm.MIXED))
    assert "md graph captured" in note
    assert abs(out["graph"]["dH"] - out["host"]["dH"]) <= 1e-6
    assert abs(out["graph"]["dH"] - out["fp64"]["dH"]) <= 1e-3
    assert abs(out["fp64"]["A0"] - out["graph"]["A0"]) <= 1e-9 * out["fp64"]["A0"]


@pytest.mark.parametrize("L,npole,c1", [((2, 2, 2, 4), 12, 0.0), ((4, 4, 4, 4), 6, -0.331)])
def test_symplectic_md_parity(L, npole, c1):
    """The exactly symplectic form of the step (momenta through dexp of the link rotation), float64,
    against the oracle's symplectic_step."""
    import paper_2112_04556_gb300 as rm
    U = inputs.random_links(L, eps=0.3, seed=52)
    P = inputs.gaussian_fields(L, 1, seed=53)[0]
    m = fit.mass_term(npole, 0.9)
    U_ref, P_ref, its = oracle.md_trajectory(L, U, P, 0.2, 3, 6.0, c1, m, tol=1e-14, fp_tol=1e-13, symplectic=True)
    U_lf, P_lf, _ = oracle.md_trajectory(L, U, P, 0.2, 3, 6.0, c1, m, tol=1e-14, fp_tol=1e-13)
    with rm.Context(L) as ctx:
        Ud, Pd = dev(U), dev(P)
        r = rm.md(ctx, Ud, Pd, _params(rm, m, c1=c1, nsteps=3, symplectic=True))
    assert np.abs(host(Ud) - U_ref).max() <= 1e-11
    assert rel_l2(host(Pd), P_ref) <= 1e-10
    assert rel_l2(P_lf, P_ref) > 1e-4          # the two forms differ at O(eps) in the momenta
    assert r["fp_iters_p"] > 0 and r["fp_iters_u"] > 0


def test_symplectic_mixed_against_fp64_and_reversible():
    """8^4, mixed precision (float32 Krylov, forces and dexp series; host-driven): the trajectory's dH
    follows the float64 one, and forward, momentum flip, forward returns to the start."""
    import paper_2112_04556_gb300 as rm
    L = (8, 8, 8, 8)
    U = inputs.random_links(L, eps=0.3, seed=75)
    xi = inputs.gaussian_fields(L, 1, seed=76)[0]
    P = inputs.gaussian_fields(L, 1, seed=77)[0]
    m = rm.mass_fit(12, 0.9)
    with rm.Context(L) as ctx:
        out = {}
        for prec in (rm.FP64, rm.MIXED):
            tol = 1e-11 if prec == rm.FP64 else 1e-7
            out[prec] = rm.rmhmc_trajectory(ctx, dev(U), _params(rm, m, tau=0.2, nsteps=4, prec=prec, tol_md=tol,
                                                                 fp_tol=tol, metropolis=False, symplectic=True),
                                            xi=dev(xi))
        Ud, Pd = dev(U), dev(P)
        p = _params(rm, m, tau=0.2, nsteps=4, prec=rm.MIXED, tol_md=1e-7, fp_tol=1e-7, symplectic=True)
        rm.md(ctx, Ud, Pd, p)
        Pd.neg_()
        rm.md(ctx, Ud, Pd, p)
        note = rm.tuning(ctx)
    assert abs(out[rm.MIXED]["dH"] - out[rm.FP64]["dH"]) <= 1e-3, (out[rm.FP64]["dH"], out[rm.MIXED]["dH"])
    assert np.abs(host(Ud) - U).max() <= 1e-5
    assert np.abs(host(Pd) + P).max() <= 1e-4
    assert "md graph captured" not in note      # the symplectic form runs host-driven
