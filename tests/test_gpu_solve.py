"""GPU parity of the rational mass term (rat_mass_solve, heatbath) against the oracle."""
import numpy as np
import pytest

import oracle
from gpu_util import dev, host, rel_l2, torch_cuda
from oracle import fit
from paper_2112_04556_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (5, 3, 4, 7)])
@pytest.mark.parametrize("prec,tol,bound", [(0, 1e-12, 1e-11), (1, 1e-10, 1e-9), (1, 1e-12, 1e-11)])
def test_rat_mass_solve_parity(L, prec, tol, bound):
    import paper_2112_04556_gb300 as rm
    U = inputs.random_links(L, eps=0.5, seed=21)
    b = inputs.gaussian_fields(L, 1, seed=22)[0]
    m = fit.mass_term(12, 0.9)
    y_ref, xs_ref = oracle.rational_apply(L, U, b, m, tol=1e-14)
    with rm.Context(L) as ctx:
        y, xs, iters, resid = rm.rat_mass_solve(ctx, dev(U), dev(b), m, tol=tol, prec=prec, want_xs=True)
        assert np.all(resid <= tol), resid
        assert rel_l2(host(y), y_ref) <= bound
        for j in range(12):
            assert rel_l2(host(xs[j]), xs_ref[j]) <= 10 * bound
        assert iters > 0


@pytest.mark.parametrize("prec,tol,bound", [(0, 1e-12, 1e-11), (1, 1e-11, 1e-10)])
def test_rat_mass_solve_nfield(prec, tol, bound):
    """Three fields in one call (Sec. 3, Eq. 6 applied field by field): every y_f, every x_fj and the
    per-field residuals against the oracle's per-field rational_apply; iterations add up over fields."""
    import paper_2112_04556_gb300 as rm
    L = (5, 3, 4, 7)
    U = inputs.random_links(L, eps=0.5, seed=25)
    b = inputs.gaussian_fields(L, 3, seed=26)
    b[1] *= 1e-3                                # a small field: tol is relative to each field's own norm
    m = fit.mass_term(12, 0.9)
    with rm.Context(L) as ctx:
        y, xs, iters, resid = rm.rat_mass_solve(ctx, dev(U), dev(b), m, tol=tol, prec=prec, want_xs=True)
        assert resid.shape == (3, 12) and np.all(resid <= tol), resid
        single = [rm.rat_mass_solve(ctx, None, dev(b[f]), m, tol=tol, prec=prec)[2] for f in range(3)]
    assert iters == sum(single)
    for f in range(3):
        y_ref, xs_ref = oracle.rational_apply(L, U, b[f], m, tol=1e-14)
        assert rel_l2(host(y[f]), y_ref) <= bound, f
        for j in range(12):
            assert rel_l2(host(xs[f, j]), xs_ref[j]) <= 10 * bound, (f, j)


def test_single_shift_is_plain_cg():
    import paper_2112_04556_gb300 as rm
    L = (4, 4, 4, 6)
    U = inputs.random_links(L, eps=0.5, seed=23)
    b = inputs.gaussian_fields(L, 1, seed=24)[0]
    x_ref, _, _ = oracle.cg(lambda v: oracle.lap(L, U, v) + 0.3 * v, b, tol=1e-14)
    with rm.Context(L) as ctx:
        y, _, _, resid = rm.rat_mass_solve(ctx, dev(U), dev(b), {"c": 0.0, "alpha": [1.0], "sigma": [0.3]},
                                          tol=1e-13, prec=rm.FP64)
    assert rel_l2(host(y), x_ref) <= 1e-12 and resid[0] <= 1e-13


def test_free_field_plane_wave():
    """U = 1: R(A) T^a cos(k.x) = R(lambda_k) T^a cos(k.x) in both precisions."""
    import paper_2112_04556_gb300 as rm
    import helpers as H
    L = (4, 4, 4, 8)
    m = fit.mass_term(12, 0.9)
    X = H.plane_wave(L, (1, 2, 0, 3), 1, 6, 0.2)
    lam = H.free_eigenvalue(L, (1, 2, 0, 3))
    with rm.Context(L) as ctx:
        for prec, tol in ((0, 1e-13), (1, 1e-11)):
            y, _, _, _ = rm.rat_mass_solve(ctx, dev(inputs.unit_links(L)), dev(X), m, tol=tol, prec=prec)
            assert np.abs(host(y) - fit.evaluate(m, lam) * X).max() < 10 * tol


def test_solve_config3_full_size():
    """24^3 x 48, 12 poles (kappa = 0.9), float32 Krylov with float64 reliable updates to 1e-10:
    reported residuals <= 1e-10, and the oracle recomputes b - (A + sigma_j) x_j at sampled sites."""
    import paper_2112_04556_gb300 as rm
    L = (24, 24, 24, 48)
    V = int(np.prod(L))
    U = inputs.random_links(L, eps=0.3, seed=0)
    b = inputs.gaussian_fields(L, 1, seed=5)[0]
    m = rm.mass_fit(12, 0.9)
    rng = np.random.default_rng(6)
    sites = np.unique(rng.integers(0, V, 3000))
    with rm.Context(L) as ctx:
        y, xs, iters, resid = rm.rat_mass_solve(ctx, dev(U), dev(b), m, tol=1e-10, prec=rm.MIXED, want_xs=True)
        assert np.all(resid <= 1e-10), resid
        for j in (0, 5, 11):
            x = host(xs[j])
            r = b[sites] - (oracle.lap_sites(L, U, x, sites) + m["sigma"][j] * x[sites])
            assert np.linalg.norm(r) <= 1e-9 * np.linalg.norm(b[sites])
        yy = host(y)
        expect = m["c"] * b + sum(a * host(xs[j]) for j, a in enumerate(m["alpha"]))
        assert rel_l2(yy, expect) <= 1e-14


@pytest.mark.parametrize("prec,bound", [(0, 1e-11), (1, 1e-5)])
def test_heatbath_parity(prec, bound):
    import paper_2112_04556_gb300 as rm
    L = (4, 4, 6, 4)
    U = inputs.random_links(L, eps=0.5, seed=25)
    xi = inputs.gaussian_fields(L, 1, seed=26)[0]
    m = fit.mass_term(12, 0.9)
    ref = oracle.heatbath(L, U, xi, m)
    with rm.Context(L) as ctx:
        P = rm.heatbath(ctx, dev(U), dev(xi), m, tol=1e-12 if prec == 0 else 1e-6, prec=prec)
    assert rel_l2(host(P), ref) <= bound


def test_solve_errors():
    import paper_2112_04556_gb300 as rm
    L = (4, 4, 4, 4)
    b = dev(inputs.gaussian_fields(L, 1, seed=1)[0])
    with rm.Context(L) as ctx:
        Ud = dev(inputs.random_links(L, 0.5, 1))
        with pytest.raises(rm.RmhmcError) as e:
            rm.rat_mass_solve(ctx, Ud, b, {"c": 1.0, "alpha": [1.0], "sigma": [-0.1]})
        assert e.value.code == rm.EINVAL
        with pytest.raises(rm.RmhmcError) as e:
            rm.rat_mass_solve(ctx, Ud, b, rm.mass_fit(12, 0.9), tol=1e-12, maxiter=2)
        assert e.value.code == rm.ENOCONV
        # zero right-hand side: zero solution, no iterations
        z = b * 0
        y, _, iters, resid = rm.rat_mass_solve(ctx, Ud, z, rm.mass_fit(12, 0.9))
        assert iters == 0 and float(y.abs().max()) == 0.0


def _fitted_mass():
    lam = (np.arange(64) + 0.5) / 64
    return fit.spectrum_mass_term(lam, 0.05 + lam ** 1.2, 8)


def test_general_heatbath_parity():
    """A mass fitted to a spectrum (kappa = 0): P = R(A)^{-1} xi from the library's inverse partial
    fraction against the oracle's CG on R(A); T(P) = |xi|^2 / 2."""
    import paper_2112_04556_gb300 as rm
    L = (4, 4, 4, 4)
    U = inputs.random_links(L, eps=0.4, seed=27)
    xi = inputs.gaussian_fields(L, 1, seed=28)[0]
    m = _fitted_mass()
    ref = oracle.heatbath(L, U, xi, m, tol=1e-13)
    with rm.Context(L) as ctx:
        P = rm.heatbath(ctx, dev(U), dev(xi), m, tol=1e-13, prec=rm.FP64)
        assert rel_l2(host(P), ref) <= 1e-11
        Pm = rm.heatbath(ctx, None, dev(xi), m, tol=1e-11, prec=rm.MIXED)
        assert rel_l2(host(Pm), ref) <= 1e-9
        _, _, T = rm.kinetic_force(ctx, None, P, m, tol=1e-13, prec=rm.FP64)
    assert abs(T - 0.5 * np.sum(xi * xi)) <= 1e-10 * T


def test_spectrum_fitted_mass_trajectory():
    """The loop of Sec. 4 on 8^4: the Wilson-force spectrum, a mass fitted to it, and a trajectory with that
    mass whose H0 = |xi|^2 / 2 + S0 (exact heatbath); float64 and mixed agree."""
    import paper_2112_04556_gb300 as rm
    import torch
    L = (8, 8, 8, 8)
    U = inputs.random_links(L, eps=0.3, seed=29)
    edges = inputs.equal_windows(16)
    with rm.Context(L) as ctx:
        Ud = dev(U)
        F, _, _ = rm.gauge_force(ctx, Ud, 6.0, 0.0, prec=rm.FP64)
        spec = rm.cheb_filter_spectrum(ctx, None, F[None], None, 64, edges, prec=rm.FP64, nnoise=16, seed=3)[0][0]
        lam = 0.5 * (edges[:-1] + edges[1:])
        ok = spec > 1e-6 * spec.max()
        m = rm.mass_fit_spectrum(lam[ok], spec[ok], 8)
        # a noisy measured spectrum need not be monotone, the fitted mass always is: R > 0 decreasing
        R = fit.evaluate(m, np.linspace(0.0, 1.0, 101))
        assert np.isfinite(m["err"]) and np.all(R > 0) and np.all(np.diff(R) < 0)
        xi = torch.from_numpy(inputs.gaussian_fields(L, 1, seed=30)[0]).cuda()
        out = {}
        for prec in (rm.FP64, rm.MIXED):
            p = rm.make_params(beta=6.0, mass=m, tau=0.1, nsteps=4, tol_md=1e-10 if prec == 0 else 1e-6, tol_h=1e-12,
                               fp_tol=1e-10 if prec == 0 else 1e-6, prec=prec, metropolis=False)
            out[prec] = rm.rmhmc_trajectory(ctx, dev(U), p, xi=xi)
    r = out[rm.FP64]
    assert abs(r["T0"] - 0.5 * float((xi * xi).sum())) <= 1e-9 * r["T0"]
    assert np.isfinite(r["dH"]) and abs(out[rm.MIXED]["dH"] - r["dH"]) <= 1e-2 * max(1.0, abs(r["dH"]))


def test_basis_cap_restarts_fitted_mass_16_4():
    """A spectrum-fitted mass with poles down to sigma = 1e-3 on smooth 16^4 links (random SU(3) close to 1,
    so A keeps eigenvalues near 0 and A + 1e-3 has a condition number near 10^3; on the thermalised links the
    adjoint Laplacian has a gap and the solves stay short), where the smallest shift needs more Krylov
    iterations than the 160 stored residuals: the first pass stops at the cap and the reliable-update loop
    continues from the true residuals (restarts).  Every shifted solution is checked against the oracle's own
    operator, |b - (A + sigma_j) x_j| / |b| with A applied by the oracle; a float64 single shift at 3e-4 to
    1e-13 must need more than 160 iterations.  The kinetic force of the MD, which has no restarts, either
    converges within the cap or reports ENOCONV."""
    import paper_2112_04556_gb300 as rm
    L = (16, 16, 16, 16)
    U = inputs.random_links(L, eps=0.05, seed=90)
    lam = (np.arange(64) + 0.5) / 64
    m = rm.mass_fit_spectrum(lam, lam, 12, 1e-3, 10.0)
    assert min(m["sigma"]) <= 1.1e-3
    b = inputs.gaussian_fields(L, 1, seed=91)[0]
    nb = np.linalg.norm(b)
    with rm.Context(L) as ctx:
        Ud = dev(U)
        y, xs, iters, resid = rm.rat_mass_solve(ctx, Ud, dev(b), m, tol=1e-10, prec=rm.MIXED, want_xs=True)
        assert np.all(resid <= 1e-10), resid
        xs = host(xs)
        for j in range(len(m["sigma"])):
            r = b - (oracle.lap(L, U, xs[j]) + m["sigma"][j] * xs[j])
            assert np.linalg.norm(r) / nb <= 2e-10, (j, np.linalg.norm(r) / nb)
        y_ref = m["c"] * b + sum(m["alpha"][j] * xs[j] for j in range(len(m["sigma"])))
        assert rel_l2(host(y), y_ref) <= 1e-12
        single = {"c": 0.0, "alpha": [1.0], "sigma": [3e-4]}
        y1, _, it1, res1 = rm.rat_mass_solve(ctx, None, dev(b), single, tol=1e-13, prec=rm.FP64)
        assert it1 > 160 and res1[0] <= 1e-13, (it1, res1)
        r = b - (oracle.lap(L, U, host(y1)) + 3e-4 * host(y1))
        assert np.linalg.norm(r) / nb <= 2e-13
        try:
            F, _, _ = rm.kinetic_force(ctx, None, dev(b), m, tol=1e-6, prec=rm.MIXED)
            assert np.all(np.isfinite(host(F)))
        except rm.RmhmcError as e:
            assert e.code == rm.ENOCONV and "cap" in str(e)


@pytest.mark.parametrize("nmu,block", [(8, 256), (2, 256), (0, 64)])
def test_cg_stencil_shapes(nmu, block):
    """The mixed solve through each pinned CG stencil shape, the link-centric kernel included, on a lattice
    with partial boxes and t-ranges (10 x 6 x 5 x 9): parity with the oracle's per-shift solves at 1e-10."""
    import paper_2112_04556_gb300 as rm
    L = (10, 6, 5, 9)
    U = inputs.random_links(L, eps=0.5, seed=27)
    b = inputs.gaussian_fields(L, 1, seed=28)[0]
    m = fit.mass_term(12, 0.9)
    y_ref, _ = oracle.rational_apply(L, U, b, m, tol=1e-14)
    with rm.Context(L) as ctx:
        rm.set_stencil_shape(ctx, rm.SHAPE_CG, rm.FP32, 18, nmu, block)
        y, _, iters, resid = rm.rat_mass_solve(ctx, dev(U), dev(b), m, tol=1e-10, prec=rm.MIXED)
        assert np.all(resid <= 1e-10) and iters > 0
        assert rel_l2(host(y), y_ref) <= 1e-9
        F, Vel, T = rm.kinetic_force(ctx, None, dev(b), m, tol=1e-7, prec=rm.MIXED)
        rm.set_stencil_shape(ctx, rm.SHAPE_CG, rm.FP32, 18, 2, 256)
        F2, Vel2, T2 = rm.kinetic_force(ctx, None, dev(b), m, tol=1e-7, prec=rm.MIXED)
    assert rel_l2(host(F), host(F2)) <= 1e-5 and rel_l2(host(Vel), host(Vel2)) <= 1e-5
    assert abs(T - T2) <= 1e-6 * abs(T2)
