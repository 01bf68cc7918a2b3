"""GPU parity of the link-adjoint kernel, the kinetic force and the autograd Functions; central
finite differences of the kinetic energy on 32 random link directions."""
import numpy as np
import pytest

import oracle
from gpu_util import dev, host, rel_l2, torch_cuda
from oracle import fit
from paper_2112_04556_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (5, 3, 4, 7)])
def test_link_grad_parity(L):
    import paper_2112_04556_gb300 as rm
    U = inputs.random_links(L, eps=0.6, seed=31)
    X = inputs.gaussian_fields(L, 3, seed=32)
    Z = inputs.gaussian_fields(L, 3, seed=33)
    w = [0.7, -1.3, 0.25]
    ref = oracle.lap_link_grad(L, U, X, Z, w)
    with rm.Context(L) as ctx:
        G = rm.lap_link_grad(ctx, dev(U), dev(X), dev(Z), w, prec=rm.FP64)
        assert rel_l2(host(G), ref) <= 1e-12
        G32 = rm.lap_link_grad(ctx, None, dev(X), dev(Z), w, prec=rm.FP32)
        assert rel_l2(host(G32), ref) <= 1e-5


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (8, 8, 8, 8)])
def test_kinetic_force_parity(L):
    import paper_2112_04556_gb300 as rm
    U = inputs.random_links(L, eps=0.4, seed=34)
    P = inputs.gaussian_fields(L, 1, seed=35)[0]
    m = fit.mass_term(12, 0.9)
    T_ref, F_ref, V_ref = oracle.kinetic(L, U, P, m, tol=1e-14)
    with rm.Context(L) as ctx:
        F, Vel, T = rm.kinetic_force(ctx, dev(U), dev(P), m, tol=1e-13, prec=rm.FP64)
        assert rel_l2(host(F), F_ref) <= 1e-10
        assert rel_l2(host(Vel), V_ref) <= 1e-11
        assert abs(T - T_ref) <= 1e-11 * T_ref
        F32, V32, T32 = rm.kinetic_force(ctx, None, dev(P), m, tol=1e-6, prec=rm.MIXED)
        assert rel_l2(host(F32), F_ref) <= 1e-5
        assert rel_l2(host(V32), V_ref) <= 1e-5
        assert abs(T32 - T_ref) <= 1e-5 * T_ref


def test_identity_mass():
    import paper_2112_04556_gb300 as rm
    L = (4, 4, 4, 4)
    P = inputs.gaussian_fields(L, 1, seed=36)[0]
    with rm.Context(L) as ctx:
        F, Vel, T = rm.kinetic_force(ctx, dev(inputs.random_links(L, 0.5, 2)), dev(P),
                                     {"c": 1.0, "alpha": [], "sigma": []})
    assert float(F.abs().max()) == 0.0 and np.abs(host(Vel) - P).max() == 0.0
    assert abs(T - 0.5 * np.sum(P * P)) <= 1e-12 * T


def _T_along(rm, ctx, U, P, m, D, h):
    """T at links exp(i h D) U (every link moved along the direction field D)."""
    Uh = rm.link_update(ctx, U, D, h, reunit=False)
    return rm.kinetic_force(ctx, Uh, P, m, tol=1e-14, prec=rm.FP64, want_force=False, want_velocity=False)[2]


def test_autograd_kinetic_finite_differences_16_4():
    """Config 4: 16^4, 12 poles.  omega.grad = dT/dw from the hand-written backward kernel, against central
    differences (h = 1e-5, float64 T) along 32 random directions in link space (every link moved by
    exp(i h d_mu(x)) at once); the float32 backward against the float64 one; the recompute mode gives the
    same gradient."""
    import paper_2112_04556_gb300 as rm
    torch = torch_cuda()
    L = (16, 16, 16, 16)
    U = dev(inputs.random_links(L, eps=0.3, seed=0))
    P0 = dev(inputs.gaussian_fields(L, 1, seed=37)[0])
    m = rm.mass_fit(12, 0.9)
    with rm.Context(L) as ctx:
        omega = torch.zeros((ctx.V, 4, 8), dtype=torch.float64, device="cuda", requires_grad=True)
        P = P0.clone().requires_grad_(True)
        T = rm.kinetic_energy(ctx, U, P, m, omega=omega, tol=1e-14)
        T.backward()
        g = omega.grad.detach()
        h = 1e-5
        dirs = torch.from_numpy(inputs.gaussian_fields(L, 32, seed=38)).cuda()
        worst = 0.0
        for k in range(32):
            D = dirs[k].contiguous()
            fd = (_T_along(rm, ctx, U, P0, m, D, h) - _T_along(rm, ctx, U, P0, m, D, -h)) / (2 * h)
            an = float((g * D).sum())
            worst = max(worst, abs(fd - an) / abs(an))
        assert worst <= 1e-5, worst
        # dT/dP = M^{-1} P
        _, Vel, _ = rm.kinetic_force(ctx, U, P0, m, tol=1e-14)
        assert rel_l2(host(P.grad), host(Vel)) <= 1e-12
        # float32 backward against float64
        om32 = torch.zeros_like(omega, requires_grad=True)
        T32 = rm.kinetic_energy(ctx, U, P0.clone(), m, omega=om32, tol=1e-6, prec=rm.MIXED)
        T32.backward()
        assert rel_l2(host(om32.grad), host(g)) <= 1e-5
        assert abs(T32.item() - T.item()) <= 1e-6 * T.item()
        # recompute mode
        om2 = torch.zeros_like(omega, requires_grad=True)
        rm.kinetic_energy(ctx, U, P0.clone(), m, omega=om2, tol=1e-14, recompute=True).backward()
        assert rel_l2(host(om2.grad), host(g)) <= 1e-12


def test_kinetic_gradient_matches_oracle_8_4():
    import paper_2112_04556_gb300 as rm
    torch = torch_cuda()
    L = (8, 8, 8, 8)
    U = inputs.random_links(L, eps=0.3, seed=0)
    P = inputs.gaussian_fields(L, 1, seed=39)[0]
    m = fit.mass_term(12, 0.9)
    _, F_ref, _ = oracle.kinetic(L, U, P, m, tol=1e-14)
    with rm.Context(L) as ctx:
        omega = torch.zeros((ctx.V, 4, 8), dtype=torch.float64, device="cuda", requires_grad=True)
        rm.kinetic_energy(ctx, dev(U), dev(P), m, omega=omega, tol=1e-14).backward()
    assert rel_l2(-host(omega.grad), F_ref) <= 1e-10


def test_autograd_laplacian():
    """Backward of Y = A(U) X: d<G, A X>/dX = A G, d/dw = lap_link_grad(X, G) vs the oracle."""
    import paper_2112_04556_gb300 as rm
    torch = torch_cuda()
    L = (4, 4, 6, 4)
    U = inputs.random_links(L, eps=0.5, seed=40)
    X = inputs.gaussian_fields(L, 1, seed=41)[0]
    G = inputs.gaussian_fields(L, 1, seed=42)[0]
    with rm.Context(L) as ctx:
        omega = torch.zeros((ctx.V, 4, 8), dtype=torch.float64, device="cuda", requires_grad=True)
        Xd = dev(X).requires_grad_(True)
        Y = rm.laplacian(ctx, dev(U), Xd, omega=omega)
        (Y * dev(G)).sum().backward()
    assert rel_l2(host(Xd.grad), oracle.lap(L, U, G)) <= 1e-12
    assert rel_l2(host(omega.grad), oracle.lap_link_grad(L, U, X, G, [1.0])) <= 1e-12


@pytest.mark.parametrize("L", [(8, 6, 4, 10), (5, 3, 4, 7), (16, 16, 16, 16)])
def test_staged_contraction_matches_global(L):
    """The four kernels of the kinetic force's basis contraction (four lanes per link reading the own basis rows
    from global memory; the same with the rows staged in shared memory; eight lanes per link splitting the
    accumulator; four lanes with the neighbour rows passed through shared memory) agree to float32 rounding
    and match the oracle's force; a tight tolerance makes the Krylov run longer than the 20 staged rows, which
    takes the global reads inside the staged kernel.  5 x 3 x 4 x 7 = 420 sites leaves a ragged last block."""
    import paper_2112_04556_gb300 as rm
    U = inputs.random_links(L, eps=0.4, seed=41)
    P = inputs.gaussian_fields(L, 1, seed=42)[0]
    m = fit.mass_term(12, 0.9)
    out = {}
    with rm.Context(L) as ctx:
        Ud, Pd = dev(U), dev(P)
        for mode, block in ((1, 128), (0, 128), (2, 256), (3, 128)):
            rm.set_stencil_shape(ctx, rm.SHAPE_KFORCE, rm.FP32, 18, mode, block)
            for tol in (1e-6, 1e-9):
                out[(mode, tol)] = host(rm.kinetic_force(ctx, Ud, Pd, m, tol=tol, prec=rm.MIXED)[0])
        for bad in ((2, 128), (3, 256), (0, 256), (4, 128)):
            with pytest.raises(rm.RmhmcError):
                rm.set_stencil_shape(ctx, rm.SHAPE_KFORCE, rm.FP32, 18, *bad)
    for tol in (1e-6, 1e-9):
        assert rel_l2(out[(1, tol)], out[(0, tol)]) <= 1e-6, tol
        assert rel_l2(out[(2, tol)], out[(0, tol)]) <= 1e-6, tol
        assert rel_l2(out[(3, tol)], out[(0, tol)]) <= 1e-6, tol
    if np.prod(L) <= 4096:
        _, ref, _ = oracle.kinetic(L, U, P, m, tol=1e-13)
        for mode in (0, 1, 2, 3):
            assert rel_l2(out[(mode, 1e-9)], ref) <= 1e-5
