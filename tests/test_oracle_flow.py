"""Pins of the oracle's Wilson gradient flow and flowed energy (the observable of Sec. 4, defined by
Luscher, JHEP 08 (2010) 071): gradient descent of the action, the initial slope fixed by the force,
third-order convergence of the Runge-Kutta scheme, gauge invariance, and the heat-equation decay of a
weak abelian plane wave."""
import math

import numpy as np

import helpers as H
from conftest import site_coords
from paper_2112_04556_gb300 import inputs

L4 = (4, 4, 4, 4)


def test_flow_is_gradient_descent(oracle_lib):
    """E(t) decreases monotonically and the flow drives a rough configuration towards smoothness."""
    U = inputs.random_links(L4, eps=0.5, seed=81)
    _, E = oracle_lib.wilson_flow(L4, U, 0.02, 10)
    assert np.all(np.diff(E) < 0), E
    assert E[-1] < 0.9 * E[0]


def test_flow_initial_slope(oracle_lib):
    """dE/dt at t = 0 is -36 |F(beta=1)|^2 / V: E = 6 s / V with s = S_W / beta, and the flow moves the
    links with velocity 6 F(beta=1), so ds/dt = -6 |F(beta=1)|^2 (central difference in t, O(eps^2))."""
    L = (2, 4, 2, 4)
    V = int(np.prod(L))
    U = inputs.random_links(L, eps=0.4, seed=82)
    F1 = oracle_lib.gauge_force(L, U, 1.0)
    slope = -36.0 * float(np.sum(F1 * F1)) / V
    eps = 2e-4
    _, Ep = oracle_lib.wilson_flow(L, U, eps, 1)
    _, Em = oracle_lib.wilson_flow(L, U, -eps, 1)
    fd = (Ep[1] - Em[1]) / (2 * eps)
    assert abs(fd - slope) < 2e-6 * abs(slope), (fd, slope)


def test_flow_third_order(oracle_lib):
    """Halving the step size shrinks the error at fixed flow time by 2^3: successive differences of the
    flowed links at t = 0.3 with eps = 0.025, 0.0125, 0.00625 fall by a factor near 8 (a second- or
    fourth-order scheme gives 4 or 16)."""
    U = inputs.random_links(L4, eps=0.4, seed=83)
    t = 0.3
    Us = [oracle_lib.wilson_flow(L4, U, t / n, n)[0] for n in (12, 24, 48)]
    d1 = np.abs(Us[0] - Us[1]).max()
    d2 = np.abs(Us[1] - Us[2]).max()
    assert 7.0 < d1 / d2 < 9.5, (d1, d2, d1 / d2)


def test_flow_gauge_invariant(oracle_lib):
    U = inputs.random_links(L4, eps=0.4, seed=84)
    g = inputs.random_su3(int(np.prod(L4)), seed=85)
    Up = H.gauge_transform_links(L4, U, g)
    _, E0 = oracle_lib.wilson_flow(L4, U, 0.05, 6)
    _, E1 = oracle_lib.wilson_flow(L4, Up, 0.05, 6)
    assert np.abs(E0 - E1).max() < 1e-12 * E0[0]


def test_flow_weak_plane_wave(oracle_lib):
    """A weak transverse abelian wave A_x(y) = a cos(k y) diag(1, -1, 0) obeys the lattice heat equation
    dA/dt = -khat^2 A (khat^2 = 4 sin^2(k/2)), so E(t) = E(0) exp(-2 khat^2 t) up to O(a^2)."""
    L = (4, 8, 4, 4)
    V = int(np.prod(L))
    k = 2 * math.pi * 1 / L[1]
    khat2 = 4 * math.sin(k / 2) ** 2
    a = 1e-3
    y = site_coords(L)[:, 1]
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    U[:, :, 0, 0] = U[:, :, 1, 1] = U[:, :, 2, 2] = 1.0
    th = a * np.cos(k * y)
    U[:, 0, 0, 0] = np.exp(1j * th)
    U[:, 0, 1, 1] = np.exp(-1j * th)
    t, n = 0.5, 50
    _, E = oracle_lib.wilson_flow(L, U, t / n, n)
    ts = np.arange(n + 1) * (t / n)
    assert np.abs(E / E[0] - np.exp(-2 * khat2 * ts)).max() < 1e-4
