"""GPU parity of lap_apply (Sec. 2, Eq. 3) against the FP64 oracle on identical seeded inputs.
Tolerances: float64 paths <= 1e-12 relative L2, float32 paths <= 1e-5."""
import numpy as np
import pytest

import oracle
from gpu_util import dev, host, rel_l2, torch_cuda
from paper_2112_04556_gb300 import inputs

pytestmark = pytest.mark.gpu

VARIANTS = [(0, 18, 1e-12), (0, 12, 1e-12), (1, 18, 1e-5), (1, 12, 1e-5)]


def _run(ctx, U_d, X, prec, linkfmt, op=0):
    import paper_2112_04556_gb300 as rm
    torch = torch_cuda()
    Xd = dev(X, torch.float64 if prec == 0 else torch.float32)
    return host(rm.lap_apply(ctx, U_d, Xd, prec=prec, linkfmt=linkfmt, op=op)).astype(np.float64)


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (2, 4, 6, 8), (5, 3, 4, 7), (3, 3, 3, 3)])
def test_lap_parity_small(L):
    """Several 128-site tiles and a ragged last tile (5x3x4x7 = 420 sites); odd extents included.  Seven
    fields: the float32 paths take the multi-field adjoint form (tiles of 32 sites, fields split by parity and
    taken in passes, so the last pass is ragged too)."""
    import paper_2112_04556_gb300 as rm
    U = inputs.random_links(L, eps=0.7, seed=1)
    X = inputs.gaussian_fields(L, 7, seed=2)
    ref = oracle.lap(L, U, X)
    with rm.Context(L) as ctx:
        Ud = dev(U)
        for prec, lf, tol in VARIANTS:
            Y = _run(ctx, Ud, X, prec, lf)
            assert rel_l2(Y, ref) <= tol, (prec, lf, rel_l2(Y, ref))
        # Delta itself: Delta = -16 A
        Y = _run(ctx, Ud, X[0], 0, 18, op=rm.OP_DELTA)
        assert rel_l2(Y, -16.0 * ref[0]) <= 1e-12


def test_lap_free_field_and_reuse_links():
    """U = 1 plane wave: exact eigenvalue; U = NULL reuses the imported links."""
    import paper_2112_04556_gb300 as rm
    torch = torch_cuda()
    L = (4, 6, 4, 8)
    from conftest import site_coords
    k = 2 * np.pi * np.array([1, 2, 0, 3]) / np.array(L)
    X = np.zeros((int(np.prod(L)), 4, 8))
    X[:, 3, 7] = np.cos(site_coords(L) @ k)
    lam = np.sum(np.sin(k / 2) ** 2) / 4
    with rm.Context(L) as ctx:
        rm.set_links(ctx, dev(inputs.unit_links(L)))
        Y = host(rm.lap_apply(ctx, None, dev(X)))
        assert np.abs(Y - lam * X).max() < 1e-14
        Y32 = host(rm.lap_apply(ctx, None, dev(X, torch.float32), prec=rm.FP32, linkfmt=12))
        assert np.abs(Y32 - lam * X).max() < 1e-6


def test_lap_parity_16_4():
    import paper_2112_04556_gb300 as rm
    L = (16, 16, 16, 16)
    U = inputs.random_links(L, eps=0.3, seed=0)
    X = inputs.gaussian_fields(L, 1, seed=3)[0]
    ref = oracle.lap(L, U, X)
    with rm.Context(L) as ctx:
        Ud = dev(U)
        for prec, lf, tol in VARIANTS:
            assert rel_l2(_run(ctx, Ud, X, prec, lf), ref) <= tol


@pytest.mark.parametrize("L", [(32, 32, 32, 32), (24, 24, 24, 48)])
def test_lap_parity_full_size_sampled(L):
    """Full-size lattices, every variant, compared on 4096 sampled sites."""
    import paper_2112_04556_gb300 as rm
    U = inputs.random_links(L, eps=0.3, seed=0)
    X = inputs.gaussian_fields(L, 1, seed=4)[0]
    rng = np.random.default_rng(5)
    V = int(np.prod(L))
    sites = np.unique(np.concatenate([rng.integers(0, V, 4000), [0, V - 1], np.arange(V - 64, V)]))
    ref = oracle.lap_sites(L, U, X, sites)
    with rm.Context(L) as ctx:
        Ud = dev(U)
        for prec, lf, tol in VARIANTS:
            Y = _run(ctx, Ud, X, prec, lf)
            assert rel_l2(Y[sites], ref) <= tol, (prec, lf)


def test_lap_errors_and_empty():
    import paper_2112_04556_gb300 as rm
    torch = torch_cuda()
    L = (4, 4, 4, 4)
    with rm.Context(L) as ctx:
        X = torch.zeros((2, 256, 4, 8), dtype=torch.float64, device="cuda")
        with pytest.raises(rm.RmhmcError):           # no links imported yet
            rm.lap_apply(ctx, None, X[0])
        rm.set_links(ctx, dev(inputs.unit_links(L)))
        with pytest.raises(rm.RmhmcError):           # overlapping input and output
            rm.lap_apply(ctx, None, X[0], Y=X[0])
        with pytest.raises(rm.RmhmcError):           # bad link format
            rm.lap_apply(ctx, None, X[0], linkfmt=9)
        code = rm.lib().lap_apply(ctx.h, None, rm._ptr(X), rm._ptr(X[1]), 0, 0, 18, 0, rm._stream())
        assert code == rm.OK                          # nothing to do for zero fields


@pytest.mark.parametrize("nf", [2, 6, 9])
def test_lap_multifield_full_size_sampled(nf):
    """32^4, several float32 fields in one launch (the adjoint form), 18- and 12-real links, on sampled sites
    of every field; each field also equals its own single-field application to float32 rounding."""
    import paper_2112_04556_gb300 as rm
    torch = torch_cuda()
    L = (32, 32, 32, 32)
    U = inputs.random_links(L, eps=0.3, seed=0)
    X = inputs.gaussian_fields(L, nf, seed=6)
    rng = np.random.default_rng(7)
    V = int(np.prod(L))
    sites = np.unique(np.concatenate([rng.integers(0, V, 3000), [0, V - 1], np.arange(V - 40, V)]))
    refs = [oracle.lap_sites(L, U, X[f], sites) for f in range(nf)]
    with rm.Context(L) as ctx:
        Ud = dev(U)
        X32 = dev(X, torch.float32)
        for lf in (18, 12):
            Y = host(rm.lap_apply(ctx, Ud, X32, prec=rm.FP32, linkfmt=lf)).astype(np.float64)
            for f in range(nf):
                assert rel_l2(Y[f][sites], refs[f]) <= 1e-5, (lf, f)
            Y1 = host(rm.lap_apply(ctx, None, X32[nf - 1].contiguous(), prec=rm.FP32, linkfmt=lf)).astype(np.float64)
            assert rel_l2(Y[nf - 1], Y1) <= 2e-6


# every pinned float32 shape, including the link-centric adjoint kernel (nmu 8): boxes of 8 x 4 x 2 sites
# swept through t-ranges of 8 slices, so these extents give full boxes (wrap inside the box), partial last
# boxes (10 = 8 + 2, 9 = 8 + 1 slices), extents 2 (both neighbours the same site) and 3
SHAPES = [(8, 256), (2, 256), (0, 128), (1, 64), (4, 256)]


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (5, 3, 4, 7), (2, 4, 6, 8), (3, 3, 3, 3), (10, 6, 5, 9), (8, 4, 2, 17)])
def test_lap_every_shape(L):
    import paper_2112_04556_gb300 as rm
    torch = torch_cuda()
    U = inputs.random_links(L, eps=0.7, seed=11)
    X = inputs.gaussian_fields(L, 1, seed=12)[0]
    ref = oracle.lap(L, U, X)
    X32 = dev(X, torch.float32)
    for nmu, block in SHAPES:
        with rm.Context(L) as ctx:
            for lf in (18, 12):
                rm.set_stencil_shape(ctx, rm.SHAPE_LAP, rm.FP32, lf, nmu, block)
            Ud = dev(U)
            for lf in (18, 12):
                Y = host(rm.lap_apply(ctx, Ud, X32, prec=rm.FP32, linkfmt=lf)).astype(np.float64)
                assert rel_l2(Y, ref) <= 1e-5, (nmu, lf, rel_l2(Y, ref))
            # Delta itself through the same shape
            Y = host(rm.lap_apply(ctx, None, X32, prec=rm.FP32, op=rm.OP_DELTA)).astype(np.float64)
            assert rel_l2(Y, -16.0 * ref) <= 1e-5


def test_lap_link_centric_full_size_sampled():
    """The link-centric kernel at 32^4 and 24^3 x 48 on sampled sites (every box full, t-ranges of 8)."""
    import paper_2112_04556_gb300 as rm
    torch = torch_cuda()
    for L in [(32, 32, 32, 32), (24, 24, 24, 48)]:
        U = inputs.random_links(L, eps=0.3, seed=0)
        X = inputs.gaussian_fields(L, 1, seed=4)[0]
        rng = np.random.default_rng(5)
        V = int(np.prod(L))
        sites = np.unique(np.concatenate([rng.integers(0, V, 3000), [0, V - 1], np.arange(V - 64, V)]))
        ref = oracle.lap_sites(L, U, X, sites)
        with rm.Context(L) as ctx:
            for lf in (18, 12):
                rm.set_stencil_shape(ctx, rm.SHAPE_LAP, rm.FP32, lf, 8, 256)
                Y = host(rm.lap_apply(ctx, dev(U), dev(X, torch.float32), prec=rm.FP32, linkfmt=lf)).astype(np.float64)
                assert rel_l2(Y[sites], ref) <= 1e-5, (L, lf)


def test_set_stencil_shape_rejects():
    import paper_2112_04556_gb300 as rm
    with rm.Context((4, 4, 4, 4)) as ctx:
        for args in [(7, rm.FP32, 18, 1, 128), (0, rm.FP64, 18, 8, 256), (0, rm.FP32, 18, 8, 128),
                     (1, rm.FP32, 12, 2, 256), (0, rm.FP32, 18, 3, 256), (0, rm.FP32, 18, 2, 100),
                     (2, rm.FP32, 18, 1, 256), (3, rm.FP32, 18, 2, 128),
                     (4, rm.FP64, 18, 2, 0), (4, rm.FP32, 18, 4, 0), (4, rm.FP32, 18, 1, 0), (4, rm.FP32, 18, 2, 5),
                     (4, rm.FP32, 18, 2, -1), (4, rm.FP32, 16, 2, 0)]:
            with pytest.raises(rm.RmhmcError):
                rm.set_stencil_shape(ctx, *args)
        for args in [(4, rm.FP32, 18, 3, 2), (4, rm.FP32, 12, 0, 0), (4, rm.FP32, 18, 2, 4)]:
            rm.set_stencil_shape(ctx, *args)


@pytest.mark.parametrize("L", [(6, 5, 7, 9), (4, 8, 6, 5), (3, 2, 2, 4)])
def test_lap_adjoint_every_shape_and_slab(L):
    """The multi-field adjoint kernel with every fields-per-pass choice and slab depths that leave a thinner
    last z block (7 = 3 + 3 + 1, 6 = 4 + 2), a slab that is not a whole number of 32-site tiles (5 x 6 x 2 =
    60 sites) and one z block holding the whole lattice; 7 fields (the last pass ragged).  The fields are
    also taken at an offset of 16 bytes within a larger buffer."""
    import paper_2112_04556_gb300 as rm
    torch = torch_cuda()
    U = inputs.random_links(L, eps=0.7, seed=21)
    X = inputs.gaussian_fields(L, 7, seed=22)
    ref = oracle.lap(L, U, X)
    X32 = dev(X, torch.float32)
    # the same fields 16 bytes into a larger buffer
    n = X32.numel()
    buf = torch.zeros(2 * n + 8, dtype=torch.float32, device=X32.device)
    Xo = buf[4:4 + n].view(X32.shape)
    Xo.copy_(X32)
    Yo = buf[n + 8:2 * n + 8].view(X32.shape)
    assert Xo.data_ptr() % 32 == 16 and Yo.data_ptr() % 32 == 0
    for ch, bz in [(2, 1), (3, 2), (2, 3), (3, 4), (2, L[2]), (3, 0)]:
        bz = min(bz, L[2])
        with rm.Context(L) as ctx:
            Ud = dev(U)
            for lf in (18, 12):
                rm.set_stencil_shape(ctx, rm.SHAPE_ADJOINT, rm.FP32, lf, ch, bz)
                Y = host(rm.lap_apply(ctx, Ud, X32, prec=rm.FP32, linkfmt=lf)).astype(np.float64)
                assert rel_l2(Y, ref) <= 1e-5, (ch, bz, lf, rel_l2(Y, ref))
                rm.lap_apply(ctx, None, Xo, Yo, prec=rm.FP32, linkfmt=lf)
                assert rel_l2(host(Yo).astype(np.float64), ref) <= 1e-5, (ch, bz, lf, "offset")
