"""Python binding of the RMHMC hot-path library (librmhmc.so, C ABI in include/rmhmc.h).

Argument marshalling only: every step of the path runs in the CUDA kernels of the library.  PyTorch
provides device memory and streams.  The binding refuses to run if the compiled library is
missing: there is no CPU fallback.

Layouts (see include/rmhmc.h): links complex128 [V,4,3,3]; su(3) fields float64 (or float32 for
lap_apply) [nfield,V,4,8] with coefficients in the basis T^a = lambda^a/2; site s = x + Lx(y + Ly(z + Lz t)).
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "librmhmc.so")
_lib = None

OK, EINVAL, ECUDA, ENOCONV, ENAN, ETIMEOUT, ENOMEM = 0, -1, -2, -3, -4, -5, -6
FP64, FP32, MIXED = 0, 1, 1
LINK18, LINK12 = 18, 12
OP_A, OP_DELTA = 0, 1
KERNEL_NONE, KERNEL_JACKSON = 0, 1

_ERRNAMES = {EINVAL: "EINVAL", ECUDA: "ECUDA", ENOCONV: "ENOCONV", ENAN: "ENAN", ETIMEOUT: "ETIMEOUT",
             ENOMEM: "ENOMEM"}


class RmhmcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_ERRNAMES.get(code, "?"), code, msg))
        self.code = code


class Mass(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double), ("npole", ctypes.c_int), ("alpha", ctypes.POINTER(ctypes.c_double)),
                ("sigma", ctypes.POINTER(ctypes.c_double)), ("kappa", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("c1", ctypes.c_double), ("mass", Mass), ("tau", ctypes.c_double),
                ("nsteps", ctypes.c_int), ("tol_md", ctypes.c_double), ("tol_h", ctypes.c_double),
                ("fp_tol", ctypes.c_double), ("fp_maxit", ctypes.c_int), ("maxiter", ctypes.c_int),
                ("prec", ctypes.c_int), ("seed", ctypes.c_uint64), ("traj_index", ctypes.c_uint32),
                ("metropolis", ctypes.c_int), ("logdet", ctypes.c_int), ("symplectic", ctypes.c_int),
                ("fp_extra", ctypes.c_int), ("fg_fp64", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("dH", ctypes.c_double), ("H0", ctypes.c_double), ("H1", ctypes.c_double),
                ("T0", ctypes.c_double), ("S0", ctypes.c_double), ("T1", ctypes.c_double), ("S1", ctypes.c_double),
                ("plaq", ctypes.c_double), ("u", ctypes.c_double), ("accepted", ctypes.c_int),
                ("md_solves", ctypes.c_int), ("md_iters", ctypes.c_longlong), ("fp_iters_p", ctypes.c_int),
                ("fp_iters_u", ctypes.c_int), ("max_fp_change", ctypes.c_double), ("A0", ctypes.c_double),
                ("A1", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def library_path():
    return _SO


def lib():
    """Load librmhmc.so (import torch first so that one CUDA context is shared)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_SO):
        raise RuntimeError("librmhmc.so is not built (run __graft_entry__.build() or "
                           "python paper_2112_04556_gb300/build.py); no CPU fallback exists")
    import torch  # noqa: F401  (creates the CUDA runtime before the library's own static runtime)
    L = ctypes.CDLL(_SO)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    DP = ctypes.POINTER(ctypes.c_double)
    sig = {
        "rmhmc_create": ([ctypes.POINTER(I), I, ctypes.POINTER(P)], I),
        "rmhmc_destroy": ([P], I),
        "rmhmc_last_error": ([P], ctypes.c_char_p),
        "rmhmc_set_links": ([P, P, P], I),
        "lap_apply": ([P, P, P, P, I, I, I, I, P], I),
        "lap_link_grad": ([P, P, P, P, I, DP, I, P, P], I),
        "cheb_filter_spectrum": ([P, P, P, I, P, I, ctypes.c_uint64, I, I, DP, I, I, DP, DP, DP, DP, P], I),
        "rat_mass_solve": ([P, P, P, I, I, DP, DP, D, D, I, I, P, P, ctypes.POINTER(I), DP, P], I),
        "rmhmc_heatbath": ([P, P, P, ctypes.POINTER(Mass), D, I, P, P], I),
        "rmhmc_mass_fit": ([I, D, DP, DP, DP, DP], I),
        "gauge_force": ([P, P, D, D, I, P, DP, DP, P], I),
        "kinetic_force": ([P, P, P, ctypes.POINTER(Mass), D, I, P, P, DP, P], I),
        "rmhmc_gauss_field": ([P, P, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, P], I),
        "rmhmc_link_update": ([P, P, P, D, I, P, P], I),
        "rmhmc_hamiltonian": ([P, P, P, ctypes.POINTER(Params), DP, DP, DP, P], I),
        "rmhmc_md": ([P, P, P, ctypes.POINTER(Params), ctypes.POINTER(Result), P], I),
        "rmhmc_trajectory": ([P, P, P, ctypes.POINTER(Params), ctypes.POINTER(Result), P, P], I),
        "rmhmc_set_profiling": ([P, I], I),
        "rmhmc_tuning": ([P, ctypes.c_char_p, I], I),
        "rmhmc_set_graphs": ([P, I], I),
        "rmhmc_set_stencil_shape": ([P, I, I, I, I, I], I),
        "wilson_flow": ([P, P, D, I, I, DP, P], I),
        "cheb_window_coeffs": ([I, DP, I, I, DP], I),
        "rmhmc_mass_fit_spectrum": ([I, DP, DP, I, D, D, DP, DP, DP, DP], I),
        "cheb_filter_apply": ([P, P, P, I, I, DP, I, P, P], I),
        "rmhmc_get_counters": ([P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                ctypes.POINTER(ctypes.c_longlong), DP, I], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name, None)
        if fn is None:
            continue
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("tensor must live on the GPU")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dbl(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Context:
    """A lattice context on one GPU (wraps rmhmc_create / rmhmc_destroy)."""

    def __init__(self, dims, device=0):
        self.dims = tuple(int(d) for d in dims)
        self.V = int(np.prod(self.dims))
        self.device = device
        h = ctypes.c_void_p()
        arr = (ctypes.c_int * 4)(*self.dims)
        code = lib().rmhmc_create(arr, int(device), ctypes.byref(h))
        if code != OK:
            raise RmhmcError(code, "rmhmc_create failed")
        self.h = h

    def check(self, code):
        if code != OK:
            raise RmhmcError(code, lib().rmhmc_last_error(self.h).decode())
        return code

    def close(self):
        if getattr(self, "h", None):
            lib().rmhmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _links(U):
    if U is None:
        return None
    import torch
    if U.dtype == torch.complex128:
        return _ptr(U)
    if U.dtype == torch.float64:
        return _ptr(U)
    raise ValueError("links must be complex128 [V,4,3,3] (or its float64 view)")


def set_profiling(ctx, on=True):
    ctx.check(lib().rmhmc_set_profiling(ctx.h, int(bool(on))))


def counters(ctx, reset=False):
    """dict(launches, krylov_iters, cg_count, cg_ms) of the context."""
    a, b, c = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
    d = ctypes.c_double()
    ctx.check(lib().rmhmc_get_counters(ctx.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d),
                                       int(bool(reset))))
    return {"launches": a.value, "krylov_iters": b.value, "cg_count": c.value, "cg_ms": d.value}


def set_graphs(ctx, on=True):
    """Run the mixed-precision MD as one CUDA graph (default) or host-driven."""
    ctx.check(lib().rmhmc_set_graphs(ctx.h, int(bool(on))))


SHAPE_LAP, SHAPE_CG, SHAPE_KFORCE, SHAPE_LINKUPDATE, SHAPE_ADJOINT = 0, 1, 2, 3, 4


def set_stencil_shape(ctx, kernel, prec, linkfmt, nmu, block):
    """Pin a stencil launch shape (see rmhmc_set_stencil_shape); nmu = 8 is the link-centric kernel."""
    ctx.check(lib().rmhmc_set_stencil_shape(ctx.h, int(kernel), int(prec), int(linkfmt), int(nmu), int(block)))


def tuning(ctx):
    """The autotuner's choices for this context (text)."""
    buf = ctypes.create_string_buffer(4096)
    ctx.check(lib().rmhmc_tuning(ctx.h, buf, 4096))
    return buf.value.decode()


def set_links(ctx, U, stream=None):
    ctx.check(lib().rmhmc_set_links(ctx.h, _links(U), _stream(stream)))


def lap_apply(ctx, U, X, Y=None, prec=None, linkfmt=LINK18, op=OP_A, stream=None):
    """Y = A X (A = -Delta_G/16) or Delta_G X; X float64 or float32 [.., V, 4, 8]."""
    import torch
    if prec is None:
        prec = FP64 if X.dtype == torch.float64 else FP32
    want = torch.float64 if prec == FP64 else torch.float32
    if X.dtype != want:
        raise ValueError("X dtype does not match prec")
    if Y is None:
        Y = torch.empty_like(X)
    nfield = X.numel() // (ctx.V * 32)
    ctx.check(lib().lap_apply(ctx.h, _links(U), _ptr(X), _ptr(Y), nfield, prec, linkfmt, op, _stream(stream)))
    return Y


def lap_link_grad(ctx, U, X, Z, w, G=None, prec=FP64, stream=None):
    import torch
    nfield = X.numel() // (ctx.V * 32)
    w, wp = _dbl(np.atleast_1d(w))
    if len(w) != nfield:
        raise ValueError("one weight per field pair")
    if G is None:
        G = torch.empty((ctx.V, 4, 8), dtype=torch.float64, device=X.device)
    ctx.check(lib().lap_link_grad(ctx.h, _links(U), _ptr(X), _ptr(Z), nfield, wp, prec, _ptr(G), _stream(stream)))
    return G


def cheb_filter_spectrum(ctx, U, F, noise, degree, edges, kernel=KERNEL_JACKSON, prec=FP64, nnoise=None, seed=0,
                         stream=None):
    """Per-mode power spectra (Eq. 4).  Returns (spec[nF,nwin], num[nF,nwin], tr[nwin], moments)."""
    nF = F.numel() // (ctx.V * 32)
    nn = noise.numel() // (ctx.V * 32) if noise is not None else int(nnoise)
    edges, ep = _dbl(edges)
    nwin = len(edges) - 1
    spec = np.zeros((nF, nwin))
    num = np.zeros((nF, nwin))
    tr = np.zeros(nwin)
    mom = np.zeros((nF + nn, degree + 1))
    ctx.check(lib().cheb_filter_spectrum(
        ctx.h, _links(U), _ptr(F), nF, _ptr(noise), nn, int(seed), int(degree), nwin, ep, int(kernel), int(prec),
        spec.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), num.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        tr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), mom.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        _stream(stream)))
    return spec, num, tr, mom


def mass_fit(npole=12, kappa=0.9):
    """Zolotarev fit R(lam) ~ ((1-kappa) + kappa lam)^{-1/2}: dict(c, alpha, sigma, kappa, err)."""
    alpha = np.zeros(max(npole, 1))
    sigma = np.zeros(max(npole, 1))
    c = ctypes.c_double()
    err = ctypes.c_double()
    code = lib().rmhmc_mass_fit(int(npole), float(kappa), ctypes.byref(c),
                                alpha.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                sigma.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(err))
    if code != OK:
        raise RmhmcError(code, "rmhmc_mass_fit failed")
    return {"c": c.value, "alpha": alpha[:npole], "sigma": sigma[:npole], "kappa": float(kappa), "err": err.value}


def _mass_struct(mass):
    alpha, ap = _dbl(mass["alpha"])
    sigma, sp = _dbl(mass["sigma"])
    m = Mass(float(mass["c"]), len(alpha), ap, sp, float(mass.get("kappa", 0.0)))
    m._keep = (alpha, sigma)
    return m


def rat_mass_solve(ctx, U, b, mass, tol=1e-10, maxiter=2000, prec=FP64, want_xs=False, stream=None):
    """y = c b + sum_j alpha_j (A + sigma_j)^{-1} b for b [V,4,8] or nfield fields [nfield,V,4,8].
    Returns (y, xs or None ([nshift,..] per field), iters summed over fields, resid[nshift] or [nfield,nshift])."""
    import torch
    alpha, ap = _dbl(mass["alpha"])
    sigma, sp = _dbl(mass["sigma"])
    n = len(alpha)
    nfield = b.numel() // (ctx.V * 32)
    single = b.dim() == 3
    y = torch.empty_like(b)
    xs = None
    if want_xs:
        shape = (n,) + tuple(b.shape) if single else (nfield, n) + tuple(b.shape[1:])
        xs = torch.empty(shape, dtype=b.dtype, device=b.device)
    iters = ctypes.c_int()
    resid = np.zeros(max(n * nfield, 1))
    ctx.check(lib().rat_mass_solve(ctx.h, _links(U), _ptr(b), nfield, n, sp, ap, float(mass["c"]), float(tol),
                                   int(maxiter), int(prec), _ptr(y), _ptr(xs), ctypes.byref(iters),
                                   resid.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream(stream)))
    res = resid[:n] if single else resid[:n * nfield].reshape(nfield, n)
    return y, xs, iters.value, res


def heatbath(ctx, U, xi, mass, tol=1e-10, prec=FP64, stream=None):
    import torch
    m = _mass_struct(mass)
    P = torch.empty_like(xi)
    ctx.check(lib().rmhmc_heatbath(ctx.h, _links(U), _ptr(xi), ctypes.byref(m), float(tol), int(prec), _ptr(P),
                                   _stream(stream)))
    return P


def gauge_force(ctx, U, beta, c1=0.0, prec=FP64, F=None, stream=None):
    """Returns (F [V,4,8], S, plaquette)."""
    import torch
    if F is None:
        F = torch.empty((ctx.V, 4, 8), dtype=torch.float64, device="cuda:%d" % ctx.device)
    S = ctypes.c_double()
    pl = ctypes.c_double()
    ctx.check(lib().gauge_force(ctx.h, _links(U), float(beta), float(c1), int(prec), _ptr(F), ctypes.byref(S),
                                ctypes.byref(pl), _stream(stream)))
    return F, S.value, pl.value


def kinetic_force(ctx, U, P, mass, tol=1e-12, prec=FP64, want_force=True, want_velocity=True, stream=None):
    """Returns (F_K or None, V = M^{-1} P or None, T)."""
    import torch
    m = _mass_struct(mass)
    F = torch.empty_like(P) if want_force else None
    Vel = torch.empty_like(P) if want_velocity else None
    T = ctypes.c_double()
    ctx.check(lib().kinetic_force(ctx.h, _links(U), _ptr(P), ctypes.byref(m), float(tol), int(prec), _ptr(F),
                                  _ptr(Vel), ctypes.byref(T), _stream(stream)))
    return F, Vel, T.value


def gauss_field(ctx, seed, stream_id, tag=0, out=None, stream=None):
    import torch
    if out is None:
        out = torch.empty((ctx.V, 4, 8), dtype=torch.float64, device="cuda:%d" % ctx.device)
    ctx.check(lib().rmhmc_gauss_field(ctx.h, _ptr(out), int(seed), int(stream_id), int(tag), _stream(stream)))
    return out


def link_update(ctx, U, V, eps, reunit=True, out=None, stream=None):
    import torch
    if out is None:
        out = torch.empty_like(U)
    ctx.check(lib().rmhmc_link_update(ctx.h, _links(U), _ptr(V), float(eps), int(bool(reunit)), _links(out),
                                      _stream(stream)))
    return out


def mass_fit_spectrum(lam, spec, npole=12, sigma_min=1e-3, sigma_max=10.0):
    """Mass term fitted to a measured power spectrum per mode (M proportional to the power, M = 1 at its
    maximum); returns a general rational mass dict (kappa = 0)."""
    import numpy as np
    la, lp = _dbl(lam)
    sa, sp = _dbl(spec)
    c = ctypes.c_double()
    err = ctypes.c_double()
    alpha = np.zeros(npole)
    sigma = np.zeros(npole)
    P = ctypes.POINTER(ctypes.c_double)
    code = lib().rmhmc_mass_fit_spectrum(len(la), lp, sp, int(npole), float(sigma_min), float(sigma_max),
                                         ctypes.byref(c), alpha.ctypes.data_as(P), sigma.ctypes.data_as(P),
                                         ctypes.byref(err))
    if code != 0:
        raise RmhmcError(code, "rmhmc_mass_fit_spectrum: bad arguments")
    return {"c": c.value, "alpha": alpha, "sigma": sigma, "kappa": 0.0, "err": err.value}


def window_coeffs(edges, degree, kernel=KERNEL_JACKSON):
    """C[w, k] of the windows [edges[w], edges[w+1]] (numpy [nwin, degree+1]), computed by the library."""
    import numpy as np
    e, ep = _dbl(edges)
    C = np.zeros((len(e) - 1, int(degree) + 1))
    code = lib().cheb_window_coeffs(len(e) - 1, ep, int(degree), int(kernel),
                                    C.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if code != 0:
        raise RmhmcError(code, "cheb_window_coeffs: bad windows, degree or kernel")
    return C


def cheb_filter_apply(ctx, U, F, coef, prec=FP64, out=None, stream=None):
    """Y = sum_k coef[k] T_k(2A - 1) F for F of shape [V,4,8] or [nfield,V,4,8] (float64, device)."""
    import numpy as np
    import torch
    c, cp = _dbl(coef)
    Fc = F.contiguous()
    nf = 1 if Fc.dim() == 3 else Fc.shape[0]
    if out is None:
        out = torch.empty_like(Fc)
    ctx.check(lib().cheb_filter_apply(ctx.h, _links(U), _ptr(Fc), nf, len(c) - 1, cp, int(prec), _ptr(out),
                                      _stream(stream)))
    return out


def band_injection(ctx, U, xi, mass, window, degree=200, md_eps=1e-4, beta=6.0, c1=0.0, flow_t=8.0,
                   flow_eps=0.01, prec=FP64, tol=1e-12):
    """The momentum-injection experiment of Sec. 4 (Fig. 2): heatbath momenta P = M^{1/2} xi filtered to the
    window [a, b] of Laplacian eigenvalues, one leapfrog step of md_eps from (U, P_w), and the change of the
    Wilson-flowed energy at flow time flow_t.  Every step runs in the library's kernels; U is not modified.
    Returns (E_t(U'), E_t(U), P_w)."""
    import numpy as np
    C = window_coeffs(np.array(window, dtype=np.float64), degree)[0]
    P = heatbath(ctx, U, xi, mass, tol=tol, prec=prec)
    Pw = cheb_filter_apply(ctx, U, P, C, prec=prec)
    U1 = U.clone()
    Pm = Pw.clone()
    md(ctx, U1, Pm, make_params(beta=beta, c1=c1, mass=mass, tau=md_eps, nsteps=1, tol_md=tol, tol_h=tol,
                                fp_tol=tol, prec=prec, metropolis=False))
    n = int(round(flow_t / flow_eps))
    U0 = U.clone()
    E0 = wilson_flow(ctx, U0, flow_eps, n, prec=prec)[-1]
    E1 = wilson_flow(ctx, U1, flow_eps, n, prec=prec)[-1]
    return E1, E0, Pw


def wilson_flow(ctx, U, eps, nsteps, prec=FP64, stream=None):
    """Wilson gradient flow of U in place (nsteps Runge-Kutta steps of size eps); returns E(t) at
    t = 0, eps, ..., nsteps*eps as a numpy array."""
    import numpy as np
    E = np.zeros(int(nsteps) + 1)
    ctx.check(lib().wilson_flow(ctx.h, _links(U), float(eps), int(nsteps), int(prec),
                                E.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream(stream)))
    return E


def make_params(beta=6.0, c1=0.0, mass=None, tau=1.0, nsteps=20, tol_md=1e-10, tol_h=1e-11, fp_tol=1e-10,
                fp_maxit=50, maxiter=2000, prec=FP64, seed=0, traj_index=0, metropolis=True, logdet=False,
                symplectic=False, fp_extra=0, fg_fp64=False):
    mass = mass if mass is not None else {"c": 1.0, "alpha": [], "sigma": [], "kappa": 0.0}
    ms = _mass_struct(mass)
    p = Params(float(beta), float(c1), ms, float(tau), int(nsteps), float(tol_md), float(tol_h),
               float(fp_tol), int(fp_maxit), int(maxiter), int(prec), int(seed), int(traj_index), int(bool(metropolis)),
               int(bool(logdet)), int(bool(symplectic)), int(fp_extra), int(bool(fg_fp64)))
    p._keep = ms._keep   # the struct copy holds raw pointers into these arrays
    return p


def hamiltonian(ctx, U, P, params, stream=None):
    H, T, S = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    ctx.check(lib().rmhmc_hamiltonian(ctx.h, _links(U), _ptr(P), ctypes.byref(params), ctypes.byref(H),
                                      ctypes.byref(T), ctypes.byref(S), _stream(stream)))
    return H.value, T.value, S.value


def md(ctx, U, P, params, stream=None):
    r = Result()
    ctx.check(lib().rmhmc_md(ctx.h, _links(U), _ptr(P), ctypes.byref(params), ctypes.byref(r), _stream(stream)))
    return r.as_dict()


def rmhmc_trajectory(ctx, U, params, xi=None, P_out=None, stream=None):
    r = Result()
    ctx.check(lib().rmhmc_trajectory(ctx.h, _links(U), _ptr(xi), ctypes.byref(params), ctypes.byref(r),
                                     _ptr(P_out), _stream(stream)))
    return r.as_dict()


# ------------------------------------------------------------------------------------------------
# autograd: derivatives with respect to the links in left-multiplication coordinates
#   U_mu(x) -> exp(i w^a T^a) U_mu(x);  "omega" is a zero tensor [V,4,8] standing for w at w = 0.
# ------------------------------------------------------------------------------------------------
def _autograd():
    import torch

    class LaplacianFn(torch.autograd.Function):
        """Y = A(U) X.  Backward: dL/dX = A gY (A is symmetric), dL/dw = lap_link_grad(X, gY)."""

        @staticmethod
        def forward(fctx, omega, X, lat, U, prec):
            fctx.lat, fctx.U, fctx.prec = lat, U, prec
            fctx.save_for_backward(X)
            return lap_apply(lat, U, X, prec=FP64 if X.dtype == torch.float64 else FP32)

        @staticmethod
        def backward(fctx, gY):
            (X,) = fctx.saved_tensors
            gY = gY.contiguous()
            gX = lap_apply(fctx.lat, fctx.U, gY, prec=FP64 if gY.dtype == torch.float64 else FP32)
            gw = lap_link_grad(fctx.lat, fctx.U, X.double(), gY.double(), [1.0], prec=fctx.prec)
            return gw, gX, None, None, None

    class KineticEnergyFn(torch.autograd.Function):
        """T(U, P) = 1/2 <P, M(U)^{-1} P>.  Backward: dT/dw = -F_K (the hand-written link-adjoint kernel),
        dT/dP = M^{-1} P.  recompute=True keeps only (U, P) and reruns the Krylov solve in backward."""

        @staticmethod
        def forward(fctx, omega, P, lat, U, mass, tol, prec, recompute):
            fctx.lat, fctx.U, fctx.mass, fctx.tol, fctx.prec, fctx.recompute = lat, U, mass, tol, prec, recompute
            if recompute:
                _, _, T = kinetic_force(lat, U, P, mass, tol, prec, want_force=False, want_velocity=False)
                fctx.save_for_backward(P)
            else:
                F, Vel, T = kinetic_force(lat, U, P, mass, tol, prec)
                fctx.save_for_backward(F, Vel)
            return torch.tensor(T, dtype=torch.float64, device=P.device)

        @staticmethod
        def backward(fctx, gT):
            if fctx.recompute:
                (P,) = fctx.saved_tensors
                F, Vel, _ = kinetic_force(fctx.lat, fctx.U, P, fctx.mass, fctx.tol, fctx.prec)
            else:
                F, Vel = fctx.saved_tensors
            return -F * gT, Vel * gT, None, None, None, None, None, None

    return LaplacianFn, KineticEnergyFn


def laplacian(lat, U, X, omega=None, prec=FP64):
    """Differentiable Y = A(U) X; omega (zero [V,4,8], requires_grad) receives dL/dw."""
    import torch
    LaplacianFn, _ = _autograd()
    if omega is None:
        omega = torch.zeros((lat.V, 4, 8), dtype=torch.float64, device=X.device)
    return LaplacianFn.apply(omega, X, lat, U, prec)


def kinetic_energy(lat, U, P, mass, omega=None, tol=1e-12, prec=FP64, recompute=False):
    """Differentiable T = 1/2 <P, M(U)^{-1} P>; omega.grad = dT/dw = -F_K, P.grad = M^{-1} P."""
    import torch
    _, KineticEnergyFn = _autograd()
    if omega is None:
        omega = torch.zeros((lat.V, 4, 8), dtype=torch.float64, device=P.device)
    return KineticEnergyFn.apply(omega, P, lat, U, mass, tol, prec, recompute)
