"""The allocation-free entry point rmhmc_action_noalloc: gauge action and average plaquette computed with a
fixed device scratch array and no context, for callers that cannot allocate device memory (an application
whose device memory is entirely handed out by another allocator, or code that must not call cudaMalloc
because it synchronises the device).  Checked through the C ABI, on two calls in a row (the scratch array
is reused and each call must reset it), against the existing entry point gauge_force's action and
plaquette and against the oracle's action."""
import ctypes

import numpy as np
import pytest

import oracle
from gpu_util import dev, torch_cuda
from paper_2112_04556_gb300 import inputs

pytestmark = pytest.mark.gpu


def _entry(rm):
    fn = rm.lib().rmhmc_action_noalloc
    fn.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                   ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


@pytest.mark.parametrize("L,c1", [((8, 6, 4, 10), 0.0), ((4, 4, 4, 4), -0.331), ((16, 16, 16, 16), 0.0),
                                  ((5, 3, 4, 6), -0.331)])
def test_noalloc_action_matches_gauge_force_and_oracle(L, c1):
    import paper_2112_04556_gb300 as rm
    torch = torch_cuda()
    fn = _entry(rm)
    Uh = inputs.random_links(L, eps=0.5, seed=3)
    U = dev(Uh)
    beta = 6.0
    with rm.Context(L) as ctx:
        _, S_ref, pl_ref = rm.gauge_force(ctx, U, beta, c1)
    S_orc, pl_orc = oracle.action(L, Uh, beta, c1)
    dims = (ctypes.c_int * 4)(*L)
    outs = [torch.zeros(2, dtype=torch.float64, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    for out in outs:
        code = fn(dims, ctypes.c_void_p(U.data_ptr()), beta, c1, ctypes.c_void_p(out.data_ptr()), rm._stream())
        assert code == 0
    torch.cuda.synchronize()
    for out in outs:
        S, pl = out.cpu().numpy()
        assert abs(S - S_ref) <= 1e-12 * abs(S_ref)
        assert abs(pl - pl_ref) <= 1e-13
        assert abs(S - S_orc) <= 1e-12 * abs(S_orc)
        assert abs(pl - pl_orc) <= 1e-13


def test_noalloc_rejects_bad_sizes():
    import paper_2112_04556_gb300 as rm
    torch = torch_cuda()
    fn = _entry(rm)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    U = torch.zeros(16, dtype=torch.float64, device="cuda")
    for dims in [(1, 4, 4, 4), (512, 512, 512, 2), (65536, 65536, 65536, 65536), (1 << 27, 2, 2, 2),
                 (2, 2, 2, -4)]:
        d = (ctypes.c_int * 4)(*dims)
        assert fn(d, ctypes.c_void_p(U.data_ptr()), 6.0, 0.0, ctypes.c_void_p(out.data_ptr()), rm._stream()) == rm.EINVAL
