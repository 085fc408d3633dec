"""logpsi_backward_noalloc: the VJP of log psi for callers that cannot
allocate device memory (its reduction scratch is a fixed array inside the
library).  Checked through the C ABI against logpsi_backward on two calls in
a row with different inputs, within the kernel-parity tolerances (float64
1e-10, float32 1e-4 relative), at the 16 x 16 lattice size near the scratch
limit (66,048 parameters, 65536 walkers in two chunks, float32 within 1e-5),
plus the size limit.  Collected last so that a
stop at the first failure has run every other test."""

import ctypes

import numpy as np
import pytest

from gpu_common import dev, host, need_gpu, relerr, torch
from paper_2103_08804_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _inputs(seed, N, M, B, cd):
    params = synth.rbm_params(seed, N, M, 0.3)
    spins = dev(synth.sz0_spins(seed + 1, B, N), torch.int8)
    g = dev(synth.rbm_params(seed + 2, B, 0, 1.0)[:B], cd)
    return params, spins, g


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4)])
@pytest.mark.parametrize("shape", [(12, 1, 12, 1024), (64, 1, 128, 3001)])
def test_noalloc_backward_matches_context_backward_twice(prec, tol, shape):
    from paper_2103_08804_gb300 import api
    Lx, Ly, M, B = shape
    N = Lx * Ly
    cd = torch.complex128 if prec == 0 else torch.complex64
    lib = api.load()
    ctx = api.Context(Lx, Ly, M, B, prec=prec)
    stream = torch.cuda.current_stream()
    err = ctypes.create_string_buffer(256)
    for call, seed in enumerate((100, 200)):
        params, spins, g = _inputs(seed, N, M, B, cd)
        th = torch.empty(B, M, dtype=cd, device="cuda")
        T = torch.empty(B, M, dtype=cd, device="cuda")
        ctx.rbm_logpsi(dev(params, cd), spins, theta_out=th)
        ctx.logderiv(dev(params, cd), spins, th, tanh_out=T)
        want = ctx.logpsi_backward(dev(params, cd), spins, T, g)
        got = torch.full((ctx.P,), float("nan"), dtype=cd, device="cuda")
        s = lib.logpsi_backward_noalloc(N, M, prec, ctypes.c_void_p(spins.data_ptr()),
                                        ctypes.c_void_p(T.data_ptr()), B,
                                        ctypes.c_void_p(g.data_ptr()),
                                        ctypes.c_void_p(got.data_ptr()),
                                        ctypes.c_void_p(stream.cuda_stream), err, len(err))
        assert s == 0, err.value
        assert relerr(host(got), host(want)) < tol, call


def test_noalloc_backward_near_its_size_limit():
    """N = M = 256: the scratch holds two partial rows, so each chunk sums
    32768 walkers; its float32 runs stay 32 walkers long (float64 carries)."""
    from paper_2103_08804_gb300 import api
    Lx = Ly = 16
    N, M, B = 256, 256, 65536
    lib = api.load()
    ctx = api.Context(Lx, Ly, M, B, prec=1)
    stream = torch.cuda.current_stream()
    err = ctypes.create_string_buffer(256)
    cd = torch.complex64
    params, spins, g = _inputs(300, N, M, B, cd)
    params = synth.rbm_params(300, N, M, 0.01)
    th = torch.empty(B, M, dtype=cd, device="cuda")
    T = torch.empty(B, M, dtype=cd, device="cuda")
    ctx.rbm_logpsi(dev(params, cd), spins, theta_out=th)
    ctx.logderiv(dev(params, cd), spins, th, tanh_out=T)
    del th
    want = ctx.logpsi_backward(dev(params, cd), spins, T, g)
    for call in range(2):
        got = torch.full((ctx.P,), float("nan"), dtype=cd, device="cuda")
        s = lib.logpsi_backward_noalloc(N, M, 1, ctypes.c_void_p(spins.data_ptr()),
                                        ctypes.c_void_p(T.data_ptr()), B,
                                        ctypes.c_void_p(g.data_ptr()),
                                        ctypes.c_void_p(got.data_ptr()),
                                        ctypes.c_void_p(stream.cuda_stream), err, len(err))
        assert s == 0, err.value
        e = relerr(host(got), host(want))
        print(f"noalloc at N = M = 256, B = 65536: {e:.2e}")
        assert e < 1e-5, call


def test_noalloc_backward_rejects_sizes_beyond_its_scratch():
    from paper_2103_08804_gb300 import api
    lib = api.load()
    err = ctypes.create_string_buffer(256)
    dummy = torch.zeros(4, dtype=torch.complex64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    # N = 1024, M = 512: 525,824 parameters, beyond the fixed scratch
    s = lib.logpsi_backward_noalloc(1024, 512, 1, p, p, 8, p, p, None, err, len(err))
    assert s == 1 and b"too large" in err.value
    s = lib.logpsi_backward_noalloc(16, 600, 1, p, p, 8, p, p, None, err, len(err))
    assert s == 1
    torch.cuda.synchronize()
    assert np.all(host(dummy) == 0)
