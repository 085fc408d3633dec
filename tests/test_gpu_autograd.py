"""The differentiable log psi (torch.autograd.Function over rbm_logpsi /
logpsi_backward): gradients of a real loss against central finite differences
on 64 random parameters (real and imaginary directions); the same gradient in
every precision against the oracle's analytic one, sum_s g_s conj(O_k(s))
with O from oracle.rbm.logderiv (float64 1e-9, float32 1e-5, mixed 1e-3
relative, the float32 and mixed tolerances of the spec parity bar);
and the gradient of the overlap loss at alpha_0 against the oracle's analytic
force bracket in every precision."""

import numpy as np
import pytest

from gpu_common import dev, host, need_gpu, relerr, torch
from oracle import rbm, sr
from paper_2103_08804_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("prec,L,alpha,B,tol", [(0, 12, 1, 1024, 1e-7), (1, 64, 2, 4096, 1e-4),
                                                (2, 64, 2, 4096, 1e-4)])
def test_gradient_matches_central_differences(prec, L, alpha, B, tol):
    """Backward of the given precision against central differences (h = 1e-6)
    of the same loss evaluated in float64 (so that the differences are exact
    to ~1e-9), on 64 random parameters, real and imaginary directions."""
    from paper_2103_08804_gb300 import api
    from paper_2103_08804_gb300.autograd import logpsi
    M = alpha * L
    cd = torch.complex128 if prec == 0 else torch.complex64
    ctx = api.Context(L, 1, M, B, prec=prec)
    ctx64 = ctx if prec == 0 else api.Context(L, 1, M, B, prec=0)
    p0n = synth.rbm_params(3, L, M, 0.05)
    spins = dev(synth.sz0_spins(4, B, L), torch.int8)
    cn = synth.rbm_params(5, B, 0, 1.0)[:B]

    def loss(c, p, cdt):
        lp = logpsi(c, p, spins)
        cc = dev(cn, cdt)
        return torch.sum((lp * cc).real) + 0.5 * torch.sum(torch.abs(lp) ** 2) / B

    p = dev(p0n, cd).requires_grad_(True)
    loss(ctx, p, cd).backward()
    g = host(p.grad)
    p64 = dev(p0n, torch.complex128)
    rng = np.random.default_rng(6)
    ks = rng.choice(ctx.P, 64, replace=False)
    h = 1e-6
    fd = []
    for k in ks:
        for step in (h, 1j * h):
            e = torch.zeros_like(p64)
            e[k] = step
            with torch.no_grad():
                d = (loss(ctx64, p64 + e, torch.complex128) -
                     loss(ctx64, p64 - e, torch.complex128)).item() / (2 * h)
            fd.append(d)
    fd = np.array(fd).reshape(64, 2)
    # torch's grad of a real loss is dL/dRe + i dL/dIm
    got = np.stack([g[ks].real, g[ks].imag], axis=1)
    assert relerr(got, fd) < tol


def test_overlap_loss_gradient_is_force_bracket():
    from paper_2103_08804_gb300 import api
    from paper_2103_08804_gb300.autograd import overlap_loss
    L, M, B = 12, 12, 2048
    ctx = api.Context(L, 1, M, B, prec=0)
    p0n = synth.rbm_params(7, L, M, 0.1)
    sp = synth.sz0_spins(8, B, L)
    g = np.random.Generator(np.random.Philox(9))
    R = 1.0 + 0.2 * (g.standard_normal(B) + 1j * g.standard_normal(B))
    p = dev(p0n, torch.complex128).requires_grad_(True)
    spins = dev(sp, torch.int8)
    lp0 = dev(rbm.logpsi(p0n, L, M, sp), torch.complex128)
    overlap_loss(ctx, p, spins, lp0, dev(R, torch.complex128)).backward()
    est = sr.estimators(rbm.logderiv(p0n, L, M, sp), R)
    bracket = est["OR"] / est["mR"] - np.conj(est["Obar"])
    # PyTorch returns dL/dRe + i dL/dIm = 2 dL/d conj(alpha) = -2 bracket
    assert relerr(host(p.grad), -2.0 * bracket) < 1e-9


GRAD_TOL = {0: 1e-9, 1: 1e-5, 2: 1e-3}
NPDT = {0: np.complex128, 1: np.complex64, 2: np.complex64}


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_gradient_matches_oracle_analytic_gradient(prec):
    """L = sum_s Re(c_s log psi_s) + |log psi_s|^2 / (2B): PyTorch's gradient is
    sum_s g_s conj(O_k(s)) with g_s = conj(c_s) + log psi_s / B (twice
    dL/d conj(log psi_s)), which the oracle forms from its own log psi and O
    at the same (context-precision) parameters."""
    from paper_2103_08804_gb300 import api
    from paper_2103_08804_gb300.autograd import logpsi
    L, M, B = 64, 128, 4096
    cd = torch.complex128 if prec == 0 else torch.complex64
    ctx = api.Context(L, 1, M, B, prec=prec)
    p0 = synth.rbm_params(11, L, M, 0.05).astype(NPDT[prec]).astype(np.complex128)
    sp = synth.sz0_spins(12, B, L)
    c = synth.rbm_params(13, B, 0, 1.0)[:B]
    p = dev(p0, cd).requires_grad_(True)
    lp = logpsi(ctx, p, dev(sp, torch.int8))
    loss = torch.sum((lp * dev(c, cd)).real) + 0.5 * torch.sum(torch.abs(lp) ** 2) / B
    loss.backward()
    g = np.conj(c) + rbm.logpsi(p0, L, M, sp) / B
    want = np.conj(rbm.logderiv(p0, L, M, sp)).T @ g
    err = relerr(host(p.grad), want)
    print(f"prec {prec}: gradient against the oracle's analytic gradient {err:.2e}")
    assert err < GRAD_TOL[prec]


@pytest.mark.parametrize("prec", [1, 2])
def test_overlap_loss_gradient_is_force_bracket_reduced_precision(prec):
    from paper_2103_08804_gb300 import api
    from paper_2103_08804_gb300.autograd import overlap_loss
    L, M, B = 12, 12, 2048
    cd = torch.complex64
    ctx = api.Context(L, 1, M, B, prec=prec)
    p0n = synth.rbm_params(7, L, M, 0.1).astype(np.complex64).astype(np.complex128)
    sp = synth.sz0_spins(8, B, L)
    g = np.random.Generator(np.random.Philox(9))
    R = (1.0 + 0.2 * (g.standard_normal(B) + 1j * g.standard_normal(B))).astype(np.complex64)
    p = dev(p0n, cd).requires_grad_(True)
    spins = dev(sp, torch.int8)
    lp0 = ctx.rbm_logpsi(dev(p0n, cd), spins)
    overlap_loss(ctx, p, spins, lp0, dev(R, cd)).backward()
    est = sr.estimators(rbm.logderiv(p0n, L, M, sp), R.astype(np.complex128))
    bracket = est["OR"] / est["mR"] - np.conj(est["Obar"])
    err = relerr(host(p.grad), -2.0 * bracket)
    print(f"prec {prec}: overlap-loss gradient against the force bracket {err:.2e}")
    assert err < GRAD_TOL[prec]
