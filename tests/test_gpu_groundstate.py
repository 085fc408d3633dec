"""Ground-state preparation on the GPU (Sec. I energy descent with the
metric of Sec. III) against the oracle: the local energy through the
Chebyshev target kernel, one energy-descent update (float64 to 1e-9, float32
to the kappa-scaled float32 error), and a sampled descent on the 12-site
chain approaching the exact ground energy."""

import numpy as np
import pytest

from gpu_common import dev, host, need_gpu, relerr, torch
from oracle import exact, groundstate, rbm
from paper_2103_08804_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def test_local_energy_through_the_target_kernel():
    from paper_2103_08804_gb300 import api
    Lx, Ly, M, B = 4, 3, 6, 333
    N = Lx * Ly
    E0, a, Wp = -7.1, 3.3, 0.9875
    p = synth.rbm_params(5, N, M, 0.3)
    spins = synth.sz0_spins(6, B, N)
    El = groundstate.local_energy(p, N, M, Lx, Ly, 1.0, spins)
    ref = (El - E0) / a - Wp
    ctx = api.Context(Lx, Ly, M, B, prec=api.FP64)
    pr, sp = dev(p, torch.complex128), dev(spins, torch.int8)
    th = torch.empty(B, M, dtype=torch.complex128, device="cuda")
    lp = torch.empty(B, dtype=torch.complex128, device="cuda")
    ctx.rbm_logpsi(pr, sp, th, lp)
    one = torch.ones(1, dtype=torch.complex128, device="cuda")
    R = host(ctx.cheb_local_target(1, ctx.state(pr), None, one, None, E0, a, Wp, sp, lp))
    ctx.sync_status()
    assert np.allclose(R, ref, rtol=0, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("prec,solver", [(0, 0), (0, 1), (1, 1), (2, 1)])
def test_energy_update_against_oracle(prec, solver):
    from paper_2103_08804_gb300 import api
    Lx, M, B = 12, 12, 1024
    N = Lx
    p = synth.rbm_params(7, N, M, 0.2)
    spins = synth.sz0_spins(8, B, N)
    O = rbm.logderiv(p, N, M, spins)
    El = groundstate.local_energy(p, N, M, Lx, 1, 1.0, spins)
    lr, shift = 0.1, 1e-2
    _, info = groundstate.sr_energy_step(p, O, El, lr, shift)
    cd = torch.complex128 if prec == 0 else torch.complex64
    ctx = api.Context(Lx, 1, M, B, prec=prec, explicit_s=solver == 0)
    pr = dev(p, cd)
    st = torch.zeros(8, dtype=torch.float64, device="cuda")
    ctx.sr_step(pr, dev(spins, torch.int8), dev(O[:, N:N + M], cd), dev(El, cd), lr, shift,
                solver=solver, cg_maxit=500, cg_tol=1e-12 if prec == 0 else 1e-6, stats_out=st,
                mode=api.SR_ENERGY)
    ctx.sync_status()
    s = host(st)
    assert s[0] == 0.0
    assert complex(s[1], s[2]) == pytest.approx(info["E"], rel=1e-9 if prec == 0 else 1e-5)
    d = host(pr).astype(np.complex128) - p
    ev = np.linalg.eigvalsh(info["S"]) + shift
    kappa = ev[-1] / ev[0]
    if prec == 0:
        tol = 1e-9 if solver == 0 else max(1e-9, 10 * kappa * 1e-12)
    else:
        tol = max(2e-3, 10 * kappa * 1e-6)
    assert relerr(d, info["delta"]) < tol


def test_sampled_descent_approaches_the_ground_energy():
    from paper_2103_08804_gb300 import api, groundstate as gsd
    Lx, M, B = 12, 24, 2048
    e0 = np.linalg.eigvalsh(exact.hamiltonian(Lx, 1, 1.0, exact.sector_basis(Lx)))[0]
    ctx = api.Context(Lx, 1, M, B, prec=api.FP32)
    g = gsd.GroundState(ctx, synth.rbm_params(9, Lx, M, 0.05), synth.sz0_spins(10, B, Lx),
                        lr=0.05, shift=1e-3, seed=11, cg_maxit=100, cg_tol=1e-5)
    g.thermalise(20)
    for _ in range(300):
        g.step()
    ctx.sync_status()
    E = g.energies()
    assert np.all(np.isfinite(E))
    assert E[0] > 0.5 * e0                     # a random RBM is far from the ground state
    assert np.mean(E[-20:]) < 0.95 * e0        # within 5% of E0 = -5.387 after 300 steps
    assert np.mean(E[-20:]) > e0 - 0.05 * abs(e0)  # and not below it beyond the sampling noise
