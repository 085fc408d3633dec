"""Explicit S and the blocked direct solve (Sec. III) against the oracle.

S: float64 contexts accumulate the Gram matrix of O in float64 (rounding
order only); float32 contexts form float32 products (relative ~1e-7); mixed
contexts form it on the tensor cores from bf16 splits of both operands with
float32 accumulation: three-term splits (six products, float32-like, held
to 2e-6 relative in the Frobenius norm) by default, two-term splits (three
products, ~2^-16 relative per product, held to 1e-4) with CR_CTX_S_BF16X3;
and element by element (the largest entry error against the largest entry,
so that one bad tile or row fails) against the oracle's S of the same
rounded inputs.

Solve: the blocked Cholesky plus float64 refinement must certify, by its
own float64 residual, that it solved the system the GPU built
(|F - S x| <= 1e-10 |F|); the float64 update must then match the oracle's
float64 Cholesky update to rounding, and the float32 / mixed updates within
the condition number times the error of S.
Shapes span several 64-row factor blocks, several 128 x 512 Gram tiles and
ragged walker counts; P = 2144 also takes the float64 blocked path."""

import numpy as np
import pytest

from gpu_common import dev, host, need_gpu, relerr, torch
from oracle import rbm, sr
from paper_2103_08804_gb300 import synth

pytestmark = pytest.mark.gpu

PREC = {"fp64": (0, torch.complex128), "fp32": (1, torch.complex64),
        "mixed": (2, torch.complex64), "mixed_x3": (2, torch.complex64)}
S_TOL = {"fp64": 1e-12, "fp32": 1e-6, "mixed": 2e-6, "mixed_x3": 1e-4}
# Element by element, max_kl |S_kl - S_kl^ref| / max |S^ref|, against the
# oracle's S built from the same (context-precision) tanh(theta) values, so
# that only the arithmetic of the build is measured: float32 products summed
# in float64 (~1e-7), tensor-core products summed in float32 per walker
# chunk (~1e-6), two-term splits (~2^-16 per product).
S_EL_TOL = {"fp64": 1e-12, "fp32": 1e-6, "mixed": 4e-6, "mixed_x3": 2e-4}
# (Lx, Ly, M, walkers): P = 560 (chain), 424 (4 x 4 square), 2144 (chain)
SHAPES = [(16, 1, 32, 2000), (4, 4, 24, 777), (32, 1, 64, 4096)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _inputs(Lx, Ly, M, B, seed):
    N = Lx * Ly
    params = synth.rbm_params(seed, N, M, 0.2)
    spins = synth.sz0_spins(seed + 1, B, N)
    O = rbm.logderiv(params, N, M, spins)
    g = np.random.Generator(np.random.Philox(seed + 2))
    R = 1.0 + 0.3 * (g.standard_normal(B) + 1j * g.standard_normal(B))
    return params, spins, O, R


def _ctx(Lx, Ly, M, B, prec):
    from paper_2103_08804_gb300 import api
    return api.Context(Lx, Ly, M, B, prec=PREC[prec][0], explicit_s=True,
                       s_bf16x3=prec == "mixed_x3")


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed", "mixed_x3"])
@pytest.mark.parametrize("shape", SHAPES)
def test_explicit_s_against_oracle(prec, shape):
    Lx, Ly, M, B = shape
    if prec == "fp64" and Lx * Ly > 16:
        pytest.skip("the float64 Gram at P = 2144 is covered by the solve test")
    N = Lx * Ly
    p, cd = PREC[prec]
    params, spins, O, R = _inputs(Lx, Ly, M, B, 50)
    shift = 1e-3
    S_ref = sr.qgt(sr.estimators(O, R)) + shift * np.eye(O.shape[1])
    ctx = _ctx(Lx, Ly, M, B, prec)
    S = host(ctx.sr_smatrix(dev(spins, torch.int8), dev(O[:, N:N + M], cd), shift))
    ctx.sync_status()
    err = np.linalg.norm(S - S_ref) / np.linalg.norm(S_ref)
    assert err < S_TOL[prec], err
    T_in = O[:, N:N + M].astype(np.complex64 if cd == torch.complex64 else np.complex128)
    S_in = sr.qgt(sr.estimators(rbm.logderiv_from_tanh(spins, T_in), R)) + shift * np.eye(O.shape[1])
    el = np.max(np.abs(S - S_in)) / np.max(np.abs(S_in))
    worst = np.unravel_index(np.argmax(np.abs(S - S_in)), S.shape)
    print(f"{prec} {shape}: S Frobenius {err:.2e}, element-wise {el:.2e} at {worst}")
    assert el < S_EL_TOL[prec], (el, worst)
    A = S - S.conj().T
    np.fill_diagonal(A, 0)
    assert not A.any()                            # off-diagonal mirrored exactly
    assert np.all(np.abs(np.diag(S).imag) <= 1e-6 * np.abs(np.diag(S).real))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed", "mixed_x3"])
@pytest.mark.parametrize("shape", SHAPES)
def test_blocked_cholesky_update(prec, shape):
    from paper_2103_08804_gb300 import api
    Lx, Ly, M, B = shape
    N = Lx * Ly
    p, cd = PREC[prec]
    params, spins, O, R = _inputs(Lx, Ly, M, B, 60)
    shift = 1e-3
    ref, info = sr.sr_step(params, O, R, shift, 0.5)
    ctx = _ctx(Lx, Ly, M, B, prec)
    P = ctx.P
    blocked = prec != "fp64" or P > 2048
    sp, T = dev(spins, torch.int8), dev(O[:, N:N + M], cd)
    S_gpu = host(ctx.sr_smatrix(sp, T, shift)).astype(np.complex128)
    pr = dev(params, cd)
    stats = torch.zeros(8, dtype=torch.float64, device="cuda")
    ctx.sr_step(pr, sp, T, dev(R, cd), 0.5, shift, solver=api.SOLVE_CHOLESKY, stats_out=stats)
    ctx.sync_status()
    st = host(stats)
    d_gpu = host(pr).astype(np.complex128) - params
    ev = np.linalg.eigvalsh(S_gpu)
    kappa = ev[-1] / ev[0]
    if blocked:
        # the refinement's own float64 residual certifies the solve of the
        # system the GPU built: |F - S x| <= 1e-10 |F|
        assert 1 <= st[5] <= 10 and st[6] <= 1e-10, st
    if prec == "fp64":
        assert relerr(d_gpu, info["delta"]) < max(1e-9, kappa * 1e-13)
    else:
        # what remains is the error of S (and of F: float32 reductions),
        # amplified by the condition number
        s_err = np.linalg.norm(S_gpu - info["S"] - shift * np.eye(P)) / np.linalg.norm(S_gpu)
        assert relerr(d_gpu, info["delta"]) < max(2e-3, 10 * kappa * max(s_err, 1e-6))
