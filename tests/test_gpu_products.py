"""The products of the matrix-free natural-gradient solve (Sec. III),
u = O v and (S + lambda I) v = O^dag (O v) / B - <O>^* (<O> . v) + lambda v,
through sr_sv (the same kernels as the CG of sr_step: tensor cores in mixed
contexts), element by element against the oracle's explicit O built from the
same tanh(theta) values, up to the 64-site chain workload shape (16384
walkers, 128 walker chunks) with a ragged walker tail; the starting
parameters of a projection step against the oracle; and the device status
paths (non-finite estimators, a singular direct solve, CG that stops at its
iteration limit)."""

import numpy as np
import pytest

from gpu_common import dev, host, need_gpu, relerr, torch
from oracle import chebyshev, rbm
from paper_2103_08804_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


PRECS = {"fp64": (0, torch.complex128, np.complex128),
         "fp32": (1, torch.complex64, np.complex64),
         "mixed": (2, torch.complex64, np.complex64)}


def _inputs(Lx, Ly, M, B, sigma, seed, npdt):
    """Spins, T = tanh(theta) in the context precision (the oracle takes the
    same rounded values), a direction v."""
    N = Lx * Ly
    params = synth.rbm_params(seed, N, M, sigma)
    spins = synth.sz0_spins(seed + 1, B, N)
    T = np.tanh(rbm.theta(params, N, M, spins)).astype(npdt).astype(np.complex128)
    v = synth.rbm_params(seed + 2, N, M, 1.0)
    return spins, T, v


def _oracle_sv(spins, T, v, shift, block=1024):
    """u = O v and (S + shift I) v from the explicit O, walker block by block."""
    B = spins.shape[0]
    u = np.empty(B, dtype=np.complex128)
    acc = np.zeros(len(v), dtype=np.complex128)
    sumO = np.zeros(len(v), dtype=np.complex128)
    for s0 in range(0, B, block):
        O = rbm.logderiv_from_tanh(spins[s0:s0 + block], T[s0:s0 + block])
        ub = O @ v
        u[s0:s0 + block] = ub
        acc += np.conj(O).T @ ub
        sumO += O.sum(axis=0)
    Obar = sumO / B
    return u, acc / B - np.conj(Obar) * (Obar @ v) + shift * v


# (Lx, Ly, M, B): several walker tiles and chunks with ragged tails; the last
# is the 64-site chain workload (P = 8384) with 16381 walkers in 128 chunks.
SHAPES = [(12, 1, 12, 1000), (10, 1, 20, 333), (8, 8, 128, 4099), (64, 1, 128, 16381)]
# float64: rounding only.  float32 and mixed: products of float32 values with
# float32 accumulation (tensor-core TMEM or FMA) over 128-walker chunks, then
# float64: about 1e-6 of the largest entry; gate 1e-5.
TOL = {"fp64": 1e-11, "fp32": 1e-5, "mixed": 1e-5}


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
@pytest.mark.parametrize("shape", SHAPES)
def test_sv_products_against_explicit_O(prec, shape):
    from paper_2103_08804_gb300 import api
    Lx, Ly, M, B = shape
    if prec == "fp64" and B > 5000:
        pytest.skip("float64 products are covered at the smaller shapes")
    p, cd, npdt = PRECS[prec]
    spins, T, v = _inputs(Lx, Ly, M, B, 0.02 if M >= 64 else 0.2, 60, npdt)
    shift = 1e-3
    u_ref, sv_ref = _oracle_sv(spins, T, v, shift)
    ctx = api.Context(Lx, Ly, M, B, prec=p)
    u = torch.empty(B, dtype=cd, device="cuda")
    out = ctx.sr_sv(dev(spins, torch.int8), dev(T, cd), dev(v, torch.complex128), shift, u_out=u)
    ctx.sync_status()
    eu, es = relerr(host(u), u_ref), relerr(host(out), sv_ref)
    print(f"{prec} {shape}: u = O v {eu:.2e}, (S + lambda) v {es:.2e}")
    assert eu < TOL[prec] and es < TOL[prec]


def _oracle_estimators(spins, T, R, block=256):
    """<R>, <|R|^2>, <O> and <O* R> from the explicit O, walker block by block."""
    B = spins.shape[0]
    Obar = OR = 0.0
    for s0 in range(0, B, block):
        O = rbm.logderiv_from_tanh(spins[s0:s0 + block], T[s0:s0 + block])
        Obar = Obar + O.sum(axis=0)
        OR = OR + (np.conj(O) * R[s0:s0 + block, None]).sum(axis=0)
    return {"mR": R.mean(), "mRR": float(np.mean(np.abs(R) ** 2)), "Obar": Obar / B, "OR": OR / B}


# the estimator sums (F, <O>, <R>, <|R|^2>) of one natural-gradient step:
# float32 path compensated float32 sums, mixed path tensor cores (bf16 splits,
# float32 accumulation over 128-walker chunks and K segments, float64 across):
# about 1e-7 of the summed terms; gate 1e-6
EST_TOL = {"fp32": 1e-6, "mixed": 1e-6}


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
@pytest.mark.parametrize("shape", [(12, 1, 12, 1000), (8, 8, 128, 4099), (16, 16, 256, 4099)])
def test_estimators_and_force_against_oracle(prec, shape):
    """F through the update of a step on a zero RBM: one CG iteration on
    (S + lambda I) x = F gives x = F |F|^2 / F^dag (S + lambda I) F (the
    oracle forms F^dag S F matrix-free), and the update writes x into the zero
    parameters (float32 rounding only); lambda = 1e9 keeps x a scaled F."""
    from oracle import sr
    from paper_2103_08804_gb300 import api
    Lx, Ly, M, B = shape
    N = Lx * Ly
    p, cd, npdt = PRECS[prec]
    spins, T, _ = _inputs(Lx, Ly, M, B, 0.05, 90, npdt)
    g = np.random.Generator(np.random.Philox(91))
    R = (1.0 + 0.3 * (g.standard_normal(B) + 1j * g.standard_normal(B))).astype(npdt)
    est = _oracle_estimators(spins, T, R.astype(np.complex128))
    F_ref, gamma = sr.force(est, 0.5)
    ctx = api.Context(Lx, Ly, M, B, prec=p)
    pr = torch.zeros(ctx.P, dtype=cd, device="cuda")
    stats = torch.zeros(api.STATS_LEN, dtype=torch.float64, device="cuda")
    ctx.sr_step(pr, dev(spins, torch.int8), dev(T, cd), dev(R, cd), 0.5, 1e9,
                solver=api.SOLVE_CG, cg_maxit=1, cg_tol=1e-12, stats_out=stats)
    ctx.sync_status()
    st = host(stats)
    assert st[0] == pytest.approx(gamma, rel=1e-6)
    assert complex(st[1], st[2]) == pytest.approx(est["mR"], rel=1e-6)
    assert st[3] == pytest.approx(est["mRR"], rel=1e-6)
    # F = c (<O* R>/<R> - <O>*) cancels (here R is independent of O): the
    # error of the two float32-accumulated sums is measured against the size
    # of the terms that are subtracted
    c = 0.5 * sr.gamma_cot_gamma(gamma)
    scale = c * np.max(np.abs(est["OR"] / est["mR"]))
    blocks = (rbm.logderiv_from_tanh(spins[s0:s0 + 256], T[s0:s0 + 256]) for s0 in range(0, B, 256))
    fsf = np.vdot(F_ref, sr.sv_matrix_free(blocks, F_ref, 1e9)).real
    x_ref = F_ref * (np.vdot(F_ref, F_ref).real / fsf)
    dF = 1e9 * np.max(np.abs(host(pr).astype(np.complex128) - x_ref))
    print(f"{prec} {shape}: F {dF / scale:.2e} of the terms, {dF / np.max(np.abs(F_ref)):.2e} of F")
    assert dF / scale < EST_TOL[prec]


def test_init_params_match_the_oracle():
    from paper_2103_08804_gb300 import api
    N, M = 12, 12
    psi = synth.rbm_params(70, N, M, 0.05)
    prev = synth.rbm_params(71, N, M, 0.05)
    for prec in ("fp64", "fp32"):
        p, cd, npdt = PRECS[prec]
        ctx = api.Context(N, 1, M, 8, prec=p)
        out = torch.empty(ctx.P, dtype=cd, device="cuda")
        for n in (1, 2, 5):
            ctx.cheb_init_params(n, dev(psi, cd), dev(prev, cd), out)
            want = chebyshev.initial_params(psi.astype(npdt), prev.astype(npdt), n)
            tol = 0.0 if prec == "fp64" else 2e-7
            assert np.max(np.abs(host(out) - want)) <= tol, (prec, n)


# ------------------------------------------------------------ status paths

def _sr_case(prec, B, N=12, M=12, seed=80, identical=False):
    from paper_2103_08804_gb300 import api
    p, cd, npdt = PRECS[prec]
    params = synth.rbm_params(seed, N, M, 0.2)
    spins = synth.sz0_spins(seed + 1, B, N)
    if identical:
        spins[:] = spins[0]
    T = np.tanh(rbm.theta(params, N, M, spins))
    g = np.random.Generator(np.random.Philox(seed + 2))
    R = 1.0 + 0.3 * (g.standard_normal(B) + 1j * g.standard_normal(B))
    return api, cd, dev(params, cd), dev(spins, torch.int8), dev(T, cd), R


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_nonfinite_local_target_sets_enonfinite(prec):
    """A NaN planted in R on the host: the force kernel reports CR_ENONFINITE."""
    api, cd, params, spins, T, R = _sr_case(prec, 256)
    R[17] = np.nan
    ctx = api.Context(12, 1, 12, 256, prec=PRECS[prec][0])
    ctx.sr_step(params, spins, T, dev(R, cd), 0.5, 1e-3, solver=api.SOLVE_CG, cg_maxit=5)
    with pytest.raises(api.CRError, match="CR_ENONFINITE"):
        ctx.sync_status()
    ctx.sync_status()  # read and cleared


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_rank_deficient_S_without_shift_sets_esingular(prec):
    """8 copies of one configuration: every O_k is constant over the samples,
    so S = 0, and its first pivot S_00 = <sigma_0^2> - <sigma_0>^2 = 1 - 1 is
    exactly 0 in any precision; with shift 0 the Cholesky factorisation meets
    it (float64 single-CTA path and the blocked float32 path)."""
    api, cd, params, spins, T, R = _sr_case(prec, 8, identical=True)
    ctx = api.Context(12, 1, 12, 8, prec=PRECS[prec][0], explicit_s=True)
    ctx.sr_step(params, spins, T, dev(R, cd), 0.5, 0.0, solver=api.SOLVE_CHOLESKY, cg_maxit=4)
    with pytest.raises(api.CRError, match="CR_ESINGULAR"):
        ctx.sync_status()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
def test_cg_iteration_cap_sets_enotconv_when_strict(prec):
    api, cd, params, spins, T, R = _sr_case(prec, 512)
    ctx = api.Context(12, 1, 12, 512, prec=PRECS[prec][0])
    stats = torch.zeros(api.STATS_LEN, dtype=torch.float64, device="cuda")
    Rd = dev(R, cd)
    # not strict: the truncated solve is reported in the stats only
    ctx.sr_step(params, spins, T, Rd, 0.5, 1e-3, solver=api.SOLVE_CG, cg_maxit=2, cg_tol=1e-12,
                stats_out=stats)
    ctx.sync_status()
    st = host(stats)
    assert st[5] == 2 and st[6] > 1e-12
    ctx.sr_step(params, spins, T, Rd, 0.5, 1e-3, solver=api.SOLVE_CG, cg_maxit=2, cg_tol=1e-12,
                cg_strict=True)
    with pytest.raises(api.CRError, match="CR_ENOTCONV"):
        ctx.sync_status()
    # a solve that converges is not flagged
    ctx.sr_step(params, spins, T, Rd, 0.5, 1.0, solver=api.SOLVE_CG, cg_maxit=500, cg_tol=1e-4,
                cg_strict=True, stats_out=stats)
    ctx.sync_status()
    assert host(stats)[6] <= 1e-4
