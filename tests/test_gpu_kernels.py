"""Kernel-by-kernel parity of the CUDA path (through the C ABI) with the oracle.

Tolerances: float64 contexts must agree to 1e-10 relative (rounding order
only).  float32 contexts: unit roundoff u = 6e-8; log psi sums N + M terms of
size O(1) (absolute error ~ (N + M) u |theta| < 2e-4 at the sizes here), a
bond ratio is a product of M factors (relative ~ M u ~ 1e-5) and R sums
N_b of them, so R, moments and reductions are held to 1e-4 relative.
Integer work (spins, accepted counts) is bit-exact.
"""

import numpy as np
import pytest

from gpu_common import dev, host, logdiff, need_gpu, relerr, torch
from oracle import exact, lattice, rbm, sampler, sr, target
from oracle.target import State
from paper_2103_08804_gb300 import synth

pytestmark = pytest.mark.gpu

PRECS = {"fp64": (0, torch.complex128, 1e-10, 1e-10), "fp32": (1, torch.complex64, 2e-4, 1e-4),
         # mixed: the CG products on the tensor cores (sigma exact in bf16, the
         # other operand split into three bf16 terms): float32-like accuracy
         "mixed": (2, torch.complex64, 2e-4, 1e-4)}
# (Lx, Ly, alpha, sigma, walkers): several tiles of every kernel plus a ragged tail
CASES = [(12, 1, 1, 0.05, 1024), (4, 3, 2, 0.1, 333), (8, 1, 3, 0.1, 37), (64, 1, 2, 0.02, 517)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _ctx(Lx, Ly, M, B, prec, explicit=False):
    from paper_2103_08804_gb300 import api
    return api.Context(Lx, Ly, M, B, prec=prec, explicit_s=explicit)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES)
def test_rbm_logpsi(prec, case):
    Lx, Ly, alpha, sig, B = case
    N, M = Lx * Ly, alpha * Lx * Ly
    p, cd, tol_lp, _ = PRECS[prec]
    params = synth.rbm_params(3, N, M, 4 * sig)
    spins = synth.sz0_spins(4, B, N)
    ctx = _ctx(Lx, Ly, M, B, p)
    th = torch.empty(B, M, dtype=cd, device="cuda")
    lp = ctx.rbm_logpsi(dev(params, cd), dev(spins, torch.int8), theta_out=th)
    ref_th = rbm.theta(params, N, M, spins)
    ref_lp = rbm.logpsi(params, N, M, spins)
    assert relerr(host(th), ref_th) < (1e-12 if prec == "fp64" else 1e-5)
    assert np.max(logdiff(host(lp), ref_lp)) < tol_lp


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_logderiv_explicit_and_tanh(prec):
    Lx, Ly, M, B = 4, 3, 10, 61
    N = Lx * Ly
    p, cd, _, tol = PRECS[prec]
    params = synth.rbm_params(5, N, M, 0.3)
    spins = synth.sz0_spins(6, B, N)
    ctx = _ctx(Lx, Ly, M, B, p)
    th = torch.empty(B, M, dtype=cd, device="cuda")
    ctx.rbm_logpsi(dev(params, cd), dev(spins, torch.int8), theta_out=th)
    T = torch.empty(B, M, dtype=cd, device="cuda")
    O = torch.empty(B, ctx.P, dtype=cd, device="cuda")
    ctx.logderiv(dev(params, cd), dev(spins, torch.int8), th, tanh_out=T, O_out=O)
    ref = rbm.logderiv(params, N, M, spins)
    assert relerr(host(O), ref) < tol
    assert relerr(host(T), ref[:, N:N + M]) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES)
def test_mc_sweep_trajectories(prec, case):
    Lx, Ly, alpha, sig, B = case
    N, M = Lx * Ly, alpha * Lx * Ly
    p, cd, tol_lp, _ = PRECS[prec]
    from paper_2103_08804_gb300 import api
    params = synth.rbm_params(7, N, M, 4 * sig)
    spins0 = synth.sz0_spins(8, B, N)
    n_sweeps = 3 if N <= 12 else 1
    ctx = _ctx(Lx, Ly, M, B, p)
    sp = dev(spins0, torch.int8)
    th = torch.empty(B, M, dtype=cd, device="cuda")
    pr = dev(params, cd)
    ctx.rbm_logpsi(pr, sp, theta_out=th)
    rng = api.Philox(1234567, 99)
    lp = torch.empty(B, dtype=cd, device="cuda")
    acc = torch.empty(B, dtype=torch.int32, device="cuda")
    ctx.mc_sweep(pr, sp, th, n_sweeps, rng, logpsi_out=lp, n_accepted=acc)
    assert rng.counter == 99 + (n_sweeps * N + 1) // 2
    # the oracle on every walker for small batches, on a sample of walkers otherwise
    ids = np.arange(B) if B <= 1024 and N <= 12 else np.arange(0, B, max(1, B // 48))
    bl = lattice.bonds(Lx, Ly)
    s_ref, acc_ref, ctr = sampler.mc_sweep(params, N, M, bl, spins0[ids], n_sweeps, 1234567, 99,
                                           walker_ids=ids)
    assert ctr == rng.counter
    s_gpu, acc_gpu = host(sp)[ids], host(acc)[ids]
    assert np.all(host(sp).sum(axis=1) == 0)
    same = np.all(s_gpu == s_ref, axis=1) & (acc_gpu == acc_ref)
    if prec == "fp64":
        assert np.all(same)
    else:
        # float32 decisions may differ from float64 only at near-ties
        assert same.mean() >= 0.98
    lp_ref = rbm.logpsi(params, N, M, s_gpu)
    assert np.max(logdiff(host(lp)[ids], lp_ref)) < tol_lp
    assert relerr(host(th)[ids], rbm.theta(params, N, M, s_gpu)) < (1e-10 if prec == "fp64" else 1e-4)


def _target_states(N, M, n, sig):
    psi = synth.rbm_params(11, N, M, sig)
    prev = State(psi, probe=True) if n == 1 else State(synth.rbm_params(12, N, M, sig))
    prev2 = State(psi, probe=True) if n == 2 else State(synth.rbm_params(13, N, M, sig))
    return prev, prev2, synth.rbm_params(14, N, M, sig)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [1, 2, 3])
@pytest.mark.parametrize("case", CASES)
def test_local_target(prec, n, case):
    Lx, Ly, alpha, sig, B = case
    N, M = Lx * Ly, alpha * Lx * Ly
    p, cd, _, tol = PRECS[prec]
    q = (np.pi / 2, np.pi) if Ly > 1 else (np.pi / 2, 0.0)
    J, E0, a, Wp = 1.0, -0.75 * len(lattice.bonds(Lx, Ly)), 3.3, 0.9875
    prev, prev2, psin = _target_states(N, M, n, 4 * sig)
    spins = synth.sz0_spins(15, B, N)
    bp, bp2 = 0.7 - 0.2j, -0.4 + 0.9j
    ctx = _ctx(Lx, Ly, M, B, p)
    sp = dev(spins, torch.int8)
    lpn = ctx.rbm_logpsi(dev(psin, cd), sp)
    betas = dev(np.array([bp, bp2]), torch.complex128)
    tp, tp2 = dev(prev.params, cd), dev(prev2.params, cd)
    mean = torch.zeros(1, dtype=torch.complex128, device="cuda")
    R = ctx.cheb_local_target(n, ctx.state(tp, prev.probe, q), ctx.state(tp2, prev2.probe, q),
                              betas[0:1], betas[1:2], E0, a, Wp, sp, lpn, mean_out=mean)
    ids = np.arange(B) if B <= 1024 else np.arange(0, B, 7)
    lp_ref = rbm.logpsi(psin, N, M, spins[ids])
    ref = target.local_target(n, prev, prev2, bp, bp2, N, M, Lx, Ly, J, E0, a, Wp, q, spins[ids],
                              lp_ref)
    Rg = host(R)[ids]
    # compare against the oracle's log psi_n at the same samples
    Rg = Rg * np.exp(host(lpn)[ids] - lp_ref)
    assert relerr(Rg, ref) < tol
    if len(ids) == B:
        assert abs(host(mean)[0] - np.mean(ref)) < tol * np.max(np.abs(ref))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_logpsi_backward(prec):
    Lx, Ly, M, B = 8, 1, 16, 300
    N = Lx * Ly
    p, cd, _, tol = PRECS[prec]
    params = synth.rbm_params(16, N, M, 0.3)
    spins = synth.sz0_spins(17, B, N)
    g = synth.rbm_params(18, B, 0, 1.0)[:B]
    ctx = _ctx(Lx, Ly, M, B, p)
    sp = dev(spins, torch.int8)
    th = torch.empty(B, M, dtype=cd, device="cuda")
    T = torch.empty(B, M, dtype=cd, device="cuda")
    ctx.rbm_logpsi(dev(params, cd), sp, theta_out=th)
    ctx.logderiv(dev(params, cd), sp, th, tanh_out=T)
    grad = ctx.logpsi_backward(dev(params, cd), sp, T, dev(g, cd))
    ref = np.conj(rbm.logderiv(params, N, M, spins)).T @ g
    assert relerr(host(grad), ref) < tol


def _sr_inputs(Lx, Ly, M, B, seed):
    N = Lx * Ly
    params = synth.rbm_params(seed, N, M, 0.2)
    spins = synth.sz0_spins(seed + 1, B, N)
    O = rbm.logderiv(params, N, M, spins)
    g = np.random.Generator(np.random.Philox(seed + 2))
    R = 1.0 + 0.3 * (g.standard_normal(B) + 1j * g.standard_normal(B))
    return params, spins, O, R


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sr_step_cholesky(prec):
    Lx, Ly, M, B = 12, 1, 12, 1024
    N = Lx * Ly
    p, cd, _, tol = PRECS[prec]
    params, spins, O, R = _sr_inputs(Lx, Ly, M, B, 20)
    ref, info = sr.sr_step(params, O, R, 1e-3, 0.5)
    ctx = _ctx(Lx, Ly, M, B, p, explicit=True)
    pr = dev(params, cd)
    T = dev(O[:, N:N + M], cd)
    stats = torch.zeros(8, dtype=torch.float64, device="cuda")
    from paper_2103_08804_gb300 import api
    ctx.sr_step(pr, dev(spins, torch.int8), T, dev(R, cd), 0.5, 1e-3, solver=api.SOLVE_CHOLESKY,
                stats_out=stats)
    ctx.sync_status()
    st = host(stats)
    assert st[0] == pytest.approx(info["gamma"], rel=1e-9 if prec == "fp64" else 1e-5)
    assert complex(st[1], st[2]) == pytest.approx(info["mR"], rel=1e-9 if prec == "fp64" else 1e-5)
    d_gpu = host(pr).astype(np.complex128) - params
    assert relerr(d_gpu, info["delta"]) < (1e-9 if prec == "fp64" else 2e-3)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
@pytest.mark.parametrize("shape", [(12, 1, 12, 1024), (16, 1, 32, 2000), (64, 1, 128, 700),
                                   (10, 1, 20, 333)])
@pytest.mark.parametrize("jacobi", [False, True])
def test_sr_step_cg_matches_oracle_cg(prec, shape, jacobi):
    """float64: the matrix-free (preconditioned) CG against the oracle's
    textbook CG on the explicit S with the same stopping rule (both stop at
    the same iteration).  float32: products in float32 limit the attainable
    residual, so the solution is held to the direct solve within
    kappa-scaled float32 error."""
    Lx, Ly, M, B = shape
    N = Lx * Ly
    p, cd, _, _ = PRECS[prec]
    params, spins, O, R = _sr_inputs(Lx, Ly, M, B, 30)
    shift = 1e-2 if M <= 32 else 1.0
    tol = 1e-10 if prec == "fp64" else 1e-5
    _, info = sr.sr_step(params, O, R, shift, 0.5, solver="cg", cg_maxit=300, cg_tol=tol,
                         jacobi=jacobi)
    _, its = sr.cg_solve(info["S"], info["F"], shift, 300, tol, jacobi)
    ctx = _ctx(Lx, Ly, M, B, p)
    pr = dev(params, cd)
    stats = torch.zeros(8, dtype=torch.float64, device="cuda")
    from paper_2103_08804_gb300 import api
    ctx.sr_step(pr, dev(spins, torch.int8), dev(O[:, N:N + M], cd), dev(R, cd), 0.5, shift,
                solver=api.SOLVE_CG, cg_maxit=300, cg_tol=tol, stats_out=stats, jacobi=jacobi)
    ctx.sync_status()
    st = host(stats)
    d_gpu = host(pr).astype(np.complex128) - params
    ev = np.linalg.eigvalsh(info["S"]) + shift
    if prec == "fp64":
        # after a long plateau near the threshold the two may stop a few steps apart;
        # two solves that stop at |r| <= tol |F| each lie within kappa tol of the
        # solution, so they may differ by 2 kappa tol
        assert abs(st[5] - its) <= max(1, 0.05 * its)
        assert relerr(d_gpu, info["delta"]) < max(1e-8, 2 * (ev[-1] / ev[0]) * tol)
    else:
        x_exact = sr.shifted_solve(info["S"], info["F"], shift)
        assert st[6] <= tol
        assert relerr(d_gpu, x_exact) < (ev[-1] / ev[0]) * 1e-5


@pytest.mark.parametrize("jacobi", [False, True])
def test_sr_step_cg_converges_to_direct_solve(jacobi):
    Lx, Ly, M, B = 16, 1, 32, 2000
    N = Lx * Ly
    params, spins, O, R = _sr_inputs(Lx, Ly, M, B, 31)
    shift = 1e-2
    _, info = sr.sr_step(params, O, R, shift, 0.5)
    ctx = _ctx(Lx, Ly, M, B, 0)
    pr = dev(params, torch.complex128)
    stats = torch.zeros(8, dtype=torch.float64, device="cuda")
    from paper_2103_08804_gb300 import api
    ctx.sr_step(pr, dev(spins, torch.int8), dev(O[:, N:N + M], torch.complex128),
                dev(R, torch.complex128), 0.5, shift, solver=api.SOLVE_CG, cg_maxit=2000,
                cg_tol=1e-12, stats_out=stats, jacobi=jacobi)
    ctx.sync_status()
    st = host(stats)
    assert st[6] <= 1e-12 and st[5] < 2000
    assert relerr(host(pr) - params, info["delta"]) < 1e-8


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("probe", [True, False])
def test_cheb_moment_columns(prec, probe):
    Lx, Ly, M, B = 4, 3, 12, 700
    N = Lx * Ly
    p, cd, _, tol = PRECS[prec]
    q = (np.pi, np.pi / 3)
    psi = synth.rbm_params(40, N, M, 0.2)
    st = State(psi if probe else synth.rbm_params(41, N, M, 0.2), probe=probe)
    spins = synth.sz0_spins(42, B, N)
    beta = 0.3 - 0.8j
    E0, a, Wp = -5.0, 4.0, 0.9875
    ctx = _ctx(Lx, Ly, M, B, p)
    sp = dev(spins, torch.int8)
    lpr = ctx.rbm_logpsi(dev(psi, cd), sp)
    Bc = torch.empty(B, dtype=cd, device="cuda")
    HBc = torch.empty(B, dtype=cd, device="cuda")
    mu = torch.zeros(1, dtype=torch.complex128, device="cuda")
    ctx.cheb_moment(ctx.state(dev(st.params, cd), probe, q), dev(np.array([beta]), torch.complex128),
                    q, sp, lpr, hprime=(E0, a, Wp), Bcol=Bc, HBcol=HBc, mu_out=mu)
    lp_ref = rbm.logpsi(psi, N, M, spins)
    scale = np.exp(host(lpr) - lp_ref)  # GPU log psi vs oracle log psi at the same samples
    Bref = beta * target.rel_amplitude(st, N, M, Lx, Ly, q, spins, lp_ref)
    HBref = beta * target.apply_hprime(st, N, M, Lx, Ly, 1.0, E0, a, Wp, q, spins, lp_ref)
    assert relerr(host(Bc) * scale, Bref) < tol
    assert relerr(host(HBc) * scale, HBref) < tol
    f = lattice.probe(Lx, Ly, q[0], q[1], spins)
    assert host(mu)[0] == pytest.approx(np.mean(np.conj(f) * Bref), rel=10 * tol, abs=1e-12)


def test_gram_and_krylov_on_exact_vectors():
    # exact Chebyshev vectors of a 10-site chain as columns (enumeration weights folded in)
    from oracle import krylov
    Lx, Nm = 10, 6
    basis = exact.sector_basis(Lx)
    H = exact.hamiltonian(Lx, 1, 1.0, basis)
    e = np.linalg.eigvalsh(H)
    a = (e[-1] - e[0]) / (2 * 0.9875)
    Hp = exact.rescaled(H, e[0], a, 0.9875)
    psi = exact.rbm_vector(synth.rbm_params(50, Lx, 10, 0.3), Lx, 10, basis)
    t0 = exact.probe_vector(Lx, 1, 0.6 * np.pi, 0.0, basis, psi)
    ts = exact.chebyshev_vectors(Hp, t0, Nm)
    w = np.abs(psi) ** 2 / np.vdot(psi, psi).real
    D = len(basis)
    # sample means over D "samples" reproduce the weighted sums if every column carries sqrt(D w)
    sq = np.sqrt(D * w)
    Bm = np.array([sq * t / psi for t in ts])
    HBm = np.array([sq * (Hp @ t) / psi for t in ts])
    G_ref, H_ref = krylov.gram(list(Bm), list(HBm))
    mu_ex = exact.chebyshev_moments(Hp, t0, psi, 2 * Nm)
    ctx = _ctx(Lx, 1, 10, D, 0)
    Gd = torch.zeros(Nm, Nm, dtype=torch.complex128, device="cuda")
    Hd = torch.zeros_like(Gd)
    ctx.cheb_gram(dev(Bm, torch.complex128), dev(HBm, torch.complex128), Gd, Hd)
    assert relerr(host(Gd), G_ref) < 1e-12
    assert relerr(host(Hd), H_ref) < 1e-12
    mu = torch.zeros(2 * Nm, dtype=torch.complex128, device="cuda")
    poles = torch.zeros(Nm, dtype=torch.float64, device="cuda")
    wts = torch.zeros(Nm, dtype=torch.float64, device="cuda")
    rank = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.cheb_krylov(Gd, Hd, 1e-13, 2 * Nm, mu, poles, wts, rank)
    assert int(host(rank)[0]) == Nm
    assert np.allclose(host(mu), mu_ex, atol=1e-8 * abs(mu_ex[0]))
    lam, wk = krylov.krylov_poles(G_ref, H_ref, cutoff=1e-13)
    assert np.allclose(host(poles), np.sort(lam), atol=1e-9)
    assert np.allclose(host(wts), wk[np.argsort(lam)], atol=1e-9 * abs(mu_ex[0]))


@pytest.mark.parametrize("Nm", [40, 100, 300])
def test_krylov_against_oracle_at_scale(Nm):
    """cheb_krylov on a well-conditioned Gram pair of Nm states (random states,
    G = X^dag X / D, H = X^dag A X / D with spec(A) in [-W', W']): poles,
    weights and corrected moments equal the oracle's, and the weights sum to
    mu'_0 = G_00."""
    from oracle import krylov
    rng = np.random.default_rng(60 + Nm)
    D = 3 * Nm
    X = (rng.standard_normal((D, Nm)) + 1j * rng.standard_normal((D, Nm))) / np.sqrt(2)
    A = rng.standard_normal((D, D)) + 1j * rng.standard_normal((D, D))
    A = (A + A.conj().T) / 2
    e = np.linalg.eigvalsh(A)
    A = (A - e[0] * np.eye(D)) / ((e[-1] - e[0]) / 1.975) - 0.9875 * np.eye(D)
    G = X.conj().T @ X / D
    H = X.conj().T @ A @ X / D
    H = (H + H.conj().T) / 2
    n_out = 2 * Nm if Nm <= 100 else 64
    ctx = _ctx(4, 1, 4, 8, 0)
    mu = torch.zeros(n_out, dtype=torch.complex128, device="cuda")
    poles = torch.zeros(Nm, dtype=torch.float64, device="cuda")
    wts = torch.zeros(Nm, dtype=torch.float64, device="cuda")
    rank = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.cheb_krylov(dev(G, torch.complex128), dev(H, torch.complex128), 1e-12, n_out, mu, poles,
                    wts, rank)
    ctx.sync_status()
    assert int(host(rank)[0]) == Nm
    lam_ref, w_ref = krylov.krylov_poles(G, H, cutoff=1e-12)
    order = np.argsort(lam_ref)
    assert np.allclose(host(poles), lam_ref[order], atol=1e-9)
    assert np.allclose(host(wts), w_ref[order], atol=1e-9 * abs(G[0, 0]))
    mc = krylov.corrected_moments(G, H, n_out, cutoff=1e-12)
    assert np.allclose(host(mu), mc, atol=1e-8 * abs(G[0, 0]))
    assert abs(np.sum(host(wts)) - G[0, 0].real) < 1e-9 * abs(G[0, 0])


def test_zero_walkers_is_a_no_op():
    from paper_2103_08804_gb300 import api
    ctx = _ctx(8, 1, 8, 16, 1)
    pr = dev(synth.rbm_params(1, 8, 8, 0.1), torch.complex64)
    sp = torch.empty(0, 8, dtype=torch.int8, device="cuda")
    th = torch.empty(0, 8, dtype=torch.complex64, device="cuda")
    rng = api.Philox(5, 10)
    ctx.mc_sweep(pr, sp, th, 2, rng)
    assert rng.counter == 10 + 8  # the stream still advances
    ctx.rbm_logpsi(pr, sp)
    ctx.sync_status()


def test_bad_arguments_raise():
    from paper_2103_08804_gb300 import api
    ctx = _ctx(8, 1, 8, 16, 1)
    pr = dev(synth.rbm_params(1, 8, 8, 0.1), torch.complex64)
    sp = dev(synth.sz0_spins(1, 32, 8), torch.int8)  # more walkers than the context allows
    with pytest.raises(api.CRError):
        ctx.rbm_logpsi(pr, sp)
    with pytest.raises(ValueError):
        ctx.rbm_logpsi(pr.to(torch.complex128), sp[:4])
