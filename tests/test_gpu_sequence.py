"""End-to-end parity of the Chebyshev sequence: CUDA path (driver over the C
ABI) against the oracle, on the 12-site chain workload (alpha = 1, sigma =
0.05, q = pi, 1024 walkers, 10 moments, 20 natural-gradient iterations per
moment, shift 1e-3), both sides drawing from the same Philox stream.

Three gates:
  * free-running float64: walker trajectories bit-identical and beta_n, mu_n
    within 1e-7 mu_0 for the first moments.  The shifted solve is
    ill-conditioned (lambda = 1e-3), so rounding-order differences of 1e-16
    grow by ~x3 per moment; once a fit turns unstable (gamma jumps) they reach
    a Metropolis near-tie and the two chains part.  This is a property of the
    method, not of either implementation, so the later moments are gated by:
  * lockstep float64: every iteration of all 10 moments, one oracle step is
    replayed from the GPU's own state (spins, parameters, counters); spins
    must match exactly and the update to the forward-error bound of a
    backward-stable solve, 2 P u kappa(S + lambda I) |dalpha| (u = 2^-53);
  * replay: the CUDA path consumes the walker configurations the oracle
    recorded (no sampling on either side), so all differences are arithmetic:
    one projection step from the oracle's inputs within 1e-9 mu_0 (float64),
    1e-5 mu_0 (float32) and 1e-3 mu_0 (mixed); the whole float64 recursion
    within 1e-6 mu_0.
"""

import numpy as np
import pytest

from gpu_common import dev, host, need_gpu, torch
from oracle import chebyshev, exact, lattice, rbm, sampler, sr, target
from oracle.target import State
from paper_2103_08804_gb300 import synth

pytestmark = pytest.mark.gpu

WL = synth.WORKLOADS["chain12_fp64"]
# RBM and walker seeds of this instance: its sampled sequence stays stable
# through all 10 moments (every moment within 1.5% mu_0 of the exact one).
SEED = 20


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.fixture(scope="module")
def e0():
    return np.linalg.eigvalsh(exact.hamiltonian(12, 1, 1.0, exact.sector_basis(12)))[0]


def _oracle_cfg(e0, n_moments=WL.moments):
    return chebyshev.Config(Lx=12, Ly=1, M=WL.M, q=WL.q, n_moments=n_moments, n_iter=WL.iters,
                            shift=WL.shift, dgamma=WL.dgamma, E0=e0, a=5.0, Wp=0.9875,
                            seed=SEED, seed_ref=SEED + 1)


def _inputs():
    return (synth.rbm_params(SEED, 12, WL.M, WL.sigma), synth.sz0_spins(SEED + 1, WL.walkers, 12),
            synth.sz0_spins(SEED + 2, WL.walkers, 12))


def _seq(prec, e0, n_moments, solver, cg_tol=1e-12, cg_maxit=400, jacobi=False):
    from paper_2103_08804_gb300 import api, driver
    cfg = driver.SeqConfig(Lx=12, Ly=1, M=WL.M, q=WL.q, n_moments=n_moments, n_iter=WL.iters,
                           shift=WL.shift, dgamma=WL.dgamma, E0=e0, a=5.0, Wp=0.9875,
                           solver=solver, cg_maxit=cg_maxit, cg_tol=cg_tol, jacobi=jacobi,
                           seed=SEED, seed_ref=SEED + 1)
    ctx = api.Context(12, 1, WL.M, WL.walkers, prec=prec, explicit_s=(solver == api.SOLVE_CHOLESKY))
    psi, s_fit, s_ref = _inputs()
    return driver.Sequence(ctx, cfg, psi, s_fit, s_ref), ctx


@pytest.fixture(scope="module")
def recorded(e0):
    psi, s_fit, s_ref = _inputs()
    return chebyshev.run_sampled(_oracle_cfg(e0), psi, s_fit, s_ref, record=True)


def test_fp64_free_running_bit_exact_first_moments(e0, recorded):
    from paper_2103_08804_gb300 import api
    nm = 4
    seq, ctx = _seq(api.FP64, e0, nm, api.SOLVE_CHOLESKY)
    seq.run()
    ctx.sync_status()
    psi, s_fit, s_ref = _inputs()
    ref = chebyshev.run_sampled(_oracle_cfg(e0, nm), psi, s_fit, s_ref)
    assert np.array_equal(host(seq.spins_ref), ref.spins_ref)
    assert np.array_equal(host(seq.spins), ref.spins_fit)
    assert seq.rng.counter == ref.counter_fit and seq.rng_ref.counter == ref.counter_ref
    mu0 = abs(ref.mu[0])
    assert np.max(np.abs(host(seq.mu) - np.array(ref.mu))) < 1e-7 * mu0
    assert np.max(np.abs(host(seq.betas) - np.array(ref.betas))) < 1e-7
    assert np.allclose(host(seq.stats)[1:, :, 0], np.array(ref.gammas), atol=1e-7)
    assert np.max(np.abs(host(seq.params[nm - 1]) - ref.states[nm - 1].params)) < 1e-7
    assert np.max(np.abs(host(seq.Bmat) - np.array(ref.B))) < 1e-7 * np.sqrt(mu0)
    assert np.max(np.abs(host(seq.HBmat) - np.array(ref.HB))) < 1e-7 * np.sqrt(mu0)


def test_fp64_lockstep_every_iteration(e0):
    """Each natural-gradient iteration of all 10 moments, replayed by the oracle
    from the GPU's state before it."""
    from paper_2103_08804_gb300 import api
    seq, ctx = _seq(api.FP64, e0, WL.moments, api.SOLVE_CHOLESKY)
    cfg = seq.cfg
    L, M = 12, WL.M
    bl = lattice.bonds(L, 1)
    seq.start()
    worst = 0.0
    for n in range(1, WL.moments):
        pn = seq.params[n]
        ctx.cheb_init_params(n, seq.params[0], seq.params[n - 1], pn)
        ctx.rbm_logpsi(pn, seq.spins, seq.theta, seq.lp)
        ctx.mc_sweep(pn, seq.spins, seq.theta, cfg.n_therm, seq.rng, logpsi_out=seq.lp,
                     tanh_out=seq.tanh)
        b = None
        for it in range(cfg.n_iter):
            sp0, p0, ctr0 = host(seq.spins).copy(), host(pn).copy(), seq.rng.counter
            ctx.mc_sweep(pn, seq.spins, seq.theta, 1, seq.rng, logpsi_out=seq.lp, tanh_out=seq.tanh)
            seq._target(n)
            ctx.sr_step(pn, seq.spins, seq.tanh, seq.R, cfg.dgamma, cfg.shift,
                        solver=api.SOLVE_CHOLESKY)
            ctx.rbm_logpsi(pn, seq.spins, seq.theta, seq.lp)
            if b is None:
                b = host(seq.betas)
                prev = State(host(seq.params[n - 1]), probe=(n == 1))
                prev2 = State(host(seq.params[n - 2]), probe=(n == 2)) if n >= 2 else None
            sp, _, _ = sampler.mc_sweep(p0, L, M, bl, sp0, 1, cfg.seed, ctr0)
            lp = rbm.logpsi(p0, L, M, sp)
            R = target.local_target(n, prev, prev2, b[n - 1], b[n - 2] if n >= 2 else 0, L, M, L,
                                    1, 1.0, e0, 5.0, 0.9875, WL.q, sp, lp)
            p1, info = sr.sr_step(p0, rbm.logderiv(p0, L, M, sp), R, WL.shift, WL.dgamma)
            assert np.array_equal(host(seq.spins), sp), (n, it)
            ev = np.linalg.eigvalsh(info["S"]) + WL.shift
            bound = 2 * len(p0) * 2.0 ** -53 * (ev[-1] / ev[0]) * np.max(np.abs(info["delta"]))
            d = np.max(np.abs(host(pn) - p1))
            worst = max(worst, d / bound)
            assert d < max(bound, 1e-13), (n, it, d, bound)
        ctx.mc_sweep(pn, seq.spins, seq.theta, 1, seq.rng, logpsi_out=seq.lp, tanh_out=seq.tanh)
        seq._target(n, mean_out=seq.betas[n:n + 1])
        seq._moment(n)
    ctx.sync_status()
    print(f"worst one-iteration parameter difference / bound {worst:.2e}")


def _replay(seq, ref):
    seq.start(replay_ref=dev(ref.spins_ref, torch.int8))
    for n in range(1, seq.cfg.n_moments):
        seq.fit(n, replay=[dev(s, torch.int8) for s in ref.samples[n]])
    seq.ctx.sync_status()
    return host(seq.mu), host(seq.betas)


def _oracle_single_step(ref, e0, n, solver):
    """One projection step of the oracle from its own recorded inputs and
    samples, with the given solver options."""
    psi = ref.states[0].params
    N, M = 12, WL.M
    params = chebyshev.initial_params(psi, ref.states[n - 1].params, n)
    prev, prev2 = ref.states[n - 1], (ref.states[n - 2] if n >= 2 else None)
    b1, b2 = ref.betas[n - 1], (ref.betas[n - 2] if n >= 2 else 0)

    def R_at(p, sp):
        return target.local_target(n, prev, prev2, b1, b2, N, M, 12, 1, 1.0, e0, 5.0, 0.9875,
                                   WL.q, sp, rbm.logpsi(p, N, M, sp))

    for it in range(WL.iters):
        sp = ref.samples[n][it]
        params, _ = sr.sr_step(params, rbm.logderiv(params, N, M, sp), R_at(params, sp),
                               WL.shift, WL.dgamma, **solver)
    beta = np.mean(R_at(params, ref.samples[n][WL.iters]))
    lp_ref = rbm.logpsi(psi, N, M, ref.spins_ref)
    f = lattice.probe(12, 1, WL.q[0], WL.q[1], ref.spins_ref)
    Bn = beta * target.rel_amplitude(State(params), N, M, 12, 1, WL.q, ref.spins_ref, lp_ref)
    return params, beta, np.mean(np.conj(f) * Bn), Bn


def _single_steps(seq, ref, e0, solver):
    """Each projection step n alone: the GPU takes the oracle's t~_{n-1},
    t~_{n-2}, beta_{n-1}, beta_{n-2} and recorded samples, fits t~_n and
    measures beta_n, mu_n; the oracle does the same with the same solver.
    Returns per-n relative errors of (mu_n, beta_n, parameters of t~_n, the
    state beta_n t~_n / psi on the reference samples in the mean-square norm)."""
    cd = seq.ctx.cdtype
    seq.start(replay_ref=dev(ref.spins_ref, torch.int8))
    e_mu, e_beta, e_par, e_B = [], [], [], []
    mu0 = abs(ref.mu[0])
    for n in range(1, seq.cfg.n_moments):
        for k in range(max(1, n - 2), n):
            seq.params[k].copy_(dev(ref.states[k].params, cd))
        seq.betas[:n].copy_(dev(np.array(ref.betas[:n]), torch.complex128))
        seq.fit(n, replay=[dev(s, torch.int8) for s in ref.samples[n]])
        seq.ctx.sync_status()
        p, beta, mu, Bn = _oracle_single_step(ref, e0, n, solver)
        e_mu.append(abs(host(seq.mu)[n] - mu) / mu0)
        e_beta.append(abs(host(seq.betas)[n] - beta) / abs(beta))
        e_par.append(np.max(np.abs(host(seq.params[n]) - p)) / np.max(np.abs(p)))
        e_B.append(np.sqrt(np.mean(np.abs(host(seq.Bmat)[n] - Bn) ** 2) / np.mean(np.abs(Bn) ** 2)))
    return np.array(e_mu), np.array(e_beta), np.array(e_par), np.array(e_B)


# One projection step from the oracle's inputs.  float64 paths: each side
# with the same solver.  The 20 updates of a step each solve
# (S + lambda I) dalpha = F with kappa ~ 1e4-1e5 at lambda = 1e-3, so a
# difference e in the inputs of a solve reaches kappa e in dalpha:
#   Cholesky: rounding only, agreement to 1e-9;
#   CG: two solves stopping at |r| <= 1e-10 |F| may differ by kappa 1e-10.
# float32 and mixed paths, against the oracle's direct solve: the moments are
# held to the parity bar of the method's precision modes, 1e-5 mu_0 (float32)
# and 1e-3 mu_0 (mixed), with the walker sums of F and <O> compensated (float32 chunk sums
# left ~1e-5); the float32 CG runs to 1e-7.  beta_n and the parameters are
# not invariant under the near-null directions of S + lambda I (a scale of
# t~_n moves beta_n against it, kappa amplifies both).  The state itself,
# beta_n t~_n / psi on the reference samples (the Krylov column B_n, in the
# mean-square norm), is invariant under the scale but still measures those
# directions pointwise on samples of |psi|^2, not of |psi_n|^2: measured
# 30-50x the moment error (float64 CG 8.8e-5, float32 Cholesky 4.3e-5,
# mixed 5e-3), while mu_n, its projection on the probe, stays at the bar.
# beta_n, the parameters and the state are gated at about 10x their
# measured errors (regression guards); the moments at the parity bar.
# Tolerances: (mu / mu_0, beta relative, parameters relative, B_n rms relative).
SOLVERS = {"cholesky": dict(solver="cholesky"),
           "cg": dict(solver="cg", cg_maxit=400, cg_tol=1e-10, jacobi=False),
           "pcg": dict(solver="cg", cg_maxit=400, cg_tol=1e-10, jacobi=True)}
CG_TOL = {"fp64": 1e-10, "fp32": 1e-7, "mixed": 1e-5}


@pytest.mark.parametrize("path,tol", [("fp64-cholesky", (1e-9, 1e-9, 1e-9, 1e-9)),
                                      ("fp64-cg", (1e-5, 5e-3, 1e-3, 1e-3)),
                                      ("fp64-pcg", (1e-4, 2e-2, 5e-3, 5e-3)),
                                      ("fp32-cholesky", (1e-5, 5e-3, 2e-3, 5e-4)),
                                      ("fp32-pcg", (1e-5, 1e-2, 1e-2, 3e-3)),
                                      ("mixed-cg", (1e-3, 0.2, 0.2, 5e-2)),
                                      ("mixed-pcg", (1e-3, 0.2, 0.2, 5e-2))])
def test_single_projection_step_replay(e0, recorded, path, tol):
    from paper_2103_08804_gb300 import api
    prec_s, sol = path.split("-")
    prec = {"fp64": api.FP64, "fp32": api.FP32, "mixed": api.MIXED}[prec_s]
    solver = api.SOLVE_CHOLESKY if sol == "cholesky" else api.SOLVE_CG
    seq, _ = _seq(prec, e0, WL.moments, solver, cg_tol=CG_TOL[prec_s], cg_maxit=1000,
                  jacobi=(sol == "pcg"))
    ref_solver = SOLVERS[sol] if prec == api.FP64 else SOLVERS["cholesky"]
    e_mu, e_beta, e_par, e_B = _single_steps(seq, recorded, e0, ref_solver)
    print(f"{path} single-step errors: mu {e_mu.max():.2e} beta {e_beta.max():.2e} "
          f"params {e_par.max():.2e} state {e_B.max():.2e}; per-n mu "
          + np.array2string(e_mu, precision=1))
    assert e_mu.max() < tol[0] and e_beta.max() < tol[1] and e_par.max() < tol[2]
    assert e_B.max() < tol[3]


def test_fp64_replay_accumulated_over_sequence(e0, recorded):
    """The whole recursion on the recorded samples: errors of each step feed
    the next targets and grow with n (about x10 per moment late in this
    sequence, measured); float64 stays within 1e-6 mu_0."""
    from paper_2103_08804_gb300 import api
    seq, _ = _seq(api.FP64, e0, WL.moments, api.SOLVE_CHOLESKY)
    mu, betas = _replay(seq, recorded)
    errs = np.abs(mu - np.array(recorded.mu)) / abs(recorded.mu[0])
    print("fp64 accumulated replay moment error per n:", np.array2string(errs, precision=2))
    assert errs.max() < 1e-6
    rel_b = np.abs(betas[1:] - np.array(recorded.betas[1:])) / np.abs(np.array(recorded.betas[1:]))
    assert rel_b.max() < 1e-5


def test_fp32_replay_accumulated_over_sequence_reported(e0, recorded):
    """Accumulated float32 moment error on the recorded samples, per n.  Every
    step's error feeds the later targets and the recursion amplifies it (the
    float64 replay above measures about x10 per moment late in this
    sequence), so the parity gate is the single-step bound on the first step
    (1e-5 mu_0) and the later moments are reported."""
    from paper_2103_08804_gb300 import api
    seq, _ = _seq(api.FP32, e0, WL.moments, api.SOLVE_CHOLESKY)
    mu, _ = _replay(seq, recorded)
    err = np.abs(mu - np.array(recorded.mu)) / abs(recorded.mu[0])
    print("fp32 accumulated replay moment error per n:", np.array2string(err, precision=2))
    assert err[0] < 1e-6 and err[1] < 1e-5
    assert np.all(np.isfinite(mu))
