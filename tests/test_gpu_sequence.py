"""End-to-end parity of the Chebyshev sequence: CUDA path (driver over the C
ABI) against the oracle, on the 12-site chain workload (alpha = 1, sigma =
0.05, q = pi, 1024 walkers, 10 moments, 20 natural-gradient iterations per
moment, shift 1e-3), with both sides drawing from the same Philox stream.

float64: walker trajectories are bit-identical and beta_n, mu_n agree to
1e-8 relative to mu_0 (only rounding order differs, amplified by the
recursion).  float32: trajectories diverge after the first near-tie
decision, so the moments are compared to the oracle within Monte Carlo error
(5% of mu_0) and to the float64 GPU run."""

import numpy as np
import pytest

from gpu_common import host, need_gpu, torch
from oracle import chebyshev, exact
from paper_2103_08804_gb300 import synth

pytestmark = pytest.mark.gpu

WL = synth.WORKLOADS["chain12_fp64"]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.fixture(scope="module")
def e0():
    return np.linalg.eigvalsh(exact.hamiltonian(12, 1, 1.0, exact.sector_basis(12)))[0]


def _run_gpu(prec, e0, n_moments, solver):
    from paper_2103_08804_gb300 import api, driver
    cfg = driver.SeqConfig(Lx=12, Ly=1, M=WL.M, q=WL.q, n_moments=n_moments, n_iter=WL.iters,
                           shift=WL.shift, dgamma=WL.dgamma, E0=e0, a=5.0, Wp=0.9875,
                           solver=solver, cg_maxit=300, cg_tol=1e-12)
    ctx = api.Context(12, 1, WL.M, WL.walkers, prec=prec, explicit_s=(solver == api.SOLVE_CHOLESKY))
    psi = synth.rbm_params(0, 12, WL.M, WL.sigma)
    seq = driver.Sequence(ctx, cfg, psi, synth.sz0_spins(1, WL.walkers, 12),
                          synth.sz0_spins(2, WL.walkers, 12))
    seq.run()
    ctx.sync_status()
    return seq


@pytest.fixture(scope="module")
def oracle_run(e0):
    cfg = chebyshev.Config(Lx=12, Ly=1, M=WL.M, q=WL.q, n_moments=WL.moments, n_iter=WL.iters,
                           shift=WL.shift, dgamma=WL.dgamma, E0=e0, a=5.0, Wp=0.9875)
    psi = synth.rbm_params(0, 12, WL.M, WL.sigma)
    return chebyshev.run_sampled(cfg, psi, synth.sz0_spins(1, WL.walkers, 12),
                                 synth.sz0_spins(2, WL.walkers, 12))


def test_fp64_sequence_matches_oracle(e0, oracle_run):
    from paper_2103_08804_gb300 import api
    seq = _run_gpu(api.FP64, e0, WL.moments, api.SOLVE_CHOLESKY)
    ref = oracle_run
    assert np.array_equal(host(seq.spins), ref.spins_fit)
    assert np.array_equal(host(seq.spins_ref), ref.spins_ref)
    assert seq.rng.counter == ref.counter_fit and seq.rng_ref.counter == ref.counter_ref
    mu0 = abs(ref.mu[0])
    assert np.max(np.abs(host(seq.mu) - np.array(ref.mu))) < 1e-8 * mu0
    assert np.max(np.abs(host(seq.betas) - np.array(ref.betas))) < 1e-8
    g = host(seq.stats)[1:, :, 0]
    assert np.allclose(g, np.array(ref.gammas), atol=1e-8)
    for n in (1, WL.moments - 1):
        assert np.max(np.abs(host(seq.params[n]) - ref.states[n].params)) < 1e-8
    # Krylov columns at the reference samples
    assert np.max(np.abs(host(seq.Bmat) - np.array(ref.B))) < 1e-8 * np.sqrt(mu0)


def test_fp64_cg_solver_tracks_cholesky(e0, oracle_run):
    from paper_2103_08804_gb300 import api
    seq = _run_gpu(api.FP64, e0, 4, api.SOLVE_CG)
    mu0 = abs(oracle_run.mu[0])
    assert np.max(np.abs(host(seq.mu) - np.array(oracle_run.mu[:4]))) < 1e-6 * mu0


def test_fp32_sequence_within_mc_error(e0, oracle_run):
    from paper_2103_08804_gb300 import api
    seq = _run_gpu(api.FP32, e0, WL.moments, api.SOLVE_CG)
    mu0 = abs(oracle_run.mu[0])
    mu = host(seq.mu)
    # same reference samples up to the odd float32 near-tie decision of the reference chain
    assert abs(mu[0] - oracle_run.mu[0]) < 2e-2 * mu0
    assert np.max(np.abs(mu - np.array(oracle_run.mu))) < 0.05 * mu0
    assert np.all(host(seq.spins).sum(axis=1) == 0)
