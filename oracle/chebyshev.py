"""The RBM-projected Chebyshev recursion and its moments (Secs. II-III).

Sec. II: mu_n = <psi|A^dag T_n(H') A|psi> = <t_0|t_n> with
|t_n> = T_n(H')|t_0>, |t_0> = A|psi>.  Sec. III: each |t_n> is approximated
by beta_n |t~_n>, with |t~_n> an RBM fitted to the target phi_n by the
natural-gradient update and beta_n = <R> after convergence; beta_0 = 1 and
t~_0 = t_0 exactly.

Readings of points the paper leaves open (see also oracle.sr, oracle.sampler):
  * A = S^z_q, so t~_0(sigma) = f_q(sigma) psi(sigma);
  * the RBM for n = 1 starts from psi with a_0 += i pi/2, which is exactly
    proportional to S^z_0 psi (e^{i pi sigma/2} = i sigma); later RBMs start
    from the previous one (warm start);
  * order within moment n: n_therm sweeps; then n_iter times
    {sweeps_per_iter sweeps, R, O, update}; then sweeps_per_iter sweeps and
    beta_n = <R> on those fresh samples;
  * the moments are averaged over one fixed sample set of |psi|^2, drawn
    once with its own random stream:
        mu_0 = <|f_q|^2>,  mu_n = beta_n < f_q* t~_n / psi >.
  * the walker chain of the fit continues across iterations and moments.

Enumeration mode replaces every sample average by the exact
|psi|^2-weighted sum over the S^z = 0 sector (no sampling).
"""

from dataclasses import dataclass, field

import numpy as np

from . import lattice, sampler, sr
from .exact import sector_basis
from .rbm import logderiv, logpsi
from .target import State, apply_hprime, local_target, rel_amplitude


@dataclass
class Config:
    Lx: int
    Ly: int
    M: int
    q: tuple
    n_moments: int
    n_iter: int
    shift: float = 1e-3
    dgamma: float = 0.5
    J: float = 1.0
    E0: float = 0.0
    a: float = 5.0
    Wp: float = 0.9875
    n_therm: int = 10
    sweeps_per_iter: int = 1
    n_therm_ref: int = 20
    seed: int = 0
    seed_ref: int = 1
    solver: str = "cholesky"
    cg_maxit: int = 100
    cg_tol: float = 1e-6
    jacobi: bool = False

    @property
    def N(self):
        return self.Lx * self.Ly


@dataclass
class Result:
    betas: list = field(default_factory=list)
    mu: list = field(default_factory=list)
    states: list = field(default_factory=list)
    gammas: list = field(default_factory=list)
    B: list = field(default_factory=list)
    HB: list = field(default_factory=list)
    spins_fit: np.ndarray = None
    spins_ref: np.ndarray = None
    counter_fit: int = 0
    counter_ref: int = 0
    samples: dict = field(default_factory=dict)  # n -> [spins of each iteration, beta spins]


def initial_params(psi_params, prev_params, n):
    if n == 1:
        p = np.array(psi_params, dtype=np.complex128, copy=True)
        p[0] += 0.5j * np.pi
        return p
    return np.array(prev_params, dtype=np.complex128, copy=True)


def _target(cfg, n, res, spins, lp):
    prev = res.states[n - 1]
    prev2 = res.states[n - 2] if n >= 2 else None
    b2 = res.betas[n - 2] if n >= 2 else 0.0
    return local_target(n, prev, prev2, res.betas[n - 1], b2, cfg.N, cfg.M, cfg.Lx, cfg.Ly,
                        cfg.J, cfg.E0, cfg.a, cfg.Wp, cfg.q, spins, lp)


def _moment_columns(cfg, state, beta, spins_ref, lp_ref):
    """B_n(s) = t_n(s)/psi(s) and (H' t_n)(s)/psi(s) on the reference samples."""
    Bn = beta * rel_amplitude(state, cfg.N, cfg.M, cfg.Lx, cfg.Ly, cfg.q, spins_ref, lp_ref)
    HBn = beta * apply_hprime(state, cfg.N, cfg.M, cfg.Lx, cfg.Ly, cfg.J, cfg.E0, cfg.a,
                              cfg.Wp, cfg.q, spins_ref, lp_ref)
    return Bn, HBn


def run_sampled(cfg, psi_params, spins_fit0, spins_ref0, n_moments=None, record=False):
    """The full sampled recursion with the Philox streams of oracle.philox.

    record: keep the walker configurations every estimator was taken on
    (res.samples[n]), so another implementation can replay them."""
    N, M = cfg.N, cfg.M
    bl = lattice.bonds(cfg.Lx, cfg.Ly)
    nm = cfg.n_moments if n_moments is None else n_moments
    res = Result()
    spins_ref, _, res.counter_ref = sampler.mc_sweep(psi_params, N, M, bl, spins_ref0,
                                                     cfg.n_therm_ref, cfg.seed_ref, 0)
    lp_ref = logpsi(psi_params, N, M, spins_ref)
    f_ref = lattice.probe(cfg.Lx, cfg.Ly, cfg.q[0], cfg.q[1], spins_ref)
    res.spins_ref = spins_ref
    res.states.append(State(np.asarray(psi_params, dtype=np.complex128), probe=True))
    res.betas.append(1.0 + 0.0j)
    res.mu.append(np.mean(np.abs(f_ref) ** 2) + 0.0j)
    B0, HB0 = _moment_columns(cfg, res.states[0], 1.0, spins_ref, lp_ref)
    res.B.append(B0)
    res.HB.append(HB0)
    spins = np.array(spins_fit0, dtype=np.int8)
    ctr = 0
    for n in range(1, nm):
        params = initial_params(psi_params, res.states[n - 1].params, n)
        g_n = []
        if cfg.n_therm:
            spins, _, ctr = sampler.mc_sweep(params, N, M, bl, spins, cfg.n_therm, cfg.seed, ctr)
        rec = res.samples.setdefault(n, []) if record else None
        for _ in range(cfg.n_iter):
            spins, _, ctr = sampler.mc_sweep(params, N, M, bl, spins, cfg.sweeps_per_iter,
                                             cfg.seed, ctr)
            if record:
                rec.append(spins.copy())
            lp = logpsi(params, N, M, spins)
            R = _target(cfg, n, res, spins, lp)
            O = logderiv(params, N, M, spins)
            params, info = sr.sr_step(params, O, R, cfg.shift, cfg.dgamma, solver=cfg.solver,
                                      cg_maxit=cfg.cg_maxit, cg_tol=cfg.cg_tol, jacobi=cfg.jacobi)
            g_n.append(info["gamma"])
        spins, _, ctr = sampler.mc_sweep(params, N, M, bl, spins, cfg.sweeps_per_iter,
                                         cfg.seed, ctr)
        if record:
            rec.append(spins.copy())
        lp = logpsi(params, N, M, spins)
        beta = np.mean(_target(cfg, n, res, spins, lp))
        state = State(params)
        res.states.append(state)
        res.betas.append(beta)
        res.gammas.append(g_n)
        Bn, HBn = _moment_columns(cfg, state, beta, spins_ref, lp_ref)
        res.B.append(Bn)
        res.HB.append(HBn)
        res.mu.append(np.mean(np.conj(f_ref) * Bn))
    res.spins_fit = spins
    res.counter_fit = ctr
    return res


def run_enumerated(cfg, psi_params, n_moments=None):
    """The same recursion with every average taken exactly over the S^z = 0 sector."""
    N, M = cfg.N, cfg.M
    nm = cfg.n_moments if n_moments is None else n_moments
    basis = sector_basis(N)
    res = Result()

    def weights(params):
        lp = logpsi(params, N, M, basis)
        w = np.exp(2.0 * (lp.real - lp.real.max()))
        return lp, w / w.sum()

    lp_ref, w_ref = weights(psi_params)
    f = lattice.probe(cfg.Lx, cfg.Ly, cfg.q[0], cfg.q[1], basis)
    res.states.append(State(np.asarray(psi_params, dtype=np.complex128), probe=True))
    res.betas.append(1.0 + 0.0j)
    res.mu.append(np.sum(w_ref * np.abs(f) ** 2) + 0.0j)
    for n in range(1, nm):
        params = initial_params(psi_params, res.states[n - 1].params, n)
        g_n = []
        for _ in range(cfg.n_iter):
            lp, w = weights(params)
            R = _target(cfg, n, res, basis, lp)
            O = logderiv(params, N, M, basis)
            params, info = sr.sr_step(params, O, R, cfg.shift, cfg.dgamma, weights=w,
                                      solver=cfg.solver, cg_maxit=cfg.cg_maxit,
                                      cg_tol=cfg.cg_tol, jacobi=cfg.jacobi)
            g_n.append(info["gamma"])
        lp, w = weights(params)
        beta = np.sum(w * _target(cfg, n, res, basis, lp))
        state = State(params)
        res.states.append(state)
        res.betas.append(beta)
        res.gammas.append(g_n)
        Bn = beta * rel_amplitude(state, N, M, cfg.Lx, cfg.Ly, cfg.q, basis, lp_ref)
        res.mu.append(np.sum(w_ref * np.conj(f) * Bn))
    return res
