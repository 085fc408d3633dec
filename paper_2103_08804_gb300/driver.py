"""The Chebyshev recursion driven through the C ABI (Secs. II-III).

Host-side orchestration only: it decides the order of library calls and
owns the device buffers.  Every arithmetic step runs in libchebrbm kernels,
and no call inside a moment waits on the host, so a whole moment can be
enqueued (or captured) in one go.

Order within moment n >= 1 (shared with the oracle):
  theta <- b + sigma W for the initial RBM_n; n_therm sweeps;
  n_iter times { sweeps_per_iter sweeps (giving log psi_n, tanh theta);
                 R = phi_n / psi_n; natural-gradient update;
                 theta, log psi_n recomputed for the new parameters };
  sweeps_per_iter sweeps; beta_n = <R> on those samples;
  mu_n = beta_n < conj(f_q) t~_n / psi > on the fixed samples of |psi|^2,
  together with the Krylov columns B_n and (H' t_n)/psi.
RBM_1 starts from psi with a_0 += i pi/2 (exactly proportional to
S^z_0 psi); RBM_n (n >= 2) starts from RBM_{n-1} (cheb_init_params).
"""

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import api


@dataclass
class SeqConfig:
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
    solver: int = api.SOLVE_CG
    cg_maxit: int = 100
    cg_tol: float = 1e-6
    jacobi: bool = False
    krylov: bool = True

    @property
    def N(self):
        return self.Lx * self.Ly


class Sequence:
    """Device state of one Chebyshev sequence (one probe momentum).

    graphs=True captures one natural-gradient iteration (sweep, target, update,
    theta refresh) in a CUDA graph per kind of step (n = 1, n = 2, n >= 3) and
    replays it; the moment's inputs are copied into fixed buffers first and
    the random stream position lives on the device, so replays reproduce the
    eager launches exactly."""

    def __init__(self, ctx, cfg, psi_params, spins_fit, spins_ref, graphs=False):
        self.ctx, self.cfg = ctx, cfg
        dev = torch.device("cuda")
        cd = ctx.cdtype
        Nm, P, M = cfg.n_moments, ctx.P, ctx.M
        self.B = spins_fit.shape[0]
        self.Bref = spins_ref.shape[0]
        psi = np.asarray(psi_params, dtype=np.complex128)
        self.params = torch.zeros(Nm, P, dtype=cd, device=dev)
        self.params[0].copy_(torch.from_numpy(psi).to(cd))
        self.spins = torch.as_tensor(spins_fit, dtype=torch.int8).to(dev).contiguous()
        self.spins_ref = torch.as_tensor(spins_ref, dtype=torch.int8).to(dev).contiguous()
        self.theta = torch.empty(self.B, M, dtype=cd, device=dev)
        self.tanh = torch.empty(self.B, M, dtype=cd, device=dev)
        self.lp = torch.empty(self.B, dtype=cd, device=dev)
        self.R = torch.empty(self.B, dtype=cd, device=dev)
        self.theta_ref = torch.empty(self.Bref, M, dtype=cd, device=dev)
        self.lp_ref = torch.empty(self.Bref, dtype=cd, device=dev)
        self.betas = torch.zeros(Nm, dtype=torch.complex128, device=dev)
        self.mu = torch.zeros(Nm, dtype=torch.complex128, device=dev)
        self.stats = torch.zeros(Nm, max(cfg.n_iter, 1), api.STATS_LEN, dtype=torch.float64,
                                 device=dev)
        if cfg.krylov:
            self.Bmat = torch.zeros(Nm, self.Bref, dtype=cd, device=dev)
            self.HBmat = torch.zeros(Nm, self.Bref, dtype=cd, device=dev)
        self.rng = api.Philox(cfg.seed, 0)
        self.rng_ref = api.Philox(cfg.seed_ref, 0)
        self.hprime = (cfg.E0, cfg.a, cfg.Wp)
        self.n_done = 0
        self.graphs = graphs
        self.graph_launches = 0
        if graphs:
            self.work = torch.zeros(P, dtype=cd, device=dev)
            self.prev_buf = torch.zeros(P, dtype=cd, device=dev)
            self.prev2_buf = torch.zeros(P, dtype=cd, device=dev)
            self.beta_buf = torch.zeros(2, dtype=torch.complex128, device=dev)
            self.stats_it = torch.zeros(api.STATS_LEN, dtype=torch.float64, device=dev)
            self.ctr = torch.zeros(1, dtype=torch.int64, device=dev)
            self.rng_dev = api.Philox(cfg.seed, 0, self.ctr.data_ptr())
            self._graph = {}
            self._eager_done = set()

    def state(self, n):
        return self.ctx.state(self.params[n], probe=(n == 0), q=self.cfg.q)

    def start(self, replay_ref=None):
        """Sample |psi|^2 once (or take the recorded samples replay_ref) and
        record mu_0 (beta_0 = 1)."""
        c, cfg = self.ctx, self.cfg
        self.betas[0] = 1.0
        if replay_ref is not None:
            self.spins_ref.copy_(replay_ref)
        c.rbm_logpsi(self.params[0], self.spins_ref, self.theta_ref, self.lp_ref)
        if replay_ref is None:
            c.mc_sweep(self.params[0], self.spins_ref, self.theta_ref, cfg.n_therm_ref,
                       self.rng_ref, logpsi_out=self.lp_ref)
        self._moment(0)
        self.n_done = 1

    def _moment(self, n):
        c, cfg = self.ctx, self.cfg
        kw = {}
        if cfg.krylov:
            kw = dict(hprime=self.hprime, Bcol=self.Bmat[n], HBcol=self.HBmat[n])
        c.cheb_moment(self.state(n), self.betas[n:n + 1], cfg.q, self.spins_ref, self.lp_ref,
                      mu_out=self.mu[n:n + 1], **kw)

    def _target(self, n, mean_out=None):
        c, cfg = self.ctx, self.cfg
        prev2 = self.state(n - 2) if n >= 2 else None
        b2 = self.betas[n - 2:n - 1] if n >= 2 else None
        c.cheb_local_target(n, self.state(n - 1), prev2, self.betas[n - 1:n], b2, cfg.E0, cfg.a,
                            cfg.Wp, self.spins, self.lp, self.R, mean_out=mean_out)

    def _samples(self, pn, n_sweeps, replay, record=None):
        """Fresh samples of |psi_n|^2: Metropolis sweeps, or, when replaying,
        the next recorded configuration set (then theta, log psi and tanh theta
        are evaluated on it).  record: list receiving a copy of each sample set."""
        c = self.ctx
        if replay is None:
            c.mc_sweep(pn, self.spins, self.theta, n_sweeps, self.rng, logpsi_out=self.lp,
                       tanh_out=self.tanh)
            if record is not None:
                record.append(self.spins.clone())
        else:
            self.spins.copy_(next(replay))
            c.rbm_logpsi(pn, self.spins, self.theta, self.lp)
            c.logderiv(pn, self.spins, self.theta, tanh_out=self.tanh)

    def fit(self, n, replay=None, record=None):
        """Projection step n: fit RBM_n, then beta_n and mu_n.

        replay: optional iterable of walker configurations (device int8
        [B, N]) to use, in order, instead of the sampler: one per iteration
        and one for beta_n (the recorded samples of another run).
        record: optional list that receives those configurations."""
        if self.graphs and replay is None and record is None:
            return self._fit_graph(n)
        c, cfg = self.ctx, self.cfg
        replay = iter(replay) if replay is not None else None
        pn = self.params[n]
        c.cheb_init_params(n, self.params[0], self.params[n - 1], pn)
        if replay is None:
            c.rbm_logpsi(pn, self.spins, self.theta, self.lp)
            if cfg.n_therm:
                c.mc_sweep(pn, self.spins, self.theta, cfg.n_therm, self.rng, logpsi_out=self.lp,
                           tanh_out=self.tanh)
        for it in range(cfg.n_iter):
            self._samples(pn, cfg.sweeps_per_iter, replay, record)
            self._target(n)
            c.sr_step(pn, self.spins, self.tanh, self.R, cfg.dgamma, cfg.shift, solver=cfg.solver,
                      cg_maxit=cfg.cg_maxit, cg_tol=cfg.cg_tol, stats_out=self.stats[n, it],
                      jacobi=cfg.jacobi)
            if replay is None:
                c.rbm_logpsi(pn, self.spins, self.theta, self.lp)
        self._samples(pn, cfg.sweeps_per_iter, replay, record)
        self._target(n, mean_out=self.betas[n:n + 1])
        self._moment(n)
        self.n_done = n + 1

    # ------------------------------------------------------------ graphs
    def counter(self):
        """Current position of the fit walkers' random stream."""
        if self.graphs:
            return int(self.ctr.item())
        return self.rng.counter

    def _iteration(self, kind):
        """One natural-gradient iteration on the fixed buffers (capturable)."""
        c, cfg = self.ctx, self.cfg
        c.mc_sweep(self.work, self.spins, self.theta, cfg.sweeps_per_iter, self.rng_dev,
                   logpsi_out=self.lp, tanh_out=self.tanh)
        self._target_fixed(kind)
        c.sr_step(self.work, self.spins, self.tanh, self.R, cfg.dgamma, cfg.shift,
                  solver=cfg.solver, cg_maxit=cfg.cg_maxit, cg_tol=cfg.cg_tol,
                  stats_out=self.stats_it, jacobi=cfg.jacobi)
        c.rbm_logpsi(self.work, self.spins, self.theta, self.lp)

    def iter_desc(self, kind):
        """The cr_seq_iter of one natural-gradient iteration on the fixed
        buffers (graph mode), for cr_batch_run; the structs it points to are
        kept alive on the sequence."""
        c, cfg, q = self.ctx, self.cfg, self.cfg.q
        prev = c.state(self.prev_buf, probe=(kind == 1), q=q)
        prev2 = c.state(self.prev2_buf, probe=(kind == 2), q=q) if kind >= 2 else None
        tg = c.target(1 if kind == 1 else 2, prev, prev2, self.beta_buf[0:1],
                      self.beta_buf[1:2] if kind >= 2 else None, cfg.E0, cfg.a, cfg.Wp)
        o = api.SROpts(cfg.dgamma, cfg.shift, cfg.solver, cfg.cg_maxit, cfg.cg_tol,
                       1 if cfg.jacobi else 0, 0, 0)
        it = api.SeqIter(c.h, self.work.data_ptr(), self.spins.data_ptr(), self.theta.data_ptr(),
                         self.tanh.data_ptr(), self.lp.data_ptr(), self.R.data_ptr(), self.B,
                         cfg.sweeps_per_iter, tg, o, ctypes.pointer(self.rng_dev),
                         self.stats_it.data_ptr())
        self._keep = getattr(self, "_keep", {})
        self._keep[kind] = (prev, prev2, tg, o, it)
        return it

    def _target_fixed(self, kind, mean_out=None):
        c, cfg, q = self.ctx, self.cfg, self.cfg.q
        prev = c.state(self.prev_buf, probe=(kind == 1), q=q)
        prev2 = c.state(self.prev2_buf, probe=(kind == 2), q=q) if kind >= 2 else None
        c.cheb_local_target(1 if kind == 1 else 2, prev, prev2, self.beta_buf[0:1],
                            self.beta_buf[1:2] if kind >= 2 else None, cfg.E0, cfg.a, cfg.Wp,
                            self.spins, self.lp, self.R, mean_out=mean_out)

    def _replay(self, kind):
        if kind not in self._graph:
            g = torch.cuda.CUDAGraph()
            side = torch.cuda.Stream()
            main = torch.cuda.current_stream()
            side.wait_stream(main)
            n0 = self.ctx.n_launches()
            with torch.cuda.graph(g, stream=side):
                self.ctx.set_stream(side)
                self._iteration(kind)
            self.ctx.set_stream(main)
            main.wait_stream(side)
            self._graph[kind] = (g, self.ctx.n_launches() - n0)
        g, nodes = self._graph[kind]
        g.replay()
        self.graph_launches += nodes

    @staticmethod
    def kind_of(n):
        """Graph kind of projection step n: the target's form differs for
        n = 1 (probe state), n = 2 (probe as t~_{n-2}) and n >= 3."""
        return 1 if n == 1 else (2 if n == 2 else 3)

    def _moment_begin(self, n):
        """Inputs of step n into the fixed buffers, theta and thermalisation."""
        c, cfg = self.ctx, self.cfg
        c.cheb_init_params(n, self.params[0], self.params[n - 1], self.work)
        self.prev_buf.copy_(self.params[n - 1])
        self.beta_buf[0:1].copy_(self.betas[n - 1:n])
        if n >= 2:
            self.prev2_buf.copy_(self.params[n - 2])
            self.beta_buf[1:2].copy_(self.betas[n - 2:n - 1])
        c.rbm_logpsi(self.work, self.spins, self.theta, self.lp)
        if cfg.n_therm:
            c.mc_sweep(self.work, self.spins, self.theta, cfg.n_therm, self.rng_dev,
                       logpsi_out=self.lp, tanh_out=self.tanh)

    def _moment_end(self, n):
        """Fresh samples, beta_n = <R>, the parameters of RBM_n and mu_n."""
        c, cfg = self.ctx, self.cfg
        c.mc_sweep(self.work, self.spins, self.theta, cfg.sweeps_per_iter, self.rng_dev,
                   logpsi_out=self.lp, tanh_out=self.tanh)
        self._target_fixed(self.kind_of(n), mean_out=self.betas[n:n + 1])
        self.params[n].copy_(self.work)
        self._moment(n)
        self.n_done = n + 1

    def _fit_graph(self, n):
        kind = self.kind_of(n)
        self._moment_begin(n)
        for it in range(self.cfg.n_iter):
            if kind in self._eager_done:
                self._replay(kind)
            else:
                self._iteration(kind)  # first of its kind: eager (loads every kernel)
                self._eager_done.add(kind)
            self.stats[n, it].copy_(self.stats_it)
        self._moment_end(n)

    def run(self, n_moments=None):
        nm = self.cfg.n_moments if n_moments is None else n_moments
        if self.n_done == 0:
            self.start()
        for n in range(self.n_done, nm):
            self.fit(n)
        return self
