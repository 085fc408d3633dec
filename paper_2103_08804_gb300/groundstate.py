"""Ground-state preparation through the C ABI (Sec. I): the RBM psi is
optimised to minimise E = <psi|H|psi> / <psi|psi> by natural-gradient
descent on samples of |psi|^2, with the metric S of Sec. III:

  per step: Metropolis sweeps of |psi|^2 (mc_sweep, giving log psi and
  tanh theta); the local H' = (H' psi)/psi from cheb_local_target with
  n = 1, t~_0 = psi (no probe) and beta_0 = 1; sr_step in CR_SR_ENERGY mode
  (F = -lr (<O* E> - <O*><E>), (S + shift I) dalpha = F); theta and log psi
  refreshed for the new parameters.

Energies are reported in the units of H: E = a (<H'> + W') + E0.  Host-side
orchestration only; every arithmetic step runs in library kernels.
"""

import numpy as np
import torch

from . import api


class GroundState:
    def __init__(self, ctx, params, spins, lr=0.05, shift=1e-3, E0=0.0, a=1.0, Wp=0.0,
                 seed=0, sweeps=1, solver=api.SOLVE_CG, cg_maxit=100, cg_tol=1e-6):
        self.ctx = ctx
        dev = torch.device("cuda")
        cd = ctx.cdtype
        self.params = torch.as_tensor(np.asarray(params, dtype=np.complex128)).to(cd).to(dev)
        self.spins = torch.as_tensor(spins, dtype=torch.int8).to(dev).contiguous()
        B, M = self.spins.shape[0], ctx.M
        self.theta = torch.empty(B, M, dtype=cd, device=dev)
        self.tanh = torch.empty(B, M, dtype=cd, device=dev)
        self.lp = torch.empty(B, dtype=cd, device=dev)
        self.R = torch.empty(B, dtype=cd, device=dev)
        self.one = torch.ones(1, dtype=torch.complex128, device=dev)
        self.rng = api.Philox(seed, 0)
        self.lr, self.shift, self.sweeps = lr, shift, sweeps
        self.E0, self.a, self.Wp = E0, a, Wp
        self.solver, self.cg_maxit, self.cg_tol = solver, cg_maxit, cg_tol
        self.stats = []
        ctx.rbm_logpsi(self.params, self.spins, self.theta, self.lp)

    def thermalise(self, n_sweeps):
        self.ctx.mc_sweep(self.params, self.spins, self.theta, n_sweeps, self.rng,
                          logpsi_out=self.lp, tanh_out=self.tanh)

    def step(self):
        c = self.ctx
        c.mc_sweep(self.params, self.spins, self.theta, self.sweeps, self.rng,
                   logpsi_out=self.lp, tanh_out=self.tanh)
        c.cheb_local_target(1, c.state(self.params), None, self.one, None, self.E0, self.a,
                            self.Wp, self.spins, self.lp, self.R)
        st = torch.zeros(api.STATS_LEN, dtype=torch.float64, device=self.params.device)
        c.sr_step(self.params, self.spins, self.tanh, self.R, self.lr, self.shift,
                  solver=self.solver, cg_maxit=self.cg_maxit, cg_tol=self.cg_tol, stats_out=st,
                  mode=api.SR_ENERGY)
        c.rbm_logpsi(self.params, self.spins, self.theta, self.lp)
        self.stats.append(st)

    def energies(self):
        """<H> before each step, in the units of H (the local H' rescaled)."""
        if not self.stats:
            return np.zeros(0)
        st = torch.stack(self.stats).cpu().numpy()
        return self.a * (st[:, 1] + self.Wp) + self.E0
