"""The local ratio R(s) = phi_s / psi_s for the projected Chebyshev targets.

Sec. III (last paragraph): with beta_0 = 1 and t~_0 = t_0,
    phi_1 = beta_0 H' t~_0,
    phi_n = 2 beta_{n-1} H' t~_{n-1} - beta_{n-2} t~_{n-2}   (n >= 2),
and the fitted RBM psi_n is sampled, so R(s) = phi_n(s) / psi_n(s).

Sec. II: H' = (H - E0) / a - W'.  Sec. V: H = J sum_b S_i . S_j, whose
action on an amplitude is
    (H v)(s) = sum_b [ (J/4) sigma_i sigma_j v(s) + (J/2) [sigma_i != sigma_j] v(s^{ij}) ]
with s^{ij} the configuration with spins i and j exchanged.

A state is an RBM, optionally multiplied by the probe factor f_q(sigma)
(the exact t_0 = S^z_q psi is f_q * psi, Sec. II and Appendix B).  Every
amplitude here is evaluated from scratch by the definitions in oracle.rbm;
no ratio identity is used.
"""

from dataclasses import dataclass

import numpy as np

from . import lattice
from .rbm import logpsi


@dataclass
class State:
    params: np.ndarray
    probe: bool = False


def rel_amplitude(state, N, M, Lx, Ly, q, spins, logpsi_ref):
    """t~(spins) / exp(logpsi_ref), elementwise over rows."""
    v = np.exp(logpsi(state.params, N, M, spins) - logpsi_ref)
    if state.probe:
        v = v * lattice.probe(Lx, Ly, q[0], q[1], spins)
    return v


def apply_hprime(state, N, M, Lx, Ly, J, E0, a, Wp, q, spins, logpsi_ref):
    """(H' t~)(s) / exp(logpsi_ref(s)) for each row s of spins."""
    spins = np.asarray(spins, dtype=np.int8)
    rows = np.arange(spins.shape[0])
    v = rel_amplitude(state, N, M, Lx, Ly, q, spins, logpsi_ref)
    Hv = lattice.bond_diagonal(Lx, Ly, J, spins) * v
    for i, j in lattice.bonds(Lx, Ly):
        anti = spins[:, i] != spins[:, j]
        if not np.any(anti):
            continue
        flipped = spins.copy()
        flipped[rows, i] = spins[:, j]
        flipped[rows, j] = spins[:, i]
        vf = rel_amplitude(state, N, M, Lx, Ly, q, flipped, logpsi_ref)
        Hv = Hv + np.where(anti, 0.5 * J * vf, 0.0)
    return (Hv - E0 * v) / a - Wp * v


def local_target(n, prev, prev2, beta_prev, beta_prev2, N, M, Lx, Ly, J, E0, a, Wp, q,
                 spins, logpsi_n):
    """R(s) = phi_n(s) / psi_n(s).

    n         index of the state being fitted (>= 1)
    prev      State t~_{n-1};  prev2: State t~_{n-2} (ignored for n == 1)
    beta_*    complex beta_{n-1}, beta_{n-2}
    logpsi_n  log psi_n at the rows of spins
    """
    if n < 1:
        raise ValueError("targets start at n = 1")
    h = apply_hprime(prev, N, M, Lx, Ly, J, E0, a, Wp, q, spins, logpsi_n)
    if n == 1:
        return beta_prev * h
    v2 = rel_amplitude(prev2, N, M, Lx, Ly, q, spins, logpsi_n)
    return 2.0 * beta_prev * h - beta_prev2 * v2
