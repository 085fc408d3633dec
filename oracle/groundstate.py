"""Ground-state preparation: the RBM psi is variationally optimised to
minimise E = <psi|H|psi> / <psi|psi> by Monte Carlo (Sec. I, after Carleo
and Troyer), here by the natural-gradient (stochastic reconfiguration)
descent with the same metric S as Sec. III:

    E_loc(s)  = (H psi)(s) / psi(s)                      (local energy)
    F_k       = <O_k* E_loc> - <O_k*> <E_loc>             (= dE / d conj(alpha_k))
    (S + lambda I) dalpha = -lr F,   alpha <- alpha + dalpha.

Any affine rescaling H' = (H - E0) / a - W' of the Hamiltonian leaves the
direction unchanged and scales F by 1 / a; the functions below take the
local values of whichever operator the caller uses (the GPU path feeds the
local H' of the Chebyshev target machinery).

THIS MODULE IS TEST INFRASTRUCTURE (see the package docstring).
"""

import numpy as np

from . import rbm, sr
from .target import State, apply_hprime


def local_energy(params, N, M, Lx, Ly, J, spins):
    """E_loc(s) = (H psi)(s) / psi(s) for the rows of spins (H unscaled:
    E0 = 0, a = 1, W' = 0 in the rescaling)."""
    lp = rbm.logpsi(params, N, M, spins)
    return apply_hprime(State(params), N, M, Lx, Ly, J, 0.0, 1.0, 0.0, (0.0, 0.0), spins, lp)


def energy_force(O, Eloc, weights=None):
    """F_k = <O_k* E> - <O_k*> <E> and <E>."""
    est = sr.estimators(O, Eloc, weights)
    mE = est["mR"]
    return est["OR"] - np.conj(est["Obar"]) * mE, mE


def sr_energy_step(params, O, Eloc, lr, shift, weights=None):
    """One descent step; returns (new params, info)."""
    F, mE = energy_force(O, Eloc, weights)
    est = sr.estimators(O, Eloc, weights)
    S = sr.qgt(est)
    delta = sr.shifted_solve(S, -lr * F, shift)
    info = {"E": mE, "F": F, "S": S, "delta": delta}
    return np.asarray(params, dtype=np.complex128) + delta, info
