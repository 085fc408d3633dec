"""Exact diagonalisation and exact Chebyshev vectors on small lattices.

These are the references the rest of the oracle is pinned to (N <= 14):
the Heisenberg Hamiltonian (Sec. V) as a dense matrix on the S^z = 0 sector,
its spectrum, the exact Chebyshev vectors |t_n> = T_n(H') |t_0> by the
three-term recursion T_{n+1} = 2x T_n - T_{n-1} (Sec. II), and the exact
moments mu_n = <t_0|t_n> / <psi|psi> (Sec. II).
"""

import itertools

import numpy as np

from . import lattice
from .rbm import logpsi


def sector_basis(N, n_up=None):
    """All configurations with n_up up-spins (default N/2) as int8 [D, N]."""
    if n_up is None:
        if N % 2:
            raise ValueError("odd N has no S^z = 0 sector")
        n_up = N // 2
    rows = []
    for ups in itertools.combinations(range(N), n_up):
        s = -np.ones(N, dtype=np.int8)
        s[list(ups)] = 1
        rows.append(s)
    return np.array(rows, dtype=np.int8)


def _key(s):
    return s.tobytes()


def hamiltonian(Lx, Ly, J, basis):
    """Dense H = J sum_b S_i . S_j on the span of `basis` (closed under exchange)."""
    D = basis.shape[0]
    index = {_key(s): k for k, s in enumerate(basis)}
    H = np.zeros((D, D))
    H[np.arange(D), np.arange(D)] = lattice.bond_diagonal(Lx, Ly, J, basis)
    for k, s in enumerate(basis):
        for i, j in lattice.bonds(Lx, Ly):
            if s[i] != s[j]:
                t = s.copy()
                t[i], t[j] = s[j], s[i]
                H[index[_key(t)], k] += 0.5 * J
    return H


def rbm_vector(params, N, M, basis):
    """The RBM amplitudes psi(s) on every basis configuration."""
    return np.exp(logpsi(params, N, M, basis))


def probe_vector(Lx, Ly, qx, qy, basis, psi_vec):
    """t_0 = S^z_q psi as a dense vector (Appendix B)."""
    return lattice.probe(Lx, Ly, qx, qy, basis) * psi_vec


def rescaled(H, E0, a, Wp):
    """H' = (H - E0) / a - W' (Sec. II)."""
    return (H - E0 * np.eye(H.shape[0])) / a - Wp * np.eye(H.shape[0])


def chebyshev_vectors(Hp, t0, n_moments):
    """[t_0, t_1, ..] with t_n = T_n(H') t_0 by the three-term recursion."""
    out = [np.asarray(t0, dtype=np.complex128)]
    if n_moments > 1:
        out.append(Hp @ out[0])
    for _ in range(2, n_moments):
        out.append(2.0 * (Hp @ out[-1]) - out[-2])
    return out


def chebyshev_moments(Hp, t0, psi_vec, n_moments):
    """Exact mu_n = <t_0|t_n> / <psi|psi>."""
    norm = np.vdot(psi_vec, psi_vec).real
    return np.array([np.vdot(t0, t) / norm for t in chebyshev_vectors(Hp, t0, n_moments)])
