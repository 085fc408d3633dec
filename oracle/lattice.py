"""Lattice geometry, the Heisenberg bond list and the probe operator.

Sec. V: H = J sum_<ij> S_i . S_j over nearest-neighbour pairs with periodic
boundaries, on a chain or a square lattice.  Appendix B: the momentum-space
operator A_k = (1/L) sum_n exp(-i 2pi k.n / L) A_n on L^2 sites; with
A_n = S^z_n and N sites the prefactor is 1/sqrt(N).

Conventions (shared by contract with the CUDA path, which builds its own
copy of the bond list):
  * site index r = x + Lx*y, 0 <= x < Lx, 0 <= y < Ly (Ly = 1 is a chain);
  * bond list = all (r, r + x-hat) in increasing r, then, for Ly > 1, all
    (r, r + y-hat) in increasing r;
  * spins sigma_r = +-1 and S^z_r = sigma_r / 2.
"""

import numpy as np


def check_dims(Lx, Ly):
    if Lx < 3 or Ly < 1 or (Ly != 1 and Ly < 3):
        raise ValueError("lattice needs Lx >= 3 and Ly == 1 or Ly >= 3")


def coords(Lx, Ly):
    """(x, y) of every site, in site order."""
    check_dims(Lx, Ly)
    r = np.arange(Lx * Ly)
    return r % Lx, r // Lx


def bonds(Lx, Ly):
    """Periodic nearest-neighbour bonds as an int array [N_b, 2]."""
    check_dims(Lx, Ly)
    out = []
    for y in range(Ly):
        for x in range(Lx):
            out.append((x + Lx * y, (x + 1) % Lx + Lx * y))
    if Ly > 1:
        for y in range(Ly):
            for x in range(Lx):
                out.append((x + Lx * y, x + Lx * ((y + 1) % Ly)))
    return np.array(out, dtype=np.int64)


def probe(Lx, Ly, qx, qy, spins):
    """f_q(sigma) = <sigma|S^z_q|psi> / <sigma|psi> = (1/sqrt N) sum_r e^{-i q.r} sigma_r / 2.

    Appendix B, momentum operator; spins is [..., N] with entries +-1.
    """
    x, y = coords(Lx, Ly)
    N = Lx * Ly
    phase = np.exp(-1j * (qx * x + qy * y))
    return (np.asarray(spins, dtype=np.float64) * 0.5) @ phase / np.sqrt(N)


def bond_diagonal(Lx, Ly, J, spins):
    """Diagonal part of H: sum_b (J/4) sigma_i sigma_j, for each row of spins."""
    bl = bonds(Lx, Ly)
    s = np.asarray(spins, dtype=np.float64)
    return 0.25 * J * np.sum(s[..., bl[:, 0]] * s[..., bl[:, 1]], axis=-1)
