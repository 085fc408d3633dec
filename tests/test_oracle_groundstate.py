"""Pins for the oracle's ground-state preparation: the local energy against
the dense Hamiltonian, the force against finite differences of the energy
functional, and convergence of the enumerated descent to the exact ground
energy of a small chain."""

import numpy as np
import pytest

from oracle import exact, groundstate, rbm


def test_local_energy_is_h_psi_over_psi():
    Lx, Ly, N, M = 4, 3, 12, 6
    basis = exact.sector_basis(N)
    p = rbm.init_params(np.random.default_rng(1), N, M, 0.3)
    psi = exact.rbm_vector(p, N, M, basis)
    H = exact.hamiltonian(Lx, Ly, 1.3, basis)
    El = groundstate.local_energy(p, N, M, Lx, Ly, 1.3, basis)
    assert np.allclose(El * psi, H @ psi, atol=1e-12 * np.abs(H @ psi).max())
    w = np.abs(psi) ** 2
    assert np.sum(w * El) / np.sum(w) == pytest.approx(
        np.vdot(psi, H @ psi) / np.vdot(psi, psi), rel=1e-12)


def test_force_is_the_wirtinger_gradient_of_the_energy():
    # E(alpha) in enumeration mode; for a holomorphic psi,
    # dE/dRe alpha_k = 2 Re F_k and dE/dIm alpha_k = 2 Im F_k
    Lx, N, M = 8, 8, 4
    basis = exact.sector_basis(N)
    H = exact.hamiltonian(Lx, 1, 1.0, basis)
    p = rbm.init_params(np.random.default_rng(2), N, M, 0.3)

    def energy(q):
        v = exact.rbm_vector(q, N, M, basis)
        return (np.vdot(v, H @ v) / np.vdot(v, v)).real

    psi = exact.rbm_vector(p, N, M, basis)
    w = np.abs(psi) ** 2
    F, _ = groundstate.energy_force(rbm.logderiv(p, N, M, basis),
                                    groundstate.local_energy(p, N, M, Lx, 1, 1.0, basis),
                                    weights=w / w.sum())
    h = 1e-6
    for k in (0, N, N + M, rbm.n_params(N, M) - 1):
        e = np.zeros(len(p), dtype=np.complex128)
        e[k] = h
        d_re = (energy(p + e) - energy(p - e)) / (2 * h)
        d_im = (energy(p + 1j * e) - energy(p - 1j * e)) / (2 * h)
        assert d_re == pytest.approx(2 * F[k].real, abs=1e-7)
        assert d_im == pytest.approx(2 * F[k].imag, abs=1e-7)


def test_enumerated_descent_reaches_the_ground_energy():
    Lx, N, M = 8, 8, 16
    basis = exact.sector_basis(N)
    H = exact.hamiltonian(Lx, 1, 1.0, basis)
    e0 = np.linalg.eigvalsh(H)[0]
    p = rbm.init_params(np.random.default_rng(3), N, M, 0.05)
    O = None
    for _ in range(150):
        psi = exact.rbm_vector(p, N, M, basis)
        w = np.abs(psi) ** 2
        O = rbm.logderiv(p, N, M, basis)
        El = groundstate.local_energy(p, N, M, Lx, 1, 1.0, basis)
        p, info = groundstate.sr_energy_step(p, O, El, 0.1, 1e-4, weights=w / w.sum())
    assert info["E"].real == pytest.approx(e0, rel=1e-2)
