"""Pins for the oracle's RBM amplitude, log-derivatives and local target."""

import numpy as np
import pytest

from oracle import exact, lattice, rbm, target
from oracle.target import State


def _params(seed, N, M, sigma):
    return rbm.init_params(np.random.default_rng(seed), N, M, sigma)


def test_logpsi_closed_forms():
    rng = np.random.default_rng(1)
    N, M = 6, 5
    s = exact.sector_basis(N)
    # W = 0: psi = exp(a.s) prod_j 2 cosh b_j, each factor independent of the others
    p = _params(2, N, M, 0.3)
    p[N + M:] = 0
    a, b = p[:N], p[N:N + M]
    ref = s @ a + np.sum(np.log(2 * np.cosh(b)))
    d = rbm.logpsi(p, N, M, s) - ref
    assert np.allclose(np.exp(d), 1, atol=1e-13)
    # N = 1, M = 1 by hand
    p1 = np.array([0.1 + 0.2j, -0.3 + 0.05j, 0.7 - 0.4j])
    for sg in (1, -1):
        v = np.exp(rbm.logpsi(p1, 1, 1, np.array([[sg]])))[0]
        assert v == pytest.approx(np.exp(p1[0] * sg) * 2 * np.cosh(p1[1] + p1[2] * sg), rel=1e-14)
    # a = b = 0: cosh is even, so psi(-s) = psi(s)
    p = _params(3, N, M, 0.4)
    p[:N + M] = 0
    assert np.allclose(np.exp(rbm.logpsi(p, N, M, s) - rbm.logpsi(p, N, M, -s)), 1, atol=1e-13)
    del rng


@pytest.mark.parametrize("h", [1e-5])
def test_logderiv_matches_central_differences(h):
    N, M = 5, 4
    p = _params(4, N, M, 0.5)
    s = exact.sector_basis(6)[:7, :5]
    O = rbm.logderiv(p, N, M, s)
    for k in range(rbm.n_params(N, M)):
        for step in (h, 1j * h):
            e = np.zeros_like(p)
            e[k] = step
            fd = (rbm.logpsi(p + e, N, M, s) - rbm.logpsi(p - e, N, M, s)) / (2 * step)
            assert np.allclose(fd, O[:, k], atol=1e-8), k


@pytest.mark.parametrize("Lx,Ly,n", [(8, 1, 1), (8, 1, 2), (8, 1, 3), (4, 3, 2)])
def test_local_target_against_dense_hamiltonian(Lx, Ly, n):
    N, M = Lx * Ly, 6
    J, E0, a, Wp = 1.0, -3.1, 2.7, 0.9875
    q = (np.pi / 2, np.pi)
    basis = exact.sector_basis(N)
    H = exact.hamiltonian(Lx, Ly, J, basis)
    Hp = exact.rescaled(H, E0, a, Wp)
    psi = _params(5, N, M, 0.3)
    s_prev = State(psi, probe=True) if n == 1 else State(_params(6, N, M, 0.3))
    s_prev2 = State(psi, probe=True) if n == 2 else State(_params(7, N, M, 0.3))
    psi_n = _params(8, N, M, 0.3)
    bp, bp2 = 0.7 - 0.2j, -0.4 + 0.9j

    def dense(st):
        v = exact.rbm_vector(st.params, N, M, basis)
        return lattice.probe(Lx, Ly, q[0], q[1], basis) * v if st.probe else v

    phi = bp * (Hp @ dense(s_prev)) if n == 1 else 2 * bp * (Hp @ dense(s_prev)) - bp2 * dense(s_prev2)
    lp = rbm.logpsi(psi_n, N, M, basis)
    R = target.local_target(n, s_prev, s_prev2, bp, bp2, N, M, Lx, Ly, J, E0, a, Wp, q, basis, lp)
    assert np.allclose(R * np.exp(lp), phi, atol=1e-12 * np.abs(phi).max())
