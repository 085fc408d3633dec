"""Pins for the oracle's lattice, Philox, exact diagonalisation and Chebyshev recursion."""

import os

import numpy as np
import pytest

from oracle import exact, lattice, philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([int(w, 16) for w in line.split()])
    assert len(rows) == 3
    for r in rows:
        out = philox.philox4x32_10(*r[:4], r[4], r[5])
        assert [int(o) for o in out] == r[6:]


def test_philox_vectorised_matches_scalar_and_uniform_range():
    w = np.arange(1000, dtype=np.uint64)
    vec = philox.proposal_words(123456789012345, 77, w)
    for k in (0, 1, 999):
        sc = philox.philox4x32_10(k, 77, 0, 0, 123456789012345 & 0xFFFFFFFF,
                                  123456789012345 >> 32)
        assert [int(v[k]) for v in vec] == [int(s) for s in sc]
    u = philox.uniform(vec[1])
    assert np.all(u > 0) and np.all(u < 1)
    assert philox.uniform(0) == 2.0 ** -24 and philox.uniform(0xFFFFFFFF) == 1 - 2.0 ** -24
    b = philox.bond_index(vec[0], 7)
    assert b.min() >= 0 and b.max() <= 6
    # 1000 uniform bond draws over 7 bins: chi-square with 6 dof far from its tail
    cnt = np.bincount(b, minlength=7)
    chi2 = np.sum((cnt - 1000 / 7) ** 2 / (1000 / 7))
    assert chi2 < 30


@pytest.mark.parametrize("Lx,Ly,deg", [(4, 1, 2), (12, 1, 2), (4, 3, 4), (4, 4, 4), (3, 3, 4)])
def test_bonds_are_periodic_nearest_neighbours(Lx, Ly, deg):
    bl = lattice.bonds(Lx, Ly)
    N = Lx * Ly
    assert len(bl) == (N if Ly == 1 else 2 * N)
    assert len({tuple(sorted(b)) for b in bl}) == len(bl)
    assert np.all(np.bincount(bl.ravel(), minlength=N) == deg)
    x, y = lattice.coords(Lx, Ly)
    for i, j in bl:
        dx = (x[j] - x[i]) % Lx
        dy = (y[j] - y[i]) % Ly
        assert (dx, dy) in ((1, 0), (0, 1))


def test_bad_lattices_rejected():
    for Lx, Ly in ((2, 1), (4, 2), (1, 1)):
        with pytest.raises(ValueError):
            lattice.bonds(Lx, Ly)


def test_ring4_spectrum_closed_form():
    gold = np.loadtxt(os.path.join(GOLDEN, "heisenberg_ring4_spectrum.txt"))
    basis = exact.sector_basis(4)
    H = exact.hamiltonian(4, 1, 1.0, basis)
    assert np.allclose(H, H.T)
    assert np.allclose(np.linalg.eigvalsh(H), np.sort(gold), atol=1e-12)


@pytest.mark.parametrize("Lx,Ly", [(8, 1), (12, 1), (4, 3)])
def test_top_of_spectrum_is_ferromagnetic_multiplet(Lx, Ly):
    # S_i.S_j <= 1/4 with equality on the fully polarised multiplet, which has
    # an S^z = 0 member: E_max = J N_b / 4 exactly.  The sector trace is
    # sum_s (J/4) sum_b s_i s_j; for each bond the antiparallel fraction in
    # the S^z = 0 sector is N/(2(N-1)), giving Tr H = D N_b (J/4)(1 - N/(N-1)).
    N = Lx * Ly
    basis = exact.sector_basis(N)
    J = 1.3
    H = exact.hamiltonian(Lx, Ly, J, basis)
    e = np.linalg.eigvalsh(H)
    Nb = len(lattice.bonds(Lx, Ly))
    assert e[-1] == pytest.approx(J * Nb / 4, abs=1e-10)
    D = basis.shape[0]
    assert np.trace(H) == pytest.approx(D * Nb * J / 4 * (1 - N / (N - 1)), rel=1e-12)


def test_probe_definition_special_cases():
    # q = 0 annihilates the S^z = 0 sector; q = pi on a chain is the staggered moment.
    basis = exact.sector_basis(8)
    assert np.allclose(lattice.probe(8, 1, 0.0, 0.0, basis), 0)
    neel = np.array([[1, -1] * 4], dtype=np.int8)
    assert lattice.probe(8, 1, np.pi, 0.0, neel)[0] == pytest.approx(8 * 0.5 / np.sqrt(8))
    # the 4x3 lattice at q = (pi, 0) with stripes along y
    s = np.array([[1 if x % 2 == 0 else -1 for y in range(3) for x in range(4)]], dtype=np.int8)
    assert lattice.probe(4, 3, np.pi, 0.0, s)[0] == pytest.approx(12 * 0.5 / np.sqrt(12))


def _cheb_T(n, x):
    return np.cos(n * np.arccos(np.clip(x, -1, 1)))


def test_chebyshev_recursion_matches_spectral_sum():
    rng = np.random.default_rng(0)
    basis = exact.sector_basis(10)
    H = exact.hamiltonian(10, 1, 1.0, basis)
    e, V = np.linalg.eigh(H)
    a = (e[-1] - e[0]) / (2 * 0.9875)
    Hp = exact.rescaled(H, e[0], a, 0.9875)
    psi = rng.standard_normal(len(basis)) + 1j * rng.standard_normal(len(basis))
    t0 = exact.probe_vector(10, 1, np.pi / 2, 0.0, basis, psi)
    mu = exact.chebyshev_moments(Hp, t0, psi, 40)
    x = (e - e[0]) / a - 0.9875
    ck = np.abs(V.T @ t0) ** 2 / np.vdot(psi, psi).real
    mu_spec = np.array([np.sum(ck * _cheb_T(n, x)) for n in range(40)])
    assert np.allclose(mu, mu_spec, atol=1e-12 * abs(mu[0]))
    # |mu_n| <= mu_0 when the spectrum of H' lies in [-1, 1]
    assert np.all(np.abs(mu) <= mu[0].real * (1 + 1e-12))
    # doubling identities from T_m T_n = (T_{m+n} + T_{|m-n|}) / 2
    t = exact.chebyshev_vectors(Hp, t0, 20)
    nrm = np.vdot(psi, psi).real
    for n in range(1, 19):
        assert np.vdot(t[n], t[n]) / nrm == pytest.approx((mu[2 * n] + mu[0]) / 2, abs=1e-10)
        assert np.vdot(t[n + 1], t[n]) / nrm == pytest.approx((mu[2 * n + 1] + mu[1]) / 2,
                                                              abs=1e-10)
