"""Pins for the oracle's moment correction and Krylov projection.

Fed the exact Chebyshev vectors of a small lattice, the projected recursion
must return the exact moments, and the generalised eigenproblem is a Gauss
quadrature of the probe's spectral measure: sum_k w_k T_n(lambda_k) = mu_n for
n <= 2 Nm - 1, sum_k w_k = mu_0, and the nodes are the Ritz values of a
plain Lanczos run from t_0."""

import numpy as np
import pytest

from oracle import exact, krylov, rbm


def _setup(Nm):
    Lx = 10
    basis = exact.sector_basis(Lx)
    H = exact.hamiltonian(Lx, 1, 1.0, basis)
    e = np.linalg.eigvalsh(H)
    a = (e[-1] - e[0]) / (2 * 0.9875)
    Hp = exact.rescaled(H, e[0], a, 0.9875)
    p = rbm.init_params(np.random.default_rng(20), Lx, 10, 0.3)
    psi = exact.rbm_vector(p, Lx, 10, basis)
    t0 = exact.probe_vector(Lx, 1, 0.6 * np.pi, 0.0, basis, psi)
    ts = exact.chebyshev_vectors(Hp, t0, Nm)
    w = np.abs(psi) ** 2 / np.vdot(psi, psi).real
    B = [t / psi for t in ts]
    HB = [(Hp @ t) / psi for t in ts]
    G, Hm = krylov.gram(B, HB, weights=w)
    mu = exact.chebyshev_moments(Hp, t0, psi, 2 * Nm)
    return Hp, t0, psi, G, Hm, mu


def _T(n, x):
    return np.cos(n * np.arccos(np.clip(x, -1, 1)))


def test_gram_matches_dense_inner_products():
    Hp, t0, psi, G, Hm, _ = _setup(6)
    ts = exact.chebyshev_vectors(Hp, t0, 6)
    Z = np.vdot(psi, psi).real
    Gd = np.array([[np.vdot(a, b) for b in ts] for a in ts]) / Z
    Hd = np.array([[np.vdot(a, Hp @ b) for b in ts] for a in ts]) / Z
    assert np.allclose(G, Gd, atol=1e-14)
    assert np.allclose(Hm, Hd, atol=1e-14)


def test_corrected_moments_reproduce_exact_moments():
    Nm = 6
    _, _, _, G, Hm, mu = _setup(Nm)
    mc = krylov.corrected_moments(G, Hm, 2 * Nm, cutoff=1e-13)
    assert np.allclose(mc, mu, atol=1e-8 * abs(mu[0]))


def test_poles_are_gauss_quadrature_and_lanczos_ritz_values():
    Nm = 6
    Hp, t0, psi, G, Hm, mu = _setup(Nm)
    lam, w = krylov.krylov_poles(G, Hm, cutoff=1e-13)
    assert len(lam) == Nm
    assert np.sum(w) == pytest.approx(mu[0].real, rel=1e-10)
    for n in range(2 * Nm):
        assert np.sum(w * _T(n, lam)) == pytest.approx(mu[n].real, abs=1e-8 * abs(mu[0]))
    # plain Lanczos with full reorthogonalisation from v0 = t0 / |t0|
    V = [t0 / np.linalg.norm(t0)]
    alpha, beta = [], []
    for k in range(Nm):
        w_ = Hp @ V[-1]
        alpha.append(np.vdot(V[-1], w_).real)
        for v in V:
            w_ = w_ - np.vdot(v, w_) * v
        if k < Nm - 1:
            beta.append(np.linalg.norm(w_))
            V.append(w_ / beta[-1])
    Tm = np.diag(alpha) + np.diag(beta, 1) + np.diag(beta, -1)
    assert np.allclose(np.sort(lam), np.linalg.eigvalsh(Tm), atol=1e-9)


def test_sampled_H_is_hermitian():
    """On sampled columns (plain means over a subset of the configurations)
    the raw estimator <conj(B_n) HB_m> is not Hermitian; the projected H
    the Krylov step uses is (its sampled form is Hermitised), with a real
    diagonal, and G is Hermitian positive semi-definite."""
    Hp, t0, psi, _, _, _ = _setup(6)
    ts = exact.chebyshev_vectors(Hp, t0, 6)
    g = np.random.default_rng(4)
    idx = g.choice(len(psi), size=60, replace=True)
    B = [(t / psi)[idx] for t in ts]
    HB = [((Hp @ t) / psi)[idx] for t in ts]
    raw = (np.conj(np.array(B)) / 60) @ np.array(HB).T
    assert np.max(np.abs(raw - raw.conj().T)) > 1e-6
    G, Hm = krylov.gram(B, HB)
    assert np.array_equal(Hm, Hm.conj().T)
    assert np.max(np.abs(G - G.conj().T)) <= 1e-14 * np.max(np.abs(G))
    assert np.min(np.linalg.eigvalsh(0.5 * (G + G.conj().T))) > -1e-12 * np.max(np.abs(G))
