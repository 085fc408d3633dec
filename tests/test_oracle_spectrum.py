"""Pins for the oracle's spectral reconstruction (Sec. II, Eq. Aw with the
Jackson damping of Sec. V) and continued fraction (Sec. IV)."""

import numpy as np
import pytest

from oracle import krylov, spectrum


def test_jackson_factors():
    for N in (2, 5, 100):
        g = spectrum.jackson(N)
        assert g[0] == pytest.approx(1.0, abs=1e-15)
        assert np.all(g > 0) and np.all(np.diff(g) < 0)
    # N = 2 by hand: g_1 = (2 cos(pi/3) + sin(pi/3) cot(pi/3)) / 3 = 1/2
    assert spectrum.jackson(2)[1] == pytest.approx(0.5, abs=1e-15)


def test_finite_chebyshev_series_is_reconstructed_exactly():
    # density rho(x) = p(x) / (pi sqrt(1 - x^2)) with p a cubic: its moments
    # int rho T_n are b_0 and b_n / 2 for p = sum b_n T_n (numpy's own
    # power-to-Chebyshev conversion); without damping, Eq. (Aw) with N > 3
    # moments must give back rho(omega') / a on any grid
    p = np.array([1.0, 0.5, -0.3, 0.2])            # 1 + x/2 - 0.3 x^2 + 0.2 x^3
    b = np.polynomial.chebyshev.poly2cheb(p)
    mu = np.zeros(7, dtype=np.complex128)
    mu[0] = b[0]
    mu[1:len(b)] = b[1:] / 2
    a, Wp = 2.5, 0.9875
    omega = np.linspace(0.01, 2 * a * Wp - 0.01, 37)
    x = omega / a - Wp
    rho = np.polynomial.polynomial.polyval(x, p) / (np.pi * np.sqrt(1 - x * x))
    A = spectrum.chebyshev_spectrum(mu, a, Wp, omega, damping=None)
    assert np.allclose(A, rho / a, rtol=1e-12, atol=0)
    assert np.all(spectrum.chebyshev_spectrum(mu, a, Wp, np.array([-1.0, 2 * a + 1])) == 0)


def test_jackson_delta_is_positive_and_keeps_the_sum_rule():
    # moments of a delta at x0: mu_n = T_n(x0).  The Jackson-damped series is
    # non-negative and integrates to mu_0 (Gauss-Chebyshev quadrature in
    # omega' is exact for the polynomial part)
    N, x0, a, Wp = 64, 0.3, 1.7, 0.9875
    mu = np.cos(np.arange(N) * np.arccos(x0)) + 0j
    K = 400
    xj = np.cos(np.pi * (np.arange(K) + 0.5) / K)
    A = spectrum.chebyshev_spectrum(mu, a, Wp, a * (xj + Wp))
    assert np.all(A.real > -1e-12) and np.allclose(A.imag, 0)
    integral = np.sum(A.real * np.sqrt(1 - xj * xj)) * np.pi / K * a
    assert integral == pytest.approx(1.0, abs=1e-12)
    fine = np.linspace(-0.99, 0.99, 2001)
    Af = spectrum.chebyshev_spectrum(mu, a, Wp, a * (fine + Wp)).real
    assert abs(fine[np.argmax(Af)] - x0) < np.pi / N


def _chebyshev_states(D, Nm, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((D, D)) + 1j * rng.standard_normal((D, D))
    A = (A + A.conj().T) / 2
    e = np.linalg.eigvalsh(A)
    A = (A - e[0] * np.eye(D)) / ((e[-1] - e[0]) / 1.9) - 0.95 * np.eye(D)
    t0 = rng.standard_normal(D) + 1j * rng.standard_normal(D)
    T = [t0, A @ t0]
    while len(T) < Nm:
        T.append(2 * A @ T[-1] - T[-2])
    T = np.array(T[:Nm]).T
    return A, t0, T.conj().T @ T, T.conj().T @ A @ T


def test_continued_fraction_is_the_resolvent_on_the_full_space():
    D = 8
    A, t0, G, H = _chebyshev_states(D, D, 3)
    a, Wp, eta = 3.0, 0.9875, 0.1
    omega = np.linspace(0.0, 2 * a * Wp, 53)
    Acf = spectrum.continued_fraction(G, H, a, Wp, omega, eta, cutoff=1e-14)
    z = omega / a - Wp + 1j * eta / a
    exact = np.array([np.vdot(t0, np.linalg.solve(zz * np.eye(D) - A, t0)) for zz in z])
    assert np.allclose(Acf, -exact.imag / (np.pi * a), rtol=1e-8, atol=1e-12)


def test_continued_fraction_equals_the_projected_pole_sum():
    # on a Krylov subspace smaller than the space, the Lanczos continued
    # fraction and the generalised eigen-decomposition of (H, G) are two
    # routes to the same projected resolvent sum_k w_k / (z - lambda_k)
    A, t0, G, H = _chebyshev_states(30, 9, 4)
    a, Wp, eta = 2.0, 0.9875, 0.05
    omega = np.linspace(0.0, 2 * a * Wp, 71)
    Acf = spectrum.continued_fraction(G, H, a, Wp, omega, eta, cutoff=1e-12)
    lam, w = krylov.krylov_poles(G, H, cutoff=1e-12)
    z = omega / a - Wp + 1j * eta / a
    poles = np.sum(w[None, :] / (z[:, None] - lam[None, :]), axis=1)
    assert np.allclose(Acf, -poles.imag / (np.pi * a), rtol=1e-8, atol=1e-12)
    assert np.sum(w) == pytest.approx(G[0, 0].real, rel=1e-10)
