"""Pins for the oracle's linear prediction of Chebyshev moments (Sec. VI;
the method of Ganahl et al. 2014 with the growing-mode treatment of
Barthel, Schollwoeck and White 2009): sequences whose continuation is known
in closed form (sums of cosines, damped complex exponentials), the fitted
roots of a known recurrence, the clipping of a growing mode, and the exact
Chebyshev moments of a 6-site Heisenberg chain (a finite set of poles, so
the prediction from 120 moments reproduces the exact moments up to 600)."""

import numpy as np
import pytest

from oracle import exact
from oracle import extrapolate as ex
from paper_2103_08804_gb300 import synth

n = np.arange(600)


def cosines():
    th = np.array([0.3, 0.9, 1.7, 2.2, 2.9])
    w = np.array([0.5, 0.2, 0.1, 0.15, 0.05])
    return (w[:, None] * np.cos(np.outer(th, n))).sum(0)


def damped():
    r = np.array([0.99, 0.97, 0.995])
    t = np.array([0.4, 1.1, 2.5])
    c = np.array([1.0, 0.5 - 0.2j, 0.3j])
    return (c[:, None] * (r[:, None] * np.exp(1j * t[:, None])) ** n).sum(0), r * np.exp(1j * t)


def chain6_moments(n_moments):
    L = 6
    basis = exact.sector_basis(L)
    H = exact.hamiltonian(L, 1, 1.0, basis)
    e = np.linalg.eigvalsh(H)
    a = (e[-1] - e[0]) / (2 * 0.9875)
    Hp = exact.rescaled(H, e[0], a, 0.9875)
    psi = exact.rbm_vector(synth.rbm_params(50, L, 6, 0.3), L, 6, basis)
    t0 = exact.probe_vector(L, 1, 0.6 * np.pi, 0.0, basis, psi)
    return exact.chebyshev_moments(Hp, t0, psi, n_moments)


def test_sum_of_cosines_is_continued_exactly():
    mu = cosines()
    out, z, w = ex.extrapolate(mu[:60], 20, 30, 400)
    assert np.array_equal(out[:60], mu[:60])
    assert np.max(np.abs(out - mu[:400])) < 1e-8


def test_damped_exponentials_and_their_roots():
    mu, poles = damped()
    out, z, w = ex.extrapolate(mu[:50], 12, 20, 500)
    assert np.max(np.abs(out - mu[:500])) < 1e-9
    # each true pole is a fitted root (inside the unit circle: unchanged)
    for q in poles:
        assert np.min(np.abs(z - q)) < 1e-8
    assert np.all(np.abs(w) <= 1.0 + 1e-15)


def test_single_cosine_roots_on_the_unit_circle():
    mu = np.cos(0.77 * n)
    _, z, _ = ex.extrapolate(mu[:40], 2, 10, 100, reg=0.0)
    assert np.allclose(np.sort_complex(z), np.sort_complex(np.exp([-0.77j, 0.77j])), atol=1e-10)


def test_growing_mode_is_put_on_the_unit_circle():
    # mu_n = 1.02^n e^{0.5 i n} + e^{1.3 i n}: the fitted root 1.02 e^{0.5 i}
    # keeps its amplitude (1.02 e^{0.5 i})^{N-p} and loses its growth, so the
    # prediction is 1.02^{N-p} e^{0.5 i n} + e^{1.3 i n} for n >= N
    N, p = 40, 2
    mu = 1.02 ** n * np.exp(0.5j * n) + np.exp(1.3j * n)
    out, z, w = ex.extrapolate(mu[:N], p, 20, 300, reg=0.0)
    assert np.min(np.abs(z - 1.02 * np.exp(0.5j))) < 1e-10
    want = 1.02 ** (N - p) * np.exp(0.5j * n[N:300]) + np.exp(1.3j * n[N:300])
    assert np.max(np.abs(out[N:] - want)) < 1e-8
    assert np.all(np.abs(w) <= 1.0 + 1e-15)


def test_exact_chain_moments_are_predicted():
    mu = chain6_moments(600)
    out, z, _ = ex.extrapolate(mu[:120], 48, 60, 600)
    assert np.max(np.abs(out - mu)) < 1e-5 * abs(mu[0])


def test_coefficients_are_the_least_squares_solution():
    """Without the Tikhonov term the coefficients minimise the one-step
    prediction error over the window: on arbitrary complex data they equal
    the library least-squares solution (SVD) of the data matrix."""
    g = np.random.Generator(np.random.Philox(17))
    mu = g.standard_normal(40) + 1j * g.standard_normal(40)
    p, n0 = 5, 10
    A = np.array([mu[n - p:n][::-1] for n in range(n0, 40)])
    want = np.linalg.lstsq(A, -mu[n0:40], rcond=None)[0]
    assert np.max(np.abs(ex.lp_coefficients(mu, p, n0, 0.0) - want)) < 1e-10


def test_bad_arguments():
    mu = cosines()[:50]
    for p, n0, n_out in ((0, 10, 60), (20, 10, 60), (10, 50, 60), (10, 20, 40)):
        with pytest.raises(ValueError):
            ex.extrapolate(mu, p, n0, n_out)


def _pins_fail():
    """True when at least one pin above fails."""
    checks = (test_sum_of_cosines_is_continued_exactly, test_damped_exponentials_and_their_roots,
              test_single_cosine_roots_on_the_unit_circle, test_growing_mode_is_put_on_the_unit_circle,
              test_exact_chain_moments_are_predicted,
              test_coefficients_are_the_least_squares_solution)
    for f in checks:
        try:
            f()
        except (AssertionError, np.linalg.LinAlgError, ValueError):
            return True
    return False


def test_planted_mistakes_fail_a_pin(monkeypatch):
    """Plausible mistakes planted in the oracle (on the CPU) each fail a pin:
    the normal equations without the conjugate, a lag off by one, the sign
    of the prediction coefficients, growing roots left in place."""
    good_ne, good_coef, good_roots = ex.normal_equations, ex.lp_coefficients, ex.lp_roots
    assert not _pins_fail()

    def no_conj(mu, p, n0, reg):
        mu = np.asarray(mu, dtype=np.complex128)
        R = np.zeros((p, p), dtype=np.complex128)
        r = np.zeros(p, dtype=np.complex128)
        for n in range(n0, len(mu)):
            past = mu[n - p:n][::-1]
            R += np.outer(past, past)
            r += past * mu[n]
        return R + reg * np.max(np.abs(np.diag(R))) * np.eye(p), r

    def lag_off(mu, p, n0, reg):
        mu = np.asarray(mu, dtype=np.complex128)
        R = np.zeros((p, p), dtype=np.complex128)
        r = np.zeros(p, dtype=np.complex128)
        for n in range(max(n0, p + 1), len(mu)):
            past = mu[n - p - 1:n - 1][::-1]
            R += np.outer(np.conj(past), past)
            r += np.conj(past) * mu[n]
        return R + reg * np.max(np.real(np.diag(R))) * np.eye(p), r

    for name, fn in (("normal_equations", no_conj), ("normal_equations", lag_off),
                     ("lp_coefficients", lambda *a: -good_coef(*a))):
        monkeypatch.setattr(ex, name, fn)
        assert _pins_fail(), name
        monkeypatch.setattr(ex, "normal_equations", good_ne)
        monkeypatch.setattr(ex, "lp_coefficients", good_coef)
    # growing roots kept: the clipped-mode pin must fail
    monkeypatch.setattr(ex, "stabilise", lambda z: z)
    with pytest.raises(AssertionError):
        test_growing_mode_is_put_on_the_unit_circle()
    monkeypatch.undo()
    assert good_roots is ex.lp_roots
