"""Plausible mistakes planted in the oracle, on the CPU, each fail one of its
pins: a dropped conjugate in the force, the estimators or O_W, a missing
gamma cot gamma factor, S without its centring term or with the conjugate on
the wrong side, an unsymmetrised sampled H, W flattened in the wrong order,
the exchange term of H at J instead of J/2, the recursion without its factor
2, the Chebyshev sum without the factor 2 of its n >= 1 terms, and Jackson
factors with the sign of the sine term flipped.  (The planted mistakes of the extrapolation oracle are in
test_oracle_extrapolate.py.)"""

import numpy as np
import pytest

import test_oracle_krylov as TK
import test_oracle_rbm as TR
import test_oracle_spectrum as TP
import test_oracle_sr as TS
from oracle import krylov, lattice, rbm, spectrum, sr, target


def _fails(*checks):
    for f, kw in checks:
        try:
            with np.errstate(all="ignore"):
                f(**kw)
        except (AssertionError, ValueError, np.linalg.LinAlgError):
            return True
    return False


def _force_no_conj(est, dgamma):
    gamma = sr.fubini_study_angle(est["mR"], est["mRR"])
    return dgamma * sr.gamma_cot_gamma(gamma) * (est["OR"] / est["mR"] - est["Obar"]), gamma


def _force_no_gamma_factor(est, dgamma):
    gamma = sr.fubini_study_angle(est["mR"], est["mRR"])
    return dgamma * (est["OR"] / est["mR"] - np.conj(est["Obar"])), gamma


def _qgt_uncentred(est):
    return est["OO"]


def _qgt_conj_swapped(est):
    return est["OO"] - np.outer(est["Obar"], np.conj(est["Obar"]))


_good_estimators = sr.estimators


def _estimators_no_conj(O, R, weights=None, with_OO=True):
    e = _good_estimators(O, R, weights, with_OO)
    e["OR"] = sr._mean(np.asarray(O, dtype=np.complex128) * np.asarray(R)[:, None], weights)
    return e


def _gram_unsymmetrised(B, HB, weights=None):
    Bm, HBm = np.array(B, dtype=np.complex128), np.array(HB, dtype=np.complex128)
    w = np.full(Bm.shape[1], 1.0 / Bm.shape[1]) if weights is None else np.asarray(weights)
    return (np.conj(Bm) * w) @ Bm.T, (np.conj(Bm) * w) @ HBm.T


def _logderiv_conj_T(spins, T):
    s = np.asarray(spins, dtype=np.float64)
    T = np.asarray(T, dtype=np.complex128)
    OW = (s[:, :, None] * np.conj(T)[:, None, :]).reshape(s.shape[0], -1)
    return np.concatenate([s.astype(np.complex128), T, OW], axis=1)


def _theta_column_major(params, N, M, spins):
    _, b, W = rbm.unpack(params, N, M)
    return b + np.asarray(spins, dtype=np.float64) @ W.reshape(M, N).T


def _hprime_full_exchange(state, N, M, Lx, Ly, J, E0, a, Wp, q, spins, logpsi_ref):
    spins = np.asarray(spins, dtype=np.int8)
    rows = np.arange(spins.shape[0])
    v = target.rel_amplitude(state, N, M, Lx, Ly, q, spins, logpsi_ref)
    Hv = lattice.bond_diagonal(Lx, Ly, J, spins) * v
    for i, j in lattice.bonds(Lx, Ly):
        anti = spins[:, i] != spins[:, j]
        flipped = spins.copy()
        flipped[rows, i] = spins[:, j]
        flipped[rows, j] = spins[:, i]
        vf = target.rel_amplitude(state, N, M, Lx, Ly, q, flipped, logpsi_ref)
        Hv = Hv + np.where(anti, J * vf, 0.0)
    return (Hv - E0 * v) / a - Wp * v


def _target_without_factor_two(n, prev, prev2, beta_prev, beta_prev2, N, M, Lx, Ly, J, E0, a,
                               Wp, q, spins, logpsi_n):
    h = target.apply_hprime(prev, N, M, Lx, Ly, J, E0, a, Wp, q, spins, logpsi_n)
    if n == 1:
        return beta_prev * h
    v2 = target.rel_amplitude(prev2, N, M, Lx, Ly, q, spins, logpsi_n)
    return beta_prev * h - beta_prev2 * v2


_good_spectrum = spectrum.chebyshev_spectrum


def _spectrum_without_factor_two(mu, a, Wp, omega, damping="jackson"):
    half = np.array(mu, dtype=np.complex128)
    half[1:] *= 0.5
    return _good_spectrum(half, a, Wp, omega, damping)


def _jackson_sine_flipped(N):
    n = np.arange(N, dtype=np.float64)
    q = np.pi / (N + 1)
    return ((N - n + 1) * np.cos(q * n) - np.sin(q * n) / np.tan(q)) / (N + 1)


FAST_SR = ((TS.test_vmc_estimators_equal_braket_forms, {}),
           (TS.test_exact_representability_gives_zero_angle_and_force, {}),
           (TS.test_matrix_free_product_and_cg_equal_the_explicit_forms, {}))
DRIVER = ((TS.test_enumerated_driver_betas_and_moments_against_dense_vectors, {}),)

CASES = {
    "force without the conjugate of <O>": (sr, "force", _force_no_conj, FAST_SR),
    "force without gamma cot gamma": (sr, "force", _force_no_gamma_factor, FAST_SR),
    "S without its centring term": (sr, "qgt", _qgt_uncentred, FAST_SR),
    "S with the conjugate on the wrong side": (sr, "qgt", _qgt_conj_swapped, FAST_SR),
    "<O* R> without the conjugate": (sr, "estimators", _estimators_no_conj, FAST_SR),
    "sampled H not Hermitised": (krylov, "gram", _gram_unsymmetrised,
                                 ((TK.test_sampled_H_is_hermitian, {}),)),
    "O_W with conj(T)": (rbm, "logderiv_from_tanh", _logderiv_conj_T, DRIVER),
    "W flattened column-major": (rbm, "theta", _theta_column_major, DRIVER),
    "exchange term at J": (target, "apply_hprime", _hprime_full_exchange,
                           ((TR.test_local_target_against_dense_hamiltonian,
                             {"Lx": 8, "Ly": 1, "n": 1}),)),
    "recursion without its factor 2": (target, "local_target", _target_without_factor_two,
                                       ((TR.test_local_target_against_dense_hamiltonian,
                                         {"Lx": 8, "Ly": 1, "n": 2}),)),
    "Chebyshev sum without the factor 2": (spectrum, "chebyshev_spectrum",
                                           _spectrum_without_factor_two,
                                           ((TP.test_finite_chebyshev_series_is_reconstructed_exactly,
                                             {}),)),
    "Jackson sine term flipped": (spectrum, "jackson", _jackson_sine_flipped,
                                  ((TP.test_jackson_factors, {}),
                                   (TP.test_jackson_delta_is_positive_and_keeps_the_sum_rule, {}))),
}


@pytest.mark.parametrize("case", list(CASES))
def test_planted_mistake_fails_a_pin(case, monkeypatch):
    mod, attr, bad, checks = CASES[case]
    assert not _fails(*checks), "the pins must pass on the oracle as written"
    monkeypatch.setattr(mod, attr, bad)
    assert _fails(*checks), case
