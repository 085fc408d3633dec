"""Plausible mistakes planted in the oracle, on the CPU, each fail one of its
pins: a dropped conjugate in the force, the estimators or O_W, a missing
gamma cot gamma factor, S without its centring term or with the conjugate on
the wrong side, an unsymmetrised sampled H, and W flattened in the wrong
order.  (The planted mistakes of the extrapolation oracle are in
test_oracle_extrapolate.py.)"""

import numpy as np
import pytest

import test_oracle_krylov as TK
import test_oracle_rbm as TR
import test_oracle_sr as TS
from oracle import krylov, rbm, sr


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
}


@pytest.mark.parametrize("case", list(CASES))
def test_planted_mistake_fails_a_pin(case, monkeypatch):
    mod, attr, bad, checks = CASES[case]
    assert not _fails(*checks), "the pins must pass on the oracle as written"
    monkeypatch.setattr(mod, attr, bad)
    assert _fails(*checks), case
