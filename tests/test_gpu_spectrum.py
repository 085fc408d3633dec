"""The spectral function on a frequency grid (Sec. II Eq. Aw with Jackson
damping; Sec. IV continued fraction) through the C ABI, against the oracle.

Float64 throughout: the GPU evaluates T_n(omega') by the three-term
recursion, the oracle as cos(n arccos omega'), so the two agree to
rounding (held to 1e-10 of the largest value).  The Krylov route compares
the GPU's pole sum (cheb_krylov, then cheb_lorentzian) with the oracle's
Lanczos continued fraction, two different evaluations of the same
projected resolvent (1e-8 relative)."""

import numpy as np
import pytest

from gpu_common import dev, host, need_gpu, torch
from oracle import spectrum

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _ctx():
    from paper_2103_08804_gb300 import api
    return api.Context(4, 1, 4, 8, prec=api.FP64)


@pytest.mark.parametrize("Nm", [1, 7, 300])
@pytest.mark.parametrize("jackson", [False, True])
def test_chebyshev_spectrum_against_oracle(Nm, jackson):
    rng = np.random.default_rng(Nm)
    mu = (rng.standard_normal(Nm) + 1j * rng.standard_normal(Nm)) / (1 + np.arange(Nm))
    a, Wp = 3.3, 0.9875
    # a ragged grid reaching outside [-1, 1] in omega' on both sides
    omega = np.sort(rng.uniform(-0.5, 2 * a + 0.5, 1001))
    ref = spectrum.chebyshev_spectrum(mu, a, Wp, omega, damping="jackson" if jackson else None)
    ctx = _ctx()
    A = host(ctx.cheb_spectrum(dev(mu, torch.complex128), a, Wp, dev(omega, torch.float64),
                               jackson=jackson))
    ctx.sync_status()
    assert np.max(np.abs(A - ref)) <= 1e-10 * np.max(np.abs(ref))
    assert np.all(A[np.abs(omega / a - Wp) >= 1] == 0)


def test_lorentzian_of_krylov_poles_equals_oracle_continued_fraction():
    from test_oracle_spectrum import _chebyshev_states
    _, _, G, H = _chebyshev_states(30, 9, 4)
    a, Wp, eta = 2.0, 0.9875, 0.05
    omega = np.linspace(0.0, 2 * a * Wp, 333)
    ref = spectrum.continued_fraction(G, H, a, Wp, omega, eta, cutoff=1e-12)
    ctx = _ctx()
    Nm = G.shape[0]
    mu = torch.zeros(2 * Nm, dtype=torch.complex128, device="cuda")
    poles = torch.zeros(Nm, dtype=torch.float64, device="cuda")
    wts = torch.zeros(Nm, dtype=torch.float64, device="cuda")
    ctx.cheb_krylov(dev(G, torch.complex128), dev(H, torch.complex128), 1e-12, 2 * Nm, mu,
                    poles, wts)
    A = host(ctx.cheb_lorentzian(poles, wts, a, Wp, eta, dev(omega, torch.float64)))
    ctx.sync_status()
    assert np.allclose(A, ref, rtol=1e-8, atol=1e-12 * np.max(np.abs(ref)))


def test_spectrum_edge_cases_and_bad_arguments():
    from paper_2103_08804_gb300 import api
    ctx = _ctx()
    mu = dev(np.ones(4), torch.complex128)
    empty = torch.empty(0, dtype=torch.float64, device="cuda")
    assert ctx.cheb_spectrum(mu, 1.0, 0.9, empty).numel() == 0
    w = dev(np.linspace(0, 1, 5), torch.float64)
    with pytest.raises(api.CRError):
        ctx.cheb_spectrum(mu, -1.0, 0.9, w)
    with pytest.raises(api.CRError):
        ctx.cheb_spectrum(mu, 1.0, 1.5, w)
    with pytest.raises(api.CRError):
        ctx.cheb_lorentzian(w, w, 1.0, 0.9, 0.0, w)
    ctx.sync_status()
