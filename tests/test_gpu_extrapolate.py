"""cheb_extrapolate (linear prediction of Chebyshev moments, Sec. VI) against
the oracle on the same moments: closed-form sequences (sums of cosines,
damped complex exponentials), the exact moments of a 6-site Heisenberg
chain, the same moments with noise of a sampled estimate, a growing mode
clipped onto the unit circle; the fitted roots; a batch of sequences equal
to each sequence alone; a singular window (CR_ESINGULAR, NaN prediction);
argument errors."""

import numpy as np
import pytest

from gpu_common import host, need_gpu, torch
from oracle import extrapolate as ex

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.fixture(scope="module")
def ctx():
    from paper_2103_08804_gb300 import api
    return api.Context(4, 1, 4, 8, prec=api.FP64)


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()


def _chain6(n_moments):
    from test_oracle_extrapolate import chain6_moments
    return chain6_moments(n_moments)


def _cases():
    from test_oracle_extrapolate import cosines, damped
    n = np.arange(600)
    noisy = _chain6(600)
    g = np.random.Generator(np.random.Philox(5))
    noisy = noisy + 1e-6 * abs(noisy[0]) * (g.standard_normal(600) + 1j * g.standard_normal(600))
    return {
        "cosines": (cosines(), 60, 20, 30, 400, 1e-12),
        "damped": (damped()[0], 50, 12, 20, 500, 1e-12),
        "chain6": (_chain6(600), 120, 48, 60, 600, 1e-12),
        "chain6_noisy": (noisy, 120, 40, 60, 600, 1e-8),
        "growing": (1.02 ** n * np.exp(0.5j * n) + np.exp(1.3j * n), 40, 2, 20, 300, 0.0),
    }


def _match_roots(zg, zo):
    """Largest distance from an oracle root to the nearest GPU root."""
    return max(np.min(np.abs(zg - q)) for q in zo)


@pytest.mark.parametrize("case", ["cosines", "damped", "chain6", "chain6_noisy", "growing"])
def test_prediction_matches_the_oracle(ctx, case):
    mu, N, p, n0, n_out, reg = _cases()[case]
    ref, z_ref, _ = ex.extrapolate(mu[:N], p, n0, n_out, reg=reg)
    roots = torch.empty(1, p, dtype=torch.complex128, device="cuda")
    info = torch.empty(1, dtype=torch.int32, device="cuda")
    got = host(ctx.cheb_extrapolate(_dev(mu[:N]), p, n0, n_out, reg=reg, roots_out=roots,
                                    info_out=info))
    ctx.sync_status()
    assert np.array_equal(got[:N], mu[:N])
    scale = np.max(np.abs(mu[:N]))
    err = np.max(np.abs(got - ref)) / scale
    print(f"{case}: prediction vs oracle {err:.2e}, root iterations {int(host(info)[0])}")
    assert 0 < int(host(info)[0]) <= 500
    assert err < (1e-9 if case != "chain6_noisy" else 1e-6)
    # the poles of the sequence are fitted roots on both sides (the remaining
    # roots of an over-sized order are fixed only by the Tikhonov term)
    from test_oracle_extrapolate import damped
    th = np.array([0.3, 0.9, 1.7, 2.2, 2.9])
    poles = {"cosines": np.concatenate([np.exp(1j * th), np.exp(-1j * th)]),
             "damped": damped()[1], "growing": z_ref}.get(case)
    if poles is not None:
        assert _match_roots(host(roots)[0], poles) < 1e-8
        assert _match_roots(z_ref, poles) < 1e-8
    if case == "chain6":
        assert np.max(np.abs(got - mu[:n_out])) < 1e-5 * scale


def test_growing_mode_closed_form(ctx):
    n = np.arange(300)
    N, p = 40, 2
    mu = 1.02 ** n * np.exp(0.5j * n) + np.exp(1.3j * n)
    got = host(ctx.cheb_extrapolate(_dev(mu[:N]), p, 20, 300, reg=0.0))
    want = 1.02 ** (N - p) * np.exp(0.5j * n[N:]) + np.exp(1.3j * n[N:])
    assert np.max(np.abs(got[N:] - want)) < 1e-8


def test_batch_equals_each_sequence_alone(ctx):
    cs = _cases()
    seqs = [cs["chain6"][0][:120], cs["chain6_noisy"][0][:120], cs["cosines"][0][:120]]
    batch = host(ctx.cheb_extrapolate(_dev(np.stack(seqs)), 40, 60, 500, reg=1e-10))
    for k, m in enumerate(seqs):
        alone = host(ctx.cheb_extrapolate(_dev(m), 40, 60, 500, reg=1e-10))
        assert np.array_equal(batch[k], alone)
    ctx.sync_status()


def test_singular_window_sets_esingular(ctx):
    from paper_2103_08804_gb300 import api
    # mu_n = 1: R_ij = 4 (window of 4 targets), so the second Cholesky pivot
    # of R without a Tikhonov term is 4 - 2 * 2 = 0 exactly
    mu = np.ones(12, dtype=np.complex128)
    info = torch.empty(1, dtype=torch.int32, device="cuda")
    got = host(ctx.cheb_extrapolate(_dev(mu), 3, 8, 20, reg=0.0, info_out=info))
    with pytest.raises(api.CRError, match="CR_ESINGULAR"):
        ctx.sync_status()
    assert int(host(info)[0]) == -2
    assert np.array_equal(got[:12], mu) and np.all(np.isnan(got[12:]))


def test_bad_arguments(ctx):
    from paper_2103_08804_gb300 import api
    mu = _dev(np.ones(50))
    for p, n0, n_out in ((0, 10, 60), (20, 10, 60), (10, 50, 60), (10, 20, 40), (513, 600, 700)):
        with pytest.raises(api.CRError):
            ctx.cheb_extrapolate(mu, p, n0, n_out)
