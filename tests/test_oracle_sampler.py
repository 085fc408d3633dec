"""Pins for the oracle's Metropolis sampler: S^z conservation, the accept rule,
and the stationary distribution |psi|^2 / Z against exact enumeration."""

import numpy as np
import scipy.stats

from oracle import exact, lattice, rbm, sampler


def _sz0(seed, B, N):
    rng = np.random.default_rng(seed)
    s = np.tile(np.array([1] * (N // 2) + [-1] * (N // 2), dtype=np.int8), (B, 1))
    return rng.permuted(s, axis=1)


def test_sz_is_conserved_and_counter_advances():
    N, M = 8, 8
    p = rbm.init_params(np.random.default_rng(0), N, M, 0.3)
    s0 = _sz0(1, 64, N)
    s1, acc, ctr = sampler.mc_sweep(p, N, M, lattice.bonds(8, 1), s0, 3, 11, 5)
    assert np.all(s1.sum(axis=1) == 0)
    assert ctr == 5 + 12
    assert np.all(acc <= 24) and acc.sum() > 0


def test_flat_amplitude_accepts_every_antiparallel_proposal():
    # psi = const: every exchange has |ratio|^2 = 1 > u, so the accepted count
    # equals the number of proposals that landed on an antiparallel bond.
    N, M = 8, 3
    p = np.zeros(rbm.n_params(N, M), dtype=np.complex128)
    bl = lattice.bonds(8, 1)
    s = _sz0(2, 32, N)
    from oracle import philox
    n_anti = np.zeros(32, dtype=int)
    cur = s.copy()
    rows = np.arange(32)
    for prop in range(N):
        words = philox.proposal_words(9, prop // 2, np.arange(32, dtype=np.uint64))
        b = philox.bond_index(words[2 * (prop % 2)], len(bl))
        i, j = bl[b, 0], bl[b, 1]
        anti = cur[rows, i] != cur[rows, j]
        n_anti += anti
        t = cur[rows, i].copy()
        cur[rows, i] = np.where(anti, cur[rows, j], t)
        cur[rows, j] = np.where(anti, t, cur[rows, j])
    s1, acc, _ = sampler.mc_sweep(p, N, M, bl, s, 1, 9, 0)
    assert np.array_equal(acc, n_anti)
    assert np.array_equal(s1, cur)


def test_stationary_distribution_matches_enumeration():
    N, M = 8, 8
    p = rbm.init_params(np.random.default_rng(3), N, M, 0.2)
    basis = exact.sector_basis(N)
    w = np.abs(exact.rbm_vector(p, N, M, basis)) ** 2
    w /= w.sum()
    s, _, ctr = sampler.mc_sweep(p, N, M, lattice.bonds(8, 1), _sz0(4, 6000, N), 40, 21, 0)
    index = {b.tobytes(): k for k, b in enumerate(basis)}
    counts = np.bincount([index[r.tobytes()] for r in s], minlength=len(basis))
    # independent walkers -> multinomial; pool sparse bins for the chi-square test
    expected = w * len(s)
    order = np.argsort(expected)
    obs, exp_ = [], []
    acc_o = acc_e = 0.0
    for k in order:
        acc_o += counts[k]
        acc_e += expected[k]
        if acc_e >= 10:
            obs.append(acc_o)
            exp_.append(acc_e)
            acc_o = acc_e = 0.0
    obs[-1] += acc_o
    exp_[-1] += acc_e
    _, pval = scipy.stats.chisquare(obs, exp_)
    assert pval > 1e-4
