"""Metropolis sampling of P(s) = |psi_s|^2 / <psi|psi> (Sec. III).

The paper fixes the target distribution only.  The move set read here: pick
one nearest-neighbour bond uniformly; if its two spins are antiparallel,
propose exchanging them (total S^z is conserved), otherwise the proposal is
a no-op that counts as rejected.  The proposal is symmetric, so the
Metropolis acceptance is min(1, |psi(s') / psi(s)|^2).

The amplitude ratio is taken by evaluating log psi from scratch at the
proposed configuration, with no incremental update of any kind.

Random stream: see oracle.philox.  Proposal p (0-based within one call)
uses call index counter + p // 2 and word pair p % 2; one sweep is N
proposals; the call returns the advanced counter.
"""

import numpy as np

from . import philox
from .rbm import logpsi


def n_calls(n_sweeps, N):
    return (n_sweeps * N + 1) // 2


def mc_sweep(params, N, M, bonds, spins, n_sweeps, seed, counter, walker_ids=None):
    """Run n_sweeps * N exchange proposals on every walker.

    spins       int8 [B, N], +-1 (not modified; a new array is returned)
    walker_ids  the walker index of each row in the random stream (default
                0..B-1), so that a subset of a large batch can be replayed
    returns (new spins, accepted-move count per walker, advanced counter)
    """
    spins = np.array(spins, dtype=np.int8, copy=True)
    B = spins.shape[0]
    walkers = (np.arange(B) if walker_ids is None else np.asarray(walker_ids)).astype(np.uint64)
    rows = np.arange(B)
    lp = logpsi(params, N, M, spins)
    accepted = np.zeros(B, dtype=np.int64)
    n_prop = n_sweeps * N
    for p in range(n_prop):
        words = philox.proposal_words(seed, counter + p // 2, walkers)
        w_bond, w_acc = words[2 * (p % 2)], words[2 * (p % 2) + 1]
        b = philox.bond_index(w_bond, len(bonds))
        i, j = bonds[b, 0], bonds[b, 1]
        anti = spins[rows, i] != spins[rows, j]
        prop = spins.copy()
        prop[rows, i] = spins[rows, j]
        prop[rows, j] = spins[rows, i]
        lp_new = logpsi(params, N, M, prop)
        with np.errstate(over="ignore"):
            ratio2 = np.exp(2.0 * (lp_new - lp).real)
        acc = anti & (philox.uniform(w_acc) < ratio2)
        spins[acc] = prop[acc]
        lp[acc] = lp_new[acc]
        accepted += acc
    return spins, accepted, counter + n_calls(n_sweeps, N)
