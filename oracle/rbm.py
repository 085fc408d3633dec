"""The complex RBM amplitude and its log-derivatives.

Sec. I: psi(sigma) = exp(sum_i a_i sigma_i) prod_j 2 cosh(theta_j),
theta_j = b_j + sum_i W_ij sigma_i, with complex a (N), b (M), W (N x M).

Parameter vector layout (the index k of O_k, S_kk' and F_k):
    alpha = [a_0 .. a_{N-1} | b_0 .. b_{M-1} | W_00, W_01, .., W_0,M-1, W_10, ..]
i.e. W row-major with the visible index i outer.

Sec. III: O_k(s) = (d psi_s / d alpha_k) / psi_s, which for this ansatz is
O_{a_i} = sigma_i, O_{b_j} = tanh(theta_j), O_{W_ij} = sigma_i tanh(theta_j).
"""

import numpy as np


def n_params(N, M):
    return N + M + N * M


def unpack(params, N, M):
    params = np.asarray(params, dtype=np.complex128)
    if params.shape[-1] != n_params(N, M):
        raise ValueError("parameter vector has the wrong length")
    return params[:N], params[N:N + M], params[N + M:].reshape(N, M)


def theta(params, N, M, spins):
    """theta_j = b_j + sum_i W_ij sigma_i, for each row of spins -> [B, M]."""
    _, b, W = unpack(params, N, M)
    return b + np.asarray(spins, dtype=np.float64) @ W


def lncosh2(z):
    """log(2 cosh z) with the principal complex logarithm (plain definition)."""
    return np.log(2.0 * np.cosh(z))


def logpsi(params, N, M, spins):
    """log psi(sigma) for each row of spins -> complex [B] (defined mod 2 pi i)."""
    a, _, _ = unpack(params, N, M)
    th = theta(params, N, M, spins)
    return np.asarray(spins, dtype=np.float64) @ a + np.sum(lncosh2(th), axis=-1)


def logderiv_from_tanh(spins, T):
    """Explicit O_k(s) from the spins and T_j(s) = tanh(theta_j(s)):
    O_a = sigma, O_b = T, O_W = sigma_i T_j -> complex [B, P]."""
    s = np.asarray(spins, dtype=np.float64)
    T = np.asarray(T, dtype=np.complex128)
    N, M = s.shape[1], T.shape[1]
    OW = (s[:, :, None] * T[:, None, :]).reshape(s.shape[0], N * M)
    return np.concatenate([s.astype(np.complex128), T, OW], axis=1)


def logderiv(params, N, M, spins):
    """Explicit O_k(s) for each row of spins -> complex [B, P]."""
    return logderiv_from_tanh(spins, np.tanh(theta(params, N, M, spins)))


def init_params(rng, N, M, sigma):
    """Reference helper for tests: Re and Im of every parameter i.i.d. N(0, sigma^2)."""
    P = n_params(N, M)
    return sigma * rng.standard_normal(P) + 1j * sigma * rng.standard_normal(P)
