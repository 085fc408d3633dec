"""Extrapolation of Chebyshev moments by linear prediction (Sec. VI).

THIS MODULE IS TEST INFRASTRUCTURE (see the package docstring).

The paper remarks that higher moments can be approximated from the known
ones by extrapolation and cites the Chebyshev-MPS literature for it; it
gives no algorithm.  The method taken here is linear prediction as applied
to Chebyshev moments by Ganahl, Thunstroem, Verstraete, Held and Evertz,
Phys. Rev. B 90, 045144 (2014), with the treatment of growing modes of
Barthel, Schollwoeck and White, Phys. Rev. B 79, 245101 (2009):

1. Model: mu_n = -sum_{i=1}^{p} a_i mu_{n-i}.  The coefficients minimise the
   squared one-step prediction error over a training window of targets
   n = n0 .. N-1 (N known moments, n0 >= p):
       sum_n |mu_n + sum_i a_i mu_{n-i}|^2,
   whose normal equations are (R + delta I) a = -r with
       R_ij = sum_n conj(mu_{n-i}) mu_{n-j},  r_i = sum_n conj(mu_{n-i}) mu_n,
   i, j = 1 .. p, and a Tikhonov term delta = reg * max_i R_ii.
2. Any sequence obeying the recursion is mu_n = sum_k c_k z_k^n with z_k the
   roots of z^p + a_1 z^{p-1} + ... + a_p (the eigenvalues of the
   companion matrix).  The amplitudes c_k follow from the last p known
   moments, sum_k c_k z_k^m = mu_{N-p+m}, m = 0 .. p-1.
3. Roots outside the unit circle would make the prediction grow without
   bound; they are put on the unit circle, z_k -> z_k / |z_k|.
4. Prediction: mu_{N-p+m} = sum_k c_k w_k^m for m >= p, w_k the roots after
   step 3 (the known moments are returned unchanged).

Library primitives serve as single steps: a linear solve for the normal
equations and for the amplitudes, the eigenvalues of the companion matrix
for the roots.
"""

import numpy as np


def normal_equations(mu, p, n0, reg):
    """R + delta I and r of step 1 (float64 sums over n = n0 .. N-1)."""
    mu = np.asarray(mu, dtype=np.complex128)
    N = len(mu)
    R = np.zeros((p, p), dtype=np.complex128)
    r = np.zeros(p, dtype=np.complex128)
    for n in range(n0, N):
        past = mu[n - p:n][::-1]  # mu_{n-1} .. mu_{n-p}
        R += np.outer(np.conj(past), past)
        r += np.conj(past) * mu[n]
    R += reg * np.max(np.real(np.diag(R))) * np.eye(p)
    return R, r


def lp_coefficients(mu, p, n0, reg):
    R, r = normal_equations(mu, p, n0, reg)
    return np.linalg.solve(R, -r)


def lp_roots(a):
    """Roots of z^p + a_1 z^{p-1} + ... + a_p: eigenvalues of the companion
    matrix (first row -a, ones on the subdiagonal)."""
    p = len(a)
    C = np.zeros((p, p), dtype=np.complex128)
    C[0, :] = -np.asarray(a)
    C[np.arange(1, p), np.arange(p - 1)] = 1.0
    return np.linalg.eigvals(C)


def stabilise(z):
    """Step 3: roots outside the unit circle are moved onto it."""
    return np.where(np.abs(z) > 1.0, z / np.abs(z), z)


def extrapolate(mu, p, n0, n_out, reg=1e-12):
    """The first n_out moments: the known ones, then the prediction.

    returns (moments [n_out], fitted roots z_k [p], stabilised roots w_k [p])"""
    mu = np.asarray(mu, dtype=np.complex128)
    N = len(mu)
    if not (1 <= p <= n0 < N and n_out >= N):
        raise ValueError("need 1 <= p <= n0 < len(mu) <= n_out")
    a = lp_coefficients(mu, p, n0, reg)
    z = lp_roots(a)
    V = np.power.outer(z, np.arange(p)).T          # V[m, k] = z_k^m
    c = np.linalg.solve(V, mu[N - p:])
    w = stabilise(z)
    out = np.empty(n_out, dtype=np.complex128)
    out[:N] = mu
    m = np.arange(p, n_out - N + p)                 # mu_{N-p+m}, m >= p
    out[N:] = np.power.outer(w, m).T @ c
    return out, z, w
