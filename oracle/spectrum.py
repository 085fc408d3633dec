"""Spectral function on a frequency grid from the Chebyshev moments (Sec. II)
and from the Krylov projection by a continued fraction (Sec. IV).

Frequencies: omega' = omega / a - W' maps the excitation energy omega =
E - E0 into [-1, 1] (Sec. II), so H' = (H - E0) / a - W'.

  chebyshev_spectrum : Eq. (Aw) of Sec. II,
      A(omega) = [g_0 mu_0 + 2 sum_{n=1}^{N-1} g_n mu_n T_n(omega')]
                 / (a pi sqrt(1 - omega'^2)),
    the prefactor 2 W' / W_* of the paper being 1 / a; zero outside
    |omega'| < 1, where the expansion is not defined.
  jackson            : the damping factors g_n of Sec. V.
  continued_fraction : Lanczos tridiagonalisation of the projected H' in
    the basis of Chebyshev states (Sec. IV: start vector t_0), then the
    continued fraction of the resolvent at z' = omega' + i eta / a,
      G'(z') = mu_0 / (z' - alpha_0 - beta_1^2 / (z' - alpha_1 - ...)),
    and A(omega) = -Im G'(z') / (pi a) (dz = a dz').

THIS MODULE IS TEST INFRASTRUCTURE (see the package docstring).
"""

import numpy as np


def jackson(N):
    """g_n, n = 0 .. N - 1, for an expansion of N moments (Sec. V)."""
    n = np.arange(N, dtype=np.float64)
    q = np.pi / (N + 1)
    return ((N - n + 1) * np.cos(q * n) + np.sin(q * n) / np.tan(q)) / (N + 1)


def chebyshev_spectrum(mu, a, Wp, omega, damping="jackson"):
    """Eq. (Aw) on the frequencies omega (complex: mu may be complex)."""
    mu = np.asarray(mu, dtype=np.complex128)
    N = len(mu)
    g = jackson(N) if damping == "jackson" else np.ones(N)
    x = np.asarray(omega, dtype=np.float64) / a - Wp
    out = np.zeros(len(x), dtype=np.complex128)
    inside = np.abs(x) < 1.0
    xi = x[inside]
    theta = np.arccos(xi)
    series = g[0] * mu[0] * np.ones(len(xi), dtype=np.complex128)
    for n in range(1, N):
        series = series + 2.0 * g[n] * mu[n] * np.cos(n * theta)  # T_n(cos t) = cos(n t)
    out[inside] = series / (a * np.pi * np.sqrt(1.0 - xi * xi))
    return out


def lanczos(Hx, v0, steps):
    """Hermitian Lanczos from v0 (full reorthogonalisation): alpha, beta."""
    D = Hx.shape[0]
    steps = min(steps, D)
    V = np.zeros((D, steps), dtype=np.complex128)
    alpha = np.zeros(steps)
    beta = np.zeros(steps)
    v = v0 / np.linalg.norm(v0)
    for j in range(steps):
        V[:, j] = v
        w = Hx @ v
        alpha[j] = np.vdot(v, w).real
        w = w - V[:, :j + 1] @ (V[:, :j + 1].conj().T @ w)
        if j + 1 < steps:
            b = np.linalg.norm(w)
            if b < 1e-14:
                return alpha[:j + 1], beta[:j + 1]
            beta[j + 1] = b
            v = w / b
    return alpha, beta


def cf_resolvent(alpha, beta, norm2, z):
    """norm2 / (z - alpha_0 - beta_1^2 / (z - alpha_1 - ...)), evaluated
    from the innermost level outwards."""
    g = np.zeros_like(z, dtype=np.complex128)
    for j in range(len(alpha) - 1, -1, -1):
        tail = beta[j + 1] ** 2 * g if j + 1 < len(alpha) else 0.0
        g = 1.0 / (z - alpha[j] - tail)
    return norm2 * g


def continued_fraction(G, H, a, Wp, omega, eta, cutoff=1e-10):
    """A(omega) from the Gram matrix G_nm = <t_n|t_m> and H_nm = <t_n|H'|t_m>
    of the Chebyshev states (Sec. IV), by canonical orthogonalisation, Lanczos
    from t_0 and the continued fraction at omega' + i eta / a."""
    G = np.asarray(G, dtype=np.complex128)
    H = np.asarray(H, dtype=np.complex128)
    lam, U = np.linalg.eigh(G)
    keep = lam > cutoff * lam.max()
    X = U[:, keep] / np.sqrt(lam[keep])
    Hx = X.conj().T @ (0.5 * (H + H.conj().T)) @ X
    v0 = X.conj().T @ G[:, 0]          # t_0 in the orthonormal basis
    mu0 = np.vdot(v0, v0).real         # = G_00
    alpha, beta = lanczos(Hx, v0, Hx.shape[0])
    z = np.asarray(omega, dtype=np.float64) / a - Wp + 1j * eta / a
    return -cf_resolvent(alpha, beta, mu0, z).imag / (np.pi * a)
