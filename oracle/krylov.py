"""Chebyshev moment correction and the Krylov projection (Secs. IV-V).

Sec. IV: with sigma_nm = <t_n|t_m> and H_nm = <t_n|H'|t_m> over the stored
Chebyshev states, the recomputed states |t'_n> = T_n(H_P)|t_0> =
sum_m c_mn |t_m> follow from
    sigma c_{.,1}   = H c_{.,0}
    sigma c_{.,n+1} = 2 H c_{.,n} - sigma c_{.,n-1}
with c_{.,0} = e_0 (|t'_0> = |t_0>), and mu_n = sum_ml c*_m0 sigma_ml c_ln.
Sec. V: the Krylov / continued-fraction route diagonalises the projected
Hamiltonian in the same non-orthogonal basis.

Readings: the recursion runs in the rescaled H' (the Chebyshev polynomials
are defined for H'); the paper indexes c_{0n} = delta_{0n}, which only makes
sense as c_{m0} = delta_{m0}; sigma^{-1} is a pseudo-inverse with a relative
eigenvalue cutoff (a sampled Gram matrix is near-singular); a sampled H is
Hermitised as (H + H^dag)/2.  Estimators on samples s of |psi|^2:
B_n(s) = t_n(s)/psi(s), sigma_nm = <B_n* B_m>, H_nm = <B_n* (H' t_m)(s)/psi(s)>.
"""

import numpy as np


def gram(B, HB, weights=None):
    """sigma and H' from the columns B_n(s), (H' t_n)(s)/psi(s) -> [Nm, Nm] each.

    weights None: plain sample means; else exact weights p_s (sum 1)."""
    Bm = np.array(B, dtype=np.complex128)        # [Nm, Ns]
    HBm = np.array(HB, dtype=np.complex128)
    w = np.full(Bm.shape[1], 1.0 / Bm.shape[1]) if weights is None else np.asarray(weights)
    G = (np.conj(Bm) * w) @ Bm.T
    H = (np.conj(Bm) * w) @ HBm.T
    return G, 0.5 * (H + H.conj().T)


def pinv_hermitian(G, cutoff):
    lam, U = np.linalg.eigh(G)
    keep = lam > cutoff * lam.max()
    return (U[:, keep] / lam[keep]) @ U[:, keep].conj().T


def corrected_moments(G, H, n_out, cutoff=1e-10):
    """mu'_n for n < n_out by the projected recursion of Sec. IV."""
    Nm = G.shape[0]
    Gp = pinv_hermitian(G, cutoff)
    c_prev = np.zeros(Nm, dtype=np.complex128)
    c_prev[0] = 1.0
    cs = [c_prev]
    if n_out > 1:
        cs.append(Gp @ (H @ c_prev))
    for _ in range(2, n_out):
        cs.append(Gp @ (2.0 * (H @ cs[-1]) - G @ cs[-2]))
    return np.array([(G @ c)[0] for c in cs[:n_out]])


def krylov_poles(G, H, cutoff=1e-10):
    """Generalised eigenproblem H c = lambda G c by canonical orthogonalisation.

    Returns (lambda_k in H' units, weights w_k = |<v_k| X^dag G e_0>|^2)."""
    lam, U = np.linalg.eigh(G)
    keep = lam > cutoff * lam.max()
    X = U[:, keep] / np.sqrt(lam[keep])
    Hx = X.conj().T @ H @ X
    e, V = np.linalg.eigh(0.5 * (Hx + Hx.conj().T))
    g0 = X.conj().T @ G[:, 0]
    w = np.abs(V.conj().T @ g0) ** 2
    return e, w
