"""Symmetry-projected Chebyshev states of the square lattice (Appendix A).

The sequence is computed once for the local probe S^z_00; every momentum
k = 2 pi (k1, k2) / L follows from translations T_m and quarter turns R:
    |t~_nk> = L P_k^(T) P^(R) |t_n00>,
    P_k^(T) = L^-2 sum_m e^{-i 2pi k.m / L} T_m,
    P^(R)   = (1 + T_(1,0) R + T_(1,1) R^2 + T_(0,1) R^3) / 4.
Operators act on basis states by moving spins: (T_m sigma)(x) = sigma(x - m),
(R sigma)(x) = sigma(R^-1 x), so T_m carries the operator S^z_x to S^z_{x+m}
and R carries it to S^z_{Rx}.

Reading of R: the paper states that P^(R) leaves the exact |t_n00> unchanged
and that each rotation is followed by the translation that brings the S^z
operator back to the origin.  Both hold when T_{d_r} R^r fixes the probe
site, d_r = (0,0), (1,0), (1,1), (0,1), i.e. when R^r takes site (0, 0) to
-d_r: R is the quarter turn about the plaquette centre (-1/2, -1/2),
    R (x, y) = (-y - 1, x) mod L,
and each term T_{d_r} R^r of P^(R) is the r-fold quarter turn about the
probe site.  Then
    B_{n,m,r}(s) = <s| T_m R^r |t_n00> / <s|psi> = t_n00(s') / psi(s),
    s'(x) = s(R^r x + m),
and, with the rotation terms of P^(R) folded into the translation sum,
    B~_nk(s) = L^-1 sum_m e^{-i 2pi k.m / L} (1/4) [B_{n,m,0} + B_{n,m+(1,0),1}
               + B_{n,m+(1,1),2} + B_{n,m+(0,1),3}].
The Gram matrix of each momentum is G^(k)_nn' = < conj(B~_nk) B~_n'k > over
samples of |psi|^2 (= <t~_nk|t~_n'k> / <psi|psi>).

The projected Hamiltonian H^(k) follows the same procedure.  H' = (H - E0)/a
- W' commutes with every translation and rotation of the periodic lattice, so
H' |t~_nk> = L P_k^(T) P^(R) H' |t_n00>, and
    HB~_nk(s) = <s|H'|t~_nk> / <s|psi>
is the projection above applied to (H' t_n00)(s') / psi(s) in place of
t_n00(s') / psi(s); then H^(k)_nn' = < conj(B~_nk) HB~_n'k >
(= <t~_nk|H'|t~_n'k> / <psi|psi>).

THIS MODULE IS TEST INFRASTRUCTURE (see the package docstring).
"""

import numpy as np

from . import rbm, target

SHIFTS = ((0, 0), (1, 0), (1, 1), (0, 1))  # translation paired with R^r in P^(R)


def rotate(x, y, r, L):
    """R^r (x, y) with R (x, y) = (-y - 1, x) mod L, the quarter turn about
    the plaquette centre (-1/2, -1/2)."""
    for _ in range(r % 4):
        x, y = (-y - 1) % L, x % L
    return x, y


def transform(spins, m, r, L):
    """Rows s'(x) = s(R^r x + m) of the configurations in spins [B, L*L]."""
    spins = np.asarray(spins)
    out = np.empty_like(spins)
    for y in range(L):
        for x in range(L):
            rx, ry = rotate(x, y, r, L)
            src = ((rx + m[0]) % L) + L * ((ry + m[1]) % L)
            out[:, x + L * y] = spins[:, src]
    return out


def _project(params_list, L, spins, value):
    """L^-1 sum_m e^{-i 2pi k.m / L} (1/4) sum_r value(t_n, s'_{m + d_r, r})
    for every state n and momentum k: complex [Nm, L*L, B]."""
    spins = np.asarray(spins, dtype=np.int8)
    Bn = spins.shape[0]
    out = np.zeros((len(params_list), L * L, Bn), dtype=np.complex128)
    ks = [(k1, k2) for k2 in range(L) for k1 in range(L)]
    for n, p in enumerate(params_list):
        for m1 in range(L):
            for m2 in range(L):
                acc = np.zeros(Bn, dtype=np.complex128)
                for r, (d1, d2) in enumerate(SHIFTS):
                    sp = transform(spins, ((m1 + d1) % L, (m2 + d2) % L), r, L)
                    acc = acc + 0.25 * value(p, sp)
                for ki, (k1, k2) in enumerate(ks):
                    ph = np.exp(-2j * np.pi * (k1 * m1 + k2 * m2) / L) / L
                    out[n, ki] += ph * acc
    return out


def b_tilde(params_list, N, M, L, spins, logpsi_ref):
    """B~_nk(s) for every stored state n and momentum k: complex [Nm, L*L, B]
    (momentum index k1 + L k2)."""
    return _project(params_list, L, spins,
                    lambda p, sp: np.exp(rbm.logpsi(p, N, M, sp) - logpsi_ref))


def hb_tilde(params_list, N, M, L, J, E0, a, Wp, spins, logpsi_ref):
    """HB~_nk(s) = <s|H'|t~_nk> / <s|psi> for every stored state n and
    momentum k: complex [Nm, L*L, B], from (H' t_n00)(s') / psi(s) at every
    transformed configuration (oracle.target.apply_hprime, no probe)."""
    return _project(params_list, L, spins,
                    lambda p, sp: target.apply_hprime(target.State(p), N, M, L, L, J, E0, a, Wp,
                                                      (0.0, 0.0), sp, logpsi_ref))


def gram_by_momentum(Bt, weights=None, HBt=None):
    """G^(k)_nn' = < conj(B~_nk) B~_n'k >, or with HBt the projected
    H^(k)_nn' = < conj(B~_nk) HB~_n'k >: complex [L*L, Nm, Nm]."""
    Nm, Nk, Bn = Bt.shape
    w = np.full(Bn, 1.0 / Bn) if weights is None else np.asarray(weights)
    return np.einsum("nks,mks,s->knm", np.conj(Bt), Bt if HBt is None else HBt, w)
