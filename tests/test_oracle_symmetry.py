"""Pins for the symmetry projection (Appendix A): the estimators of the
projected Gram and Hamiltonian matrices against the projected dense vectors
built from the operator definitions (and the dense H' of exact
diagonalisation), projector identities, and a state that is already
symmetric."""

import numpy as np
import pytest

from oracle import exact, lattice, rbm, symmetry


def _perm_op(basis, L, f):
    """Permutation matrix of the operator that maps configuration sigma to
    sigma' with sigma'(x) = sigma(f(x)) (as a basis-index map)."""
    index = {b.tobytes(): k for k, b in enumerate(basis)}
    src = [f(x, y) for y in range(L) for x in range(L)]
    dst = np.array([index[b[[sx + L * sy for sx, sy in src]].tobytes()] for b in basis])
    return dst


def _apply(dst, v):
    # (A v)[dst[k]] = v[k]: A moves the amplitude of basis state k to dst[k]
    out = np.zeros_like(v)
    out[dst] = v
    return out


def _dense_projector(basis, L):
    """v -> L P_k^(T) P^(R) v on dense vectors over `basis`, from the
    permutation operators themselves."""
    # operators on states: (T_m v)(sigma) = v(T_m^-1 sigma): T_m moves the spin at
    # x - m to x, i.e. maps sigma to sigma'(x) = sigma(x - m)
    def T(m):
        return _perm_op(basis, L, lambda x, y: ((x - m[0]) % L, (y - m[1]) % L))
    Rop = _perm_op(basis, L, lambda x, y: symmetry.rotate(x, y, -1, L))  # sigma'(x) = sigma(R^-1 x)
    Ts = {(m1, m2): T((m1, m2)) for m1 in range(L) for m2 in range(L)}

    def proj(v, k):
        vr = v.copy()
        acc = 0.25 * v
        for r, sh in enumerate(symmetry.SHIFTS[1:], start=1):
            vr = _apply(Rop, vr)                 # R^r v
            acc = acc + 0.25 * _apply(Ts[sh], vr)
        out = np.zeros_like(v)
        for (m1, m2), Tm in Ts.items():
            ph = np.exp(-2j * np.pi * (k[0] * m1 + k[1] * m2) / L)
            out = out + ph * _apply(Tm, acc)
        return out / L
    return proj


def test_projected_gram_equals_dense_projection():
    L, M = 4, 6
    N = L * L
    basis = exact.sector_basis(N)
    rng = np.random.default_rng(3)
    psi_p = rbm.init_params(rng, N, M, 0.2)
    states = [rbm.init_params(rng, N, M, 0.2) for _ in range(3)]
    psi = exact.rbm_vector(psi_p, N, M, basis)
    Z = np.vdot(psi, psi).real
    proj = _dense_projector(basis, L)
    dense = [exact.rbm_vector(p, N, M, basis) for p in states]
    Bt = symmetry.b_tilde(states, N, M, L, basis, rbm.logpsi(psi_p, N, M, basis))
    G = symmetry.gram_by_momentum(Bt, weights=np.abs(psi) ** 2 / Z)
    for k in ((0, 0), (1, 0), (2, 1), (2, 2), (3, 1)):
        ki = k[0] + L * k[1]
        tk = [proj(v, k) for v in dense]
        Gd = np.array([[np.vdot(a, b) for b in tk] for a in tk]) / Z
        assert np.allclose(G[ki], Gd, atol=1e-12 * np.abs(Gd).max()), k
        # B~ is the amplitude ratio of the projected state: <s|t~_nk> / <s|psi>
        assert np.allclose(Bt[0, ki] * psi, tk[0], atol=1e-12 * np.abs(tk[0]).max())


def test_projected_hamiltonian_equals_dense_projection():
    # 3 x 3 lattice, sector of 4 up-spins (126 states): the dense H' of exact
    # diagonalisation applied to the projected dense vectors
    L, M, J, E0, a, Wp = 3, 5, 1.0, -4.1, 3.7, 0.3
    N = L * L
    basis = exact.sector_basis(N, n_up=4)
    rng = np.random.default_rng(11)
    psi_p = rbm.init_params(rng, N, M, 0.3)
    states = [rbm.init_params(rng, N, M, 0.3) for _ in range(3)]
    psi = exact.rbm_vector(psi_p, N, M, basis)
    Z = np.vdot(psi, psi).real
    Hp = exact.rescaled(exact.hamiltonian(L, L, J, basis), E0, a, Wp)
    proj = _dense_projector(basis, L)
    lref = rbm.logpsi(psi_p, N, M, basis)
    Bt = symmetry.b_tilde(states, N, M, L, basis, lref)
    HBt = symmetry.hb_tilde(states, N, M, L, J, E0, a, Wp, basis, lref)
    w = np.abs(psi) ** 2 / Z
    H = symmetry.gram_by_momentum(Bt, weights=w, HBt=HBt)
    dense = [exact.rbm_vector(p, N, M, basis) for p in states]
    for k1 in range(L):
        for k2 in range(L):
            ki = k1 + L * k2
            tk = [proj(v, (k1, k2)) for v in dense]
            Hd = np.array([[np.vdot(u, Hp @ v) for v in tk] for u in tk]) / Z
            assert np.allclose(H[ki], Hd, atol=1e-12 * np.abs(Hd).max()), (k1, k2)
            assert np.allclose(H[ki], H[ki].conj().T, atol=1e-12 * np.abs(Hd).max())
            # HB~ is the amplitude ratio of H' applied to the projected state
            for n in range(len(states)):
                assert np.allclose(HBt[n, ki] * psi, Hp @ tk[n],
                                   atol=1e-12 * np.abs(Hp @ tk[n]).max()), (k1, k2, n)


def test_momentum_sum_and_symmetric_state():
    L, M = 4, 4
    N = L * L
    basis = exact.sector_basis(N)[:300]
    rng = np.random.default_rng(5)
    p = rbm.init_params(rng, N, M, 0.3)
    lref = rbm.logpsi(p, N, M, basis)
    Bt = symmetry.b_tilde([p], N, M, L, basis, lref)
    # sum_k L P_k = L: the momenta add up to L times the rotation average at m = 0
    rot = sum(0.25 * np.exp(rbm.logpsi(p, N, M, symmetry.transform(basis, sh, r, L)) - lref)
              for r, sh in enumerate(symmetry.SHIFTS))
    assert np.allclose(Bt[0].sum(axis=0), L * rot, atol=1e-12)
    # an RBM with W = 0 and uniform a, b is invariant under every lattice map:
    # only k = 0 survives, with B~ = L
    q = np.zeros(rbm.n_params(N, M), dtype=np.complex128)
    q[:N] = 0.1 + 0.2j
    q[N:N + M] = -0.3 + 0.1j
    Bq = symmetry.b_tilde([q], N, M, L, basis, rbm.logpsi(q, N, M, basis))
    assert np.allclose(Bq[0, 0], L)
    assert np.allclose(Bq[0, 1:], 0, atol=1e-12)


def _turn_about_origin(x, y, L):
    # quarter turn about site (0, 0), written out independently of the oracle
    return (L - y) % L, x % L


def test_rotation_is_a_quarter_turn_paired_to_fix_the_probe_site():
    L = 5
    for x in range(L):
        for y in range(L):
            assert symmetry.rotate(x, y, 4, L) == (x, y)
    # R^r takes the probe site to -d_r, so T_{d_r} R^r fixes it (Appendix A)
    for r, (d1, d2) in enumerate(symmetry.SHIFTS):
        assert symmetry.rotate(0, 0, r, L) == ((-d1) % L, (-d2) % L)
    # and T_{d_r} R^r is the r-fold quarter turn about the probe site
    for r, (d1, d2) in enumerate(symmetry.SHIFTS):
        for x in range(L):
            for y in range(L):
                rx, ry = symmetry.rotate(x, y, r, L)
                qx, qy = x, y
                for _ in range(r):
                    qx, qy = _turn_about_origin(qx, qy, L)
                assert ((rx + d1) % L, (ry + d2) % L) == (qx, qy)
    # R maps the nearest-neighbour bonds of the periodic lattice onto themselves
    bonds = {frozenset(b) for b in lattice.bonds(L, L)}
    site = lambda x, y: x + L * y
    for i, j in lattice.bonds(L, L):
        a = symmetry.rotate(i % L, i // L, 1, L)
        b = symmetry.rotate(j % L, j // L, 1, L)
        assert frozenset((site(*a), site(*b))) in bonds
    s = np.arange(L * L)[None, :]
    assert np.array_equal(symmetry.transform(symmetry.transform(s, (0, 0), 1, L), (0, 0), 3, L), s)


def test_rotation_projector_leaves_a_probe_site_symmetric_state_unchanged():
    # Appendix A: in the exact calculation P^(R) leaves |t_n00> unchanged.  An
    # RBM invariant under quarter turns about the probe site (visible biases
    # symmetric about it, hidden units in orbits of four with the weight
    # columns turned) must give B~ = the translation projection alone.
    L, N = 4, 16
    rng = np.random.default_rng(9)
    turn = np.array([(lambda q: q[0] + L * q[1])(_turn_about_origin(i % L, i // L, L))
                     for i in range(N)])                 # site i -> its quarter turn
    dist = np.array([min(i % L, L - i % L) ** 2 + min(i // L, L - i // L) ** 2
                     for i in range(N)], dtype=float)
    a = (0.05 + 0.03j) * dist
    w = 0.2 * (rng.standard_normal(N) + 1j * rng.standard_normal(N))
    cols = [w]
    for _ in range(3):
        nxt = np.empty(N, dtype=complex)
        nxt[turn] = cols[-1]                               # weight carried to the turned site
        cols.append(nxt)
    M = 4
    W = np.stack(cols, axis=1)                             # [N, M]
    b = np.full(M, 0.1 - 0.2j)
    p = np.concatenate([a, b, W.reshape(-1)])
    basis = exact.sector_basis(N)[:400]
    turned = basis[:, np.argsort(turn)]                    # s(turn^-1 x): the turned configuration
    assert np.allclose(rbm.logpsi(p, N, M, turned), rbm.logpsi(p, N, M, basis))
    q = rbm.init_params(rng, N, M, 0.2)                    # reference psi, no symmetry needed
    lref = rbm.logpsi(q, N, M, basis)
    Bt = symmetry.b_tilde([p], N, M, L, basis, lref)
    for k1 in range(L):
        for k2 in range(L):
            bt = sum(np.exp(-2j * np.pi * (k1 * m1 + k2 * m2) / L)
                     * np.exp(rbm.logpsi(p, N, M, symmetry.transform(basis, (m1, m2), 0, L)) - lref)
                     for m1 in range(L) for m2 in range(L)) / L
            assert np.allclose(Bt[0, k1 + L * k2], bt, atol=1e-12 * np.abs(bt).max() + 1e-14)


def test_projected_local_probe_is_the_momentum_probe():
    # For a psi invariant under every lattice map, t_0 = psi with a_0 += i pi/2
    # is exactly 2i S^z_00 psi, and L P_k^(T) P^(R) S^z_00 psi = S^z_k psi, the
    # momentum probe of Sec. II, f_k(s) = N^-1/2 sum_r e^{-i k.r} s_r / 2: so
    # B~_0k(s) = 2i f_k(s) at every momentum (phase convention included).
    L, M = 4, 3
    N = L * L
    psi = np.zeros(rbm.n_params(N, M), dtype=np.complex128)
    psi[:N] = 0.07 - 0.02j
    psi[N:N + M] = 0.3 + 0.1j
    t0 = psi.copy()
    t0[0] += 0.5j * np.pi
    spins = exact.sector_basis(N)[::37]
    lref = rbm.logpsi(psi, N, M, spins)
    Bt = symmetry.b_tilde([t0], N, M, L, spins, lref)
    for k1 in range(L):
        for k2 in range(L):
            f = lattice.probe(L, L, 2 * np.pi * k1 / L, 2 * np.pi * k2 / L, spins)
            assert np.allclose(Bt[0, k1 + L * k2], 2j * f, atol=1e-12), (k1, k2)
