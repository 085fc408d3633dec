"""Pins for the oracle's natural-gradient estimators and its Chebyshev driver.

The VMC forms (sample averages of O_k and R) are checked against the
bra-ket forms of the same quantities, built from dense vectors and
finite-difference parameter derivatives; the driver's beta_n and mu_n are
checked against dense inner products."""

import numpy as np
import pytest

from oracle import chebyshev, exact, rbm, sr


def _dense_psi(p, N, M, basis):
    return exact.rbm_vector(p, N, M, basis)


def test_vmc_estimators_equal_braket_forms():
    N, M = 6, 4
    basis = exact.sector_basis(N)
    rng = np.random.default_rng(10)
    p = rbm.init_params(rng, N, M, 0.4)
    psi = _dense_psi(p, N, M, basis)
    phi = psi * (1 + 0.3 * rng.standard_normal(len(basis))) + 0.2 * rng.standard_normal(len(basis))
    Z = np.vdot(psi, psi).real
    # finite-difference derivative vectors d psi / d alpha_k (holomorphic, real step)
    P = rbm.n_params(N, M)
    h = 1e-6
    dpsi = np.empty((P, len(basis)), dtype=np.complex128)
    for k in range(P):
        e = np.zeros(P, dtype=np.complex128)
        e[k] = h
        dpsi[k] = (_dense_psi(p + e, N, M, basis) - _dense_psi(p - e, N, M, basis)) / (2 * h)
    dgamma = 0.37
    gamma_d = np.arccos(abs(np.vdot(psi, phi)) / np.sqrt(Z * np.vdot(phi, phi).real))
    c = dgamma * gamma_d / np.tan(gamma_d)
    dpsi_vec = c * ((Z / np.vdot(psi, phi)) * phi - psi)
    # rotation properties of the update direction
    assert abs(np.vdot(psi, dpsi_vec)) < 1e-12 * Z
    assert np.vdot(dpsi_vec, dpsi_vec).real == pytest.approx((dgamma * gamma_d) ** 2 * Z, rel=1e-10)
    S_bk = (np.conj(dpsi) @ dpsi.T) / Z - np.outer(np.conj(dpsi) @ psi, np.conj(psi) @ dpsi.T) / Z ** 2
    F_bk = (np.conj(dpsi) @ dpsi_vec) / Z - (np.conj(dpsi) @ psi) / Z * np.vdot(psi, dpsi_vec) / Z
    # VMC forms in enumeration mode
    w = np.abs(psi) ** 2 / Z
    O = rbm.logderiv(p, N, M, basis)
    est = sr.estimators(O, phi / psi, weights=w)
    F, gamma = sr.force(est, dgamma)
    S = sr.qgt(est)
    assert gamma == pytest.approx(gamma_d, rel=1e-12)
    assert np.allclose(S, S_bk, atol=1e-7)
    assert np.allclose(F, F_bk, atol=1e-7)
    assert np.allclose(S, S.conj().T, atol=1e-14)
    assert np.linalg.eigvalsh(S).min() > -1e-12


def test_exact_representability_gives_zero_angle_and_force():
    N, M = 6, 4
    basis = exact.sector_basis(N)
    p = rbm.init_params(np.random.default_rng(11), N, M, 0.4)
    c = 0.3 - 1.7j
    O = rbm.logderiv(p, N, M, basis)
    w = np.abs(_dense_psi(p, N, M, basis)) ** 2
    est = sr.estimators(O, np.full(len(basis), c), weights=w / w.sum())
    F, gamma = sr.force(est, 0.5)
    assert gamma < 1e-7 and np.allclose(F, 0, atol=1e-12)
    assert est["mR"] == pytest.approx(c)


def test_shifted_solve_residual():
    rng = np.random.default_rng(12)
    O = rng.standard_normal((50, 20)) + 1j * rng.standard_normal((50, 20))
    est = sr.estimators(O, rng.standard_normal(50) + 0j)
    S = sr.qgt(est)
    F = rng.standard_normal(20) + 1j * rng.standard_normal(20)
    x = sr.shifted_solve(S, F, 1e-3)
    assert np.linalg.norm((S + 1e-3 * np.eye(20)) @ x - F) < 1e-10 * np.linalg.norm(F)


@pytest.mark.parametrize("jacobi", [False, True])
def test_cg_reaches_the_direct_solution(jacobi):
    # conjugate gradients on an n x n SPD system terminate in at most n steps in
    # exact arithmetic; with a badly scaled diagonal the Jacobi variant needs fewer
    rng = np.random.default_rng(40)
    O = rng.standard_normal((400, 30)) + 1j * rng.standard_normal((400, 30))
    O[:, :10] *= 30.0
    est = sr.estimators(O, rng.standard_normal(400) + 0j)
    S = sr.qgt(est)
    F = rng.standard_normal(30) + 1j * rng.standard_normal(30)
    x_direct = sr.shifted_solve(S, F, 1e-2)
    x, it = sr.cg_solve(S, F, 1e-2, 200, 1e-12, jacobi)
    assert np.linalg.norm(x - x_direct) < 1e-9 * np.linalg.norm(x_direct)
    assert it <= 120
    _, it1 = sr.cg_solve(S, F, 1e-2, 1, 0.0, jacobi)
    assert it1 == 1
    if jacobi:
        _, it_plain = sr.cg_solve(S, F, 1e-2, 200, 1e-12, False)
        assert it < it_plain


def test_natural_gradient_fit_converges_on_representable_target():
    # phi = i sigma_0 psi0 is exactly the RBM psi0 with a_0 += i pi / 2.
    N, M = 8, 8
    basis = exact.sector_basis(N)
    rng = np.random.default_rng(13)
    p0 = rbm.init_params(rng, N, M, 0.3)
    phi = 1j * basis[:, 0] * _dense_psi(p0, N, M, basis)
    p = chebyshev.initial_params(p0, None, 1)
    p = p + 0.02 * (rng.standard_normal(len(p)) + 1j * rng.standard_normal(len(p)))
    gammas = []
    for _ in range(40):
        psi = _dense_psi(p, N, M, basis)
        w = np.abs(psi) ** 2
        p, info = sr.sr_step(p, rbm.logderiv(p, N, M, basis), phi / psi, 1e-6, 0.5, weights=w / w.sum())
        gammas.append(info["gamma"])
    assert gammas[-1] < 1e-3 * gammas[0]


def test_matrix_free_product_and_cg_equal_the_explicit_forms():
    """The matrix-free (S + shift) v from blocks of O equals the explicit
    qgt product, and CG through it takes the explicit CG's steps."""
    N, M, B = 6, 5, 300
    rng = np.random.default_rng(15)
    p = rbm.init_params(rng, N, M, 0.3)
    spins = np.where(rng.random((B, N)) < 0.5, 1, -1).astype(np.int8)
    O = rbm.logderiv(p, N, M, spins)
    R = 1.0 + 0.3 * (rng.standard_normal(B) + 1j * rng.standard_normal(B))
    est = sr.estimators(O, R)
    S = sr.qgt(est)
    v = rng.standard_normal(O.shape[1]) + 1j * rng.standard_normal(O.shape[1])
    blocks = [O[:100], O[100:170], O[170:]]
    assert np.allclose(sr.sv_matrix_free(blocks, v, 0.01), (S + 0.01 * np.eye(len(v))) @ v,
                       atol=1e-12)
    F, _ = sr.force(est, 0.5)
    x1, it1 = sr.cg_solve(S, F, 0.1, 300, 1e-11)
    x2, it2 = sr.cg_solve_op(lambda u: sr.sv_matrix_free(blocks, u, 0.1), F,
                             np.ones(len(F)), 300, 1e-11)
    assert it1 < 300 and abs(it1 - it2) <= 1
    assert np.max(np.abs(x1 - x2)) <= 1e-9 * np.max(np.abs(x1))
    assert np.allclose(x1, sr.shifted_solve(S, F, 0.1), rtol=0, atol=1e-9 * np.max(np.abs(x1)))


def test_initial_params_start_from_the_probe_site_operator():
    """The start of projection step 1 (Sec. III leaves it open): the RBM with
    a_0 += i pi/2 is exactly i sigma_0 psi = 2i S^z_0 psi on every
    configuration (e^{i pi sigma/2} = i sigma); step n >= 2 starts from a copy
    of RBM_{n-1}."""
    N, M = 8, 6
    basis = exact.sector_basis(N)
    rng = np.random.default_rng(14)
    psi = rbm.init_params(rng, N, M, 0.3)
    prev = rbm.init_params(rng, N, M, 0.3)
    p1 = chebyshev.initial_params(psi, prev, 1)
    ratio = _dense_psi(p1, N, M, basis) / _dense_psi(psi, N, M, basis)
    assert np.allclose(ratio, 1j * basis[:, 0], atol=1e-13)
    p3 = chebyshev.initial_params(psi, prev, 3)
    assert np.array_equal(p3, prev) and p3 is not prev
    assert np.array_equal(chebyshev.initial_params(psi, prev, 2), prev)


def _cfg(**kw):
    # E0 and a from the exact spectrum, so that H' maps it onto [-W', W']
    e = np.linalg.eigvalsh(exact.hamiltonian(8, 1, 1.0, exact.sector_basis(8)))
    base = dict(Lx=8, Ly=1, M=8, q=(np.pi / 2, 0.0), n_moments=4, n_iter=12, shift=1e-3,
                dgamma=0.5, E0=e[0], a=(e[-1] - e[0]) / (2 * 0.9875), Wp=0.9875, n_therm=5,
                sweeps_per_iter=1)
    base.update(kw)
    return chebyshev.Config(**base)


def test_enumerated_driver_betas_and_moments_against_dense_vectors():
    cfg = _cfg(M=16, n_iter=40)
    N, M = cfg.N, cfg.M
    basis = exact.sector_basis(N)
    psi_p = rbm.init_params(np.random.default_rng(14), N, M, 0.2)
    res = chebyshev.run_enumerated(cfg, psi_p)
    H = exact.hamiltonian(cfg.Lx, cfg.Ly, cfg.J, basis)
    Hp = exact.rescaled(H, cfg.E0, cfg.a, cfg.Wp)
    psi = _dense_psi(psi_p, N, M, basis)
    Z = np.vdot(psi, psi).real
    t0 = exact.probe_vector(cfg.Lx, cfg.Ly, cfg.q[0], cfg.q[1], basis, psi)
    assert res.mu[0] == pytest.approx(np.vdot(t0, t0).real / Z, rel=1e-12)
    dense = [t0] + [_dense_psi(s.params, N, M, basis) for s in res.states[1:]]
    for n in range(1, cfg.n_moments):
        phi = res.betas[n - 1] * (Hp @ dense[n - 1]) if n == 1 else \
            2 * res.betas[n - 1] * (Hp @ dense[n - 1]) - res.betas[n - 2] * dense[n - 2]
        beta = np.vdot(dense[n], phi) / np.vdot(dense[n], dense[n])
        assert res.betas[n] == pytest.approx(beta, rel=1e-10)
        assert res.mu[n] == pytest.approx(res.betas[n] * np.vdot(t0, dense[n]) / Z, rel=1e-10)
    # accuracy report, not a parity gate: with alpha = 2 the fits of t_1 and
    # t_2 converge (gamma -> 1e-4) and their moments match the exact ones;
    # t_3 stalls at a large angle from its warm start (force ~ cot gamma -> 0).
    mu_ex = exact.chebyshev_moments(Hp, t0, psi, cfg.n_moments)
    assert res.gammas[0][-1] < 1e-3 and res.gammas[1][-1] < 1e-2
    for n in (1, 2):
        assert abs(res.mu[n] - mu_ex[n]) < 0.01 * abs(mu_ex[0])


def test_sampled_driver_tracks_enumeration_within_mc_error():
    # 12-site chain, q = pi, alpha = 1, weights sigma = 0.05, paper rescaling
    # (a = 5, E0 = exact ground energy): the shape of the FP64 chain workload.
    basis = exact.sector_basis(12)
    e0 = np.linalg.eigvalsh(exact.hamiltonian(12, 1, 1.0, basis))[0]
    cfg = chebyshev.Config(Lx=12, Ly=1, M=12, q=(np.pi, 0.0), n_moments=3, n_iter=20,
                           E0=e0, a=5.0, Wp=0.9875, n_therm=10, n_therm_ref=40)
    N, M = cfg.N, cfg.M
    psi_p = rbm.init_params(np.random.default_rng(0), N, M, 0.05)
    rng = np.random.default_rng(1)
    base = np.array([1] * (N // 2) + [-1] * (N // 2), dtype=np.int8)
    s_fit = rng.permuted(np.tile(base, (1024, 1)), axis=1)
    s_ref = rng.permuted(np.tile(base, (1024, 1)), axis=1)
    res_s = chebyshev.run_sampled(cfg, psi_p, s_fit, s_ref)
    res_e = chebyshev.run_enumerated(cfg, psi_p)
    mu0 = abs(res_e.mu[0])
    for n in range(cfg.n_moments):
        assert abs(res_s.mu[n] - res_e.mu[n]) < 0.05 * mu0, n
    assert np.all(res_s.spins_fit.sum(axis=1) == 0)
    # and the enumerated moments sit close to the exact ones (fit error only)
    Hp = exact.rescaled(exact.hamiltonian(12, 1, 1.0, basis), cfg.E0, cfg.a, cfg.Wp)
    psi = exact.rbm_vector(psi_p, N, M, basis)
    t0 = exact.probe_vector(12, 1, np.pi, 0.0, basis, psi)
    mu_ex = exact.chebyshev_moments(Hp, t0, psi, cfg.n_moments)
    assert np.max(np.abs(np.array(res_e.mu) - mu_ex)) < 0.01 * mu0
