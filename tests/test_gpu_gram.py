"""The Krylov Gram estimators of Sec. IV, G_nm = <conj(B_n) B_m> and
H_nm = <conj(B_n) HB_m> (then (H + H^dag)/2), in mixed contexts on the tensor
cores, element by element against the oracle's float64 sums of the same
complex64 columns: sizes spanning several 128-row tiles, K segments and a
ragged sample tail, a leading dimension larger than the sample count, one
column and one sample, columns of very different norms (error measured
against sqrt(G_nn G_mm)), G exactly Hermitian, and the exact Chebyshev
vectors of a 10-site chain through the moment correction."""

import numpy as np
import pytest

from gpu_common import dev, host, need_gpu, relerr, torch
from oracle import exact, krylov
from paper_2103_08804_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _columns(seed, Nm, B, ld, spread=0.0):
    g = np.random.Generator(np.random.Philox(seed))
    X = (g.standard_normal((Nm, ld)) + 1j * g.standard_normal((Nm, ld))).astype(np.complex64)
    if spread:
        X *= np.exp(spread * g.standard_normal((Nm, 1))).astype(np.float32)
    return X


def _normalised(Gd, Gr):
    d = np.sqrt(np.abs(np.real(np.diag(Gr))))
    return np.max(np.abs(Gd - Gr) / np.maximum(np.outer(d, d), 1e-300))


# float32 inputs split into three bf16 terms (about 2^-24 relative each),
# float32 accumulation over 128-sample chunks and over the chunks of a K
# segment, float64 across segments: about 1e-6 of sqrt(G_nn G_mm); gate 1e-5.
TOL = 1e-5


@pytest.mark.parametrize("Nm,B,ld,spread", [(1, 1, 1, 0.0), (6, 1000, 1003, 0.0),
                                            (37, 4099, 4099, 3.0), (130, 20011, 20016, 0.0),
                                            (300, 65536, 65536, 1.0)])
@pytest.mark.parametrize("with_h", [False, True])
def test_mixed_gram_against_oracle(Nm, B, ld, spread, with_h):
    from paper_2103_08804_gb300 import api
    X = _columns(100 + Nm, Nm, B, ld, spread)
    Y = _columns(200 + Nm, Nm, B, ld, spread) if with_h else None
    G_ref, H_ref = krylov.gram(list(X[:, :B]), list((Y if with_h else X)[:, :B]))
    ctx = api.Context(4, 1, 4, 8, prec=api.MIXED)
    G = torch.zeros(Nm, Nm, dtype=torch.complex128, device="cuda")
    H = torch.zeros_like(G) if with_h else None
    ctx.cheb_gram(dev(X, torch.complex64), dev(Y, torch.complex64) if with_h else None, G, H,
                  n_samples=B)
    ctx.sync_status()
    Gh = host(G)
    eg = _normalised(Gh, G_ref)
    print(f"Nm={Nm} B={B}: G {eg:.2e}")
    assert eg < TOL
    assert np.array_equal(Gh, Gh.conj().T) and np.all(np.imag(np.diag(Gh)) == 0)
    if with_h:
        Hh = host(H)
        # H' entries are bounded by |B_n| |HB_m|: measure against both norms
        dx = np.sqrt(np.sum(np.abs(X[:, :B].astype(np.complex128)) ** 2, axis=1) / B)
        dy = np.sqrt(np.sum(np.abs(Y[:, :B].astype(np.complex128)) ** 2, axis=1) / B)
        scale = 0.5 * (np.outer(dx, dy) + np.outer(dy, dx))
        eh = np.max(np.abs(Hh - H_ref) / scale)
        print(f"  H {eh:.2e}")
        assert eh < TOL
        assert np.array_equal(Hh, Hh.conj().T)


def test_mixed_gram_repeated_calls_and_sizes():
    """Calls of different sizes on one context (the scratch grows, the tile
    list follows Nm) give the same results as fresh contexts, bit for bit."""
    from paper_2103_08804_gb300 import api
    ctx = api.Context(4, 1, 4, 8, prec=api.MIXED)
    out = []
    for Nm, B in ((20, 3000), (150, 4096), (20, 3000), (7, 50000)):
        X, Y = _columns(Nm, Nm, B, B), _columns(Nm + 1, Nm, B, B)
        G = torch.zeros(Nm, Nm, dtype=torch.complex128, device="cuda")
        H = torch.zeros_like(G)
        ctx.cheb_gram(dev(X, torch.complex64), dev(Y, torch.complex64), G, H)
        fresh = api.Context(4, 1, 4, 8, prec=api.MIXED)
        G2, H2 = torch.zeros_like(G), torch.zeros_like(G)
        fresh.cheb_gram(dev(X, torch.complex64), dev(Y, torch.complex64), G2, H2)
        ctx.sync_status()
        fresh.sync_status()
        assert torch.equal(G, G2) and torch.equal(H, H2)
        out.append(host(G))
    assert np.array_equal(out[0], out[2])


def test_mixed_gram_of_exact_chebyshev_vectors():
    """Exact Chebyshev vectors of a 10-site chain as columns (enumeration
    weights folded in): G and H' against the oracle, then the corrected
    moments of the mixed G, H' against the exact moments."""
    Lx, Nm = 10, 6
    basis = exact.sector_basis(Lx)
    Hm = exact.hamiltonian(Lx, 1, 1.0, basis)
    e = np.linalg.eigvalsh(Hm)
    a = (e[-1] - e[0]) / (2 * 0.9875)
    Hp = exact.rescaled(Hm, e[0], a, 0.9875)
    psi = exact.rbm_vector(synth.rbm_params(50, Lx, 10, 0.3), Lx, 10, basis)
    t0 = exact.probe_vector(Lx, 1, 0.6 * np.pi, 0.0, basis, psi)
    ts = exact.chebyshev_vectors(Hp, t0, Nm)
    w = np.abs(psi) ** 2 / np.vdot(psi, psi).real
    D = len(basis)
    sq = np.sqrt(D * w)
    Bm = np.array([sq * t / psi for t in ts]).astype(np.complex64)
    HBm = np.array([sq * (Hp @ t) / psi for t in ts]).astype(np.complex64)
    G_ref, H_ref = krylov.gram(list(Bm), list(HBm))
    from paper_2103_08804_gb300 import api
    ctx = api.Context(Lx, 1, 10, D, prec=api.MIXED)
    Gd = torch.zeros(Nm, Nm, dtype=torch.complex128, device="cuda")
    Hd = torch.zeros_like(Gd)
    ctx.cheb_gram(dev(Bm, torch.complex64), dev(HBm, torch.complex64), Gd, Hd)
    ctx.sync_status()
    assert relerr(host(Gd), G_ref) < TOL
    assert relerr(host(Hd), H_ref) < TOL
    mu_ex = exact.chebyshev_moments(Hp, t0, psi, 2 * Nm)
    mu = krylov.corrected_moments(host(Gd), host(Hd), 2 * Nm, cutoff=1e-6)
    assert np.max(np.abs(mu - mu_ex)) < 1e-3 * abs(mu_ex[0])
