"""Symmetry projection (Appendix A) through the C ABI against the oracle:
B~_nk(s) and HB~_nk(s) = <s|H'|t~_nk> / psi(s) for every momentum of a 4 x 4
lattice at sampled configurations (float64 to 1e-10, float32 to 1e-4 of the
largest value), and the per-momentum Gram and Hamiltonian matrices through
cheb_gram; B~ and HB~ at the 6 x 6 workload size (M = 72, 4096 samples,
float32) on 16 sampled outputs."""

import numpy as np
import pytest

from gpu_common import dev, host, need_gpu, torch
from oracle import krylov, rbm, symmetry
from paper_2103_08804_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4)])
def test_btilde_and_momentum_grams_against_oracle(prec, tol):
    from paper_2103_08804_gb300 import api
    L, M, B, Nm = 4, 8, 517, 3
    N = L * L
    psi = synth.rbm_params(20, N, M, 0.2)
    states = [synth.rbm_params(21 + n, N, M, 0.2) for n in range(Nm)]
    spins = synth.sz0_spins(30, B, N)
    lref = rbm.logpsi(psi, N, M, spins)
    Bt_ref = symmetry.b_tilde(states, N, M, L, spins, lref)          # [Nm, N, B]
    G_ref = symmetry.gram_by_momentum(Bt_ref)                          # [N, Nm, Nm]
    cd = torch.complex128 if prec == 0 else torch.complex64
    ctx = api.Context(L, L, M, B, prec=prec)
    Bt = ctx.sym_btilde(dev(np.array(states), cd), dev(spins, torch.int8), dev(lref, cd))
    Bh = host(Bt).astype(np.complex128)                                # [N, Nm, B]
    scale = np.abs(Bt_ref).max()
    assert np.max(np.abs(Bh - np.transpose(Bt_ref, (1, 0, 2)))) <= tol * scale
    for k in (0, 1, 5, 10, 15):
        G = torch.zeros(Nm, Nm, dtype=torch.complex128, device="cuda")
        ctx.cheb_gram(Bt[k], None, G, None)
        assert np.allclose(host(G), G_ref[k], rtol=0, atol=10 * tol * np.abs(G_ref).max()), k
    ctx.sync_status()


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4)])
def test_hbtilde_and_momentum_hamiltonians_against_oracle(prec, tol):
    from paper_2103_08804_gb300 import api
    L, M, B, Nm = 4, 8, 389, 3
    J, E0, a, Wp = 1.0, -11.2, 9.5, 0.15
    N = L * L
    psi = synth.rbm_params(40, N, M, 0.2)
    states = [synth.rbm_params(41 + n, N, M, 0.2) for n in range(Nm)]
    spins = synth.sz0_spins(50, B, N)
    lref = rbm.logpsi(psi, N, M, spins)
    Bt_ref = symmetry.b_tilde(states, N, M, L, spins, lref)                        # [Nm, N, B]
    HBt_ref = symmetry.hb_tilde(states, N, M, L, J, E0, a, Wp, spins, lref)
    # per momentum, the estimators of cheb_gram (sampled H Hermitised)
    GH_ref = [krylov.gram(Bt_ref[:, k], HBt_ref[:, k]) for k in range(N)]
    cd = torch.complex128 if prec == 0 else torch.complex64
    ctx = api.Context(L, L, M, B, prec=prec, J=J)
    Bt, HBt = ctx.sym_hbtilde(dev(np.array(states), cd), dev(spins, torch.int8), dev(lref, cd),
                              (E0, a, Wp))
    for got, ref in ((Bt, Bt_ref), (HBt, HBt_ref)):
        gh = host(got).astype(np.complex128)                                       # [N, Nm, B]
        assert np.max(np.abs(gh - np.transpose(ref, (1, 0, 2)))) <= tol * np.abs(ref).max()
    for k in (0, 1, 5, 10, 15):
        G = torch.zeros(Nm, Nm, dtype=torch.complex128, device="cuda")
        H = torch.zeros_like(G)
        ctx.cheb_gram(Bt[k], HBt[k], G, H)
        G_ref, H_ref = GH_ref[k]
        assert np.allclose(host(G), G_ref, rtol=0, atol=10 * tol * np.abs(G_ref).max()), k
        assert np.allclose(host(H), H_ref, rtol=0, atol=10 * tol * np.abs(H_ref).max()), k
    # B~ of the H call is the B~ of sym_btilde (to rounding: the rotation
    # kernel's two variants may contract their arithmetic differently)
    Bt2 = ctx.sym_btilde(dev(np.array(states), cd), dev(spins, torch.int8), dev(lref, cd))
    assert float((Bt - Bt2).abs().max()) <= 1e-2 * tol * float(Bt.abs().max())
    ctx.sync_status()


def test_hbtilde_at_the_6x6_workload_size_on_sampled_outputs():
    # the bench's sym6 configuration (6 x 6, M = 72, 4096 samples, float32):
    # N, M and the bond count exceed a warp, so every strided loop of the
    # kernels takes several passes; B~ and HB~ of a sample depend on that
    # sample alone, so the oracle checks 16 of them (the last one included)
    from paper_2103_08804_gb300 import api
    L, M, B, Nm, Wp = 6, 72, 4096, 2, 0.9875
    N = L * L
    E0, a = synth.safe_rescaling(L, L)
    psi = synth.rbm_params(60, N, M, 0.02)
    states = [synth.rbm_params(61 + n, N, M, 0.02) for n in range(Nm)]
    spins = synth.sz0_spins(70, B, N)
    lref = rbm.logpsi(psi, N, M, spins)
    ctx = api.Context(L, L, M, B, prec=api.FP32)
    Bt, HBt = ctx.sym_hbtilde(dev(np.array(states), torch.complex64), dev(spins, torch.int8),
                              dev(lref, torch.complex64), (E0, a, Wp))
    idx = np.append(np.sort(np.random.default_rng(1).choice(B - 1, 15, replace=False)), B - 1)
    Bt_ref = symmetry.b_tilde(states, N, M, L, spins[idx], lref[idx])
    HBt_ref = symmetry.hb_tilde(states, N, M, L, 1.0, E0, a, Wp, spins[idx], lref[idx])
    for got, ref in ((Bt, Bt_ref), (HBt, HBt_ref)):
        gh = host(got)[:, :, idx].astype(np.complex128)                           # [N, Nm, 16]
        assert np.all(np.isfinite(gh))
        assert np.max(np.abs(gh - np.transpose(ref, (1, 0, 2)))) <= 1e-4 * np.abs(ref).max()
    ctx.sync_status()


def test_btilde_rejects_chains_and_probe_states():
    from paper_2103_08804_gb300 import api
    ctx = api.Context(8, 1, 4, 16, prec=1)
    p = torch.zeros(1, ctx.P, dtype=torch.complex64, device="cuda")
    sp = dev(synth.sz0_spins(1, 16, 8), torch.int8)
    with pytest.raises(api.CRError):
        ctx.sym_btilde(p, sp, torch.zeros(16, dtype=torch.complex64, device="cuda"))
    sq = api.Context(4, 4, 4, 16, prec=1)
    p = torch.zeros(1, sq.P, dtype=torch.complex64, device="cuda")
    sp = dev(synth.sz0_spins(2, 16, 16), torch.int8)
    with pytest.raises(api.CRError):
        sq.sym_hbtilde(p, sp, torch.zeros(16, dtype=torch.complex64, device="cuda"), (0.0, 0.0, 0.0))
