"""Many sequences in one graph: the batched schedule (every sequence's
iteration in one CUDA graph through cr_batch_run, each sequence on its own
stream) and the one-sequence-after-another schedule give the same moments,
bit for bit, as each sequence run alone (also with tuned fused-CG CTA
counts), a vanishing probe (q = 0) is skipped with zero moments, and
cr_batch_run itself reproduces the oracle's sequences on a small float64
instance."""

import numpy as np
import pytest

from gpu_common import host, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _specs():
    from paper_2103_08804_gb300 import api, batch
    return batch.momentum_scan_specs(L=4, alpha=2, chains=(8,), walkers=1024, n_moments=4,
                                     n_iter=4, sigma=0.05, n_therm=2, solver=api.SOLVE_CG,
                                     cg_maxit=20, cg_tol=1e-5)


def _alone(spec, chunks=None):
    from paper_2103_08804_gb300 import api, driver
    c = spec.cfg
    ctx = api.Context(c.Lx, c.Ly, c.M, spec.spins_fit.shape[0], api.FP32)
    if chunks is not None:
        ctx.set_chunks(chunks)
    seq = driver.Sequence(ctx, c, spec.psi, spec.spins_fit, spec.spins_ref, graphs=True)
    seq.run()
    ctx.sync_status()
    return seq


def test_batched_graph_equals_sequences_alone():
    from paper_2103_08804_gb300 import api, batch
    specs = _specs()
    assert len(specs) == 7
    b = batch.Batch(specs, prec=api.FP32, tune=False)
    assert len(b.seqs) == 6 and b.skipped == [specs[0].name]
    b.start()
    for n in range(1, 4):
        b.fit(n)
    for ctx in b.ctxs:
        ctx.sync_status()
    assert b.graph_launches > 0
    mom = b.moments()
    assert np.all(mom[specs[0].name] == 0)
    for spec, seq in zip(specs[1:], b.seqs):
        ref = _alone(spec)
        assert np.array_equal(mom[spec.name], host(ref.mu)), spec.name
        assert np.array_equal(host(seq.params), host(ref.params)), spec.name
        assert np.array_equal(host(seq.stats), host(ref.stats)), spec.name
        assert seq.counter() == ref.counter()
        assert np.all(np.isfinite(mom[spec.name])) and abs(mom[spec.name][0]) > 0


def test_per_q_schedule_equals_batched_and_autotune():
    from paper_2103_08804_gb300 import api, batch
    specs = _specs()[3:]
    runs = {}
    for schedule in ("batched", "per_q"):
        b = batch.Batch(specs, prec=api.FP32, tune=False)
        b.set_chunks([4] * len(b.ctxs))
        b.start()
        for n in range(1, 4):
            b.fit(n, schedule=schedule)
        for ctx in b.ctxs:
            ctx.sync_status()
        runs[schedule] = b.moments()
    for k in runs["batched"]:
        assert np.array_equal(runs["batched"][k], runs["per_q"][k]), k
    t = batch.Batch(specs, prec=api.FP32, tune=True, chunk_candidates=(2, 4, 8), tune_reps=2)
    assert all(1 <= n <= c.max_chunks() for n, c in zip(t.chunks, t.ctxs))
    assert t.tuned_ms > 0 and ("all", 4) in t.timings


@pytest.mark.parametrize("prec", [1, 2])
def test_chunk_count_changes_only_the_summation_order(prec):
    # one natural-gradient update on identical inputs with the largest and a
    # small chunk count.  float32: the float64 combination of float32 partial
    # sums in a different grouping, so the updates agree to float32 rounding
    # (a strong shift keeps the solve well conditioned).  mixed: the estimator
    # sums run on the tensor cores over K segments and the CG is fused, so
    # the chunk count does not enter the step at all.
    import torch
    from gpu_common import dev
    from paper_2103_08804_gb300 import api, synth
    N, M, B = 16, 32, 4096
    ctx = api.Context(N, 1, M, B, prec)
    assert ctx.max_chunks() == 32
    rng = np.random.default_rng(3)
    spins = dev(synth.sz0_spins(4, B, N), torch.int8)
    p0 = dev(synth.rbm_params(5, N, M, 0.1), ctx.cdtype)
    theta = torch.empty(B, M, dtype=ctx.cdtype, device="cuda")
    ctx.rbm_logpsi(p0, spins, theta)
    T = torch.empty_like(theta)
    ctx.logderiv(p0, spins, theta, tanh_out=T)
    R = dev(1 + 0.3 * rng.standard_normal(B) + 0.3j * rng.standard_normal(B), ctx.cdtype)
    out = {}
    for n in (32, 3):
        ctx.set_chunks(n)
        p = p0.clone()
        ctx.sr_step(p, spins, T, R, 0.5, 0.1, cg_maxit=200, cg_tol=1e-6)
        ctx.sync_status()
        out[n] = host(p - p0)
    d = out[32]
    if prec == 2:
        assert np.array_equal(out[3], d)
    else:
        assert np.linalg.norm(out[3] - d) < 1e-4 * np.linalg.norm(d)
        assert not np.array_equal(out[3], d)
    with pytest.raises(api.CRError):
        ctx.set_chunks(33)
    with pytest.raises(api.CRError):
        ctx.set_chunks(0)


def test_mixed_contexts_of_different_sizes_coexist():
    # the tensor-core kernels' shared-memory opt-in belongs to the function,
    # not the context: a smaller mixed context created after a larger one
    # must leave the larger one launchable
    import torch
    from gpu_common import dev
    from paper_2103_08804_gb300 import api, synth
    big = api.Context(64, 1, 128, 1024, api.MIXED)
    small = api.Context(48, 1, 96, 1024, api.MIXED)
    for ctx, N, M in ((big, 64, 128), (small, 48, 96), (big, 64, 128)):
        spins = dev(synth.sz0_spins(1, 1024, N), torch.int8)
        p = dev(synth.rbm_params(2, N, M, 0.05), ctx.cdtype)
        theta = torch.empty(1024, M, dtype=ctx.cdtype, device="cuda")
        ctx.rbm_logpsi(p, spins, theta)
        T = torch.empty_like(theta)
        ctx.logderiv(p, spins, theta, tanh_out=T)
        R = torch.ones(1024, dtype=ctx.cdtype, device="cuda") * 0.5
        ctx.sr_step(p, spins, T, R + 0.1 * T[:, 0], 0.5, 1e-2, cg_maxit=10, cg_tol=1e-4)
        ctx.sync_status()
        assert torch.isfinite(torch.view_as_real(p)).all()


def test_batch_run_reproduces_the_oracle_sequences():
    """Two 12-site chains at different momenta advanced by cr_batch_run
    (float64, Cholesky): walker trajectories bit-identical to the oracle's
    shared Philox stream and the moments within 1e-8 mu_0, as each sequence
    alone in smoke()."""
    from oracle import chebyshev, exact
    from paper_2103_08804_gb300 import api, batch, driver, synth
    L, M, B = 12, 12, 256
    e0 = np.linalg.eigvalsh(exact.hamiltonian(L, 1, 1.0, exact.sector_basis(L)))[0]
    specs, refs = [], []
    for k, q in enumerate(((np.pi, 0.0), (np.pi / 2, 0.0))):
        kw = dict(Lx=L, Ly=1, M=M, q=q, n_moments=3, n_iter=2, shift=1e-3, dgamma=0.5, E0=e0,
                  a=5.0, Wp=0.9875, n_therm=2, n_therm_ref=4, seed=10 + 2 * k, seed_ref=11 + 2 * k)
        psi = synth.rbm_params(20 + k, L, M, 0.05)
        s_fit, s_ref = synth.sz0_spins(30 + k, B, L), synth.sz0_spins(40 + k, B, L)
        specs.append(batch.SeqSpec(f"q{k}", driver.SeqConfig(solver=api.SOLVE_CHOLESKY, **kw), psi,
                                   s_fit, s_ref))
        refs.append(chebyshev.run_sampled(chebyshev.Config(**kw), psi, s_fit, s_ref))
    b = batch.Batch(specs, prec=api.FP64, tune=False)
    b.start()
    for n in (1, 2):
        b.fit(n)
    for ctx in b.ctxs:
        ctx.sync_status()
    assert b.graph_launches > 0
    for seq, ref in zip(b.seqs, refs):
        assert np.array_equal(host(seq.spins), ref.spins_fit)
        mu = host(seq.mu)
        assert np.max(np.abs(mu - np.array(ref.mu))) < 1e-8 * abs(ref.mu[0])


def test_tuned_fused_cg_ctas_keep_batched_equal_to_alone():
    """Mixed contexts (the fused CG) with a smaller CTA count: the batched
    graph equals each sequence run alone with the same CTA count, bit for
    bit; a different CTA count changes the sums' grouping only (rounding)."""
    import torch
    from gpu_common import dev
    from paper_2103_08804_gb300 import api, batch, driver, synth
    specs = _specs()[3:5]
    b = batch.Batch(specs, prec=api.MIXED, tune=False)
    b.set_ctas([16] * len(b.ctxs))
    b.start()
    for n in range(1, 4):
        b.fit(n)
    for ctx in b.ctxs:
        ctx.sync_status()
    mom = b.moments()
    for spec in specs:
        c = spec.cfg
        ctx = api.Context(c.Lx, c.Ly, c.M, spec.spins_fit.shape[0], api.MIXED)
        assert ctx.fused_cg()
        ctx.set_fcg_ctas(16)
        seq = driver.Sequence(ctx, c, spec.psi, spec.spins_fit, spec.spins_ref, graphs=True)
        seq.run()
        ctx.sync_status()
        assert np.array_equal(mom[spec.name], host(seq.mu)), spec.name
    # one product with the default and with 16 CTAs
    N, M, B = 16, 32, 4096
    ctx = api.Context(N, 1, M, B, api.MIXED)
    spins = dev(synth.sz0_spins(4, B, N), torch.int8)
    p0 = dev(synth.rbm_params(5, N, M, 0.1), ctx.cdtype)
    theta = torch.empty(B, M, dtype=ctx.cdtype, device="cuda")
    ctx.rbm_logpsi(p0, spins, theta)
    T = torch.empty_like(theta)
    ctx.logderiv(p0, spins, theta, tanh_out=T)
    v = dev(synth.rbm_params(6, N, M, 1.0), torch.complex128)
    out = {}
    for n in (0, 16):
        ctx.set_fcg_ctas(n)
        out[n] = host(ctx.sr_sv(spins, T, v, 1e-2))
    ctx.sync_status()
    assert np.max(np.abs(out[16] - out[0])) < 1e-6 * np.max(np.abs(out[0]))
    with pytest.raises(api.CRError):
        ctx.set_fcg_ctas(100000)
