"""Many Chebyshev sequences (probe momenta, lattices) advanced together (Sec. V).

The spectral function S(q, omega) needs one Chebyshev sequence per probe
momentum q (Sec. II), and the sequences are independent: nothing is
exchanged between them.  A Batch gives every sequence its own library
context (its own workspace), its own CUDA stream and the fixed buffers of a
graph-mode Sequence, and captures one natural-gradient iteration of ALL
sequences into a single CUDA graph through one cr_batch_run call (the
library forks every sequence onto its context's stream, interleaves their
launches and joins them back).  One replay then launches every sequence's
kernels at once, so small sequences that cannot fill the GPU alone run side
by side.

schedule="per_q" is the baseline: each sequence replays its own iteration
graph, one sequence after another on one stream.

Both schedules launch the same kernels with the same arguments on the same
data, so they give bit-identical moments; only the overlap differs.  Two
knobs shape the kernels of a sequence that shares the GPU: the CTA count
(walker-block shape) of its fused CG kernel (cr_set_fcg_ctas: fewer, wider
blocks leave SMs to the other sequences' cooperative launches) and the
walker chunks of its split-K reductions (cr_set_chunks).  The autotuner
times the batched iteration graph on throwaway copies of the sequences,
first the CTA counts, then the chunk counts, each for all sequences and
then per lattice group, and applies the fastest setting.

A sequence whose probe vanishes identically (q = 0 on the S^z = 0 sector,
where f_q = 0 and R is undefined) is not run: its moments are zero.
"""

from dataclasses import dataclass, field

import numpy as np
import torch

from . import api
from .driver import Sequence, SeqConfig


@dataclass
class SeqSpec:
    """One sequence of a batch: its configuration, the RBM psi and the
    initial walkers (fit walkers and the fixed |psi|^2 samples)."""
    name: str
    cfg: SeqConfig
    psi: np.ndarray
    spins_fit: np.ndarray
    spins_ref: np.ndarray


def square_irreducible_momenta(L):
    """q = 2 pi (k1, k2) / L with 0 <= k2 <= k1 <= L/2: the momenta of an
    L x L lattice up to its point-group symmetry ((L/2 + 1)(L/2 + 2)/2 of them)."""
    return [(2 * np.pi * k1 / L, 2 * np.pi * k2 / L)
            for k1 in range(L // 2 + 1) for k2 in range(k1 + 1)]


def zero_momentum(cfg):
    """True where f_q vanishes on every S^z = 0 configuration: q = 0 mod 2 pi
    along every lattice direction (then f_q is proportional to the total S^z)."""
    def zero(v):
        r = np.remainder(v, 2 * np.pi)
        return min(r, 2 * np.pi - r) < 1e-9
    return zero(cfg.q[0]) and (cfg.Ly == 1 or zero(cfg.q[1]))


@dataclass
class Batch:
    specs: list
    prec: int = api.FP32
    tune: bool = True
    chunk_candidates: tuple = (8, 16, 32, 64, 128)
    cta_divisors: tuple = (1, 2, 4, 8)
    tune_reps: int = 5
    timings: dict = field(default_factory=dict)

    def __post_init__(self):
        if len({s.cfg.n_iter for s in self.specs}) > 1:
            raise ValueError("sequences of a batch share n_iter")
        self.active = [s for s in self.specs if not zero_momentum(s.cfg)]
        self.skipped = [s.name for s in self.specs if zero_momentum(s.cfg)]
        self.ctxs, self.streams, self.seqs = [], [], []
        for s in self.active:
            st = torch.cuda.Stream()
            B = max(s.spins_fit.shape[0], s.spins_ref.shape[0])
            ctx = api.Context(s.cfg.Lx, s.cfg.Ly, s.cfg.M, B, self.prec, J=s.cfg.J, stream=st,
                              explicit_s=s.cfg.solver == api.SOLVE_CHOLESKY)
            with torch.cuda.stream(st):
                seq = Sequence(ctx, s.cfg, s.psi, s.spins_fit, s.spins_ref, graphs=True)
            self.ctxs.append(ctx)
            self.streams.append(st)
            self.seqs.append(seq)
        torch.cuda.synchronize()
        self._graphs = {}
        self.chunks = [c.max_chunks() for c in self.ctxs]
        self.ctas = [0] * len(self.ctxs)
        self.graph_launches = 0
        if self.tune:
            self.autotune()

    # -------------------------------------------------------------- streams
    def _fork(self):
        main = torch.cuda.current_stream()
        for st in self.streams:
            st.wait_stream(main)

    def _join(self):
        main = torch.cuda.current_stream()
        for st in self.streams:
            main.wait_stream(st)

    def set_chunks(self, chunks):
        for ctx, n in zip(self.ctxs, chunks):
            ctx.set_chunks(min(n, ctx.max_chunks()))
        self.chunks = [c for c in chunks]
        self._graphs = {}

    def set_ctas(self, ctas):
        """CTA counts of the contexts' fused CG kernels (0: one per SM)."""
        for ctx, n in zip(self.ctxs, ctas):
            if ctx.fused_cg():
                ctx.set_fcg_ctas(n)
        self.ctas = list(ctas)
        self._graphs = {}

    # -------------------------------------------------------------- graphs
    def _capture(self, seqs, kind):
        """One iteration of every sequence in seqs, each on its own stream,
        captured as one graph (fork from and join into the capture stream)."""
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream()
        main = torch.cuda.current_stream()
        cap.wait_stream(main)
        self._fork()
        n0 = sum(c.n_launches() for c in self.ctxs)
        for seq, st in zip(seqs, self.streams):
            seq.ctx.set_stream(st)
        iters = [seq.iter_desc(kind) for seq in seqs]
        with torch.cuda.graph(g, stream=cap):
            api.batch_run(iters, 1, cap)
        main.wait_stream(cap)
        return g, sum(c.n_launches() for c in self.ctxs) - n0

    def _eager(self, seqs, kind):
        self._fork()
        for seq, st in zip(seqs, self.streams):
            with torch.cuda.stream(st):
                seq._iteration(kind)
                seq._eager_done.add(kind)
        self._join()

    def _each(self, fn):
        """Run fn(seq) for every sequence on its own stream (eager work)."""
        self._fork()
        for seq, st in zip(self.seqs, self.streams):
            with torch.cuda.stream(st):
                fn(seq)
        self._join()

    # -------------------------------------------------------------- tuning
    def _throwaway(self):
        seqs = []
        for s, ctx, st in zip(self.active, self.ctxs, self.streams):
            with torch.cuda.stream(st):
                seqs.append(Sequence(ctx, s.cfg, s.psi, s.spins_fit, s.spins_ref, graphs=True))
        self._fork()
        for seq, st in zip(seqs, self.streams):
            with torch.cuda.stream(st):
                seq.start()
                seq._moment_begin(1)
        self._join()
        self._eager(seqs, 1)
        return seqs

    def _time_graph(self, seqs, chunks, ctas):
        for ctx, n, m in zip(self.ctxs, chunks, ctas):
            ctx.set_chunks(min(n, ctx.max_chunks()))
            if ctx.fused_cg():
                ctx.set_fcg_ctas(m)
        g, _ = self._capture(seqs, 1)
        for _ in range(2):
            g.replay()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(self.tune_reps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / self.tune_reps

    def autotune(self):
        """Pick each context's fused-CG CTA count and reduction chunk count by
        timing the batched iteration graph on throwaway sequences (the real
        ones are not touched), then apply them."""
        seqs = self._throwaway()
        n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        groups = {}
        for i, s in enumerate(self.active):
            groups.setdefault((s.cfg.Lx, s.cfg.Ly, s.cfg.M), []).append(i)
        best_ch, best_ct = list(self.chunks), list(self.ctas)
        t_best = self._time_graph(seqs, best_ch, best_ct)
        self.timings = {("max",): t_best}

        def trial(key, ch, ct):
            nonlocal best_ch, best_ct, t_best
            if (ch, ct) == (best_ch, best_ct):
                return
            t = self._time_graph(seqs, ch, ct)
            self.timings[key] = t
            if t < t_best:
                best_ch, best_ct, t_best = ch, ct, t

        # walker-block shape of the fused CG: n_sm / d CTAs per sequence
        fcg = any(c.fused_cg() for c in self.ctxs)
        for d in self.cta_divisors[1:] if fcg else ():
            trial(("ctas", d), best_ch, [max(1, n_sm // d)] * len(self.ctxs))
        if fcg and len(groups) > 1:
            for key, idx in groups.items():
                for d in self.cta_divisors:
                    ct = list(best_ct)
                    for i in idx:
                        ct[i] = 0 if d == 1 else max(1, n_sm // d)
                    trial(("ctas", key, d), best_ch, ct)
        # walker chunks of the split-K reductions
        for n in self.chunk_candidates:
            trial(("all", n), [min(n, c.max_chunks()) for c in self.ctxs], best_ct)
        if len(groups) > 1:
            for key, idx in groups.items():
                for n in self.chunk_candidates:
                    ch = list(best_ch)
                    for i in idx:
                        ch[i] = min(n, self.ctxs[i].max_chunks())
                    trial((key, n), ch, best_ct)
        self.tuned_ms = t_best
        del seqs
        # the throwaway sequences replayed one iteration many times over; a
        # device status they raised (e.g. a non-finite update of an overfitted
        # RBM) says nothing about the real sequences, so read and clear it
        for ctx in self.ctxs:
            try:
                ctx.sync_status()
            except api.CRError:
                pass
        self.set_chunks(best_ch)
        self.set_ctas(best_ct)
        torch.cuda.synchronize()
        return best_ch, best_ct

    # -------------------------------------------------------------- driving
    def start(self):
        self._each(lambda seq: seq.start())

    def _fit_batched(self, n):
        kind = Sequence.kind_of(n)
        self._each(lambda seq: seq._moment_begin(n))
        for it in range(self.seqs[0].cfg.n_iter):
            if kind not in self.seqs[0]._eager_done:
                self._eager(self.seqs, kind)
            else:
                if kind not in self._graphs:
                    self._graphs[kind] = self._capture(self.seqs, kind)
                g, nodes = self._graphs[kind]
                g.replay()
                self.graph_launches += nodes
            for seq in self.seqs:
                seq.stats[n, it].copy_(seq.stats_it)
        self._each(lambda seq: seq._moment_end(n))

    def _fit_per_q(self, n):
        main = torch.cuda.current_stream()
        for seq in self.seqs:
            seq.ctx.set_stream(main)
            seq.graph_launches = 0
            seq.fit(n)
            self.graph_launches += seq.graph_launches
        for seq, st in zip(self.seqs, self.streams):
            seq.ctx.set_stream(st)

    def fit(self, n, schedule="batched"):
        """Projection step n of every sequence."""
        if schedule == "batched":
            self._fit_batched(n)
        elif schedule == "per_q":
            self._fit_per_q(n)
        else:
            raise ValueError(schedule)

    def moments(self):
        """Moments of every sequence by name (zeros for a vanishing probe)."""
        out = {}
        it = iter(self.seqs)
        for s in self.specs:
            if s.name in self.skipped:
                out[s.name] = np.zeros(s.cfg.n_moments, dtype=np.complex128)
            else:
                out[s.name] = next(it).mu.cpu().numpy()
        return out


def momentum_scan_specs(L=8, alpha=2, chains=(48, 96), walkers=8192, n_moments=150, n_iter=50,
                        sigma=0.02, seed=0, **cfg_kw):
    """Every irreducible momentum of an L x L lattice plus chains of the given
    lengths at q = pi/2, alpha = M/N hidden units per site, random RBMs and
    walkers from synth; rescaling from the rigorous spectrum bounds; the
    shift from synth.default_shift unless given."""
    from . import synth
    lat = [((L, L), q) for q in square_irreducible_momenta(L)]
    lat += [((n, 1), (np.pi / 2, 0.0)) for n in chains]
    specs = []
    for k, ((Lx, Ly), q) in enumerate(lat):
        N, M = Lx * Ly, alpha * Lx * Ly
        E0, a = synth.safe_rescaling(Lx, Ly)
        kw = dict(cfg_kw)
        kw.setdefault("shift", synth.default_shift(N + M + N * M, walkers))
        cfg = SeqConfig(Lx=Lx, Ly=Ly, M=M, q=q, n_moments=n_moments, n_iter=n_iter, E0=E0, a=a,
                        seed=2 * k, seed_ref=2 * k + 1, **kw)
        name = f"square{L}_q{q[0]:.4f}_{q[1]:.4f}" if Ly > 1 else f"chain{Lx}_q{q[0]:.4f}"
        specs.append(SeqSpec(name, cfg, synth.rbm_params(seed + 100 + k, N, M, sigma),
                             synth.sz0_spins(seed + 200 + k, walkers, N),
                             synth.sz0_spins(seed + 300 + k, walkers, N)))
    return specs
