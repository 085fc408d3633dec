"""Throughput of the RBM-Chebyshev projection step on one GB300.

One step = one Chebyshev moment n: fit RBM_n to
phi_n = 2 beta_{n-1} H' t~_{n-1} - beta_{n-2} t~_{n-2} by 50 natural-gradient
iterations (each: one Metropolis sweep, the local target R, the estimators,
the matrix-free shifted solve by CG, theta refresh), then beta_n = <R> and
mu_n with its Krylov columns.  Inputs are synthetic random complex RBMs and
seeded S^z = 0 walkers, resident in HBM; L2 is flushed between timed steps.

Default workload (the largest single-GPU configuration): the 16 x 16
periodic lattice, alpha = 1 (M = 256, P = 66,048), 65536 walkers,
q = (pi, 0).  The mixed path (the CG as one persistent tensor-core kernel)
is the headline; the plain float32 path is timed beside it on fewer steps;
the moment error of the timed configuration against the float64 GPU path
and against a converged CG is reported, and the Krylov step over 300
states (once per sequence) is timed separately.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload square16|chain64|batch|square10|sym6]

--workload chain64: the 64-site chain (alpha = 2, 16384 walkers, q = pi/2),
mixed and plain float32 paths, timed steps cycling through moments 3-5.

--workload batch times the momentum scan instead: all 15 irreducible momenta
of an 8 x 8 square lattice (q = 0 has a vanishing probe and is skipped) plus
chains of 48 and 96 sites at q = pi/2, alpha = 2, 8192 walkers each; one step
= one moment of every sequence, with every sequence's iteration in one CUDA
graph, against one sequence after another.

--workload square10 times the explicit-S path: 10 x 10 square lattice,
alpha = 1 (P = 10,200), 32768 walkers, q = (pi, pi); S built on the tensor
cores (three-term bf16 splits), blocked Cholesky in float32 refined in
float64; it also reports |S_mixed - S_fp64|_F / |S_fp64|_F on a walker
sample, for the default splits and for the cheaper two-term (bf16x3) form.

--workload sym6 times the symmetry projection of Appendix A on the 6 x 6
lattice (alpha = 2): B~ and HB~ of 150 stored states at 4096 samples for
all 36 momenta, then G^(k) and H^(k) of every momentum.

--impl reference times the float64 oracle on the host cores on a walker
sample of the same workload (extrapolated to the workload's walkers and
iterations).  Prints one JSON line.  Under torchrun every rank runs an
independent sequence (a different seed): weak scaling with no data-path
collective.
"""

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "square16"
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cg-maxit", type=int, default=50)
    ap.add_argument("--cg-tol", type=float, default=1e-4)
    ap.add_argument("--jacobi", action="store_true", help="Jacobi-preconditioned CG")
    ap.add_argument("--iters", type=int, default=None,
                    help="natural-gradient iterations per moment (profiling runs only; the "
                         "workload's own count otherwise)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the replayed moment-error check against the float64 path")
    ap.add_argument("--eager", action="store_true",
                    help="launch every kernel from the host instead of replaying CUDA graphs")
    ap.add_argument("--cpu-walkers", type=int, default=None,
                    help="walkers of the oracle sample (default 2048 for chain64, 64 for square16)")
    ap.add_argument("--chunks", type=int, default=None,
                    help="walker chunks of the split-K reductions (default: the context's)")
    ap.add_argument("--only-mixed", action="store_true",
                    help="chain64: skip the plain float32 path (tuning runs)")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=["chain64", "batch", "square10", "square16", "sym6"])
    ap.add_argument("--s-error-walkers", type=int, default=2048,
                    help="square10: walkers of the tensor-core S vs float64 S comparison")
    return ap.parse_args()


def dist_setup():
    from paper_2103_08804_gb300 import replicas
    return replicas.init()


def barrier(ws):
    from paper_2103_08804_gb300 import replicas
    replicas.barrier(ws)


def max_over_ranks(ws, x):
    from paper_2103_08804_gb300 import replicas
    return replicas.max_over_ranks(ws, x)


def clock_path(name, rank):
    """Where the nvidia-smi samples of a timed region go: $CHEBRBM_CLOCKS_DIR
    when set (to keep them), else the system temporary directory."""
    d = os.environ.get("CHEBRBM_CLOCKS_DIR") or tempfile.gettempdir()
    return os.path.join(d, f"clocks_{name}_r{rank}.csv")


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    def __init__(self, path, index):
        self.path, self.index, self.p = path, index, None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            self.p.wait()
            self.f.close()

    def summary(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(np.max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except ValueError:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def make_config(wl, E0, a, args, n_moments, seed, solver=None):
    from paper_2103_08804_gb300 import api, driver
    return driver.SeqConfig(Lx=wl.Lx, Ly=wl.Ly, M=wl.M, q=wl.q, n_moments=n_moments,
                            n_iter=wl.iters if args.iters is None else args.iters,
                            shift=wl.shift, dgamma=wl.dgamma, E0=E0, a=a,
                            Wp=0.9875, n_therm=2, sweeps_per_iter=1, n_therm_ref=20, seed=seed,
                            seed_ref=seed + 1,
                            solver=api.SOLVE_CG if solver is None else solver,
                            cg_maxit=args.cg_maxit, cg_tol=args.cg_tol, jacobi=args.jacobi,
                            krylov=True)


# Timed steps are moments 3, 4, 5 of a sequence, then the sequence is
# restarted (sample |psi|^2, fit moments 1 and 2, untimed) and the cycle
# repeats.  Every timed step is a full projection step with the n >= 3
# target (the largest per-moment work); later moments are avoided because on
# random RBMs the late fits degrade (gamma near 1, growing forces) until a
# float32 ratio overflows, at a moment that depends on rounding.
CYCLE = (3, 4, 5)


CYCLE_NOTE = ("timed steps cycle through moments 3, 4, 5 (the n >= 3 target); the sequence is "
              "restarted (|psi|^2 sampled, moments 1-2 fitted) untimed before each cycle")


def restart(seq, first=CYCLE[0]):
    """Sample |psi|^2 and fit the moments before `first` (untimed)."""
    seq.start()
    for n in range(1, first):
        seq.fit(n)


def cycle_moment(k, cyc=CYCLE):
    """Moment index of timed step k; a restart precedes k % len(cyc) == 0."""
    return cyc[k % len(cyc)]


# The momentum scan and the 16 x 16 lattice time moment 3 only (a restart
# before every step): on their random RBMs some fits already degrade by
# moment 5 (gamma above 1 rad on the 8 x 8 scan; non-finite on 16 x 16).
EARLY_CYCLE = (3,)
BATCH_CYCLE = EARLY_CYCLE
# The 16 x 16 random RBM already fails at moment 3 for some trajectories:
# its steps are moment 2 (the n = 2 target, with the same terms to evaluate).
SQ16_CYCLE = (2,)
SQ16_CYCLE_NOTE = ("every timed step is moment 2 (the n = 2 target) after an untimed restart "
                   "(|psi|^2 sampled, moment 1 fitted)")
BATCH_CYCLE_NOTE = ("every timed step is moment 3 (the n >= 3 target) of every sequence, after an "
                    "untimed restart (|psi|^2 sampled, moments 1-2 fitted)")


def reduce_flops(wl):
    """Algorithmic flops of one launch of the O-reduction over all walkers:
    per (walker, i, j) one real x complex FMA for O_W (4 flops), per (walker, j)
    conj(T) g (6 flops) and its b-sum (2 flops), per (walker, i) 4 flops."""
    B, N, M = wl.walkers, wl.N, wl.M
    return B * (4 * N * M + 8 * M + 4 * N)


def sm_count():
    """Multiprocessors of the current device (the library sizes its grids the same way)."""
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def fp32_peak(f_sm):
    return sm_count() * FP32_LANES_PER_SM * 2 * f_sm * 1e6 / 1e12


def fcg_bytes_per_iter(wl):
    """Algorithmic bytes of one CG iteration of the fused solve: T = tanh theta
    (complex64 [B][M]) and the spins (int8 [B][N]) read once; the P-vectors
    are negligible beside them."""
    return wl.walkers * (8 * wl.M + wl.N)


def fcg_flops_per_iter(wl):
    """Algorithmic flops of one CG iteration: the two contractions sigma V
    (B x N x M, real sigma times complex V: 4 flops per term) and
    sigma^T (conj(T) w) (the same), before the three-term bf16 splits."""
    return 8.0 * wl.walkers * wl.N * wl.M


def roofline_fcg(ctx, seq, wl, kind, clocks, n_eager=3):
    """Live CUDA-event timing of the fused CG kernel on eagerly launched
    natural-gradient iterations of the current step (graph replays record no
    host-side events), with the CG iteration count of each solve."""
    import torch
    ctx.time_kernel("fcg", 64)
    its = []
    for _ in range(n_eager):
        seq._iteration(kind)
        its.append(float(seq.stats_it[5].item()))
    torch.cuda.synchronize()
    times = ctx.kernel_times()
    ctx.time_kernel(None, 1)
    k_ms = float(np.mean(times)) if times else None
    it = float(np.mean(its))
    peaks, src = measured_peaks()
    bw_peak = float(peaks["hbm_gbs"])
    tf_peak = float(peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]))
    work = fcg_bytes_per_iter(wl) * it
    achieved = work / (k_ms * 1e-3) / 1e9 if k_ms else None
    flops = fcg_flops_per_iter(wl) * it
    tf = flops / (k_ms * 1e-3) / 1e12 if k_ms else None
    return {"kernel": "cg_fused_kernel (one persistent launch per CG solve: tcgen05 O v and "
                      "O^dag w products from bf16 splits, float64 CG vectors)",
            "bound": "hbm", "achieved": achieved, "peak": bw_peak, "unit": "GB/s",
            "frac": achieved / bw_peak if achieved else None, "traffic": None,
            "work_per_launch": work, "cg_iters_per_launch": it,
            "work_note": "algorithmic bytes: T (complex64 B x M) and spins (int8 B x N) once per "
                         "CG iteration, times the CG iterations of the launch",
            "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({src})",
            "launches_timed": len(times), "avg_launch_ms": k_ms,
            "us_per_cg_iteration": k_ms * 1e3 / it if k_ms else None,
            "tensor_view": {"achieved": tf, "peak": tf_peak, "unit": "TFLOP/s",
                            "frac": tf / tf_peak if tf else None, "work_per_launch": flops,
                            "note": "algorithmic flops of the two contractions (8 B N M per CG "
                                    "iteration); the three-term splits execute 3x that on the "
                                    "tensor cores; peak: MEASURED_PEAKS.json "
                                    "bf16_tflops_sustained"}}


def roofline_oreduce2(ctx, seq, wl, kind, clocks, n_eager=3):
    """Live timing of the float32 O-reduction (the plain path's top kernel)."""
    import torch
    ctx.time_kernel("reduce", 4096)
    for _ in range(n_eager):
        seq._iteration(kind)
    torch.cuda.synchronize()
    ktimes = ctx.kernel_times()
    ctx.time_kernel(None, 1)
    k_ms = float(np.mean(ktimes)) if ktimes else None
    f_sm = clocks.get("sm_mhz") or 2070.0
    peak = fp32_peak(f_sm)
    achieved = reduce_flops(wl) / (k_ms * 1e-3) / 1e12 if k_ms else None
    return {"kernel": "oreduce2_kernel (sum_s sigma_si conj(T_sj) g_s, FP32 FMA)", "bound": "alu",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if achieved else None, "traffic": None,
            "work_per_launch": reduce_flops(wl),
            "peak_source": f"{sm_count()} SMs x 128 FP32 lanes x 2 flop x median SM clock under load",
            "launches_timed": len(ktimes), "avg_launch_ms": k_ms}


def cg_summary(st, cg_maxit, cg_tol):
    """CG convergence over the timed natural-gradient iterations (stats
    [5] iterations, [6] relative residual)."""
    its, res = st[..., 5].ravel(), st[..., 6].ravel()
    trunc = (its >= cg_maxit) & (res > cg_tol)
    return {"cg_iters_mean": float(its.mean()), "cg_iters_max": float(its.max()),
            "cg_rel_residual_median": float(np.median(res)), "cg_rel_residual_max": float(res.max()),
            "cg_truncated_fraction": float(trunc.mean()),
            "cg_note": f"CG stops at |r| <= {cg_tol} |F| or after {cg_maxit} iterations; truncated = "
                       f"stopped at the limit above tolerance (a fixed CG budget per update)"}


def measure(args, prec_name, ws, rank, local, wl_name, cyc, K=None, W=None):
    """Time K moments of one precision path; returns (result dict, config, workload)."""
    import torch

    from paper_2103_08804_gb300 import api, driver, replicas, synth

    wl = synth.WORKLOADS[wl_name]
    E0, a = synth.safe_rescaling(wl.Lx, wl.Ly)
    K = args.steps if K is None else K
    W = args.warmup if W is None else W
    n_moments = 1 + max(cyc)
    seed = replicas.replica_seed(1000, rank)
    prec = {"fp32": api.FP32, "mixed": api.MIXED}[prec_name]
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = api.Context(wl.Lx, wl.Ly, wl.M, wl.walkers, prec=prec, stream=stream)
    if args.chunks:
        ctx.set_chunks(min(args.chunks, ctx.max_chunks()))
    psi = synth.rbm_params(seed, wl.N, wl.M, wl.sigma)
    cfg = make_config(wl, E0, a, args, n_moments, seed)
    seq = driver.Sequence(ctx, cfg, psi, synth.sz0_spins(seed + 2, wl.walkers, wl.N),
                          synth.sz0_spins(seed + 3, wl.walkers, wl.N), graphs=not args.eager)
    # warm-up: W moments of the cycle (at least one of each target kind, so
    # every graph is captured before the timed region)
    restart(seq, cyc[0])
    for k in range(max(W, len(cyc))):
        if k and k % len(cyc) == 0:
            restart(seq, cyc[0])
        seq.fit(cycle_moment(k, cyc))
    ctx.sync_status()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    barrier(ws)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    clk_path = clock_path(f"{prec_name}_{wl_name}", rank)
    stats = []
    launches = 0  # kernels inside the timed event pairs (restarts excluded)
    with ClockSampler(clk_path, local) as clk:
        for k in range(K):
            if k % len(cyc) == 0:
                restart(seq, cyc[0])  # untimed: outside the event pair
            flush.zero_()
            l0 = ctx.n_launches() + seq.graph_launches
            ev[k][0].record(stream)
            seq.fit(cycle_moment(k, cyc))
            ev[k][1].record(stream)
            launches += ctx.n_launches() + seq.graph_launches - l0
            stats.append(seq.stats[cycle_moment(k, cyc)].clone())
        torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    barrier(ws)
    ctx.sync_status()
    step_ms = [e[0].elapsed_time(e[1]) for e in ev]
    ms = max_over_ranks(ws, float(np.mean(step_ms)))
    st = torch.stack(stats).cpu().numpy()
    clocks = clk.summary()
    kind = seq.kind_of(cycle_moment(K - 1, cyc))  # the graph buffers hold the last fitted moment
    if args.eager:
        roof = None
    elif prec_name == "mixed" and ctx.fused_cg():
        roof = roofline_fcg(ctx, seq, wl, kind, clocks)
    else:
        roof = roofline_oreduce2(ctx, seq, wl, kind, clocks)
    ctx.sync_status()
    sweeps_per_moment = cfg.n_therm + cfg.n_iter * cfg.sweeps_per_iter + cfg.sweeps_per_iter
    res = {"value": ws * 3600.0 * 1000.0 / ms, "ms_per_step": ms, "steps": K, "warmup": W,
           "mc_samples_per_s": ws * wl.walkers * sweeps_per_moment / (ms * 1e-3),
           "gpu_launches": int(round(launches)), "gpu_launches_per_step": launches / K,
           "wall_s_timed": wall, "clocks": clocks, "roofline": roof,
           **cg_summary(st, args.cg_maxit, args.cg_tol)}
    e2e_ms, Bi, Bo = e2e(seq, ctx, K, stream, cyc)
    e2e_ms = max_over_ranks(ws, e2e_ms)
    res["e2e"] = {"value": ws * 3600.0 * 1000.0 / e2e_ms, "unit": "moments/hour",
                  "h2d_bytes_per_step": Bi, "d2h_bytes_per_step": Bo}
    del flush
    return res, cfg, wl


def moment_error(args, wl_name, cyc, walkers_fp64):
    """Moment error of the timed configuration, max over the moments fitted
    in a timed cycle (mu_1 .. mu_max(cyc)), |mu_n - mu_n^ref| / mu_0:
      precision: mixed and plain float32 against the float64 GPU path, all
        three with the timed natural-gradient and CG settings, on the same
        walker configurations (replay of the float64 run's samples), at
        walkers_fp64 walkers (the full count where float64 is affordable);
      truncation: the timed mixed and plain float32 runs against the same run
        with four times the CG budget (4 cg_maxit iterations, |r| <= 1e-6 |F|),
        on the same samples, at the full walker count.
    The error of the timed configuration against a float64 solve with the
    larger budget is at most their sum.  A reference run that fails (a fit
    that turns non-finite) is reported as such instead of a number: on random
    RBMs the closer-to-exact natural-gradient step at a small shift can be
    unstable, the CG budget acting as a regulariser."""
    import torch

    from paper_2103_08804_gb300 import api, driver, synth

    wl = synth.WORKLOADS[wl_name]
    E0, a = synth.safe_rescaling(wl.Lx, wl.Ly)
    nm = 1 + max(cyc)
    seed = 4242

    class _A:
        pass

    def cfg_of(maxit, tol):
        a_ = _A()
        a_.cg_maxit, a_.cg_tol, a_.jacobi, a_.iters = maxit, tol, args.jacobi, args.iters
        return make_config(wl, E0, a, a_, nm, seed)

    torch.cuda.set_stream(torch.cuda.default_stream())
    psi = synth.rbm_params(seed, wl.N, wl.M, wl.sigma)
    out = {"moments": f"1..{nm - 1} of a sequence started as the timed cycles start"}

    def run(prec, B, cfg, s_fit, s_ref, replay=None, record=None):
        ctx = api.Context(wl.Lx, wl.Ly, wl.M, B, prec=prec)
        seq = driver.Sequence(ctx, cfg, psi, s_fit, s_ref)
        seq.start(replay_ref=None if replay is None else replay[0])
        for n in range(1, nm):
            seq.fit(n, replay=None if replay is None else replay[1][n],
                    record=None if record is None else record.setdefault(n, []))
        try:
            ctx.sync_status()
            mu = seq.mu.cpu().numpy()
        except api.CRError as e:
            mu = str(e).split(":")[1].strip()  # the status name of the failure
        ref_spins = seq.spins_ref
        del seq, ctx
        return mu, ref_spins

    def err(mu, ref):
        if isinstance(mu, str) or isinstance(ref, str):
            return f"run failed: {mu if isinstance(mu, str) else ref}"
        return float(np.max(np.abs(mu[1:] - ref[1:])) / abs(ref[0]))

    timed = cfg_of(args.cg_maxit, args.cg_tol)
    conv = cfg_of(4 * args.cg_maxit, 1e-6)
    # precision against float64, same settings, same samples
    Bp = min(walkers_fp64, wl.walkers)
    s_fit, s_ref = synth.sz0_spins(seed + 2, Bp, wl.N), synth.sz0_spins(seed + 3, Bp, wl.N)
    rec = {}
    mu64, sref = run(api.FP64, Bp, timed, s_fit, s_ref, record=rec)
    prec_err = {}
    for name, prec in (("mixed", api.MIXED), ("plain_fp32", api.FP32)):
        mu, _ = run(prec, Bp, timed, s_fit, s_ref, replay=(sref, rec))
        prec_err[name] = err(mu, mu64)
    out["precision_vs_fp64"] = {**prec_err, "walkers": Bp,
                                "reference": "float64 GPU path, same samples and settings"}
    # truncation of the timed CG, full walker count
    s_fit, s_ref = (synth.sz0_spins(seed + 2, wl.walkers, wl.N),
                    synth.sz0_spins(seed + 3, wl.walkers, wl.N))
    trunc = {}
    for name, prec in (("mixed", api.MIXED), ("plain_fp32", api.FP32)):
        rec = {}
        mu_t, sref = run(prec, wl.walkers, timed, s_fit, s_ref, record=rec)
        mu_c, _ = run(prec, wl.walkers, conv, s_fit, s_ref, replay=(sref, rec))
        trunc[name] = err(mu_t, mu_c)
    out["cg_truncation"] = {**trunc, "walkers": wl.walkers,
                            "reference": f"the same path with {4 * args.cg_maxit} CG iterations "
                                         f"(tolerance 1e-6) on the same samples"}
    for name in ("mixed", "plain_fp32"):
        a_, b_ = prec_err[name], trunc[name]
        out[name] = a_ + b_ if isinstance(a_, float) and isinstance(b_, float) else None
    out["bound"] = 1e-3
    out["note"] = ("mixed / plain_fp32: precision + truncation, an upper estimate of the error of "
                   "the timed configuration against a float64 solve with four times the CG budget "
                   "(null where a reference run failed)")
    return out


WL_TEXT = {
    "chain64": "chain64: periodic Heisenberg chain N=64, RBM alpha=2 (M=128, P=8384), 16384 "
               "walkers, q=pi/2, 50 natural-gradient iterations per moment, matrix-free CG "
               "shifted solve",
    "square16": "square16: periodic 16x16 Heisenberg lattice, RBM alpha=1 (M=256, P=66048), 65536 "
                "walkers, q=(pi,0), 50 natural-gradient iterations per moment, matrix-free CG "
                "shifted solve, then the Krylov step over 300 states",
}


def krylov_300(wl):
    """cheb_gram over 300 sampled columns of all the walkers and the float64
    generalized eigenproblem of Sec. IV (once per sequence): the mixed
    context's tensor-core Gram (timed live, with its tensor-pipe figure)
    beside the float32 context's FFMA Gram."""
    import torch

    from paper_2103_08804_gb300 import api
    Nm, Bref = 300, wl.walkers
    g = torch.Generator(device="cuda")
    g.manual_seed(7)
    Bm = torch.randn(Nm, Bref, dtype=torch.complex64, device="cuda", generator=g)
    HBm = torch.randn(Nm, Bref, dtype=torch.complex64, device="cuda", generator=g)
    G = torch.empty(Nm, Nm, dtype=torch.complex128, device="cuda")
    H = torch.empty_like(G)
    mu = torch.zeros(2 * Nm, dtype=torch.complex128, device="cuda")
    poles = torch.zeros(Nm, dtype=torch.float64, device="cuda")
    wts = torch.zeros(Nm, dtype=torch.float64, device="cuda")
    out = {}
    for name, prec in (("mixed", api.MIXED), ("fp32", api.FP32)):
        ctx = api.Context(wl.Lx, wl.Ly, wl.M, 64, prec=prec)
        ctx.cheb_gram(Bm, HBm, G, H)  # sizes the mixed path's scratch
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        reps = 5 if prec == api.MIXED else 1
        if prec == api.MIXED:
            ctx.time_kernel("gram", reps)
        ev[0].record()
        for _ in range(reps):
            ctx.cheb_gram(Bm, HBm, G, H)
        ev[1].record()
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / reps
        out[f"gram_ms_{name}"] = ms
        if prec == api.MIXED:
            kt = ctx.kernel_times()
            ctx.time_kernel(None, 0)
            kms = float(np.mean(kt)) if len(kt) else None
            flops = 2 * 8.0 * Nm * Nm * Bref
            out["gram_tc"] = {
                "kernel": "sgram_tc_kernel (G and H' tiles over K segments)",
                "kernel_ms": kms, "algorithmic_tflops": flops / (kms * 1e9) if kms else None,
                "peak_tflops": float(measured_peaks()[0]["bf16_tflops"]),
                "note": "algorithmic flops 8 Nm^2 B per matrix (G, H'); the three-term splits "
                        "execute 6x that on the tensor cores; peak: MEASURED_PEAKS.json "
                        "bf16_tflops (burst)"}
            ev2 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev2[0].record()
            ctx.cheb_krylov(G, H, 1e-10, 2 * Nm, mu, poles, wts)
            ev2[1].record()
            torch.cuda.synchronize()
            out["eigen_ms"] = ev2[0].elapsed_time(ev2[1])
        ctx.sync_status()
    out["gram_ms"] = out["gram_ms_mixed"]
    out["note"] = ("cheb_gram over 300 columns x the walkers, then cheb_krylov (pseudo-inverse, "
                   "generalized eigenproblem, 600 corrected moments); once per sequence, not in "
                   "the per-moment steps")
    return out


def extrapolation_report(n_seq=36, n_known=300, order=100, n_out=3000):
    """cheb_extrapolate (linear prediction, Sec. VI) on n_seq synthetic
    moment sequences whose continuation is known: each the moments of 40
    Lorentzian-broadened poles, mu_n = sum_k w_k r_k^n cos(n theta_k)."""
    import torch

    from paper_2103_08804_gb300 import api
    g = np.random.Generator(np.random.Philox(11))
    n = np.arange(n_out)
    mu = np.empty((n_seq, n_out), dtype=np.complex128)
    for s in range(n_seq):
        th = g.uniform(0.05, np.pi - 0.05, 40)
        w = g.exponential(1.0, 40)
        r = 1.0 - g.uniform(1e-4, 5e-3, 40)
        mu[s] = ((w[:, None] * r[:, None] ** n) * np.cos(np.outer(th, n))).sum(0) / w.sum()
    ctx = api.Context(4, 1, 4, 8, prec=api.FP64)
    x = torch.from_numpy(np.ascontiguousarray(mu[:, :n_known])).cuda()
    out = ctx.cheb_extrapolate(x, order, n_known // 2, n_out)  # sizes the scratch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = ctx.cheb_extrapolate(x, order, n_known // 2, n_out)
    e1.record()
    torch.cuda.synchronize()
    ctx.sync_status()
    got = out.cpu().numpy()
    err = float(np.max(np.abs(got - mu)) / np.max(np.abs(mu[:, 0])))
    return {"ms": e0.elapsed_time(e1), "sequences": n_seq, "known": n_known, "order": order,
            "predicted_to": n_out, "max_error_vs_closed_form": err,
            "note": "one launch, one CTA per sequence, float64: normal equations, Cholesky, "
                    "Aberth roots, Vandermonde LU, prediction; error relative to mu_0"}


def run_ours(args):
    import torch

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    wl_name = args.workload
    cyc = CYCLE if wl_name == "chain64" else SQ16_CYCLE
    cyc_note = CYCLE_NOTE if wl_name == "chain64" else SQ16_CYCLE_NOTE
    mixed, cfg, wl = measure(args, "mixed", ws, rank, local, wl_name, cyc)
    plain = None
    if not args.only_mixed:
        # the plain float32 path is 5-10x slower on the 16 x 16 lattice: fewer steps
        kp = args.steps if wl_name == "chain64" else max(2, min(args.steps, 3))
        plain = measure(args, "fp32", ws, rank, local, wl_name, cyc, K=kp,
                        W=min(args.warmup, 1))[0]
    merr = None
    if rank == 0 and not args.no_accuracy:
        merr = moment_error(args, wl_name, cyc, 16384 if wl_name == "chain64" else 4096)
    kry = krylov_300(wl) if wl_name == "square16" else None
    lp = extrapolation_report() if rank == 0 and wl_name == "square16" else None
    cgkeys = ("cg_iters_mean", "cg_iters_max", "cg_rel_residual_median", "cg_rel_residual_max",
              "cg_truncated_fraction", "cg_note")
    out = {
        "metric": "Chebyshev moments/hour",
        "value": mixed["value"],
        "unit": "moments/hour",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": mixed["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "mixed: bf16x3 tensor-core contractions with f32 accumulation, f32 elsewhere, "
                 "f64 sums and CG",
        "data": f"synthetic (random complex RBM, sigma={wl.sigma}; seeded S^z=0 walkers)",
        "config": {"workload": WL_TEXT[wl_name], "path": "mixed", "walkers": wl.walkers,
                   "iters_per_moment": cfg.n_iter, "cg_maxit": args.cg_maxit,
                   "cg_tol": args.cg_tol, "jacobi": args.jacobi,
                   "l2": "256 MiB buffer written between timed steps",
                   "launch": "eager" if args.eager else "CUDA graph per natural-gradient iteration",
                   "chunks": args.chunks, "moments": cyc_note,
                   "parallelism": f"replicas x{ws}"},
        "mc_samples_per_s": mixed["mc_samples_per_s"],
        "mc_samples_unit": "walker-sweeps/s (one sweep = N exchange proposals)",
        "gpu_launches": mixed["gpu_launches"],
        "gpu_launches_per_step": mixed["gpu_launches_per_step"],
        **{k: mixed[k] for k in cgkeys},
        "wall_s_timed": mixed["wall_s_timed"],
        "clocks": mixed["clocks"],
        "e2e": mixed["e2e"],
        "roofline": mixed["roofline"],
        "moment_error": merr,
    }
    if plain is not None:
        out["plain_fp32"] = {k: plain[k] for k in ("value", "ms_per_step", "steps", "warmup",
                                                   "mc_samples_per_s", "gpu_launches_per_step",
                                                   "e2e", "roofline", "clocks") + cgkeys}
        out["mixed_over_plain"] = mixed["value"] / plain["value"]
    if kry is not None:
        out["krylov_300"] = kry
    if lp is not None:
        out["extrapolation"] = lp
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def e2e(seq, ctx, K, stream, cyc=CYCLE):
    """Moments through the public API with host buffers: per step, copy the
    step's inputs (the two previous RBMs, their betas, the walkers) from pinned
    host memory, run the moment, read back RBM_n, beta_n and mu_n.  Steps
    follow the same moment cycle as the device-timed steps."""
    import torch
    P = ctx.P
    cd = ctx.cdtype
    h_prev = torch.empty(2, P, dtype=cd).pin_memory()
    h_beta = torch.empty(2, dtype=torch.complex128).pin_memory()
    h_spins = torch.empty_like(seq.spins, device="cpu").pin_memory()
    h_out = torch.empty(P, dtype=cd).pin_memory()
    h_res = torch.empty(2, dtype=torch.complex128).pin_memory()
    times = []
    for k in range(K):
        if k % len(cyc) == 0:
            restart(seq, cyc[0])
        n = cycle_moment(k, cyc)
        h_prev.copy_(seq.params[n - 2:n])
        h_beta.copy_(seq.betas[n - 2:n])
        h_spins.copy_(seq.spins)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        seq.params[n - 2:n].copy_(h_prev, non_blocking=True)
        seq.betas[n - 2:n].copy_(h_beta, non_blocking=True)
        seq.spins.copy_(h_spins, non_blocking=True)
        seq.fit(n)
        h_out.copy_(seq.params[n], non_blocking=True)
        h_res[0:1].copy_(seq.betas[n:n + 1], non_blocking=True)
        h_res[1:2].copy_(seq.mu[n:n + 1], non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    item = 8 if cd == torch.complex64 else 16
    Bi = 2 * P * item + 2 * 16 + seq.spins.numel()
    Bo = P * item + 2 * 16
    return float(np.mean(times)), Bi, Bo


def oracle_iteration_time(wl_name, n_walkers, seed=5, cg_sample=3, cg_maxit=50):
    """One natural-gradient iteration of the float64 oracle at the full sizes
    of the workload on n_walkers walkers: a sweep, the local target,
    the log-derivatives, the estimators and F, then the shifted solve:
    chain64 builds S and solves by Cholesky (walker-independent P x P work);
    square16 (S would take 70 GB) runs the oracle's matrix-free CG for
    cg_sample iterations, each two products with the walkers' O.
    Returns (walker part, solve part) in seconds, both scaled to the
    workload's walker count (the CG to cg_maxit iterations)."""
    from oracle import lattice, rbm, sampler, sr, target
    from oracle.target import State
    from paper_2103_08804_gb300 import synth
    wl = synth.WORKLOADS[wl_name]
    E0, a = synth.safe_rescaling(wl.Lx, wl.Ly)
    N, M = wl.N, wl.M
    psi = synth.rbm_params(seed, N, M, wl.sigma)
    p1 = synth.rbm_params(seed + 1, N, M, wl.sigma)
    p2 = synth.rbm_params(seed + 2, N, M, wl.sigma)
    spins = synth.sz0_spins(seed + 3, n_walkers, N)
    bl = lattice.bonds(wl.Lx, wl.Ly)
    scale = wl.walkers / n_walkers
    explicit = wl_name != "square16"
    t0 = time.perf_counter()
    spins, _, _ = sampler.mc_sweep(psi, N, M, bl, spins, 1, seed, 0)
    lp = rbm.logpsi(psi, N, M, spins)
    R = target.local_target(3, State(p1), State(p2), 0.5, 0.25, N, M, wl.Lx, wl.Ly, 1.0, E0, a,
                            0.9875, wl.q, spins, lp)
    O = rbm.logderiv(psi, N, M, spins)
    est = sr.estimators(O, R, with_OO=explicit)
    F, _ = sr.force(est, wl.dgamma)
    if explicit:
        S = sr.qgt(est)
    t1 = time.perf_counter()
    if explicit:
        sr.shifted_solve(S, F, wl.shift)
        t_solve = time.perf_counter() - t1
    else:
        sr.cg_solve_op(lambda v: sr.sv_matrix_free([O], v, wl.shift), F, np.ones(len(F)),
                       cg_sample, 0.0)
        t_solve = (time.perf_counter() - t1) / cg_sample * cg_maxit * scale
    return (t1 - t0) * scale, t_solve


def _moment_seconds(t_walk, t_solve, wl):
    return (t_walk + t_solve) * (wl.iters + 2)


def _oracle_sample_text(wl_name, n, tw, ts, wl):
    solve = ("Cholesky solve of the explicit S" if wl_name != "square16" else
             "matrix-free CG (3 iterations timed, scaled to 50)")
    return (f"one natural-gradient iteration of the float64 numpy oracle at N={wl.N}, M={wl.M}, "
            f"P={wl.P} on {n} walkers (walker part {tw:.1f} s and {solve} {ts:.1f} s after "
            f"scaling to {wl.walkers} walkers), times {wl.iters + 2} iterations per moment "
            f"(extrapolated)")


def default_cpu_walkers(wl_name, args):
    return args.cpu_walkers if args.cpu_walkers else (2048 if wl_name == "chain64" else 64)


def cpu_baseline(args):
    from paper_2103_08804_gb300 import synth
    wl_name = args.workload
    wl = synth.WORKLOADS[wl_name]
    cores = len(os.sched_getaffinity(0))
    n = default_cpu_walkers(wl_name, args)
    tw, ts = oracle_iteration_time(wl_name, n, cg_maxit=args.cg_maxit)
    t_moment = _moment_seconds(tw, ts, wl)
    return {"value": 3600.0 / t_moment, "unit": "moments/hour", "cores": cores, "kind": "oracle",
            "sample": _oracle_sample_text(wl_name, n, tw, ts, wl)}


def run_reference(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2103_08804_gb300 import synth
    cores = len(os.sched_getaffinity(0))
    if args.workload == "sym6":
        run_reference_sym6(args, ws, cores)
        return
    wl_name = args.workload if args.workload in ("chain64", "square16") else "chain64"
    wl = synth.WORKLOADS[wl_name]
    nw = default_cpu_walkers(wl_name, args)
    for _ in range(max(0, min(args.warmup, 1))):
        oracle_iteration_time(wl_name, 16, cg_sample=1, cg_maxit=args.cg_maxit)
    ts, walls = [], []
    for k in range(args.steps):
        t0 = time.perf_counter()
        ts.append(oracle_iteration_time(wl_name, nw, seed=5 + k, cg_maxit=args.cg_maxit))
        walls.append(time.perf_counter() - t0)
    tw, tsv = float(np.mean([t[0] for t in ts])), float(np.mean([t[1] for t in ts]))
    t_moment = _moment_seconds(tw, tsv, wl)
    value = 3600.0 / t_moment
    note = {} if args.workload == wl_name else {
        "note": f"--workload {args.workload}: the oracle arm times {wl_name}"}
    print(json.dumps({
        "impl": "reference", "metric": "Chebyshev moments/hour", "value": value,
        "unit": "moments/hour", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": float(np.mean(walls)) * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WL_TEXT[wl_name], "walkers_sampled": nw,
                   "step": "one bounded sample (one natural-gradient iteration of the oracle on "
                           "the sampled walkers); value scales it to a full moment",
                   "ms_per_moment_extrapolated": t_moment * 1e3, **note},
        "cpu_baseline": {"value": value, "unit": "moments/hour", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} samples, each " +
                                   _oracle_sample_text(wl_name, nw, tw, tsv, wl)},
        "e2e": {"value": value, "unit": "moments/hour", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def run_reference_sym6(args, ws, cores, n_samples=24):
    """The oracle's symmetry projection of the sym6 workload on the host
    cores: each step one state at n_samples samples, scaled linearly to the
    workload's states x samples."""
    Nm, B, N = SYM6["states"], SYM6["walkers"], SYM6["L"] ** 2
    for _ in range(max(0, min(args.warmup, 1))):
        sym6_oracle_seconds(4)
    per_step = float(np.mean([sym6_oracle_seconds(n_samples) for _ in range(args.steps)]))
    t_step = per_step * Nm * (B / n_samples)  # one full step of the workload, extrapolated
    value = Nm * N * 3600.0 / t_step
    sample = f"one state at {n_samples} samples per step, scaled linearly to {Nm} states x {B} samples"
    print(json.dumps({
        "impl": "reference", "metric": "symmetry-projected Chebyshev moments/hour", "value": value,
        "unit": "moments/hour", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "sym6 (see ours)", "samples_evaluated": n_samples,
                   "step": "one bounded sample (one state at the sampled configurations); "
                           "value scales it to the full step",
                   "ms_per_step_extrapolated": t_step * 1e3},
        "cpu_baseline": {"value": value, "unit": "moments/hour", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "moments/hour", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


SYM6 = {"L": 6, "M": 72, "walkers": 4096, "states": 150, "sigma": 0.02, "Wp": 0.9875}
# sym_hprime_kernel work per (antiparallel bond, hidden unit): cosh(theta - s D)
# = cosh(theta) cosh(D) - s sinh(theta) sinh(D), two complex multiplies and
# one complex subtract, then one complex multiply into the running product
SYM6_FLOP_PER_BOND_UNIT = 20


def sym6_oracle_seconds(n_samples=48):
    """The oracle's B~, HB~, G^(k) and H^(k) for one state at n_samples
    samples of the sym6 workload (host cores): seconds."""
    from oracle import rbm, symmetry
    from paper_2103_08804_gb300 import synth
    L, M = SYM6["L"], SYM6["M"]
    N = L * L
    E0, a = synth.safe_rescaling(L, L)
    st = [synth.rbm_params(1, N, M, SYM6["sigma"])]
    psi = synth.rbm_params(2, N, M, SYM6["sigma"])
    sp = synth.sz0_spins(3, n_samples, N)
    lref = rbm.logpsi(psi, N, M, sp)
    t0 = time.perf_counter()
    Bt = symmetry.b_tilde(st, N, M, L, sp, lref)
    HBt = symmetry.hb_tilde(st, N, M, L, 1.0, E0, a, SYM6["Wp"], sp, lref)
    symmetry.gram_by_momentum(Bt)
    symmetry.gram_by_momentum(Bt, HBt=HBt)
    return time.perf_counter() - t0


def run_sym6(args):
    """Symmetry projection (Appendix A) on the 6 x 6 lattice: one step =
    sym_hbtilde for 150 stored states at 4096 samples (4 N = 144 transformed
    configurations each) and cheb_gram (G and H) for each of the 36 momenta."""
    import torch

    from paper_2103_08804_gb300 import api, replicas, synth

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    L, M, B, Nm = SYM6["L"], SYM6["M"], SYM6["walkers"], SYM6["states"]
    N = L * L
    E0, a = synth.safe_rescaling(L, L)
    hp = (E0, a, SYM6["Wp"])
    seed = replicas.replica_seed(11, rank)
    ctx = api.Context(L, L, M, B, prec=api.FP32)
    stream = torch.cuda.current_stream()
    params_h = np.array([synth.rbm_params(seed + n, N, M, SYM6["sigma"]) for n in range(Nm)])
    psi_h = synth.rbm_params(seed + 1000, N, M, SYM6["sigma"])
    spins_h = synth.sz0_spins(seed + 2000, B, N)
    params = torch.tensor(params_h, dtype=torch.complex64, device="cuda")
    psi = torch.tensor(psi_h, dtype=torch.complex64, device="cuda")
    spins = torch.tensor(spins_h, device="cuda")
    lref = ctx.rbm_logpsi(psi, spins)
    wsbuf = torch.empty(int(ctx.lib.sym_h_workspace_bytes(ctx.h, B)), dtype=torch.uint8,
                        device="cuda")
    G = torch.empty(N, Nm, Nm, dtype=torch.complex128, device="cuda")
    H = torch.empty_like(G)

    def step(p, sp, lr):
        Bt, HBt = ctx.sym_hbtilde(p, sp, lr, hp, workspace=wsbuf)
        for k in range(N):
            ctx.cheb_gram(Bt[k], HBt[k], G[k], H[k])

    K, W = args.steps, max(args.warmup, 3)
    for _ in range(W):
        step(params, spins, lref)
    torch.cuda.synchronize()
    ctx.sync_status()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    clk_path = clock_path("sym6", rank)
    launches = 0
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(clk_path, local) as clk:
        for k in range(K):
            flush.zero_()
            l0 = ctx.n_launches()
            ev[k][0].record(stream)
            step(params, spins, lref)
            ev[k][1].record(stream)
            launches += ctx.n_launches() - l0
        torch.cuda.synchronize()
    barrier(ws)
    ctx.sync_status()
    ms = max_over_ranks(ws, float(np.mean([e[0].elapsed_time(e[1]) for e in ev])))
    clocks = clk.summary()
    moments = Nm * N  # mu_nk = G^(k)_0n for every state and momentum
    value = ws * moments * 3600.0 * 1000.0 / ms

    # end to end through the public API: stored states, samples and log psi
    # from pinned host memory, G^(k) and H^(k) back to pinned host memory
    pin = {"p": torch.from_numpy(params_h.astype(np.complex64)).pin_memory(),
           "s": torch.from_numpy(spins_h).pin_memory(),
           "l": lref.cpu().pin_memory()}
    G_h = torch.empty(G.shape, dtype=G.dtype).pin_memory()
    H_h = torch.empty_like(G_h).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(K):
        p = pin["p"].to("cuda", non_blocking=True)
        sp = pin["s"].to("cuda", non_blocking=True)
        lr = pin["l"].to("cuda", non_blocking=True)
        step(p, sp, lr)
        G_h.copy_(G, non_blocking=True)
        H_h.copy_(H, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(ws, e0.elapsed_time(e1) / K)
    Bi = sum(t.numel() * t.element_size() for t in pin.values())
    Bo = 2 * G_h.numel() * G_h.element_size()

    # live timing of the dominant kernel (sym_hprime_kernel, (H' t_n)(s') /
    # psi(s) at every transformed configuration), as an FP32 ALU roofline
    ctx.time_kernel("target", 4096)
    step(params, spins, lref)
    torch.cuda.synchronize()
    kt = ctx.kernel_times()
    ctx.time_kernel(None, 1)
    k_ms = float(np.mean(kt)) if kt else None
    bonds = [(r, (r % L + 1) % L + L * (r // L)) for r in range(N)]
    bonds += [(r, (r + L) % N) for r in range(N)]
    anti = sum(int(np.sum(spins_h[:, i] != spins_h[:, j])) for i, j in bonds)
    flop = 4 * N * anti * M * SYM6_FLOP_PER_BOND_UNIT  # lattice maps keep every bond
    f_sm = clocks.get("sm_mhz") or 2070.0
    peak = fp32_peak(f_sm)
    achieved = flop / (k_ms * 1e-3) / 1e12 if k_ms else None
    roof = {"kernel": "sym_hprime_kernel ((H' t_n)(s') / psi(s) of one state at 4 N B "
                      "transformed configurations, FP32 FMA over cosh/sinh bond tables)",
            "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": (achieved / peak) if achieved else None, "traffic": None,
            "work_per_launch": flop,
            "work_note": f"{SYM6_FLOP_PER_BOND_UNIT} flop per (antiparallel bond, hidden unit)",
            "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x median SM clock under load",
            "launches_timed": len(kt), "avg_launch_ms": k_ms}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        n_s = 48
        t = sym6_oracle_seconds(n_s)
        per_step = t * Nm * (B / n_s)
        cpu = {"value": moments * 3600.0 / per_step, "unit": "moments/hour",
               "cores": torch.get_num_threads(), "kind": "oracle",
               "sample": f"one state at {n_s} samples, scaled linearly to {Nm} states x {B} samples"}
    out = {
        "metric": "symmetry-projected Chebyshev moments/hour", "value": value,
        "unit": "moments/hour", "n_gpus": ws, "steps": K, "warmup": W, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (f64 local-H' sums and Gram sums)",
        "data": "synthetic (random complex RBMs, sigma=0.02; seeded S^z=0 samples)",
        "config": {"workload": f"sym6: periodic 6x6 Heisenberg lattice, alpha=2 (M={M}), "
                               f"{Nm} stored states, {B} samples, all {N} momenta: B~, HB~ "
                               "(4N = 144 transformed configurations per sample), G^(k), H^(k)",
                   "moments_per_step": moments,
                   "l2": "256 MiB buffer written between timed steps",
                   "parallelism": f"replicas x{ws}"},
        "gpu_launches": launches, "clocks": clocks,
        "e2e": {"value": ws * moments * 3600.0 * 1000.0 / e2e_ms, "unit": "moments/hour",
                "h2d_bytes_per_step": Bi, "d2h_bytes_per_step": Bo},
        "roofline": roof, "cpu_baseline": cpu,
    }
    del flush, wsbuf
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_explicit(args):
    """Explicit-S workload: one step = one moment with the Cholesky solve."""
    import torch

    from paper_2103_08804_gb300 import api, driver, replicas, synth

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    wl = synth.WORKLOADS["square10"]
    E0, a = synth.safe_rescaling(wl.Lx, wl.Ly)
    K, W = args.steps, args.warmup
    n_moments = 1 + max(CYCLE)
    seed = replicas.replica_seed(2000, rank)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = api.Context(wl.Lx, wl.Ly, wl.M, wl.walkers, prec=api.MIXED, explicit_s=True,
                      stream=stream)
    cfg = make_config(wl, E0, a, args, n_moments, seed, solver=api.SOLVE_CHOLESKY)
    psi = synth.rbm_params(seed, wl.N, wl.M, wl.sigma)
    seq = driver.Sequence(ctx, cfg, psi, synth.sz0_spins(seed + 2, wl.walkers, wl.N),
                          synth.sz0_spins(seed + 3, wl.walkers, wl.N), graphs=not args.eager)
    restart(seq)
    for k in range(max(W, len(CYCLE))):
        if k and k % len(CYCLE) == 0:
            restart(seq)
        seq.fit(cycle_moment(k))
    ctx.sync_status()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    barrier(ws)
    torch.cuda.synchronize()
    launches0 = ctx.n_launches() + seq.graph_launches
    clk_path = clock_path("square10", rank)
    stats = []
    launches = 0  # kernels inside the timed event pairs (restarts excluded)
    with ClockSampler(clk_path, local) as clk:
        for k in range(K):
            if k % len(CYCLE) == 0:
                restart(seq)  # untimed: outside the event pair
            flush.zero_()
            l0 = ctx.n_launches() + seq.graph_launches
            ev[k][0].record(stream)
            seq.fit(cycle_moment(k))
            ev[k][1].record(stream)
            launches += ctx.n_launches() + seq.graph_launches - l0
            stats.append(seq.stats[cycle_moment(k)].clone())
        torch.cuda.synchronize()
    barrier(ws)
    del launches0
    ms = max_over_ranks(ws, float(np.mean([e[0].elapsed_time(e[1]) for e in ev])))
    clocks = clk.summary()
    st = torch.stack(stats).cpu().numpy()
    # live kernel times on eager iterations of the same step: the Gram kernel,
    # and the whole natural-gradient update (S, factor, refined solve)
    if args.eager:
        raise SystemExit("--workload square10 times its kernels on the graph-mode buffers")
    # (on a restarted sequence: a few more iterations of moment 2, whose fit is
    # settled, rather than of the last timed moment, whose later iterations
    # can turn non-finite on these random RBMs)
    restart(seq)
    torch.cuda.synchronize()
    ctx.time_kernel("sbuild", 64)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    n_eager = 2
    kind = seq.kind_of(CYCLE[0] - 1)  # the graph buffers hold the last fitted moment
    for _ in range(n_eager):
        seq._iteration(kind)
    e1.record(stream)
    torch.cuda.synchronize()
    gram_ms = float(np.mean(ctx.kernel_times()))
    iter_ms = e0.elapsed_time(e1) / n_eager
    ctx.time_kernel("chol", 20000)
    seq._iteration(kind)
    torch.cuda.synchronize()
    chol_ms = float(np.sum(ctx.kernel_times()))
    ctx.time_kernel("trsv", 20000)
    seq._iteration(kind)
    torch.cuda.synchronize()
    trsv_ms = float(np.sum(ctx.kernel_times()))
    ctx.time_kernel(None, 1)
    ctx.sync_status()
    # tensor-core S against a float64 context on a walker sample
    Bs = min(args.s_error_walkers, wl.walkers)
    ref = api.Context(wl.Lx, wl.Ly, wl.M, Bs, prec=api.FP64, explicit_s=True, stream=stream)
    sp = seq.spins[:Bs].contiguous()
    th = torch.empty(Bs, wl.M, dtype=torch.complex128, device="cuda")
    p_last = seq.params[cycle_moment(K - 1)].to(torch.complex128)
    ref.rbm_logpsi(p_last, sp, th)
    T64 = torch.empty_like(th)
    ref.logderiv(p_last, sp, th, tanh_out=T64)
    S64 = ref.sr_smatrix(sp, T64, wl.shift)
    nrm = torch.linalg.norm(S64)
    S32 = ctx.sr_smatrix(sp, T64.to(torch.complex64), wl.shift)
    ctx.sync_status()
    s_err = float(torch.linalg.norm(S32 - S64) / nrm)
    del S32
    x3 = api.Context(wl.Lx, wl.Ly, wl.M, Bs, prec=api.MIXED, explicit_s=True, stream=stream,
                     s_bf16x3=True)
    S32 = x3.sr_smatrix(sp, T64.to(torch.complex64), wl.shift)
    x3.sync_status()
    ref.sync_status()
    s_err_x3 = float(torch.linalg.norm(S32 - S64) / nrm)
    del S64, S32, ref, x3
    P, B = wl.P, wl.walkers
    flops = 8.0 * P * (P + 1) / 2 * B          # Hermitian half of O^dag O, complex MACs x 8
    peaks, peak_src = measured_peaks()
    peak = float(peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]))
    achieved = flops / (gram_ms * 1e-3) / 1e12
    roof = {"kernel": "sgram_tc_kernel<3> (tcgen05, three-term bf16 splits: six bf16 "
                      "products per float32 product, float32 accumulation in TMEM)",
            "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None, "work_per_launch": flops,
            "avg_launch_ms": gram_ms,
            "peak_source": f"MEASURED_PEAKS.json bf16_tflops_sustained ({peak_src}); six bf16 "
                           f"products per product, so frac <= 1/6"}
    sweeps_per_moment = cfg.n_therm + cfg.n_iter * cfg.sweeps_per_iter + cfg.sweeps_per_iter
    e2e_ms, Bi, Bo = e2e(seq, ctx, K, stream)
    e2e_ms = max_over_ranks(ws, e2e_ms)
    out = {
        "metric": "Chebyshev moments/hour", "value": ws * 3600.0 * 1000.0 / ms,
        "unit": "moments/hour", "n_gpus": ws, "steps": K, "warmup": W, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "mixed: S on tensor cores from three-term bf16 splits (six products, f32 "
                 "accumulation), f32 Cholesky factor, f64 refinement, f32 elsewhere",
        "data": "synthetic (random complex RBM, sigma=0.01; seeded S^z=0 walkers)",
        "config": {"workload": "square10: periodic 10x10 Heisenberg lattice, RBM alpha=1 (M=100, "
                               "P=10200), 32768 walkers, q=(pi,pi), explicit S + Cholesky",
                   "iters_per_moment": cfg.n_iter, "l2": "256 MiB buffer written between timed steps",
                   "launch": "eager" if args.eager else "CUDA graph per natural-gradient iteration",
                   "moments": CYCLE_NOTE, "parallelism": f"replicas x{ws}"},
        "mc_samples_per_s": ws * wl.walkers * sweeps_per_moment / (ms * 1e-3),
        "gpu_launches": int(launches), "clocks": clocks,
        "e2e": {"value": ws * 3600.0 * 1000.0 / e2e_ms, "unit": "moments/hour",
                "h2d_bytes_per_step": Bi, "d2h_bytes_per_step": Bo},
        "roofline": roof,
        "s_rel_error_vs_fp64": s_err,
        "s_rel_error_vs_fp64_bf16x3": s_err_x3,
        "s_error_sample": f"{Bs} walkers of the fit set, RBM of the last fitted moment",
        "iteration_ms": iter_ms, "sbuild_ms": gram_ms,
        "factor_ms": chol_ms, "trsv_ms": trsv_ms,
        "factor_note": "factor_ms: blocked factor (potrf, trsm, syrk kernels) of one iteration; "
                       "trsv_ms: the triangular solves of all its refinement steps",
        "refine_steps_mean": float(st[..., 5].mean()),
        "refine_residual_max": float(st[..., 6].max()),
    }
    del flush
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_batch(args):
    """Momentum scan: every sequence advances one moment per step."""
    import torch

    from paper_2103_08804_gb300 import api, batch, replicas, synth

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    K, W = args.steps, args.warmup
    n_moments = 1 + max(CYCLE)
    iters = 50 if args.iters is None else args.iters
    specs = batch.momentum_scan_specs(L=8, alpha=2, chains=(48, 96), walkers=8192,
                                      n_moments=n_moments, n_iter=iters, sigma=0.02,
                                      seed=1000, n_therm=2, n_therm_ref=20,
                                      solver=api.SOLVE_CG, cg_maxit=args.cg_maxit,
                                      cg_tol=args.cg_tol, jacobi=args.jacobi)
    specs = replicas.shard_specs(specs, rank, ws)  # sequence sharding: disjoint shares
    main = torch.cuda.Stream()
    torch.cuda.set_stream(main)
    t0 = time.perf_counter()
    b = batch.Batch(specs, prec=api.MIXED, tune=True)
    tune_s = time.perf_counter() - t0
    n_seq = len(b.seqs)
    n_seq_all = int(replicas.sum_over_ranks(ws, n_seq))
    # The autotuner timed the batched iteration graph on throwaway sequences
    # over the fused-CG CTA counts and the reduction chunk counts, and applied
    # the fastest setting.
    tuned = {"chunks": dict(zip([s.name for s in b.active], b.chunks)),
             "fcg_ctas": dict(zip([s.name for s in b.active], b.ctas)),
             "iteration_ms_default": b.timings[("max",)],
             "iteration_ms_tuned": b.tuned_ms,
             "speedup": b.timings[("max",)] / b.tuned_ms, "applied": True}

    def brestart():
        b.start()
        b.fit(1)
        b.fit(2)

    for k in range(max(W, 1)):
        brestart()
        b.fit(cycle_moment(k, BATCH_CYCLE))
    for c in b.ctxs:
        c.sync_status()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    clk_path = clock_path("batch", rank)
    res = {}
    with ClockSampler(clk_path, local) as clk:
        for schedule in ("batched", "per_q"):
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(K)]
            barrier(ws)
            torch.cuda.synchronize()
            launches = 0
            for k in range(K):
                brestart()  # untimed: outside the event pair
                flush.zero_()
                l0 = sum(c.n_launches() for c in b.ctxs) + b.graph_launches
                ev[k][0].record(main)
                b.fit(cycle_moment(k, BATCH_CYCLE), schedule=schedule)
                ev[k][1].record(main)
                launches += sum(c.n_launches() for c in b.ctxs) + b.graph_launches - l0
            torch.cuda.synchronize()
            barrier(ws)
            ms = max_over_ranks(ws, float(np.mean([e[0].elapsed_time(e[1]) for e in ev])))
            res[schedule] = {"ms_per_step": ms, "value": n_seq_all * 3600.0 * 1000.0 / ms,
                             "gpu_launches": int(launches)}
    clocks = clk.summary()
    for c in b.ctxs:
        c.sync_status()
    # end to end: every sequence's inputs from pinned host buffers, results back
    seqs = b.seqs
    h_in = [(torch.empty(2, s.ctx.P, dtype=s.ctx.cdtype).pin_memory(),
             torch.empty(2, dtype=torch.complex128).pin_memory(),
             torch.empty_like(s.spins, device="cpu").pin_memory()) for s in seqs]
    h_out = [(torch.empty(s.ctx.P, dtype=s.ctx.cdtype).pin_memory(),
              torch.empty(2, dtype=torch.complex128).pin_memory()) for s in seqs]
    e2e_ms = []
    for k in range(K):
        brestart()
        m = cycle_moment(k, BATCH_CYCLE)
        for s, (hp, hb, hs) in zip(seqs, h_in):
            hp.copy_(s.params[m - 2:m])
            hb.copy_(s.betas[m - 2:m])
            hs.copy_(s.spins)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main)
        for s, (hp, hb, hs) in zip(seqs, h_in):
            s.params[m - 2:m].copy_(hp, non_blocking=True)
            s.betas[m - 2:m].copy_(hb, non_blocking=True)
            s.spins.copy_(hs, non_blocking=True)
        b.fit(m)
        for s, (ho, hr) in zip(seqs, h_out):
            ho.copy_(s.params[m], non_blocking=True)
            hr[0:1].copy_(s.betas[m:m + 1], non_blocking=True)
            hr[1:2].copy_(s.mu[m:m + 1], non_blocking=True)
        e1.record(main)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_v = max_over_ranks(ws, float(np.mean(e2e_ms)))
    Bi = sum(hp.numel() * hp.element_size() + 32 + hs.numel() for hp, _, hs in h_in)
    Bo = sum(ho.numel() * ho.element_size() + 32 for ho, _ in h_out)
    sq = next(i for i, s in enumerate(b.active) if s.cfg.Ly > 1)
    b._fork()
    with torch.cuda.stream(b.streams[sq]):
        roof = roofline_fcg(b.ctxs[sq], seqs[sq], synth.WORKLOADS["square8"],
                            seqs[sq].kind_of(cycle_moment(K - 1, BATCH_CYCLE)), clocks)
    b._join()
    for c in b.ctxs:
        c.sync_status()
    bt, pq = res["batched"], res["per_q"]
    out = {
        "metric": "Chebyshev moments/hour", "value": bt["value"], "unit": "moments/hour",
        "n_gpus": ws, "steps": K, "warmup": W, "ms_per_step": bt["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "mixed: bf16x3 tensor-core contractions with f32 accumulation, f32 elsewhere, "
                 "f64 sums and CG",
        "data": "synthetic (random complex RBMs, sigma=0.02; seeded S^z=0 walkers)",
        "config": {"workload": "momentum scan: 8x8 square lattice at its 15 irreducible q "
                               "(q=0 skipped: vanishing probe) + chains N=48 and N=96 at q=pi/2, "
                               "alpha=2, 8192 walkers each, one moment of every sequence per step",
                   "sequences": n_seq_all, "sequences_per_rank": n_seq, "skipped": b.skipped,
                   "iters_per_moment": iters,
                   "cg_maxit": args.cg_maxit, "cg_tol": args.cg_tol,
                   "chunks": dict(zip([s.name for s in b.active], b.chunks)),
                   "autotune": tuned, "autotune_s": tune_s, "l2": "256 MiB buffer written between timed steps",
                   "launch": "one CUDA graph per iteration holding every sequence (forked streams)",
                   "moments": BATCH_CYCLE_NOTE,
                   "parallelism": f"sequences sharded over {ws} rank(s), no collective"},
        "gpu_launches": bt["gpu_launches"],
        "clocks": clocks,
        "e2e": {"value": n_seq_all * 3600.0 * 1000.0 / e2e_v, "unit": "moments/hour",
                "h2d_bytes_per_step": Bi, "d2h_bytes_per_step": Bo},
        "roofline": roof,
        "per_q": pq,
        "batched_over_per_q": bt["value"] / pq["value"],
    }
    del flush
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "batch":
        run_batch(a)
    elif a.workload == "square10":
        run_explicit(a)
    elif a.workload == "sym6":
        run_sym6(a)
    else:
        run_ours(a)
