"""Thin Python binding of libchebrbm (include/chebrbm.h).

Argument marshalling only: every function here checks tensor shapes and
dtypes, takes raw device pointers and calls the C function of the same name.
All compute runs in the library's CUDA kernels.  There is no CPU fallback:
if the library is missing or CUDA is unavailable, loading fails loudly.
"""

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libchebrbm.so")

FP64, FP32, MIXED = 0, 1, 2
SOLVE_CHOLESKY, SOLVE_CG = 0, 1
CTX_EXPLICIT_S = 1
CTX_S_BF16X3 = 2
SR_FIT = 0
SR_ENERGY = 1
STATS_LEN = 8
STATUS = {0: "CR_OK", 1: "CR_EINVAL", 2: "CR_ENOMEM", 3: "CR_ECUDA", 4: "CR_ETIMEOUT",
          5: "CR_ENOTCONV", 6: "CR_ESINGULAR", 7: "CR_ENONFINITE"}

# Every exported symbol of include/chebrbm.h.
SYMBOLS = ("cr_create", "cr_destroy", "cr_set_stream", "cr_last_error", "cr_sync_status",
           "cr_n_sites", "cr_n_hidden", "cr_n_params", "cr_n_bonds", "rbm_logpsi", "mc_sweep",
           "cheb_local_target", "logderiv", "logpsi_backward", "sr_step", "cheb_moment",
           "cheb_gram", "cheb_krylov", "cr_n_launches", "cr_time_kernel", "cr_kernel_times",
           "logpsi_backward_noalloc", "cr_set_chunks", "cr_max_chunks", "sr_smatrix",
           "cheb_spectrum", "cheb_lorentzian", "cheb_extrapolate", "sym_workspace_bytes", "sym_btilde",
           "sym_h_workspace_bytes", "sym_hbtilde", "cheb_init_params", "sr_sv", "cr_fused_cg",
           "cr_set_fcg_ctas", "cr_batch_run")
KERNEL = {"sweep": 0, "target": 1, "theta": 2, "ov": 3, "reduce": 4, "cg": 5, "sbuild": 6,
          "chol": 7, "trsv": 8, "fcg": 9, "gram": 10}


class Lattice(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_int), ("Ly", ctypes.c_int), ("J", ctypes.c_double)]


class State(ctypes.Structure):
    _fields_ = [("params", ctypes.c_void_p), ("probe", ctypes.c_int),
                ("qx", ctypes.c_double), ("qy", ctypes.c_double)]


class Philox(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("counter", ctypes.c_uint64),
                ("device_counter", ctypes.c_void_p)]


class Target(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("prev", State), ("prev2", State),
                ("beta_prev", ctypes.c_void_p), ("beta_prev2", ctypes.c_void_p),
                ("E0", ctypes.c_double), ("a", ctypes.c_double), ("Wp", ctypes.c_double)]


class SROpts(ctypes.Structure):
    _fields_ = [("dgamma", ctypes.c_double), ("shift", ctypes.c_double),
                ("solver", ctypes.c_int), ("cg_maxit", ctypes.c_int),
                ("cg_tol", ctypes.c_double), ("cg_precond", ctypes.c_int), ("mode", ctypes.c_int),
                ("cg_strict", ctypes.c_int)]


class SeqIter(ctypes.Structure):
    """cr_seq_iter: one sequence's part of a cr_batch_run call."""
    _fields_ = [("ctx", ctypes.c_void_p), ("params", ctypes.c_void_p), ("spins", ctypes.c_void_p),
                ("theta", ctypes.c_void_p), ("tanh_theta", ctypes.c_void_p),
                ("logpsi", ctypes.c_void_p), ("R", ctypes.c_void_p), ("B", ctypes.c_int),
                ("n_sweeps", ctypes.c_int), ("target", Target), ("opts", SROpts),
                ("rng", ctypes.POINTER(Philox)), ("stats", ctypes.c_void_p)]


_lib = None


def load(path=None):
    """Load libchebrbm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libchebrbm.so not built ({p}); run paper_2103_08804_gb300.build")
    lib = ctypes.CDLL(p)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.cr_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Lattice), i, i, i, i, vp]
    lib.cr_destroy.argtypes = [vp]
    lib.cr_set_stream.argtypes = [vp, vp]
    lib.cr_last_error.argtypes = [vp]
    lib.cr_last_error.restype = ctypes.c_char_p
    lib.cr_sync_status.argtypes = [vp]
    for f in ("cr_n_sites", "cr_n_hidden", "cr_n_params", "cr_n_bonds", "cr_fused_cg"):
        getattr(lib, f).argtypes = [vp]
    lib.rbm_logpsi.argtypes = [vp, ctypes.POINTER(State), vp, i, vp, vp]
    lib.mc_sweep.argtypes = [vp, ctypes.POINTER(State), vp, vp, i, i, ctypes.POINTER(Philox),
                             vp, vp, vp]
    lib.cheb_local_target.argtypes = [vp, ctypes.POINTER(Target), vp, vp, i, vp, vp]
    lib.logderiv.argtypes = [vp, ctypes.POINTER(State), vp, vp, i, vp, vp]
    lib.logpsi_backward.argtypes = [vp, ctypes.POINTER(State), vp, vp, i, vp, vp]
    lib.sr_step.argtypes = [vp, vp, vp, vp, vp, i, ctypes.POINTER(SROpts), vp]
    lib.cheb_moment.argtypes = [vp, ctypes.POINTER(State), vp, d, d, vp, vp, i,
                                ctypes.POINTER(d), vp, vp, vp]
    lib.cheb_gram.argtypes = [vp, vp, vp, i, i, i, vp, vp]
    lib.cheb_krylov.argtypes = [vp, vp, vp, i, d, i, vp, vp, vp, vp]
    lib.cr_n_launches.argtypes = [vp]
    lib.cr_n_launches.restype = ctypes.c_longlong
    lib.cr_time_kernel.argtypes = [vp, i, i]
    lib.cr_kernel_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float), i]
    lib.cr_set_chunks.argtypes = [vp, i]
    lib.sr_smatrix.argtypes = [vp, vp, vp, i, d, vp]
    lib.cheb_spectrum.argtypes = [vp, vp, i, d, d, i, vp, i, vp]
    lib.sym_workspace_bytes.argtypes = [vp, i]
    lib.sym_workspace_bytes.restype = ctypes.c_size_t
    lib.sym_btilde.argtypes = [vp, ctypes.POINTER(State), i, vp, vp, i, vp, ctypes.c_size_t, vp]
    lib.sym_h_workspace_bytes.argtypes = [vp, i]
    lib.sym_h_workspace_bytes.restype = ctypes.c_size_t
    lib.sym_hbtilde.argtypes = [vp, ctypes.POINTER(State), i, vp, vp, i,
                                ctypes.POINTER(ctypes.c_double), vp, ctypes.c_size_t, vp, vp]
    lib.cheb_lorentzian.argtypes = [vp, vp, vp, i, d, d, d, vp, i, vp]
    lib.cheb_extrapolate.argtypes = [vp, vp, i, i, i, i, d, i, vp, vp, vp]
    lib.cr_max_chunks.argtypes = [vp]
    lib.logpsi_backward_noalloc.argtypes = [i, i, i, vp, vp, i, vp, vp, vp, ctypes.c_char_p, i]
    lib.cheb_init_params.argtypes = [vp, i, vp, vp, vp]
    lib.sr_sv.argtypes = [vp, vp, vp, i, vp, d, vp, vp]
    lib.cr_set_fcg_ctas.argtypes = [vp, i]
    lib.cr_batch_run.argtypes = [ctypes.POINTER(SeqIter), i, i, vp]
    for f in SYMBOLS:
        if f not in ("cr_last_error", "cr_n_sites", "cr_n_hidden", "cr_n_params", "cr_n_bonds", "cr_fused_cg",
                     "cr_n_launches", "cr_max_chunks", "sym_workspace_bytes",
                     "sym_h_workspace_bytes"):
            getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


class CRError(RuntimeError):
    pass


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Context:
    """One lattice, one hidden width, one precision; owns the library context."""

    def __init__(self, Lx, Ly, M, max_walkers, prec=FP32, explicit_s=False, J=1.0, stream=None,
                 s_bf16x3=False):
        if not torch.cuda.is_available():
            raise RuntimeError("libchebrbm needs a CUDA device")
        self.lib = load()
        self.Lx, self.Ly, self.M, self.J = Lx, Ly, M, J
        self.N = Lx * Ly
        self.prec = prec
        self.max_walkers = max_walkers
        self.cdtype = torch.complex128 if prec == FP64 else torch.complex64
        st = torch.cuda.current_stream() if stream is None else stream
        self._stream = st
        h = ctypes.c_void_p()
        lat = Lattice(Lx, Ly, J)
        s = self.lib.cr_create(ctypes.byref(h), ctypes.byref(lat), M, max_walkers, prec,
                               (CTX_EXPLICIT_S if explicit_s else 0) |
                               (CTX_S_BF16X3 if s_bf16x3 else 0), ctypes.c_void_p(st.cuda_stream))
        if s != 0:
            raise CRError(f"cr_create failed: {STATUS.get(s, s)}")
        self.h = h
        self.P = self.lib.cr_n_params(h)
        self.n_bonds = self.lib.cr_n_bonds(h)

    def close(self):
        if getattr(self, "h", None):
            self.lib.cr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ helpers
    def _check(self, s, what):
        if s != 0:
            msg = self.lib.cr_last_error(self.h).decode(errors="replace")
            raise CRError(f"{what}: {STATUS.get(s, s)}: {msg}")

    def set_stream(self, stream):
        self._stream = stream
        self._check(self.lib.cr_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream)),
                    "cr_set_stream")

    def set_chunks(self, n_chunks):
        """Walker chunks of the split-K reductions (1 .. max_chunks())."""
        self._check(self.lib.cr_set_chunks(self.h, int(n_chunks)), "cr_set_chunks")

    def max_chunks(self):
        return int(self.lib.cr_max_chunks(self.h))

    def fused_cg(self):
        """True when sr_step's CG runs as one fused persistent kernel here."""
        return int(self.lib.cr_fused_cg(self.h)) == 1

    def set_fcg_ctas(self, n_ctas):
        """CTAs of the fused CG kernel (0: one per SM)."""
        self._check(self.lib.cr_set_fcg_ctas(self.h, int(n_ctas)), "cr_set_fcg_ctas")

    def target(self, n, prev, prev2, beta_prev, beta_prev2, E0, a, Wp):
        """The cr_target of projection step n (prev / prev2: State structs,
        beta_*: device complex128 scalars)."""
        tg = Target()
        tg.n = n
        tg.prev = prev
        if prev2 is not None:
            tg.prev2 = prev2
        tg.beta_prev = beta_prev.data_ptr()
        tg.beta_prev2 = beta_prev2.data_ptr() if beta_prev2 is not None else None
        tg.E0, tg.a, tg.Wp = E0, a, Wp
        return tg

    def sync_status(self):
        self._check(self.lib.cr_sync_status(self.h), "device status")

    def n_launches(self):
        return int(self.lib.cr_n_launches(self.h))

    def time_kernel(self, kernel, capacity):
        """Arm event timing of one kernel family (name in KERNEL, or None to disarm)."""
        kid = -1 if kernel is None else KERNEL[kernel]
        self._check(self.lib.cr_time_kernel(self.h, kid, capacity), "cr_time_kernel")
        self._kt_cap = capacity

    def kernel_times(self):
        """Durations (ms) of the timed launches so far."""
        cap = getattr(self, "_kt_cap", 0)
        buf = (ctypes.c_float * max(cap, 1))()
        n = self.lib.cr_kernel_times(self.h, buf, cap)
        if n < 0:
            raise CRError("cr_kernel_times failed")
        return [buf[k] for k in range(n)]

    def _c(self, t, shape, name):
        if t is None:
            return
        if not (t.is_cuda and t.dtype == self.cdtype and t.is_contiguous()):
            raise ValueError(f"{name}: need a contiguous CUDA {self.cdtype} tensor")
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name}: shape {tuple(t.shape)} != {tuple(shape)}")

    def _spins(self, s):
        if not (s.is_cuda and s.dtype == torch.int8 and s.is_contiguous() and s.dim() == 2
                and s.shape[1] == self.N):
            raise ValueError("spins: need a contiguous CUDA int8 [B, N] tensor")
        return s.shape[0]

    def state(self, params, probe=False, q=(0.0, 0.0)):
        self._c(params, (self.P,), "params")
        st = State(params.data_ptr(), 1 if probe else 0, float(q[0]), float(q[1]))
        st._keep = params
        return st

    # ---------------------------------------------------------- hot path
    def rbm_logpsi(self, params, spins, theta_out=None, logpsi_out=None):
        B = self._spins(spins)
        if logpsi_out is None:
            logpsi_out = torch.empty(B, dtype=self.cdtype, device=spins.device)
        self._c(theta_out, (B, self.M), "theta_out")
        self._c(logpsi_out, (B,), "logpsi_out")
        st = self.state(params)
        self._check(self.lib.rbm_logpsi(self.h, ctypes.byref(st), _ptr(spins), B, _ptr(theta_out),
                                        _ptr(logpsi_out)), "rbm_logpsi")
        return logpsi_out

    def mc_sweep(self, params, spins, theta, n_sweeps, rng, logpsi_out=None, tanh_out=None,
                 n_accepted=None):
        B = self._spins(spins)
        self._c(theta, (B, self.M), "theta")
        self._c(logpsi_out, (B,), "logpsi_out")
        self._c(tanh_out, (B, self.M), "tanh_out")
        if n_accepted is not None and not (n_accepted.dtype == torch.int32 and n_accepted.is_cuda
                                           and n_accepted.shape == (B,)):
            raise ValueError("n_accepted: need a CUDA int32 [B] tensor")
        st = self.state(params)
        self._check(self.lib.mc_sweep(self.h, ctypes.byref(st), _ptr(spins), _ptr(theta), B,
                                      n_sweeps, ctypes.byref(rng), _ptr(logpsi_out),
                                      _ptr(tanh_out), _ptr(n_accepted)), "mc_sweep")

    def cheb_local_target(self, n, prev, prev2, beta_prev, beta_prev2, E0, a, Wp, spins,
                          logpsi_n, R_out=None, mean_out=None):
        """prev / prev2: State structs (see state()); beta_*: device complex128 scalars."""
        B = self._spins(spins)
        self._c(logpsi_n, (B,), "logpsi_n")
        if R_out is None:
            R_out = torch.empty(B, dtype=self.cdtype, device=spins.device)
        self._c(R_out, (B,), "R_out")
        for bt in (beta_prev, beta_prev2, mean_out):
            if bt is not None and not (bt.is_cuda and bt.dtype == torch.complex128):
                raise ValueError("beta / mean_out: need CUDA complex128 scalars")
        tg = self.target(n, prev, prev2, beta_prev, beta_prev2, E0, a, Wp)
        self._check(self.lib.cheb_local_target(self.h, ctypes.byref(tg), _ptr(spins),
                                               _ptr(logpsi_n), B, _ptr(R_out), _ptr(mean_out)),
                    "cheb_local_target")
        return R_out

    def logderiv(self, params, spins, theta, tanh_out=None, O_out=None):
        B = self._spins(spins)
        self._c(theta, (B, self.M), "theta")
        self._c(tanh_out, (B, self.M), "tanh_out")
        self._c(O_out, (B, self.P), "O_out")
        st = self.state(params)
        self._check(self.lib.logderiv(self.h, ctypes.byref(st), _ptr(spins), _ptr(theta), B,
                                      _ptr(tanh_out), _ptr(O_out)), "logderiv")

    def logpsi_backward(self, params, spins, tanh_theta, grad_logpsi, grad_params=None):
        B = self._spins(spins)
        self._c(tanh_theta, (B, self.M), "tanh_theta")
        self._c(grad_logpsi, (B,), "grad_logpsi")
        if grad_params is None:
            grad_params = torch.empty(self.P, dtype=self.cdtype, device=spins.device)
        self._c(grad_params, (self.P,), "grad_params")
        st = self.state(params)
        self._check(self.lib.logpsi_backward(self.h, ctypes.byref(st), _ptr(spins),
                                             _ptr(tanh_theta), B, _ptr(grad_logpsi),
                                             _ptr(grad_params)), "logpsi_backward")
        return grad_params

    def cheb_init_params(self, n, psi, prev, out):
        """Starting parameters of projection step n into out (n == 1: psi with
        a_0 += i pi/2; n >= 2: prev)."""
        self._c(out, (self.P,), "out")
        self._c(psi, (self.P,), "psi")
        self._c(prev, (self.P,), "prev")
        self._check(self.lib.cheb_init_params(self.h, int(n), _ptr(psi), _ptr(prev), _ptr(out)),
                    "cheb_init_params")
        return out

    def sr_sv(self, spins, tanh_theta, v, shift, u_out=None, out=None):
        """(S + shift I) v through the CG's product kernels (v, out complex128 [P]);
        u_out (context precision [B]) receives O v."""
        B = self._spins(spins)
        self._c(tanh_theta, (B, self.M), "tanh_theta")
        self._c(u_out, (B,), "u_out")
        for t, name in ((v, "v"), (out, "out")):
            if t is not None and not (t.is_cuda and t.dtype == torch.complex128
                                      and t.is_contiguous() and tuple(t.shape) == (self.P,)):
                raise ValueError(f"{name}: need a contiguous CUDA complex128 [P] tensor")
        if out is None:
            out = torch.empty(self.P, dtype=torch.complex128, device=spins.device)
        self._check(self.lib.sr_sv(self.h, _ptr(spins), _ptr(tanh_theta), B, _ptr(v), float(shift),
                                   _ptr(u_out), _ptr(out)), "sr_sv")
        return out

    def sr_step(self, params, spins, tanh_theta, R, dgamma, shift, solver=SOLVE_CG, cg_maxit=100,
                cg_tol=1e-6, stats_out=None, jacobi=False, mode=0, cg_strict=False):
        B = self._spins(spins)
        self._c(params, (self.P,), "params")
        self._c(tanh_theta, (B, self.M), "tanh_theta")
        self._c(R, (B,), "R")
        if stats_out is not None and not (stats_out.dtype == torch.float64 and stats_out.is_cuda
                                          and stats_out.numel() >= STATS_LEN):
            raise ValueError("stats_out: need a CUDA float64 tensor of 8 entries")
        o = SROpts(dgamma, shift, solver, cg_maxit, cg_tol, 1 if jacobi else 0, int(mode),
                   1 if cg_strict else 0)
        self._check(self.lib.sr_step(self.h, _ptr(params), _ptr(spins), _ptr(tanh_theta), _ptr(R),
                                     B, ctypes.byref(o), _ptr(stats_out)), "sr_step")

    def sr_smatrix(self, spins, tanh_theta, shift, S_out=None):
        """Explicit S + shift I (complex128 [P, P]) as built by the Cholesky path."""
        B = self._spins(spins)
        self._c(tanh_theta, (B, self.M), "tanh_theta")
        if S_out is None:
            S_out = torch.empty(self.P, self.P, dtype=torch.complex128, device=spins.device)
        if not (S_out.dtype == torch.complex128 and S_out.is_cuda and S_out.is_contiguous()
                and tuple(S_out.shape) == (self.P, self.P)):
            raise ValueError("S_out: need a contiguous CUDA complex128 [P, P] tensor")
        self._check(self.lib.sr_smatrix(self.h, _ptr(spins), _ptr(tanh_theta), B, float(shift),
                                        _ptr(S_out)), "sr_smatrix")
        return S_out

    def _sym_args(self, params, spins, logpsi_ref):
        B = self._spins(spins)
        self._c(logpsi_ref, (B,), "logpsi_ref")
        Nm = params.shape[0]
        if params.dtype != self.cdtype or tuple(params.shape) != (Nm, self.P) \
                or not params.is_contiguous():
            raise ValueError("params: contiguous [Nm, P] in the context precision")
        sts = (State * Nm)(*[self.state(params[n]) for n in range(Nm)])
        return B, Nm, sts

    def sym_btilde(self, params, spins, logpsi_ref, workspace=None):
        """Appendix A: B~_nk(s) for the stored states params [Nm, P] (plain
        RBMs) at the samples; returns [L*L, Nm, B] (momentum k1 + L k2)."""
        B, Nm, sts = self._sym_args(params, spins, logpsi_ref)
        need = int(self.lib.sym_workspace_bytes(self.h, B))
        if workspace is None or workspace.numel() < need:
            workspace = torch.empty(need, dtype=torch.uint8, device=spins.device)
        out = torch.empty(self.N, Nm, B, dtype=self.cdtype, device=spins.device)
        self._check(self.lib.sym_btilde(self.h, sts, Nm, _ptr(spins), _ptr(logpsi_ref), B,
                                        _ptr(workspace), need, _ptr(out)), "sym_btilde")
        return out

    def sym_hbtilde(self, params, spins, logpsi_ref, hprime, workspace=None):
        """Appendix A: (B~_nk(s), HB~_nk(s) = <s|H'|t~_nk> / psi(s)) for the
        stored states params [Nm, P] at the samples, H' from hprime =
        (E0, a, W'); each [L*L, Nm, B] (momentum k1 + L k2)."""
        B, Nm, sts = self._sym_args(params, spins, logpsi_ref)
        need = int(self.lib.sym_h_workspace_bytes(self.h, B))
        if workspace is None or workspace.numel() < need:
            workspace = torch.empty(need, dtype=torch.uint8, device=spins.device)
        Bt = torch.empty(self.N, Nm, B, dtype=self.cdtype, device=spins.device)
        HBt = torch.empty_like(Bt)
        hp = (ctypes.c_double * 3)(*[float(v) for v in hprime])
        self._check(self.lib.sym_hbtilde(self.h, sts, Nm, _ptr(spins), _ptr(logpsi_ref), B, hp,
                                         _ptr(workspace), need, _ptr(Bt), _ptr(HBt)),
                    "sym_hbtilde")
        return Bt, HBt

    def cheb_spectrum(self, mu, a, Wp, omega, jackson=True):
        """A(omega) of Eq. (Aw) (complex128 [len(omega)]) from the moments mu."""
        for t, name in ((mu, "mu"), (omega, "omega")):
            if not (t.is_cuda and t.is_contiguous()):
                raise ValueError(f"{name}: need a contiguous CUDA tensor")
        if mu.dtype != torch.complex128 or omega.dtype != torch.float64:
            raise ValueError("mu: complex128, omega: float64")
        out = torch.empty(omega.numel(), dtype=torch.complex128, device=omega.device)
        self._check(self.lib.cheb_spectrum(self.h, _ptr(mu), mu.numel(), float(a), float(Wp),
                                           1 if jackson else 0, _ptr(omega), omega.numel(),
                                           _ptr(out)), "cheb_spectrum")
        return out

    def cheb_extrapolate(self, mu, order, n0, n_out, reg=1e-12, roots_out=None, info_out=None):
        """Linear prediction of the moments mu (CUDA complex128 [n_known] or
        [n_seq, n_known]) to n_out moments; returns complex128 [.., n_out]."""
        if not (mu.dtype == torch.complex128 and mu.is_cuda and mu.is_contiguous()):
            raise ValueError("mu: need contiguous CUDA complex128")
        m2 = mu.reshape(-1, mu.shape[-1])
        n_seq, n_known = m2.shape
        out = torch.empty(n_seq, n_out, dtype=torch.complex128, device=mu.device)
        for t, shape, dt in ((roots_out, (n_seq, order), torch.complex128),
                             (info_out, (n_seq,), torch.int32)):
            if t is not None and not (t.dtype == dt and t.is_cuda and t.numel() == shape[0] * (
                    shape[1] if len(shape) > 1 else 1)):
                raise ValueError("roots_out / info_out: wrong shape or dtype")
        self._check(self.lib.cheb_extrapolate(self.h, _ptr(m2), n_seq, n_known, order, n0,
                                              float(reg), n_out, _ptr(out), _ptr(roots_out),
                                              _ptr(info_out)), "cheb_extrapolate")
        return out.reshape(*mu.shape[:-1], n_out)

    def cheb_lorentzian(self, poles, weights, a, Wp, eta, omega):
        """The eta-broadened spectral function of the Krylov projection."""
        for t in (poles, weights, omega):
            if not (t.is_cuda and t.is_contiguous() and t.dtype == torch.float64):
                raise ValueError("poles, weights, omega: contiguous CUDA float64")
        out = torch.empty(omega.numel(), dtype=torch.float64, device=omega.device)
        self._check(self.lib.cheb_lorentzian(self.h, _ptr(poles), _ptr(weights), poles.numel(),
                                             float(a), float(Wp), float(eta), _ptr(omega),
                                             omega.numel(), _ptr(out)), "cheb_lorentzian")
        return out

    def cheb_moment(self, state, beta, q, spins, logpsi_ref, hprime=None, Bcol=None, HBcol=None,
                    mu_out=None):
        B = self._spins(spins)
        self._c(logpsi_ref, (B,), "logpsi_ref")
        self._c(Bcol, (B,), "Bcol")
        self._c(HBcol, (B,), "HBcol")
        if mu_out is not None and not (mu_out.dtype == torch.complex128 and mu_out.is_cuda):
            raise ValueError("mu_out: need a CUDA complex128 tensor")
        if not (beta.is_cuda and beta.dtype == torch.complex128):
            raise ValueError("beta: need a CUDA complex128 scalar")
        hp = (ctypes.c_double * 3)(*hprime) if hprime is not None else None
        self._check(self.lib.cheb_moment(self.h, ctypes.byref(state), _ptr(beta), float(q[0]),
                                         float(q[1]),
                                         _ptr(spins), _ptr(logpsi_ref), B, hp, _ptr(Bcol),
                                         _ptr(HBcol), _ptr(mu_out)), "cheb_moment")

    def cheb_gram(self, Bmat, HBmat, G_out, H_out, n_samples=None):
        """HBmat and H_out may both be None (G only)."""
        Nm, ld = Bmat.shape
        B = ld if n_samples is None else n_samples
        self._c(Bmat, (Nm, ld), "Bmat")
        self._c(HBmat, (Nm, ld), "HBmat")
        for t in (G_out, H_out):
            if t is not None and not (t.dtype == torch.complex128 and t.is_cuda
                                      and tuple(t.shape) == (Nm, Nm)):
                raise ValueError("G_out / H_out: need CUDA complex128 [Nm, Nm]")
        self._check(self.lib.cheb_gram(self.h, _ptr(Bmat), _ptr(HBmat), Nm, B, ld, _ptr(G_out),
                                       _ptr(H_out)), "cheb_gram")

    def cheb_krylov(self, G, H, cutoff, n_out, mu_out, poles_out, weights_out, rank_out=None):
        Nm = G.shape[0]
        self._check(self.lib.cheb_krylov(self.h, _ptr(G), _ptr(H), Nm, cutoff, n_out, _ptr(mu_out),
                                         _ptr(poles_out), _ptr(weights_out), _ptr(rank_out)),
                    "cheb_krylov")


def batch_run(iters, n_iter, stream):
    """cr_batch_run over a list of SeqIter structs (from Sequence.iter_desc);
    stream: the torch stream to fork from and join into."""
    lib = load()
    arr = (SeqIter * len(iters))(*iters)
    st = lib.cr_batch_run(arr, len(iters), int(n_iter), ctypes.c_void_p(stream.cuda_stream))
    if st != 0:
        msgs = {lib.cr_last_error(it.ctx).decode(errors="replace") for it in iters}
        raise CRError(f"cr_batch_run: {STATUS.get(st, st)}: {'; '.join(m for m in msgs if m)}")
